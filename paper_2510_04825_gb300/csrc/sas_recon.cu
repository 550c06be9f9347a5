// Reconstruction x_hat = S y for a batch of coefficient vectors (Alg. 1 step 4:
// "output X c").  out[j*n + i] = sum_k S[i, k] Y[j, k].
//
// float64 form: CUDA-core DFMA, bound by the float64 pipe (2 n r flops per
// parameter).  Each thread owns one row i of S and JB columns of the output;
// the JB x r slab of Y sits in shared memory and is read as broadcasts.
#include "sas_internal.cuh"

namespace sas {

template <int JB, int NT>
__global__ void __launch_bounds__(NT) reconstruct_f64_kernel(const double* __restrict__ S,
                                                             int64_t ldS, int64_t n, int r,
                                                             const double* __restrict__ Y,
                                                             int64_t m, double* __restrict__ out) {
  __shared__ __align__(16) double Ys[kMaxR * JB];
  const int64_t j0 = (int64_t)blockIdx.y * JB;
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int jb = (int)(m - j0 < JB ? m - j0 : JB);
  for (int idx = threadIdx.x; idx < r * JB; idx += NT) {
    const int k = idx / JB, jj = idx % JB;
    Ys[idx] = jj < jb ? Y[(j0 + jj) * r + k] : 0.0;
  }
  __syncthreads();
  if (i >= n) return;
  double acc[JB];
#pragma unroll
  for (int jj = 0; jj < JB; ++jj) acc[jj] = 0.0;
  const double* srow = S + i;
  for (int k = 0; k < r; ++k) {
    const double sk = srow[(int64_t)k * ldS];
    const double2* yk = reinterpret_cast<const double2*>(Ys + k * JB);
#pragma unroll
    for (int jj = 0; jj < JB / 2; ++jj) {
      const double2 yy = yk[jj];
      acc[2 * jj] = fma(sk, yy.x, acc[2 * jj]);
      acc[2 * jj + 1] = fma(sk, yy.y, acc[2 * jj + 1]);
    }
  }
#pragma unroll
  for (int jj = 0; jj < JB; ++jj)
    if (jj < jb) out[(j0 + jj) * n + i] = acc[jj];
}

cudaError_t launch_reconstruct_f64(const sas_ctx* c, const void* Y, int64_t m, void* out,
                                   cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  constexpr int JB = 16, NT = 256;
  if ((m + JB - 1) / JB > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((c->n + NT - 1) / NT), (unsigned)((m + JB - 1) / JB));
  reconstruct_f64_kernel<JB, NT><<<grid, NT, 0, st>>>((const double*)c->S, c->ldS, c->n, c->r,
                                                       (const double*)Y, m, (double*)out);
  return cudaGetLastError();
}

// Mixed form, CUDA-core fallback: float32 FMA on the split operands
// (hi + lo of S and of y).  Rows of S are K-major (n x rpad).
template <int JB, int NT>
__global__ void __launch_bounds__(NT) reconstruct_mixed_simt_kernel(
    const float* __restrict__ Shi, const float* __restrict__ Slo, int64_t n, int r, int rpad,
    const float* __restrict__ ys, int64_t m, float* __restrict__ out) {
  __shared__ float Ys[kMaxR * JB];
  const int64_t j0 = (int64_t)blockIdx.y * JB;
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int jb = (int)(m - j0 < JB ? m - j0 : JB);
  for (int idx = threadIdx.x; idx < r * JB; idx += NT) {
    const int k = idx / JB, jj = idx % JB;
    Ys[idx] = jj < jb ? ys[(j0 + jj) * rpad + k] + ys[(size_t)m * rpad + (j0 + jj) * rpad + k] : 0.f;
  }
  __syncthreads();
  if (i >= n) return;
  float acc[JB];
#pragma unroll
  for (int jj = 0; jj < JB; ++jj) acc[jj] = 0.f;
  for (int k = 0; k < r; ++k) {
    const float sk = Shi[i * rpad + k] + Slo[i * rpad + k];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) acc[jj] = fmaf(sk, Ys[k * JB + jj], acc[jj]);
  }
#pragma unroll
  for (int jj = 0; jj < JB; ++jj)
    if (jj < jb) out[(j0 + jj) * n + i] = acc[jj];
}

cudaError_t launch_reconstruct_mixed(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                                     cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  if (c->recon_kernel != 1 && reconstruct_tc_supported(c))
    return launch_reconstruct_tc(c, ysplit, m, out, st);
  if (c->recon_kernel >= 2) return cudaErrorNotSupported;
  constexpr int JB = 16, NT = 256;
  const int rpad = (c->r + 31) / 32 * 32;
  if ((m + JB - 1) / JB > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((c->n + NT - 1) / NT), (unsigned)((m + JB - 1) / JB));
  reconstruct_mixed_simt_kernel<JB, NT><<<grid, NT, 0, st>>>(c->Shi, c->Slo, c->n, c->r, rpad,
                                                              ysplit, m, out);
  return cudaGetLastError();
}

// y (m x r float64) -> tf32 split [2][m][rpad]: the rounded part and the
// float32 remainder, zero padded to rpad columns.
__global__ void split_y_kernel(const double* Y, int64_t m, int r, int rpad, float* ys) {
  const int64_t total = m * rpad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx / rpad;
    const int i = (int)(idx % rpad);
    float hi = 0.f, lo = 0.f;
    if (i < r) {
      const float yf = (float)Y[q * r + i];
      uint32_t u = __float_as_uint(yf);
      u = (u + 0x1000u) & 0xffffe000u;
      hi = __uint_as_float(u);
      lo = yf - hi;
    }
    ys[idx] = hi;
    ys[total + idx] = lo;
  }
}

cudaError_t launch_split_y(const double* Y, int64_t m, int r, int rpad, float* ysplit,
                           cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  const int64_t total = m * rpad;
  const unsigned grid = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  split_y_kernel<<<grid, 256, 0, st>>>(Y, m, r, rpad, ysplit);
  return cudaGetLastError();
}

}  // namespace sas
