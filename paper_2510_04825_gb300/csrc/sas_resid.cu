// True relative residual ||A(p) x - b|| / ||b|| of full-length solutions for
// the affine family (the (max, median) statistic of Tables 3-4).  Two passes:
// per-(parameter, row-chunk) partial sums of squares, then a fixed-order sum
// per parameter, so the result does not depend on scheduling.
#include "sas_internal.cuh"

namespace sas {

struct ResTable {
  const int64_t* rp[SAS_MAX_TERMS];
  const int32_t* ci[SAS_MAX_TERMS];
  const double* va[SAS_MAX_TERMS];
};

template <typename T> __device__ inline T theta_res(int rule, int k, const double* p);
template <> __device__ inline double theta_res<double>(int rule, int k, const double* p) {
  (void)rule;
  return k == 0 ? 1.0 : p[k - 1];
}
template <> __device__ inline zd theta_res<zd>(int rule, int k, const double* p) {
  if (rule == SAS_THETA_PENCIL) return k == 0 ? mkz(-1.0, 0.0) : mkz(0.0, p[0]);
  if (rule == SAS_THETA_DELAY) {  // p = (omega, tau): (i omega, -1, -e^{i omega tau})
    if (k == 0) return mkz(0.0, p[0]);
    if (k == 1) return mkz(-1.0, 0.0);
    double sn, cs;
    sincos(p[0] * p[1], &sn, &cs);
    return mkz(-cs, -sn);
  }
  return mkz(k == 0 ? 1.0 : p[k - 1], 0.0);
}

constexpr int kResThreads = 256;
constexpr int kResChunks = 512;

template <typename T>
__global__ void __launch_bounds__(kResThreads) true_residual_partial(
    ResTable tb, int K, int rule, int dp, const double* params, int64_t n, const T* X, const T* b,
    double* part) {
  __shared__ double red[kResThreads / 32];
  const int64_t q = blockIdx.y;
  const T* x = X + q * n;
  T th[SAS_MAX_TERMS];
  for (int k = 0; k < K; ++k) th[k] = theta_res<T>(rule, k, params + q * dp);
  const int64_t per = (n + kResChunks - 1) / kResChunks;
  const int64_t i0 = blockIdx.x * per;
  const int64_t i1 = i0 + per < n ? i0 + per : n;
  double acc = 0.0, bacc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kResThreads) {
    T ax = zero<T>();
    for (int k = 0; k < K; ++k) {
      T row = zero<T>();
      for (int64_t e = tb.rp[k][i]; e < tb.rp[k][i + 1]; ++e) row += rscale(tb.va[k][e], x[tb.ci[k][e]]);
      ax += th[k] * row;
    }
    acc += absq(ax - b[i]);
    bacc += absq(b[i]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  acc = warp_sum(acc);
  bacc = warp_sum(bacc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) t += red[w];
    part[(q * kResChunks + blockIdx.x) * 2] = t;
  }
  __syncthreads();
  if (lane == 0) red[warp] = bacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kResThreads / 32; ++w) t += red[w];
    part[(q * kResChunks + blockIdx.x) * 2 + 1] = t;
  }
}

__global__ void true_residual_final(const double* part, int64_t m, double* rho) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m;
       q += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int c = 0; c < kResChunks; ++c) {
      a += part[(q * kResChunks + c) * 2];
      b += part[(q * kResChunks + c) * 2 + 1];
    }
    rho[q] = sqrt(a) / sqrt(b);
  }
}

cudaError_t launch_true_residual(const sas_ctx* c, const double* params, int64_t m, const void* X,
                                 double* rho, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  if (m > 65535) return cudaErrorInvalidValue;
  ResTable tb;
  for (int k = 0; k < SAS_MAX_TERMS; ++k) {
    tb.rp[k] = c->rowptr[k];
    tb.ci[k] = c->colind[k];
    tb.va[k] = c->values[k];
  }
  double* part = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&part, sizeof(double) * 2 * kResChunks * m, st);
  if (e != cudaSuccess) return e;
  dim3 grid(kResChunks, (unsigned)m);
  if (c->dtype == SAS_COMPLEX128)
    true_residual_partial<zd><<<grid, kResThreads, 0, st>>>(tb, c->K, c->theta_rule, c->dp, params,
                                                            c->n, (const zd*)X, (const zd*)c->b_full,
                                                            part);
  else
    true_residual_partial<double><<<grid, kResThreads, 0, st>>>(
        tb, c->K, c->theta_rule, c->dp, params, c->n, (const double*)X, (const double*)c->b_full,
        part);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    true_residual_final<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(part, m, rho);
    e = cudaGetLastError();
  }
  cudaFreeAsync(part, st);
  return e;
}

}  // namespace sas
