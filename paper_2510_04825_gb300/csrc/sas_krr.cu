// Gaussian-kernel rows for kernel ridge regression (Sec. 5.3):
//     M(sigma, lambda) = K_sigma(X_J, X) S + lambda S_J,
//     K_sigma(x, x') = exp(-|x - x'|^2 / (2 sigma^2)),
// formed on the fly for a batch of parameters without materialising any
// s x N kernel block in global memory (only the s rows at J are ever
// evaluated, the point of Sec. 3.1 "Computing S A(p*) X").
//
// One CTA computes a 32-row slab of M for one parameter, reducing over all N
// points in chunks of 64: the 32 x 64 kernel entries of a chunk are formed in
// shared memory from direct coordinate differences, then multiplied into the
// 32 x rpad accumulator (4 x 4 outputs per thread).
//  float64 form: exact differences, exp() of double, DFMA accumulation.
//  float32 form: float differences, ex2.approx, FFMA inside a chunk; every
//                chunk's partial sum is added to a float64 accumulator, so
//                the reduction over 200k points does not grow float32 error.
#include "sas_internal.cuh"

namespace sas {

constexpr int kKrrRows = 32;
constexpr int kKrrChunk = 64;
constexpr int kKrrThreads = 256;
constexpr int kKrrMaxD = 16;

template <typename T>
struct KrrArgs {
  const double* X;    // N x d row-major
  const double* XJ;   // s x d
  const double* S;    // N x r column-major, ldS
  const double* SJ;   // s x r column-major (ld s)
  const double* params;  // m x 2 (sigma, lambda)
  int64_t N;
  int64_t ldS;
  int d, r, s;
  int64_t m;
  double* M;          // m x (s x r) column-major per parameter (ld s)
};

__device__ inline float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Dynamic shared memory: coordinates of the 32 rows and of the 64 points of a
// chunk (float32 form: hi/lo pairs so that differences of nearby points keep
// float32 relative accuracy), the 32 x 64 kernel block and the 64 x 128 slab
// of S.
template <typename T>
__host__ __device__ constexpr size_t krr_smem_bytes() {
  return sizeof(T) * (2 * (kKrrRows + kKrrChunk) * kKrrMaxD + kKrrRows * (kKrrChunk + 1) +
                      kKrrChunk * kMaxR);
}

template <typename T>
__global__ void __launch_bounds__(kKrrThreads) krr_assemble_kernel(KrrArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xj_hi = reinterpret_cast<T*>(smem_raw);
  T* Xj_lo = Xj_hi + kKrrRows * kKrrMaxD;
  T* Xc_hi = Xj_lo + kKrrRows * kKrrMaxD;
  T* Xc_lo = Xc_hi + kKrrChunk * kKrrMaxD;
  T* E = Xc_lo + kKrrChunk * kKrrMaxD;       // [32][65]
  T* Sc = E + kKrrRows * (kKrrChunk + 1);    // [64][128]
  const int64_t q = blockIdx.x;
  const int row0 = blockIdx.y * kKrrRows;
  const int tid = threadIdx.x;
  const int d = a.d, r = a.r;
  const double sigma = a.params[q * 2], lambda = a.params[q * 2 + 1];
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const float scale2 = (float)(inv2s2 * 1.4426950408889634);  // log2(e) / (2 sigma^2)
  // thread tile: rows ty*4 + u (u < 4), columns tx + 32 v (v < 4)
  const int ty = tid >> 5, tx = tid & 31;
  for (int idx = tid; idx < kKrrRows * d; idx += kKrrThreads) {
    const int i = idx / d, k = idx % d;
    const double x = row0 + i < a.s ? a.XJ[(int64_t)(row0 + i) * d + k] : 0.0;
    Xj_hi[idx] = (T)x;
    Xj_lo[idx] = (T)(x - (double)(T)x);
  }
  double acc[4][4];
  T part[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int64_t c0 = 0; c0 < a.N; c0 += kKrrChunk) {
    const int cn = (int)(a.N - c0 < kKrrChunk ? a.N - c0 : kKrrChunk);
    __syncthreads();
    for (int idx = tid; idx < kKrrChunk * d; idx += kKrrThreads) {
      const int i = idx / d, k = idx % d;
      const double x = i < cn ? a.X[(c0 + i) * d + k] : 0.0;
      Xc_hi[idx] = (T)x;
      Xc_lo[idx] = (T)(x - (double)(T)x);
    }
    for (int idx = tid; idx < kKrrChunk * kMaxR; idx += kKrrThreads) {
      const int l = idx / kKrrChunk, i = idx % kKrrChunk;
      Sc[i * kMaxR + l] = (i < cn && l < r) ? (T)a.S[(c0 + i) + (int64_t)l * a.ldS] : T(0);
    }
    __syncthreads();
    for (int idx = tid; idx < kKrrRows * kKrrChunk; idx += kKrrThreads) {
      const int i = idx / kKrrChunk, k = idx % kKrrChunk;
      T d2 = T(0);
      for (int t = 0; t < d; ++t) {
        const T df = (Xj_hi[i * d + t] - Xc_hi[k * d + t]) + (Xj_lo[i * d + t] - Xc_lo[k * d + t]);
        d2 = fma(df, df, d2);
      }
      T e;
      if constexpr (sizeof(T) == 8) {
        e = exp(-d2 * inv2s2);
      } else {
        e = ex2_approx(-d2 * scale2);
      }
      E[i * (kKrrChunk + 1) + k] = k < cn ? e : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) part[u][v] = T(0);
    for (int k = 0; k < kKrrChunk; ++k) {
      T ev[4], sv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ev[u] = E[(ty * 4 + u) * (kKrrChunk + 1) + k];
#pragma unroll
      for (int v = 0; v < 4; ++v) sv[v] = Sc[k * kMaxR + tx + 32 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) part[u][v] = fma(ev[u], sv[v], part[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += (double)part[u][v];
  }
  double* Mq = a.M + q * (int64_t)a.s * r;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = row0 + ty * 4 + u;
    if (i >= a.s) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int l = tx + 32 * v;
      if (l < r) Mq[i + (int64_t)l * a.s] = acc[u][v] + lambda * a.SJ[i + (int64_t)l * a.s];
    }
  }
}

cudaError_t launch_krr_assemble(const sas_ctx* c, const double* params, int64_t m, double* M,
                                bool f32, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  if (m > 2147483647) return cudaErrorInvalidValue;
  dim3 grid((unsigned)m, (unsigned)((c->s + kKrrRows - 1) / kKrrRows));
  cudaError_t e;
  if (f32) {
    KrrArgs<float> a{c->X, c->XJ, (const double*)c->S, c->SJ, params, c->n, c->ldS, c->d, c->r, c->s, m, M};
    const size_t sm = krr_smem_bytes<float>();
    e = cudaFuncSetAttribute(krr_assemble_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    krr_assemble_kernel<float><<<grid, kKrrThreads, sm, st>>>(a);
  } else {
    KrrArgs<double> a{c->X, c->XJ, (const double*)c->S, c->SJ, params, c->n, c->ldS, c->d, c->r, c->s, m, M};
    const size_t sm = krr_smem_bytes<double>();
    e = cudaFuncSetAttribute(krr_assemble_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    krr_assemble_kernel<double><<<grid, kKrrThreads, sm, st>>>(a);
  }
  return cudaGetLastError();
}

__global__ void gather_kernel_rows(const int64_t* J, int s, int d, int r, const double* X,
                                   const double* S, int64_t ldS, const double* b, double* XJ,
                                   double* SJ, double* bJ) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < s * (d + r + 1);
       idx += gridDim.x * blockDim.x) {
    const int i = idx % s, c = idx / s;
    const int64_t row = J[i];
    if (c < d)
      XJ[(int64_t)i * d + c] = X[row * d + c];
    else if (c < d + r)
      SJ[i + (int64_t)(c - d) * s] = S[row + (int64_t)(c - d) * ldS];
    else
      bJ[i] = b[row];
  }
}

cudaError_t launch_gather_kernel_rows(const sas_ctx* c, cudaStream_t st) {
  gather_kernel_rows<<<64, 256, 0, st>>>(c->J_dev, c->s, c->d, c->r, c->X, (const double*)c->S,
                                         c->ldS, (const double*)c->b_full, c->XJ, c->SJ,
                                         (double*)c->bJ);
  return cudaGetLastError();
}

}  // namespace sas
