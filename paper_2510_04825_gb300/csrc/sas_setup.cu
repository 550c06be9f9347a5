// Setup-time kernels: the precomputed pieces of the online stage.
//
//  G_k = (A_k)_{J,:} S  for every affine term (Sec. 3.1: with A(p) affine in
//        theta, S A(p*) X is a theta-combination of matrices computed once;
//        Sec. 5.2.2 precomputes S X, S A_0 X, S A_1 X the same way),
//  b_J, the QoI vector c^T S (Sec. 5.2.2), and the float32 / tf32-split
//  copies used by the mixed form.
#include "sas_internal.cuh"

namespace sas {

// One CTA per (row of J, term k); threads over the r columns of S.
template <typename T>
__global__ void gather_blocks_kernel(const int64_t* __restrict__ J, int s, int r, int K,
                                     const T* __restrict__ S, int64_t ldS, const int64_t* const* rp,
                                     const int32_t* const* ci, const double* const* va, T* G) {
  const int i = blockIdx.x, k = blockIdx.y;
  const int64_t row = J[i];
  const int64_t e0 = rp[k][row], e1 = rp[k][row + 1];
  const int32_t* cols = ci[k];
  const double* vals = va[k];
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    T acc = zero<T>();
    for (int64_t e = e0; e < e1; ++e) acc += rscale(vals[e], S[(int64_t)cols[e] + (int64_t)j * ldS]);
    G[(size_t)k * s * r + (size_t)j * s + i] = acc;
  }
}

struct PtrTable {
  const int64_t* rp[SAS_MAX_TERMS];
  const int32_t* ci[SAS_MAX_TERMS];
  const double* va[SAS_MAX_TERMS];
};

cudaError_t launch_gather_blocks(const sas_ctx* c, cudaStream_t st) {
  PtrTable h;
  for (int k = 0; k < SAS_MAX_TERMS; ++k) {
    h.rp[k] = c->rowptr[k];
    h.ci[k] = c->colind[k];
    h.va[k] = c->values[k];
  }
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(PtrTable));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, &h, sizeof(PtrTable), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    PtrTable* dt = (PtrTable*)d;
    dim3 grid(c->s, c->K);
    if (c->dtype == SAS_COMPLEX128)
      gather_blocks_kernel<zd><<<grid, 128, 0, st>>>(c->J_dev, c->s, c->r, c->K, (const zd*)c->S,
                                                     c->ldS, dt->rp, dt->ci, dt->va, (zd*)c->G);
    else
      gather_blocks_kernel<double><<<grid, 128, 0, st>>>(c->J_dev, c->s, c->r, c->K,
                                                         (const double*)c->S, c->ldS, dt->rp,
                                                         dt->ci, dt->va, (double*)c->G);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(d);
  return e;
}

template <typename T>
__global__ void gather_rhs_kernel(const int64_t* J, int s, const T* b, T* bJ) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x) bJ[i] = b[J[i]];
}

// w_j = sum_i c_i S_ij (kind 1) or (1/n) sum_i S_ij (kind 2): one CTA per column,
// fixed-order reduction.
template <typename T, int NT>
__global__ void qoi_vector_kernel(const T* S, int64_t ldS, int64_t n, const double* cvec, int kind,
                                  T* w) {
  __shared__ T red[NT];
  const int j = blockIdx.x;
  T acc = zero<T>();
  for (int64_t i = threadIdx.x; i < n; i += NT) {
    const T v = S[i + (int64_t)j * ldS];
    acc += kind == SAS_QOI_TRANSPOSE ? rscale(cvec[i], v) : v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) w[j] = kind == SAS_QOI_MEAN ? rscale(1.0 / (double)n, red[0]) : red[0];
}

cudaError_t launch_gather_vectors(const sas_ctx* c, const double* cvec, cudaStream_t st) {
  const bool cplx = c->dtype == SAS_COMPLEX128;
  if (cplx)
    gather_rhs_kernel<zd><<<(c->s + 255) / 256, 256, 0, st>>>(c->J_dev, c->s, (const zd*)c->b_full,
                                                              (zd*)c->bJ);
  else
    gather_rhs_kernel<double><<<(c->s + 255) / 256, 256, 0, st>>>(
        c->J_dev, c->s, (const double*)c->b_full, (double*)c->bJ);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->qoi_kind != SAS_QOI_NONE) {
    if (cplx)
      qoi_vector_kernel<zd, 256><<<c->r, 256, 0, st>>>((const zd*)c->S, c->ldS, c->n, cvec,
                                                       c->qoi_kind, (zd*)c->wq);
    else
      qoi_vector_kernel<double, 256><<<c->r, 256, 0, st>>>((const double*)c->S, c->ldS, c->n, cvec,
                                                           c->qoi_kind, (double*)c->wq);
    e = cudaGetLastError();
  }
  return e;
}

__global__ void to_float_kernel(const double* a, float* b, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__device__ inline float tf32_round_d(float x) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// S (n x r column-major, float64) -> two float32 arrays laid out row-major
// n x rpad (row i's r values contiguous, zero padded): the tf32 high part and
// the float32 remainder.  This is the K-major operand layout of the
// tensor-core reconstruction.
__global__ void split_basis_kernel(const double* S, int64_t ldS, int64_t n, int r, int rpad,
                                   float* hi, float* lo) {
  const int64_t total = n * rpad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / rpad;
    const int k = (int)(idx % rpad);
    float h = 0.f, l = 0.f;
    if (k < r) {
      const float x = (float)S[i + (int64_t)k * ldS];
      h = tf32_round_d(x);
      l = x - h;
    }
    hi[idx] = h;
    lo[idx] = l;
  }
}

cudaError_t launch_make_mixed_copies(const sas_ctx* c, cudaStream_t st) {
  const int64_t mult = c->dtype == SAS_COMPLEX128 ? 2 : 1;
  const int64_t gcount = (int64_t)c->K * c->s * c->r * mult;
  to_float_kernel<<<256, 256, 0, st>>>((const double*)c->G, (float*)c->G32, gcount);
  to_float_kernel<<<8, 256, 0, st>>>((const double*)c->bJ, (float*)c->bJ32, (int64_t)c->s * mult);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->Shi) {
    const int rpad = (c->r + 31) / 32 * 32;
    split_basis_kernel<<<c->num_sms * 8, 256, 0, st>>>((const double*)c->S, c->ldS, c->n, c->r,
                                                        rpad, c->Shi, c->Slo);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace sas
