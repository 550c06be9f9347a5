// Row selection: column-pivoted QR on (A(p_sel) S)^T in rounds (Sec. 4.3 and
// Alg. 1 step 3; for s > r the union of pivot sets of Sec. 4.3.2).
//
// W holds V = A(p_sel) S row-major (row i = column i of V^T, r entries).  A
// step of round-local index t picks the alive row with the largest trailing
// norm ||W[i, t:r]|| (float64, summed in the fixed order j = t..r-1; exact
// ties go to the lowest row index), builds the Householder reflector of that
// row's trailing part and applies it to every alive row.  The trailing norm
// of a row after t reflectors equals its residual norm after projecting out
// the t rows already picked in the round.  Every round restarts from V with
// all earlier picks removed.  The whole loop runs on the device; the host
// only enqueues launches and reads J back once.
#include <cstring>
#include <vector>

#include "sas_internal.cuh"

namespace sas {

template <typename T> __device__ inline T theta_sel(int rule, int k, const double* p);
template <> __device__ inline double theta_sel<double>(int rule, int k, const double* p) {
  (void)rule;
  return k == 0 ? 1.0 : p[k - 1];
}
template <> __device__ inline zd theta_sel<zd>(int rule, int k, const double* p) {
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

struct SelTable {
  const int64_t* rp[SAS_MAX_TERMS];
  const int32_t* ci[SAS_MAX_TERMS];
  const double* va[SAS_MAX_TERMS];
  double p[SAS_MAX_TERMS];
};

// V[i*r + j] = sum_k theta_k (A_k S)[i, j]
template <typename T>
__global__ void apply_operator_kernel(const SelTable* tb, int K, int rule, const T* S, int64_t ldS,
                                      int64_t n, int r, T* V, int ldv) {
  const int64_t total = n * r;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / r;
    const int j = (int)(idx % r);
    T acc = zero<T>();
    for (int k = 0; k < K; ++k) {
      const int64_t* rp = tb->rp[k];
      const int32_t* ci = tb->ci[k];
      const double* va = tb->va[k];
      T part = zero<T>();
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) part += rscale(va[e], S[(int64_t)ci[e] + (int64_t)j * ldS]);
      acc += theta_sel<T>(rule, k, tb->p) * part;
    }
    V[i * ldv + j] = acc;
  }
}

struct Top2 {
  double v1;
  int64_t i1;
  double v2;
  int64_t i2;
};

__device__ inline bool better(double va, int64_t ia, double vb, int64_t ib) {
  return va > vb || (va == vb && ia < ib);
}

__device__ inline void top2_push(Top2& t, double v, int64_t i) {
  if (better(v, i, t.v1, t.i1)) {
    t.v2 = t.v1;
    t.i2 = t.i1;
    t.v1 = v;
    t.i1 = i;
  } else if (better(v, i, t.v2, t.i2)) {
    t.v2 = v;
    t.i2 = i;
  }
}

__device__ inline Top2 top2_merge(Top2 a, const Top2& b) {
  top2_push(a, b.v1, b.i1);
  top2_push(a, b.v2, b.i2);
  return a;
}

__device__ inline Top2 top2_empty() {
  Top2 t;
  t.v1 = -1.0;
  t.i1 = INT64_MAX;
  t.v2 = -1.0;
  t.i2 = INT64_MAX;
  return t;
}

constexpr int kSelThreads = 256;

// Optionally apply the reflector of the previous step (t-1) to every alive row,
// then compute trailing squared norms from index t and reduce the top two.
template <typename T>
__global__ void __launch_bounds__(kSelThreads) apply_and_norms_kernel(
    T* W, int64_t n, int r, int t, const uint8_t* alive, const T* refl, const double* tau,
    int apply, Top2* partial) {
  __shared__ Top2 red[kSelThreads / 32];
  Top2 best = top2_empty();
  const double tv = apply ? tau[0] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!alive[i]) continue;
    T* w = W + i * r;
    if (apply) {
      // reflector of step t-1 acts on entries t-1..r-1
      T d = zero<T>();
      for (int j = t - 1; j < r; ++j) d += conjv(refl[j - (t - 1)]) * w[j];
      const T f = rscale(tv, d);
      for (int j = t - 1; j < r; ++j) w[j] -= f * refl[j - (t - 1)];
    }
    double s2 = 0.0;
    for (int j = t; j < r; ++j) s2 += absq(w[j]);
    top2_push(best, s2, i);
  }
  // warp reduction of top-2 lists
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    Top2 other;
    other.v1 = __shfl_down_sync(0xffffffffu, best.v1, o);
    other.i1 = __shfl_down_sync(0xffffffffu, best.i1, o);
    other.v2 = __shfl_down_sync(0xffffffffu, best.v2, o);
    other.i2 = __shfl_down_sync(0xffffffffu, best.i2, o);
    if (lane + o < 32) best = top2_merge(best, other);
  }
  if (lane == 0) red[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    Top2 b = red[0];
    for (int w2 = 1; w2 < kSelThreads / 32; ++w2) b = top2_merge(b, red[w2]);
    partial[blockIdx.x] = b;
  }
}

// One block: final top-2, record the pick, build the reflector of row i* from t.
template <typename T>
__global__ void pick_kernel(T* W, int r, int t, uint8_t* alive, const Top2* partial, int nparts,
                            int64_t* J, double* gaps, int step, T* refl, double* tau, int* status) {
  __shared__ Top2 red[32];
  __shared__ int64_t piv;
  Top2 b = top2_empty();
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) b = top2_merge(b, partial[p]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    Top2 other;
    other.v1 = __shfl_down_sync(0xffffffffu, b.v1, o);
    other.i1 = __shfl_down_sync(0xffffffffu, b.i1, o);
    other.v2 = __shfl_down_sync(0xffffffffu, b.v2, o);
    other.i2 = __shfl_down_sync(0xffffffffu, b.i2, o);
    if (lane + o < 32) b = top2_merge(b, other);
  }
  if (lane == 0) red[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    Top2 f = red[0];
    const int nw = (blockDim.x + 31) / 32;
    for (int w2 = 1; w2 < nw; ++w2) f = top2_merge(f, red[w2]);
    if (!(f.v1 > 0.0) || f.i1 == INT64_MAX) {
      *status = SAS_ERANK;
      piv = -1;
    } else {
      const double top = sqrt(f.v1);
      const double second = f.v2 >= 0.0 ? sqrt(f.v2) : -1.0;
      gaps[step] = (top - second) / top;
      J[step] = f.i1;
      alive[f.i1] = 0;
      piv = f.i1;
    }
  }
  __syncthreads();
  if (piv < 0) return;
  if (threadIdx.x == 0) {
    const T* w = W + piv * r;
    double nrm2 = 0.0;
    for (int j = t; j < r; ++j) nrm2 += absq(w[j]);
    const T alpha = w[t];
    const double aa = sqrt(absq(alpha));
    const double nrm = sqrt(nrm2);
    const T beta = rscale(-nrm, phase(alpha));
    refl[0] = alpha - beta;
    for (int j = t + 1; j < r; ++j) refl[j - t] = w[j];
    tau[0] = nrm > 0.0 ? 1.0 / (nrm * (nrm + aa)) : 0.0;
  }
}

template <typename T>
__global__ void copy_kernel(const T* a, T* b, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void fill_u8_kernel(uint8_t* a, int64_t count, uint8_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// CPQR in rounds on V (device, n x r row-major); J_out / gap_out on the host.
template <typename T>
static sas_status cpqr_rounds(const T* V0, int64_t n, int r, int s, int64_t* J_out,
                              double* gap_out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nparts = sms * 4;
  void *W = nullptr, *alive = nullptr, *partial = nullptr;
  void *refl = nullptr, *tau = nullptr, *Jd = nullptr, *gd = nullptr, *stat = nullptr;
  sas_status rc = SAS_OK;
  cudaError_t e = cudaSuccess;
  const size_t vbytes = (size_t)n * r * sizeof(T);
#define SAS_TRY(x)                  \
  do {                              \
    e = (x);                        \
    if (e != cudaSuccess) goto done; \
  } while (0)
  SAS_TRY(cudaMalloc(&W, vbytes));
  SAS_TRY(cudaMalloc(&alive, (size_t)n));
  SAS_TRY(cudaMalloc(&partial, sizeof(Top2) * nparts));
  SAS_TRY(cudaMalloc(&refl, sizeof(T) * r));
  SAS_TRY(cudaMalloc(&tau, sizeof(double)));
  SAS_TRY(cudaMalloc(&Jd, sizeof(int64_t) * s));
  SAS_TRY(cudaMalloc(&gd, sizeof(double) * s));
  SAS_TRY(cudaMalloc(&stat, sizeof(int)));
  SAS_TRY(cudaMemset(stat, 0, sizeof(int)));
  fill_u8_kernel<<<sms * 4, 256>>>((uint8_t*)alive, n, 1);
  SAS_TRY(cudaGetLastError());
  {
    int step = 0;
    while (step < s) {
      copy_kernel<T><<<sms * 8, 256>>>(V0, (T*)W, (int64_t)n * r);
      const int k = (s - step) < r ? (s - step) : r;
      for (int t = 0; t < k; ++t, ++step) {
        apply_and_norms_kernel<T><<<nparts, kSelThreads>>>((T*)W, n, r, t, (const uint8_t*)alive,
                                                           (const T*)refl, (const double*)tau,
                                                           t > 0 ? 1 : 0, (Top2*)partial);
        pick_kernel<T><<<1, 512>>>((T*)W, r, t, (uint8_t*)alive, (const Top2*)partial, nparts,
                                   (int64_t*)Jd, (double*)gd, step, (T*)refl, (double*)tau,
                                   (int*)stat);
      }
      SAS_TRY(cudaGetLastError());
    }
  }
  SAS_TRY(cudaDeviceSynchronize());
  {
    int st = 0;
    SAS_TRY(cudaMemcpy(&st, stat, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
      rc = SAS_ERANK;
      set_error("select_rows: a round ran out of non-zero residuals (rank deficient A(p_sel) S)");
    }
  }
  SAS_TRY(cudaMemcpy(J_out, Jd, sizeof(int64_t) * s, cudaMemcpyDeviceToHost));
  if (gap_out) SAS_TRY(cudaMemcpy(gap_out, gd, sizeof(double) * s, cudaMemcpyDeviceToHost));
#undef SAS_TRY
done:
  if (e != cudaSuccess) {
    rc = e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
    set_error(std::string("select_rows: ") + cudaGetErrorString(e));
  }
  cudaFree(W);
  cudaFree(alive);
  cudaFree(partial);
  cudaFree(refl);
  cudaFree(tau);
  cudaFree(Jd);
  cudaFree(gd);
  cudaFree(stat);
  return rc;
}

template <typename T>
static sas_status select_t(const sas_affine_desc* d, const double* p_sel, int64_t* J_out,
                           double* gap_out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int dp = d->theta_rule == SAS_THETA_PENCIL ? 1 : d->theta_rule == SAS_THETA_DELAY ? 2 : d->K - 1;
  SelTable h;
  for (int k = 0; k < SAS_MAX_TERMS; ++k) {
    h.rp[k] = d->rowptr[k];
    h.ci[k] = d->colind[k];
    h.va[k] = d->values[k];
    h.p[k] = k < dp ? p_sel[k] : 0.0;
  }
  void *dtab = nullptr, *V0 = nullptr;
  cudaError_t e = cudaMalloc(&dtab, sizeof(SelTable));
  if (e == cudaSuccess) e = cudaMalloc(&V0, (size_t)d->n * d->r * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(dtab, &h, sizeof(SelTable), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    apply_operator_kernel<T><<<sms * 8, 256>>>((const SelTable*)dtab, d->K, d->theta_rule,
                                               (const T*)d->S, d->ldS, d->n, d->r, (T*)V0, d->r);
    e = cudaGetLastError();
  }
  sas_status rc = SAS_OK;
  if (e != cudaSuccess) {
    rc = e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
    set_error(std::string("select_rows: ") + cudaGetErrorString(e));
  } else {
    rc = cpqr_rounds<T>((const T*)V0, d->n, d->r, d->s, J_out, gap_out);
  }
  cudaFree(dtab);
  cudaFree(V0);
  return rc;
}

// Rows of A(p_sel) S (row-major, row stride ldv) for the leverage scores.
template <typename T>
static cudaError_t operator_rows_t(const sas_affine_desc* d, const double* p_sel, T* V, int ldv) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int dp = d->theta_rule == SAS_THETA_PENCIL ? 1 : d->theta_rule == SAS_THETA_DELAY ? 2 : d->K - 1;
  SelTable h;
  for (int k = 0; k < SAS_MAX_TERMS; ++k) {
    h.rp[k] = d->rowptr[k];
    h.ci[k] = d->colind[k];
    h.va[k] = d->values[k];
    h.p[k] = k < dp ? p_sel[k] : 0.0;
  }
  void* dtab = nullptr;
  cudaError_t e = cudaMalloc(&dtab, sizeof(SelTable));
  if (e == cudaSuccess) e = cudaMemcpy(dtab, &h, sizeof(SelTable), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    apply_operator_kernel<T><<<sms * 8, 256>>>((const SelTable*)dtab, d->K, d->theta_rule,
                                               (const T*)d->S, d->ldS, d->n, d->r, V, ldv);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dtab);
  return e;
}

cudaError_t operator_rows_affine(const sas_affine_desc* d, const double* p_sel, void* V, int ldv) {
  if (d->dtype == SAS_COMPLEX128) return operator_rows_t<zd>(d, p_sel, (zd*)V, ldv);
  return operator_rows_t<double>(d, p_sel, (double*)V, ldv);
}

// column-major n x r (ld n) -> row-major n x r
__global__ void to_row_major_kernel(const double* A, int64_t n, int r, double* B) {
  const int64_t total = n * r;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / r;
    const int j = (int)(idx % r);
    B[idx] = A[i + (int64_t)j * n];
  }
}

sas_status select_rows_kernel(const sas_kernel_desc* d, const double* p_sel, int64_t* J_out,
                              double* gap_out) {
  // V = (K_sigma + lambda I) S at p_sel, from the float64 kernel rows of every point
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sas_ctx tmp;
  std::memset((void*)&tmp, 0, sizeof(tmp));
  tmp.n = d->n;
  tmp.r = d->r;
  tmp.s = (int)d->n;
  tmp.d = d->d;
  tmp.X = d->X;
  tmp.XJ = const_cast<double*>(d->X);
  tmp.S = d->S;
  tmp.SJ = const_cast<double*>(d->S);
  tmp.ldS = d->ldS;
  void *Vc = nullptr, *Vr = nullptr, *pd = nullptr;
  cudaError_t e = cudaMalloc(&Vc, (size_t)d->n * d->r * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Vr, (size_t)d->n * d->r * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&pd, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(pd, p_sel, 2 * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d->ldS != d->n) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = launch_krr_assemble(&tmp, (const double*)pd, 1, (double*)Vc, false, 0);
  if (e == cudaSuccess) {
    to_row_major_kernel<<<sms * 8, 256>>>((const double*)Vc, d->n, d->r, (double*)Vr);
    e = cudaGetLastError();
  }
  sas_status rc = SAS_OK;
  if (e != cudaSuccess) {
    rc = e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
    set_error(std::string("select_rows_kernel: ") + cudaGetErrorString(e));
  } else {
    rc = cpqr_rounds<double>((const double*)Vr, d->n, d->r, d->s, J_out, gap_out);
  }
  cudaFree(Vc);
  cudaFree(Vr);
  cudaFree(pd);
  return rc;
}

sas_status select_rows_affine(const sas_affine_desc* d, const double* p_sel, int64_t* J_out,
                              double* gap_out) {
  if (d->dtype == SAS_COMPLEX128) return select_t<zd>(d, p_sel, J_out, gap_out);
  return select_t<double>(d, p_sel, J_out, gap_out);
}

}  // namespace sas
