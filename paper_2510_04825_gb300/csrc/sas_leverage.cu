// Leverage-score row sampling with weights (Sec. 4.3.2 and its footnote) and
// the weighted subsampled rows it leads to (Sec. 4.3.3).
//
// Scores: V = [A(p_sel) S, b] (n x (r+1)), thin QR V = QR, score_i = ||Q_i,:||^2,
// computed on the device in float64 by shifted CholeskyQR3 (Fukaya, Kannan,
// Nakatsukasa, Yamamoto, Yanagisawa 2020): three times G = V^H V (a reduction
// over the n rows), G (+ sigma I on the first pass) = R^H R on the host, and
// V <- V R^{-1}.  The first, shifted pass with sigma = 11 (n c + c (c+1)) u
// trace(G) brings kappa(V) down to ~u^{-1/2} whatever it was, so that the two
// plain passes that follow leave V = Q to working accuracy.
//
// Sampling (host): s draws with replacement by inverse CDF of pi = score /
// total on caller-supplied uniforms u in [0, 1).  C_i is the running sum of the
// scores in row order, total = C_{n-1}, cdf_i = C_i / total, and draw t is the
// first row with cdf_i > u_t.  A row drawn k times is kept once with weight
// sqrt(k / (s pi_i)), which is the same least-squares objective as k copies of
// weight 1/sqrt(s pi_i).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "sas_internal.cuh"

namespace sas {
namespace lev {

constexpr int kThreads = 256;
constexpr int kRows = 16;           // rows staged per block iteration of the Gram reduction
constexpr int kMaxPairs = 40;       // (129 * 130 / 2) / 256 rounded up: pairs per thread

__device__ inline double re_of(double v) { return v; }
__device__ inline double re_of(zd v) { return v.re; }
__device__ inline double im_of(double) { return 0.0; }
__device__ inline double im_of(zd v) { return v.im; }

template <typename T>
__global__ void put_rhs_kernel(const T* b, int64_t n, int ldv, T* V) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    V[i * ldv + ldv - 1] = b[i];
}

// G[a][b] += sum_rows conj(V[i][a]) V[i][b] for a <= b, float64 atomics into
// G (c x c real parts, then c x c imaginary parts).
template <typename T>
__global__ void __launch_bounds__(kThreads) gram_kernel(const T* V, int64_t n, int c, double* G) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* tile = reinterpret_cast<T*>(smraw);  // kRows x c
  const int npairs = c * (c + 1) / 2;
  int pa[kMaxPairs], pb[kMaxPairs];
  T acc[kMaxPairs];
  int mine = 0;
  for (int p = threadIdx.x; p < npairs && mine < kMaxPairs; p += kThreads) {
    int a = 0, off = 0;
    while (off + (c - a) <= p) {
      off += c - a;
      ++a;
    }
    pa[mine] = a;
    pb[mine] = a + (p - off);
    acc[mine] = zero<T>();
    ++mine;
  }
  for (int64_t r0 = (int64_t)blockIdx.x * kRows; r0 < n; r0 += (int64_t)gridDim.x * kRows) {
    const int rows = (int)(n - r0 < kRows ? n - r0 : kRows);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kRows * c; idx += kThreads) {
      const int rr = idx / c;
      tile[idx] = rr < rows ? V[(r0 + rr) * c + (idx % c)] : zero<T>();
    }
    __syncthreads();
    for (int q = 0; q < mine; ++q) {
      T sum = zero<T>();
      for (int rr = 0; rr < kRows; ++rr) sum += conjv(tile[rr * c + pa[q]]) * tile[rr * c + pb[q]];
      acc[q] += sum;
    }
  }
  for (int q = 0; q < mine; ++q) {
    atomicAdd(&G[pa[q] * c + pb[q]], re_of(acc[q]));
    if (sizeof(T) == 16) atomicAdd(&G[c * c + pa[q] * c + pb[q]], im_of(acc[q]));
  }
}

// W[i][j] = sum_{k <= j} V[i][k] Rinv[k][j] (row vector times an upper-triangular matrix)
template <typename T>
__global__ void right_trsm_kernel(const T* V, int64_t n, int c, const T* Rinv, T* W) {
  const int64_t total = n * c;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / c;
    const int j = (int)(idx % c);
    T sum = zero<T>();
    for (int k = 0; k <= j; ++k) sum += V[i * c + k] * Rinv[k * c + j];
    W[idx] = sum;
  }
}

template <typename T>
__global__ void row_norms_kernel(const T* V, int64_t n, int c, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s2 = 0.0;
    for (int j = 0; j < c; ++j) s2 += absq(V[i * c + j]);
    out[i] = s2;
  }
}

// Row weights of the subsample: G_k rows and b_J scaled by w.
template <typename T>
__global__ void weight_rows_kernel(T* G, int K, int s, int r, T* bJ, const double* w) {
  const int64_t total = (int64_t)K * s * r + s;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < (int64_t)K * s * r) {
      const int i = (int)(idx % s);
      G[idx] = rscale(w[i], G[idx]);
    } else {
      const int i = (int)(idx - (int64_t)K * s * r);
      bJ[i] = rscale(w[i], bJ[i]);
    }
  }
}

inline double conj_h(double v) { return v; }
inline std::complex<double> conj_h(std::complex<double> v) { return std::conj(v); }

// Host: upper Cholesky G = R^H R (G Hermitian positive definite, c x c), then R^{-1}.
template <typename C>
static bool cholesky_inverse(std::vector<C>& G, int c, std::vector<C>& Rinv) {
  std::vector<C> R((size_t)c * c, C(0));
  for (int j = 0; j < c; ++j) {
    double d = std::real(G[(size_t)j * c + j]);
    for (int k = 0; k < j; ++k) d -= std::norm(R[(size_t)k * c + j]);
    if (!(d > 0.0)) return false;
    const double rjj = std::sqrt(d);
    R[(size_t)j * c + j] = C(rjj);
    for (int l = j + 1; l < c; ++l) {
      C v = G[(size_t)j * c + l];
      for (int k = 0; k < j; ++k) v -= conj_h(R[(size_t)k * c + j]) * R[(size_t)k * c + l];
      R[(size_t)j * c + l] = v / rjj;
    }
  }
  Rinv.assign((size_t)c * c, C(0));
  for (int j = 0; j < c; ++j) {  // column j of R^{-1}: R x = e_j, upper triangular
    for (int i = j; i >= 0; --i) {
      C v = i == j ? C(1) : C(0);
      for (int k = i + 1; k <= j; ++k) v -= R[(size_t)i * c + k] * Rinv[(size_t)k * c + j];
      Rinv[(size_t)i * c + j] = v / R[(size_t)i * c + i];
    }
  }
  return true;
}

template <typename T, typename C>
static sas_status scores_t(const sas_affine_desc* d, const double* p_sel, double* scores) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int c = d->r + 1;
  const int64_t n = d->n;
  T *V = nullptr, *W = nullptr, *Rinv_d = nullptr;
  double *G = nullptr, *sc = nullptr;
  sas_status rc = SAS_OK;
  cudaError_t e = cudaMalloc(&V, (size_t)n * c * sizeof(T));
  if (e == cudaSuccess) e = cudaMalloc(&W, (size_t)n * c * sizeof(T));
  if (e == cudaSuccess) e = cudaMalloc(&Rinv_d, (size_t)c * c * sizeof(T));
  if (e == cudaSuccess) e = cudaMalloc(&G, (size_t)2 * c * c * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sc, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = operator_rows_affine(d, p_sel, V, c);
  if (e == cudaSuccess) {
    put_rhs_kernel<T><<<sms * 4, 256>>>((const T*)d->b, n, c, V);
    e = cudaGetLastError();
  }
  for (int pass = 0; pass < 3 && e == cudaSuccess && rc == SAS_OK; ++pass) {
    e = cudaMemset(G, 0, (size_t)2 * c * c * sizeof(double));
    if (e != cudaSuccess) break;
    const size_t smem = (size_t)kRows * c * sizeof(T);
    gram_kernel<T><<<sms * 4, kThreads, smem>>>(V, n, c, G);
    e = cudaGetLastError();
    std::vector<double> Gh((size_t)2 * c * c);
    if (e == cudaSuccess) e = cudaMemcpy(Gh.data(), G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    std::vector<C> Gc((size_t)c * c), Rinv;
    for (int a = 0; a < c; ++a)
      for (int b = a; b < c; ++b) {
        C v;
        if constexpr (sizeof(T) == 16)
          v = C(Gh[(size_t)a * c + b], Gh[(size_t)c * c + a * c + b]);
        else
          v = C(Gh[(size_t)a * c + b]);
        Gc[(size_t)a * c + b] = v;
        Gc[(size_t)b * c + a] = conj_h(v);
      }
    if (pass == 0) {  // the shift of the first pass
      double tr = 0.0;
      for (int a = 0; a < c; ++a) tr += std::real(Gc[(size_t)a * c + a]);
      const double sigma = 11.0 * ((double)n * c + (double)c * (c + 1)) * 0x1p-53 * tr;
      for (int a = 0; a < c; ++a) Gc[(size_t)a * c + a] += sigma;
    }
    if (!cholesky_inverse<C>(Gc, c, Rinv)) {
      rc = SAS_ERANK;
      set_error("leverage scores: [A(p_sel) S, b] is numerically rank deficient");
      break;
    }
    static_assert(sizeof(C) == sizeof(T), "host and device scalar layouts");
    e = cudaMemcpy(Rinv_d, Rinv.data(), (size_t)c * c * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    right_trsm_kernel<T><<<sms * 8, 256>>>(V, n, c, Rinv_d, W);
    e = cudaGetLastError();
    std::swap(V, W);
  }
  if (e == cudaSuccess && rc == SAS_OK) {
    row_norms_kernel<T><<<sms * 4, 256>>>(V, n, c, sc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(scores, sc, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess && rc == SAS_OK) {
    rc = e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
    set_error(std::string("leverage scores: ") + cudaGetErrorString(e));
  }
  cudaFree(V);
  cudaFree(W);
  cudaFree(Rinv_d);
  cudaFree(G);
  cudaFree(sc);
  return rc;
}

}  // namespace lev

cudaError_t launch_weight_rows(sas_ctx* c, const double* w_host, cudaStream_t st) {
  double* wd = nullptr;
  cudaError_t e = cudaMalloc(&wd, sizeof(double) * c->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(wd, w_host, sizeof(double) * c->s, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    if (c->dtype == SAS_COMPLEX128)
      lev::weight_rows_kernel<zd><<<c->num_sms * 2, 256, 0, st>>>((zd*)c->G, c->K, c->s, c->r,
                                                                  (zd*)c->bJ, wd);
    else
      lev::weight_rows_kernel<double><<<c->num_sms * 2, 256, 0, st>>>((double*)c->G, c->K, c->s,
                                                                      c->r, (double*)c->bJ, wd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(wd);
  return e;
}

}  // namespace sas

using namespace sas;

static sas_status lev_fail(sas_status code, const std::string& msg) {
  set_error(msg);
  return code;
}

static bool lev_is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

sas_status subapsnap_leverage_scores_affine(const sas_affine_desc* d, const double* p_sel,
                                            double* scores) {
  if (!d || !p_sel || !scores) return lev_fail(SAS_EINVAL, "NULL argument");
  if (d->n < 1 || d->r < 1 || d->r > kMaxR) return lev_fail(SAS_EINVAL, "need n >= 1 and 1 <= r <= 128");
  if ((int64_t)d->r + 1 > d->n) return lev_fail(SAS_EINVAL, "need r + 1 <= n");
  if (d->K < 1 || d->K > SAS_MAX_TERMS) return lev_fail(SAS_EINVAL, "K must be in [1, 8]");
  if (d->dtype != SAS_REAL64 && d->dtype != SAS_COMPLEX128) return lev_fail(SAS_EINVAL, "bad dtype");
  if (d->ldS < d->n) return lev_fail(SAS_EINVAL, "ldS < n");
  if (!lev_is_device(d->S) || !lev_is_device(d->b)) return lev_fail(SAS_EINVAL, "S and b must be device pointers");
  for (int k = 0; k < d->K; ++k)
    if (!lev_is_device(d->rowptr[k]) || !lev_is_device(d->colind[k]) || !lev_is_device(d->values[k]))
      return lev_fail(SAS_EINVAL, "CSR arrays must be device pointers");
  if (d->dtype == SAS_COMPLEX128) return lev::scores_t<zd, std::complex<double>>(d, p_sel, scores);
  return lev::scores_t<double, double>(d, p_sel, scores);
}

sas_status subapsnap_sample_rows_leverage(const double* scores, int64_t n, int32_t s,
                                          const double* u, int64_t* J_out, double* w_out,
                                          int32_t* count_out) {
  if (!scores || !u || !J_out || !w_out || !count_out) return lev_fail(SAS_EINVAL, "NULL argument");
  if (n < 1 || s < 1) return lev_fail(SAS_EINVAL, "need n >= 1 and s >= 1");
  std::vector<double> C((size_t)n);
  double run = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(scores[i] >= 0.0) || !std::isfinite(scores[i]))
      return lev_fail(SAS_EINVAL, "scores must be finite and non-negative");
    run += scores[i];
    C[(size_t)i] = run;
  }
  const double total = run;
  if (!(total > 0.0)) return lev_fail(SAS_EINVAL, "scores sum to zero");
  std::vector<double> cdf((size_t)n);
  for (int64_t i = 0; i < n; ++i) cdf[(size_t)i] = C[(size_t)i] / total;
  std::vector<int64_t> draws((size_t)s);
  for (int32_t t = 0; t < s; ++t) {
    if (!(u[t] >= 0.0 && u[t] < 1.0)) return lev_fail(SAS_EINVAL, "uniforms must lie in [0, 1)");
    int64_t i = (int64_t)(std::upper_bound(cdf.begin(), cdf.end(), u[t]) - cdf.begin());
    draws[(size_t)t] = i < n ? i : n - 1;
  }
  std::sort(draws.begin(), draws.end());
  int32_t k = 0;
  for (size_t a = 0; a < draws.size();) {
    size_t b = a;
    while (b < draws.size() && draws[b] == draws[a]) ++b;
    const int64_t i = draws[a];
    const double pi = scores[i] / total;
    J_out[k] = i;
    w_out[k] = std::sqrt((double)(b - a) / ((double)s * pi));
    ++k;
    a = b;
  }
  *count_out = k;
  return SAS_OK;
}
