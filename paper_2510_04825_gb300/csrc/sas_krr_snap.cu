// Snapshots of the Gaussian-kernel family (Alg. 1 step 1 for Sec. 5.3):
//     (K_sigma + lambda I) x = b,  K_sigma(x, x') = exp(-|x - x'|^2 / (2 sigma^2)),
// on a grid of sigma values x lambda values, by multishift conjugate gradients.
//
// For one sigma the systems of all lambda_j differ by a multiple of the identity, so they
// share one Krylov space: CG runs on the seed system with the smallest lambda_0, and every
// other shift s_j = lambda_j - lambda_0 follows from scalar recurrences (its residual is
// zeta_j times the seed's; Jegerlehner's shifted CG).  Each iteration costs one product
// K_sigma p per sigma, whatever the number of lambda values; all sigma of the grid advance
// together, so one launch forms each distance once for every sigma.  A shift stops (its
// iterate, direction and scalars are frozen) once its recurrence residual |zeta_j| ||r|| is
// at most tol ||b||; a sigma stops when all of its shifts have.
//
// Arithmetic: float64 throughout.  The kernel product forms the squared distances from direct
// coordinate differences (no norm expansion, so nearby points keep full accuracy) and the
// entries with exp(): the snapshots are float64-accurate solutions.  The product is a
// matrix-vector product per sigma (one Krylov vector), whose cost is the N^2 distances and
// exponentials, not the multiply-adds; it runs on the CUDA cores.  The returned residuals
// are true float64 residuals ||(K + lambda I) x - b|| / ||b|| from one more product.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sas_internal.cuh"

namespace sas {
namespace ksnap {

constexpr int kRowsPerCta = 128;
constexpr int kChunk = 64;    // points staged in shared memory per step
constexpr int kMaxSig = 16;   // sigma values per product launch
constexpr int kMaxCols = 32;  // columns per product launch
constexpr int kMaxD = 16;

struct MatvecArgs {
  const double* X;  // N x d row-major
  int64_t N;
  int d, ns, nc;
  double inv2s2[kMaxSig];  // 1 / (2 sigma^2)
  int colsig[kMaxCols];    // sigma index of each column
  const double* P;         // column c at P + c * ld
  double* Q;               // Q[c] = K_{sigma(c)} P[c]
  int64_t ld;
};

// Q[c][i] = sum_j exp(-|x_i - x_j|^2 inv2s2[colsig[c]]) P[c][j]: one thread per row i; the
// points and the columns' values stream through shared memory in chunks.  Columns must come
// grouped by sigma (colsig nondecreasing).
__global__ void __launch_bounds__(kRowsPerCta) kmatvec_kernel(MatvecArgs a) {
  __shared__ double xs[kChunk * kMaxD];
  __shared__ double ps[kMaxCols * kChunk];
  const int64_t i = (int64_t)blockIdx.x * kRowsPerCta + threadIdx.x;
  const bool row_ok = i < a.N;
  double xi[kMaxD];
#pragma unroll
  for (int k = 0; k < kMaxD; ++k) xi[k] = (row_ok && k < a.d) ? a.X[i * a.d + k] : 0.0;
  double acc[kMaxCols];
#pragma unroll
  for (int c = 0; c < kMaxCols; ++c) acc[c] = 0.0;
  for (int64_t j0 = 0; j0 < a.N; j0 += kChunk) {
    const int nj = (int)(a.N - j0 < kChunk ? a.N - j0 : kChunk);
    __syncthreads();
    for (int t = threadIdx.x; t < nj * a.d; t += kRowsPerCta) xs[t] = a.X[j0 * a.d + t];
    for (int t = threadIdx.x; t < a.nc * kChunk; t += kRowsPerCta) {
      const int c = t / kChunk, jj = t % kChunk;
      ps[t] = jj < nj ? a.P[c * a.ld + j0 + jj] : 0.0;
    }
    __syncthreads();
    for (int jj = 0; jj < nj; ++jj) {
      double d2 = 0.0;
#pragma unroll
      for (int k = 0; k < kMaxD; ++k) {
        if (k < a.d) {
          const double df = xi[k] - xs[jj * a.d + k];
          d2 = fma(df, df, d2);
        }
      }
      // columns come grouped by sigma: one exponential per group
      double e = 0.0;
      int cur = -1;
#pragma unroll
      for (int c = 0; c < kMaxCols; ++c) {
        if (c < a.nc) {
          const int q = a.colsig[c];
          if (q != cur) {
            e = exp(-d2 * a.inv2s2[q]);
            cur = q;
          }
          acc[c] = fma(e, ps[c * kChunk + jj], acc[c]);
        }
      }
    }
  }
  if (row_ok) {
#pragma unroll
    for (int c = 0; c < kMaxCols; ++c)
      if (c < a.nc) a.Q[c * a.ld + i] = acc[c];
  }
}

// out[c] = partial sums of a[c] . b[c] per block (gridDim.x blocks per column c = blockIdx.y)
__global__ void dots_kernel(const double* A, const double* B, int64_t N, int64_t ld, double* out) {
  __shared__ double red[8];
  const int c = blockIdx.y;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(A[c * ld + i], B[c * ld + i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
    out[c * gridDim.x + blockIdx.x] = t;
  }
}

// Ap[s] = Q[s] + lambda0 pseed[s] (in place in Q)
__global__ void add_shift_kernel(double* Q, const double* Ps, double lam0, int64_t N, int64_t ld, int ns) {
  const int64_t total = (int64_t)ns * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / N, i = t % N;
    Q[s * ld + i] = fma(lam0, Ps[s * ld + i], Q[s * ld + i]);
  }
}

// x[s, j] += as[s, j] p[s, j] (as = 0 for frozen shifts); r[s] -= a[s] Ap[s]
__global__ void update_xr_kernel(double* Xs, int64_t ldx, const double* Pj, const double* as, int nl, double* R,
                                 const double* Ap, const double* a, int64_t N, int64_t ld, int ns) {
  const int64_t total = (int64_t)ns * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / N, i = t % N;
    if (a[s] == 0.0) continue;  // this sigma has stopped
    for (int j = 0; j < nl; ++j) {
      const double c = as[s * nl + j];
      if (c != 0.0) {
        const int64_t col = s * nl + j;
        Xs[col * ldx + i] = fma(c, Pj[col * ld + i], Xs[col * ldx + i]);
      }
    }
    R[s * ld + i] = fma(-a[s], Ap[s * ld + i], R[s * ld + i]);
  }
}

// p[s, j] = zeta[s, j] r[s] + bs[s, j] p[s, j] (active shifts); pseed[s] = r[s] + b[s] pseed[s]
__global__ void update_p_kernel(double* Pj, const double* zeta, const double* bs, const int* act, int nl,
                                const double* R, double* Ps, const double* b, const int* sact, int64_t N,
                                int64_t ld, int ns) {
  const int64_t total = (int64_t)ns * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / N, i = t % N;
    if (!sact[s]) continue;
    const double rv = R[s * ld + i];
    for (int j = 0; j < nl; ++j) {
      const int64_t col = s * nl + j;
      if (act[col]) Pj[col * ld + i] = fma(zeta[col], rv, bs[col] * Pj[col * ld + i]);
    }
    Ps[s * ld + i] = fma(b[s], Ps[s * ld + i], rv);
  }
}

// columns c of C = b (every column starts from the same right-hand side)
__global__ void fill_cols_kernel(double* C, const double* b, int64_t N, int64_t ld, int nc) {
  const int64_t total = (int64_t)nc * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    C[(t / N) * ld + t % N] = b[t % N];
}

// res[c] = (K x)[c] + lambda[c] x[c] - b (in place in Q)
__global__ void residual_cols_kernel(double* Q, const double* Xs, int64_t ldx, const double* lam, const double* b,
                                     int64_t N, int64_t ld, int nc) {
  const int64_t total = (int64_t)nc * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / N, i = t % N;
    Q[c * ld + i] = fma(lam[c], Xs[c * ldx + i], Q[c * ld + i]) - b[i];
  }
}

}  // namespace ksnap

namespace {

template <typename T>
struct Buf {
  T* p = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { cudaFree(p); }
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * (n ? n : 1)); }
};

int ew_grid(int64_t total) { return (int)std::min<int64_t>(4096, (total + 255) / 256); }

// Q[c] = K_{sigma(c)} P[c] for nc <= kMaxCols columns grouped by sigma
cudaError_t matvec(const double* X, int64_t N, int d, const std::vector<double>& sig, const int* colsig, int nc,
                   const double* P, int64_t ldp, double* Q, int64_t ldq, cudaStream_t st) {
  ksnap::MatvecArgs a{};
  a.X = X;
  a.N = N;
  a.d = d;
  a.ns = (int)sig.size();
  a.nc = nc;
  for (int q = 0; q < a.ns; ++q) a.inv2s2[q] = 1.0 / (2.0 * sig[q] * sig[q]);
  for (int c = 0; c < nc; ++c) a.colsig[c] = colsig[c];
  // the kernel reads P and writes Q with one leading dimension: copy-free when they agree
  if (ldp != ldq) return cudaErrorInvalidValue;
  a.P = P;
  a.Q = Q;
  a.ld = ldq;
  ksnap::kmatvec_kernel<<<(unsigned)((N + ksnap::kRowsPerCta - 1) / ksnap::kRowsPerCta), ksnap::kRowsPerCta, 0,
                          st>>>(a);
  return cudaGetLastError();
}

// host sums of the per-block partial dot products of ncols column pairs
cudaError_t dots(const double* A, const double* B, int64_t N, int64_t ld, int ncols, double* part,
                 std::vector<double>& out, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>(256, (N + 255) / 256);
  ksnap::dots_kernel<<<dim3(nb, ncols), 256, 0, st>>>(A, B, N, ld, part);
  cudaError_t e = cudaGetLastError();
  std::vector<double> h((size_t)nb * ncols);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  out.assign(ncols, 0.0);
  for (int c = 0; c < ncols; ++c)
    for (int b = 0; b < nb; ++b) out[c] += h[(size_t)c * nb + b];
  return e;
}

}  // namespace

sas_status krr_snapshots(const sas_kernel_desc* d, const double* sigma, int32_t ns, const double* lambda,
                         int32_t nl, double tol, int32_t maxit, double* Xout, int64_t ldx, int32_t* iters_out,
                         double* relres_out, cudaStream_t st) {
  const int64_t N = d->n;
  const int dim = d->d;
  const int nc = ns * nl;
  std::vector<double> sig(sigma, sigma + ns), lam(lambda, lambda + nl);
  const double lam0 = *std::min_element(lam.begin(), lam.end());
  std::vector<double> shift(nl);
  for (int j = 0; j < nl; ++j) shift[j] = lam[j] - lam0;
  Buf<double> Pj, R, Ps, Q, part, coef;
  Buf<int> flags;
  const int nbmax = (int)std::min<int64_t>(256, (N + 255) / 256);
  const int qcols = std::max(ns, std::min(nc, ksnap::kMaxCols));
  cudaError_t e = Pj.alloc((size_t)nc * N);
  if (e == cudaSuccess) e = R.alloc((size_t)ns * N);
  if (e == cudaSuccess) e = Ps.alloc((size_t)ns * N);
  if (e == cudaSuccess) e = Q.alloc((size_t)qcols * N);
  if (e == cudaSuccess) e = part.alloc((size_t)nbmax * qcols);
  if (e == cudaSuccess) e = coef.alloc((size_t)3 * nc + 2 * ns + nc);  // as, zeta, bs, a, b, lam per column
  if (e == cudaSuccess) e = flags.alloc((size_t)nc + ns);              // act per shift, sact per sigma
  if (e != cudaSuccess) {
    set_error(std::string("krr_snapshots: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
  }
  double* d_as = coef.p;
  double* d_zeta = d_as + nc;
  double* d_bs = d_zeta + nc;
  double* d_a = d_bs + nc;
  double* d_b = d_a + ns;
  double* d_lam = d_b + ns;
  int* d_act = flags.p;
  int* d_sact = flags.p + nc;
  // x = 0, r = p_seed = p_j = b
  for (int c = 0; c < nc && e == cudaSuccess; ++c)
    e = cudaMemsetAsync(Xout + (int64_t)c * ldx, 0, sizeof(double) * N, st);
  if (e == cudaSuccess) {
    ksnap::fill_cols_kernel<<<ew_grid((int64_t)nc * N), 256, 0, st>>>(Pj.p, d->b, N, N, nc);
    ksnap::fill_cols_kernel<<<ew_grid((int64_t)ns * N), 256, 0, st>>>(R.p, d->b, N, N, ns);
    ksnap::fill_cols_kernel<<<ew_grid((int64_t)ns * N), 256, 0, st>>>(Ps.p, d->b, N, N, ns);
    e = cudaGetLastError();
  }
  std::vector<double> bb;
  if (e == cudaSuccess) e = dots(d->b, d->b, N, 0, 1, part.p, bb, st);
  if (e != cudaSuccess) {
    set_error(std::string("krr_snapshots: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  const double bnorm = std::sqrt(bb[0]);
  if (!(bnorm > 0.0)) {
    set_error("krr_snapshots: b = 0");
    return SAS_EINVAL;
  }
  // host scalars of the seed CG per sigma and of every shift
  std::vector<double> rr(ns, bb[0]), a_old(ns, 1.0), b_old(ns, 0.0);
  std::vector<double> zeta(nc, 1.0), zeta_old(nc, 1.0), zeta_new(nc, 1.0), as(nc), bs(nc), av(ns), bv(ns);
  std::vector<int> act(nc, 1), sact(ns, 1), its(nc, 0), broke(ns, 0);
  std::vector<int> ident(ns);
  for (int s = 0; s < ns; ++s) ident[s] = s;
  std::vector<double> pAp, rrn;
  int k = 0;
  for (; k < maxit && e == cudaSuccess; ++k) {
    bool any = false;
    for (int s = 0; s < ns; ++s) any = any || sact[s];
    if (!any) break;
    // Ap = (K + lambda_0 I) p_seed for every sigma
    e = matvec(d->X, N, dim, sig, ident.data(), ns, Ps.p, N, Q.p, N, st);
    if (e != cudaSuccess) break;
    ksnap::add_shift_kernel<<<ew_grid((int64_t)ns * N), 256, 0, st>>>(Q.p, Ps.p, lam0, N, N, ns);
    e = dots(Ps.p, Q.p, N, N, ns, part.p, pAp, st);
    if (e != cudaSuccess) break;
    for (int s = 0; s < ns; ++s) {
      av[s] = 0.0;
      for (int j = 0; j < nl; ++j) as[s * nl + j] = 0.0;
      if (!sact[s]) continue;
      if (!(pAp[s] > 0.0) || !std::isfinite(pAp[s])) {  // breakdown: stop this sigma
        sact[s] = 0;
        broke[s] = 1;
        continue;
      }
      const double a = rr[s] / pAp[s];
      av[s] = a;
      for (int j = 0; j < nl; ++j) {
        const int c = s * nl + j;
        if (!act[c]) continue;
        const double den = a * b_old[s] * (zeta_old[c] - zeta[c]) + zeta_old[c] * a_old[s] * (1.0 + shift[j] * a);
        zeta_new[c] = zeta[c] * zeta_old[c] * a_old[s] / den;
        as[c] = a * zeta_new[c] / zeta[c];
      }
    }
    e = cudaMemcpyAsync(d_as, as.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_a, av.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
    ksnap::update_xr_kernel<<<ew_grid((int64_t)ns * N), 256, 0, st>>>(Xout, ldx, Pj.p, d_as, nl, R.p, Q.p, d_a, N,
                                                                        N, ns);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = dots(R.p, R.p, N, N, ns, part.p, rrn, st);
    if (e != cudaSuccess) break;
    for (int s = 0; s < ns; ++s) {
      bv[s] = 0.0;
      if (!sact[s]) continue;
      const double b = rrn[s] / rr[s];
      bv[s] = b;
      bool still = false;
      for (int j = 0; j < nl; ++j) {
        const int c = s * nl + j;
        if (!act[c]) continue;
        bs[c] = b * (zeta_new[c] / zeta[c]) * (zeta_new[c] / zeta[c]);
        zeta_old[c] = zeta[c];
        zeta[c] = zeta_new[c];
        its[c] = k + 1;
        if (std::fabs(zeta[c]) * std::sqrt(rrn[s]) <= tol * bnorm || !std::isfinite(zeta[c])) act[c] = 0;
        still = still || act[c];
      }
      a_old[s] = av[s];
      b_old[s] = b;
      rr[s] = rrn[s];
      sact[s] = still ? 1 : 0;
    }
    e = cudaMemcpyAsync(d_zeta, zeta.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bs, bs.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_b, bv.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_act, act.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sact, sact.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
    ksnap::update_p_kernel<<<ew_grid((int64_t)ns * N), 256, 0, st>>>(Pj.p, d_zeta, d_bs, d_act, nl, R.p, Ps.p, d_b,
                                                                       d_sact, N, N, ns);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors above are reused
  }
  if (e != cudaSuccess) {
    set_error(std::string("krr_snapshots: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  // true residuals ||(K_sigma + lambda I) x - b|| / ||b||, up to kMaxCols columns per product
  std::vector<double> lamc(nc);
  for (int c = 0; c < nc; ++c) lamc[c] = lam[c % nl];
  e = cudaMemcpyAsync(d_lam, lamc.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, st);
  const int per = std::max(1, std::min(ksnap::kMaxCols, qcols) / nl) * nl;  // whole sigma groups
  std::vector<double> res(nc, 0.0);
  for (int c0 = 0; c0 < nc && e == cudaSuccess; c0 += per) {
    const int cn = std::min(per, nc - c0);
    std::vector<int> cs(cn);
    for (int c = 0; c < cn; ++c) cs[c] = (c0 + c) / nl;
    std::vector<double> sub(sig);
    // column c0 + c of Xout: copy into Pj's first columns with leading dimension N
    for (int c = 0; c < cn && e == cudaSuccess; ++c)
      e = cudaMemcpyAsync(Pj.p + (int64_t)c * N, Xout + (int64_t)(c0 + c) * ldx, sizeof(double) * N,
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = matvec(d->X, N, dim, sub, cs.data(), cn, Pj.p, N, Q.p, N, st);
    if (e != cudaSuccess) break;
    ksnap::residual_cols_kernel<<<ew_grid((int64_t)cn * N), 256, 0, st>>>(Q.p, Pj.p, N, d_lam + c0, d->b, N, N, cn);
    std::vector<double> rq;
    e = dots(Q.p, Q.p, N, N, cn, part.p, rq, st);
    for (int c = 0; c < cn && e == cudaSuccess; ++c) res[c0 + c] = std::sqrt(rq[c]) / bnorm;
  }
  if (e != cudaSuccess) {
    set_error(std::string("krr_snapshots: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  int failed = 0;
  for (int c = 0; c < nc; ++c) {
    if (iters_out) iters_out[c] = its[c];
    if (relres_out) relres_out[c] = res[c];
    if (act[c] || broke[c / nl]) ++failed;
  }
  if (failed) {
    set_error("krr_snapshots: " + std::to_string(failed) + " of " + std::to_string(nc) +
              " systems did not reach the tolerance; X holds the last iterates");
    return SAS_ENOCONV;
  }
  return SAS_OK;
}

}  // namespace sas
