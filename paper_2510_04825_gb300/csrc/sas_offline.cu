// Offline stage on the device (Alg. 1 steps 1-2): the snapshot solves
// A(p_j) x_j = b for a batch of snapshot parameters, and an orthonormal basis
// of their span.
//
// Snapshot solves.  Alg. 1 lets the snapshots be computed "fully or
// approximately".  Every family here is symmetric in the bilinear sense
// (A^T = A, complex entries allowed), so one Krylov method covers them:
// conjugate gradients with the unconjugated form x^T y (COCG; for a real SPD
// matrix this is plain CG), preconditioned by the diagonal of A(p_j) or, on
// grid families, by a fast Poisson solve; BiCGStab serves nonsymmetric A(p).  The
// batch runs every column at once: column j has its own theta(p_j), scalars
// alpha_j, beta_j and stopping test, and one launch of each kernel covers all
// active columns.  Convergence is declared on the float64 true residual only.
// In the mixed form the iterates are float32 and the residual is replaced by
// the float64 true one whenever it has fallen 10x.  The same routine refines
// any start vector, e.g. the SubApSnap output x_hat, which Sec. 3.2 names as
// the initial guess of an outer Krylov solve when x_hat is not accurate
// enough.
//
// Orthonormalisation.  The snapshot matrices are very ill conditioned: their
// singular values decay fast, and condition numbers reach 1e22 on these
// workloads.  Cholesky-based QR is out, and the basis comes from TSQR:
// Householder QR of row panels held in shared memory, then of stacks of g of
// their R factors, level by level up a tree; Q is formed top-down by applying
// each node's reflectors to the r x r block its parent hands it.  The column
// signs are fixed so that diag(R) >= 0, which makes Q unique for a full-rank X.
#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "sas_internal.cuh"

namespace sas {
namespace off {

constexpr int kThreads = 256;

struct Ops {
  const int64_t* rp[SAS_MAX_TERMS];
  const int32_t* ci[SAS_MAX_TERMS];
  const double* va[SAS_MAX_TERMS];
  const float* va32[SAS_MAX_TERMS];  // float copies of the values (mixed iterations)
};

__device__ inline double re_of(double v) { return v; }
__device__ inline double re_of(zd v) { return v.re; }

template <typename T> __device__ inline T from_re(double v);
template <> __device__ inline double from_re<double>(double v) { return v; }
template <> __device__ inline zd from_re<zd>(double v) { return mkz(v, 0.0); }

// conversions between the float64 scalar type T and the storage type of the iterates
template <typename To> __device__ inline To cvt(double x);
template <typename To> __device__ inline To cvt(float x);
template <typename To> __device__ inline To cvt(zd x);
template <typename To> __device__ inline To cvt(zf x);
template <> __device__ inline double cvt<double>(double x) { return x; }
template <> __device__ inline double cvt<double>(float x) { return (double)x; }
template <> __device__ inline float cvt<float>(double x) { return (float)x; }
template <> __device__ inline float cvt<float>(float x) { return x; }
template <> __device__ inline zd cvt<zd>(zd x) { return x; }
template <> __device__ inline zd cvt<zd>(zf x) { return to_hi(x); }
template <> __device__ inline zf cvt<zf>(zd x) { return to_lo(x); }
template <> __device__ inline zf cvt<zf>(zf x) { return x; }

template <typename V> __device__ inline const V* vals(const Ops& o, int k);
template <> __device__ inline const double* vals<double>(const Ops& o, int k) { return o.va[k]; }
template <> __device__ inline const float* vals<float>(const Ops& o, int k) { return o.va32[k]; }

// Block-wide sum of one value per thread (kThreads threads); result valid in thread 0.
template <typename T>
__device__ inline T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T s = zero<T>();
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];
  return s;
}

// Block-wide sum of per-warp values held by lane 0 of each warp; result valid in thread 0.
template <typename T>
__device__ inline T block_sum_warps(T v, T* red) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T s = zero<T>();
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];
  return s;
}

// D[k*n + i] = (A_k)_{ii}
__global__ void diag_kernel(Ops ops, int K, int64_t n, double* D) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < K; ++k) {
      double d = 0.0;
      for (int64_t e = ops.rp[k][i]; e < ops.rp[k][i + 1]; ++e)
        if (ops.ci[k][e] == i) d += ops.va[k][e];
      D[k * n + i] = d;
    }
}

__global__ void to_float_kernel(const double* a, int64_t count, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)a[i];
}

// The iteration's vectors (x_lo, r, p, q, D^-1) are stored quad-interleaved:
// columns 4g .. 4g+3 of row i sit together at ((g * n + i) * 4 + j), so that one
// 16-byte load gathers a row of four columns (columns past B are zero padding).
__host__ __device__ inline int64_t qidx(int64_t n, int b, int64_t i) { return (((int64_t)(b >> 2) * n + i) << 2) + (b & 3); }

template <typename TL> struct Quad { TL v[4]; };
template <typename TL> __device__ inline Quad<TL> ldq(const TL* p);
template <typename TL> __device__ inline void stq(TL* p, const Quad<TL>& q);
template <> __device__ inline Quad<float> ldq<float>(const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  return Quad<float>{{a.x, a.y, a.z, a.w}};
}
template <> __device__ inline void stq<float>(float* p, const Quad<float>& q) {
  *reinterpret_cast<float4*>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
template <> __device__ inline Quad<zf> ldq<zf>(const zf* p) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  return Quad<zf>{{mkzf(a.x, a.y), mkzf(a.z, a.w), mkzf(b.x, b.y), mkzf(b.z, b.w)}};
}
template <> __device__ inline void stq<zf>(zf* p, const Quad<zf>& q) {
  reinterpret_cast<float4*>(p)[0] = make_float4(q.v[0].re, q.v[0].im, q.v[1].re, q.v[1].im);
  reinterpret_cast<float4*>(p)[1] = make_float4(q.v[2].re, q.v[2].im, q.v[3].re, q.v[3].im);
}
template <> __device__ inline Quad<double> ldq<double>(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return Quad<double>{{a.x, a.y, b.x, b.y}};
}
template <> __device__ inline void stq<double>(double* p, const Quad<double>& q) {
  reinterpret_cast<double2*>(p)[0] = make_double2(q.v[0], q.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(q.v[2], q.v[3]);
}
template <> __device__ inline Quad<zd> ldq<zd>(const zd* p) {
  Quad<zd> q;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double2 a = reinterpret_cast<const double2*>(p)[j];
    q.v[j] = mkz(a.x, a.y);
  }
  return q;
}
template <> __device__ inline void stq<zd>(zd* p, const Quad<zd>& q) {
#pragma unroll
  for (int j = 0; j < 4; ++j) reinterpret_cast<double2*>(p)[j] = make_double2(q.v[j].re, q.v[j].im);
}

// invD (quad layout, TL) = 1 / sum_k theta[b*K + k] D[k*n + i]; a zero diagonal sets *bad.
template <typename T, typename TL>
__global__ void inv_diag_kernel(const double* D, int K, int64_t n, const T* theta, TL* invD, int* bad) {
  const int b = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T d = zero<T>();
    for (int k = 0; k < K; ++k) d += rscale(D[k * n + i], theta[b * K + k]);
    if (absq(d) == 0.0 || !finitev(d)) {
      atomicExch(bad, 1);
      invD[qidx(n, b, i)] = zero<TL>();
    } else {
      invD[qidx(n, b, i)] = cvt<TL>(divv(from_re<T>(1.0), d));
    }
  }
}

// Per-column state of the batched COCG.
template <typename T>
struct Col {
  T rz;           // r^T D^{-1} r of the current residual (BiCGStab: rho = <r_hat, r>)
  T alpha, beta;
  T omega;        // BiCGStab only
  double relres;  // ||r|| / ||b|| of the iterated residual
  double rmax;    // relres at the last replacement by the true residual
  int active;     // 1 while iterating
  int iters;
  int status;     // 0 running, 1 converged, 2 breakdown, 3 iteration limit, 4 stagnation
  int upd;        // 1: replace the residual by the true one in this iteration
  int nrel;       // replacements so far
  int nstag;      // consecutive replacements that did not halve the true residual
  int restart;    // BiCGStab: restart from the current residual in this iteration
};

// Column selection of the product kernels.
enum { kSelAll = 0, kSelActive = 1, kSelUpd = 2 };

// Both product kernels take one CTA per tile of kTileRows rows.  The tile's CSR
// segments (contiguous in every block) are staged in shared memory once and
// reused for every column, so the matrix leaves HBM once per product of the
// whole batch; the two halves of the CTA take alternate column groups.  Dots
// are summed per warp, then over the four warps of a half in a fixed order.
constexpr int kTileRows = 128;
constexpr int kStage = 4096;

template <typename V>
struct TileStage {
  int32_t ci[kStage];
  V va[kStage];
  int rps[SAS_MAX_TERMS][kTileRows + 1];  // staged row starts per block
  int seg_off[SAS_MAX_TERMS];
  int64_t seg_base[SAS_MAX_TERMS];
  int staged, nsel;
  int list[256];
};

// Selects the columns (or quads of columns) to work on and stages the tile.
// Returns false when there is nothing to do (the same for the whole CTA).
template <typename T, typename V>
__device__ inline bool tile_prologue(const Ops& ops, int K, int64_t r0, int64_t r1, int B, bool quads,
                                     const Col<T>* st, int sel, int* act, TileStage<V>& ts) {
  for (int b = threadIdx.x; b < B; b += kThreads)
    act[b] = sel == kSelAll ? 1 : sel == kSelActive ? st[b].active : st[b].upd;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    if (quads) {
      for (int q = 0; 4 * q < B; ++q) {
        bool any = false;
        for (int j = 0; j < 4 && 4 * q + j < B; ++j) any = any || act[4 * q + j];
        if (any) ts.list[m++] = q;
      }
    } else {
      for (int b = 0; b < B; ++b)
        if (act[b]) ts.list[m++] = b;
    }
    ts.nsel = m;
    int64_t total = 0;
    for (int k = 0; k < K && m > 0; ++k) {
      ts.seg_base[k] = ops.rp[k][r0];
      ts.seg_off[k] = (int)(total < kStage ? total : kStage);
      total += ops.rp[k][r1] - ts.seg_base[k];
    }
    ts.staged = total <= kStage;
  }
  __syncthreads();
  if (ts.nsel == 0) return false;
  if (ts.staged) {
    const int rows = (int)(r1 - r0);
    for (int k = 0; k < K; ++k) {
      const int64_t base = ts.seg_base[k];
      const int cnt = (int)(ops.rp[k][r1] - base);
      const V* va = vals<V>(ops, k);
      for (int e = threadIdx.x; e < cnt; e += kThreads) {
        ts.ci[ts.seg_off[k] + e] = ops.ci[k][base + e];
        ts.va[ts.seg_off[k] + e] = va[base + e];
      }
      for (int j = threadIdx.x; j <= rows; j += kThreads)
        ts.rps[k][j] = (int)(ops.rp[k][r0 + j] - base) + ts.seg_off[k];
    }
  }
  __syncthreads();
  return true;
}

// Q = A(theta_b) P for the active columns, P and Q quad-interleaved in the
// storage type TL (the arithmetic too), values of type V; part[b*G + tile] =
// sum over the tile of P_ib Q_ib.  Each half takes kQ quads per pass: one
// 16-byte gather serves four columns.  theta is [quad][k][4] in TL.
// Dynamic shared memory: B * 4 values of T and B ints.
template <typename T, typename TL, typename V>
__global__ void __launch_bounds__(kThreads) product_kernel(Ops ops, int K, int64_t n, int B, const TL* theta,
                                                           const TL* P, TL* Q, const Col<T>* st, T* part) {
  constexpr int kQ = sizeof(TL) >= 16 ? 1 : 2;
  __shared__ TileStage<V> ts;
  extern __shared__ __align__(16) unsigned char dyn[];
  T* wpart = reinterpret_cast<T*>(dyn);
  int* act = reinterpret_cast<int*>(wpart + (size_t)B * 4);
  const int64_t r0 = (int64_t)blockIdx.x * kTileRows;
  const int64_t r1 = r0 + kTileRows < n ? r0 + kTileRows : n;
  if (!tile_prologue<T, V>(ops, K, r0, r1, B, true, st, kSelActive, act, ts)) return;
  const int half = threadIdx.x >> 7, t = threadIdx.x & 127;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = r0 + t;
  const bool valid = i < r1;
  const int nq = ts.nsel;
  for (int g0 = half * kQ; g0 < nq; g0 += 2 * kQ) {
    const int nj = nq - g0 < kQ ? nq - g0 : kQ;
    int qa[kQ];
    const TL* xp[kQ];
#pragma unroll
    for (int u = 0; u < kQ; ++u) {
      qa[u] = ts.list[g0 + (u < nj ? u : nj - 1)];
      xp[u] = P + (int64_t)qa[u] * n * 4;
    }
    Quad<TL> acc[kQ];
#pragma unroll
    for (int u = 0; u < kQ; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[u].v[j] = zero<TL>();
    if (valid) {
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        Quad<TL> sum[kQ];
#pragma unroll
        for (int u = 0; u < kQ; ++u)
#pragma unroll
          for (int j = 0; j < 4; ++j) sum[u].v[j] = zero<TL>();
        if (ts.staged) {
          const int e1 = ts.rps[k][t + 1];
#pragma unroll 2
          for (int e = ts.rps[k][t]; e < e1; ++e) {
            const V v = ts.va[e];
            const int64_t c4 = (int64_t)ts.ci[e] * 4;
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
              const Quad<TL> x = ldq<TL>(xp[u] + c4);
#pragma unroll
              for (int j = 0; j < 4; ++j) sum[u].v[j] += rscale(v, x.v[j]);
            }
          }
        } else {
          const V* va = vals<V>(ops, k);
          const int64_t e1 = ops.rp[k][i + 1];
          for (int64_t e = ops.rp[k][i]; e < e1; ++e) {
            const V v = va[e];
            const int64_t c4 = (int64_t)ops.ci[k][e] * 4;
#pragma unroll
            for (int u = 0; u < kQ; ++u) {
              const Quad<TL> x = ldq<TL>(xp[u] + c4);
#pragma unroll
              for (int j = 0; j < 4; ++j) sum[u].v[j] += rscale(v, x.v[j]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kQ; ++u) {
          const Quad<TL> th = ldq<TL>(theta + ((int64_t)qa[u] * K + k) * 4);
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[u].v[j] += th.v[j] * sum[u].v[j];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kQ; ++u) {
      if (u >= nj) break;  // uniform
      Quad<TL> xi;
      if (valid) {
        stq<TL>(Q + ((int64_t)qa[u] * n + i) * 4, acc[u]);
        xi = ldq<TL>(xp[u] + i * 4);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b = 4 * qa[u] + j;
        if (b >= B || !act[b]) continue;  // uniform
        TL d = valid ? xi.v[j] * acc[u].v[j] : zero<TL>();
        d = warp_sum(d);  // in the storage arithmetic, widened once per warp
        if (lane == 0) wpart[b * 4 + (warp & 3)] = cvt<T>(d);
      }
    }
  }
  __syncthreads();
  const int G = gridDim.x;
  for (int b = threadIdx.x; b < B; b += kThreads)
    if (act[b]) part[(int64_t)b * G + blockIdx.x] = ((wpart[b * 4] + wpart[b * 4 + 1]) + wpart[b * 4 + 2]) + wpart[b * 4 + 3];
}

// ---------------------------------------------------------------- merged blocks
// The K blocks merged into one pattern: row i lists the union of the blocks'
// column indices (each block's row sorted, no repeats), with K values per
// stored entry (zero where a block has none).  The product then gathers each x
// entry once for all K blocks; per column the entry's coefficient
// sum_k theta_k v_k costs K multiply-adds, against one gather per block
// without merging.

// per row: the number of distinct columns; *bad set when a block row is unsorted
// or repeats a column (the product then keeps the blocks apart)
__global__ void merge_count_kernel(Ops ops, int K, int64_t n, int* cnt, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t cur[SAS_MAX_TERMS], end[SAS_MAX_TERMS];
    for (int k = 0; k < K; ++k) {
      cur[k] = ops.rp[k][i];
      end[k] = ops.rp[k][i + 1];
      for (int64_t e = cur[k] + 1; e < end[k]; ++e)
        if (ops.ci[k][e] <= ops.ci[k][e - 1]) atomicExch(bad, 1);
    }
    int count = 0;
    for (;;) {
      int cmin = INT_MAX;
      for (int k = 0; k < K; ++k)
        if (cur[k] < end[k] && ops.ci[k][cur[k]] < cmin) cmin = ops.ci[k][cur[k]];
      if (cmin == INT_MAX) break;
      ++count;
      for (int k = 0; k < K; ++k)
        while (cur[k] < end[k] && ops.ci[k][cur[k]] <= cmin) ++cur[k];
    }
    cnt[i] = count;
  }
}

// fills the merged pattern: mci[e], mva[e*K + k] (float32 values)
__global__ void merge_fill_kernel(Ops ops, int K, int64_t n, const int64_t* mrp, int32_t* mci, float* mva) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t cur[SAS_MAX_TERMS], end[SAS_MAX_TERMS];
    for (int k = 0; k < K; ++k) {
      cur[k] = ops.rp[k][i];
      end[k] = ops.rp[k][i + 1];
    }
    int64_t o = mrp[i];
    for (;;) {
      int cmin = INT_MAX;
      for (int k = 0; k < K; ++k)
        if (cur[k] < end[k] && ops.ci[k][cur[k]] < cmin) cmin = ops.ci[k][cur[k]];
      if (cmin == INT_MAX) break;
      mci[o] = cmin;
      for (int k = 0; k < K; ++k) {
        float v = 0.0f;
        if (cur[k] < end[k] && ops.ci[k][cur[k]] == cmin) v = (float)ops.va[k][cur[k]++];
        mva[o * K + k] = v;
      }
      ++o;
    }
  }
}

struct Merged {
  const int64_t* rp;
  const int32_t* ci;
  const float* va;  // K values per entry
};

constexpr int kStageM = 1024;  // merged entries staged per tile (K values each, at most 4096 values)

// Q = A(theta_b) P over the merged pattern, float32 (TL = float or zf), one quad of
// columns per pass of a half CTA; otherwise as product_kernel.
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) product_merged_kernel(Merged mg, int K, int64_t n, int B,
                                                                  const TL* theta, const TL* P, TL* Q,
                                                                  const Col<T>* st, T* part) {
  __shared__ int32_t ci_s[kStageM];
  __shared__ float va_s[4096];
  __shared__ int rps_s[kTileRows + 1];
  __shared__ int s_staged, s_nq;
  __shared__ int qlist[64];
  extern __shared__ __align__(16) unsigned char dyn[];
  T* wpart = reinterpret_cast<T*>(dyn);
  int* act = reinterpret_cast<int*>(wpart + (size_t)B * 4);
  const int64_t r0 = (int64_t)blockIdx.x * kTileRows;
  const int64_t r1 = r0 + kTileRows < n ? r0 + kTileRows : n;
  const int rows = (int)(r1 - r0);
  for (int b = threadIdx.x; b < B; b += kThreads) act[b] = st[b].active;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int q = 0; 4 * q < B; ++q) {
      bool any = false;
      for (int j = 0; j < 4 && 4 * q + j < B; ++j) any = any || act[4 * q + j];
      if (any) qlist[m++] = q;
    }
    s_nq = m;
    const int64_t cnt = mg.rp[r1] - mg.rp[r0];
    s_staged = cnt <= kStageM && cnt * K <= 4096;
  }
  __syncthreads();
  if (s_nq == 0) return;
  const bool staged = s_staged;
  const int64_t base = mg.rp[r0];
  if (staged) {
    const int cnt = (int)(mg.rp[r1] - base);
    for (int e = threadIdx.x; e < cnt; e += kThreads) ci_s[e] = mg.ci[base + e];
    for (int e = threadIdx.x; e < cnt * K; e += kThreads) va_s[e] = mg.va[base * K + e];
    for (int j = threadIdx.x; j <= rows; j += kThreads) rps_s[j] = (int)(mg.rp[r0 + j] - base);
  }
  __syncthreads();
  const int half = threadIdx.x >> 7, t = threadIdx.x & 127;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = r0 + t;
  const bool valid = t < rows;
  const int nq = s_nq;
  for (int g = half; g < nq; g += 2) {
    const int qa = qlist[g];
    const TL* xp = P + (int64_t)qa * n * 4;
    TL th[SAS_MAX_TERMS][4];
#pragma unroll
    for (int k = 0; k < SAS_MAX_TERMS; ++k) {
      Quad<TL> tq;
      if (k < K) tq = ldq<TL>(theta + ((int64_t)qa * K + k) * 4);
#pragma unroll
      for (int j = 0; j < 4; ++j) th[k][j] = k < K ? tq.v[j] : zero<TL>();
    }
    Quad<TL> acc;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc.v[j] = zero<TL>();
    if (valid) {
      const int64_t e0 = staged ? rps_s[t] : mg.rp[i] - base;
      const int64_t e1 = staged ? rps_s[t + 1] : mg.rp[i + 1] - base;
      for (int64_t e = e0; e < e1; ++e) {
        const int c = staged ? ci_s[e] : mg.ci[base + e];
        const float* v = staged ? va_s + e * K : mg.va + (base + e) * K;
        const Quad<TL> x = ldq<TL>(xp + (int64_t)c * 4);
        TL coef[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) coef[j] = zero<TL>();
#pragma unroll
        for (int k = 0; k < SAS_MAX_TERMS; ++k) {
          if (k >= K) break;
          const float vk = v[k];
#pragma unroll
          for (int j = 0; j < 4; ++j) coef[j] += rscale(vk, th[k][j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) acc.v[j] += coef[j] * x.v[j];
      }
    }
    Quad<TL> xi;
    if (valid) {
      stq<TL>(Q + ((int64_t)qa * n + i) * 4, acc);
      xi = ldq<TL>(xp + i * 4);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = 4 * qa + j;
      if (b >= B || !act[b]) continue;  // uniform
      TL d = valid ? xi.v[j] * acc.v[j] : zero<TL>();
      d = warp_sum(d);
      if (lane == 0) wpart[b * 4 + (warp & 3)] = cvt<T>(d);
    }
  }
  __syncthreads();
  const int G = gridDim.x;
  for (int b = threadIdx.x; b < B; b += kThreads)
    if (act[b]) part[(int64_t)b * G + blockIdx.x] = ((wpart[b * 4] + wpart[b * 4 + 1]) + wpart[b * 4 + 2]) + wpart[b * 4 + 3];
}

// R = b - A(theta_b) X in float64 for the selected columns (X column-major,
// the caller's), written to R in the quad layout as TL; part0[b*G + tile] =
// sum R_ib D^-1_ib R_ib and part1 = sum |R_ib|^2, both in float64.
// Dynamic shared memory: B * 4 values of T, B * 4 doubles and B ints.
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) residual_kernel(Ops ops, int K, int64_t n, int B, const T* theta,
                                                            const T* X, TL* R, const T* bvec, const TL* invD,
                                                            const Col<T>* st, int sel, T* part0, double* part1) {
  constexpr int kCB = 4;
  __shared__ TileStage<double> ts;
  extern __shared__ __align__(16) unsigned char dyn[];
  T* wpart = reinterpret_cast<T*>(dyn);
  double* wpart1 = reinterpret_cast<double*>(wpart + (size_t)B * 4);
  int* act = reinterpret_cast<int*>(wpart1 + (size_t)B * 4);
  const int64_t r0 = (int64_t)blockIdx.x * kTileRows;
  const int64_t r1 = r0 + kTileRows < n ? r0 + kTileRows : n;
  if (!tile_prologue<T, double>(ops, K, r0, r1, B, false, st, sel, act, ts)) return;
  const int half = threadIdx.x >> 7, t = threadIdx.x & 127;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = r0 + t;
  const bool valid = i < r1;
  const int na = ts.nsel;
  for (int g0 = half * kCB; g0 < na; g0 += 2 * kCB) {
    const int nj = na - g0 < kCB ? na - g0 : kCB;
    const T* xp[kCB];
    int bj[kCB];
#pragma unroll
    for (int j = 0; j < kCB; ++j) {
      bj[j] = ts.list[g0 + (j < nj ? j : nj - 1)];
      xp[j] = X + (int64_t)bj[j] * n;
    }
    T acc[kCB];
#pragma unroll
    for (int j = 0; j < kCB; ++j) acc[j] = zero<T>();
    if (valid) {
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        T sum[kCB];
#pragma unroll
        for (int j = 0; j < kCB; ++j) sum[j] = zero<T>();
        if (ts.staged) {
          const int e1 = ts.rps[k][t + 1];
          for (int e = ts.rps[k][t]; e < e1; ++e) {
            const double v = ts.va[e];
            const int c = ts.ci[e];
#pragma unroll
            for (int j = 0; j < kCB; ++j) sum[j] += rscale(v, xp[j][c]);
          }
        } else {
          const int64_t e1 = ops.rp[k][i + 1];
          for (int64_t e = ops.rp[k][i]; e < e1; ++e) {
            const double v = ops.va[k][e];
            const int c = ops.ci[k][e];
#pragma unroll
            for (int j = 0; j < kCB; ++j) sum[j] += rscale(v, xp[j][c]);
          }
        }
#pragma unroll
        for (int j = 0; j < kCB; ++j) acc[j] += theta[(int64_t)bj[j] * K + k] * sum[j];
      }
    }
#pragma unroll
    for (int j = 0; j < kCB; ++j) {
      if (j >= nj) break;  // uniform
      const int b = bj[j];
      T d0 = zero<T>();
      double d1 = 0.0;
      if (valid) {
        const T r = bvec[i] - acc[j];
        R[qidx(n, b, i)] = cvt<TL>(r);
        d0 = r * (cvt<T>(invD[qidx(n, b, i)]) * r);
        d1 = absq(r);
      }
      d0 = warp_sum(d0);
      d1 = warp_sum(d1);
      if (lane == 0) {
        wpart[b * 4 + (warp & 3)] = d0;
        wpart1[b * 4 + (warp & 3)] = d1;
      }
    }
  }
  __syncthreads();
  const int G = gridDim.x;
  for (int b = threadIdx.x; b < B; b += kThreads) {
    if (!act[b]) continue;
    if (part0) part0[(int64_t)b * G + blockIdx.x] = ((wpart[b * 4] + wpart[b * 4 + 1]) + wpart[b * 4 + 2]) + wpart[b * 4 + 3];
    if (part1)
      part1[(int64_t)b * G + blockIdx.x] = ((wpart1[b * 4] + wpart1[b * 4 + 1]) + wpart1[b * 4 + 2]) + wpart1[b * 4 + 3];
  }
}

// One CTA per column: sums of the G partials in a fixed order.
template <typename T>
__device__ inline T column_sum(const T* part, int b, int G, T* red) {
  T s = zero<T>();
  for (int g = threadIdx.x; g < G; g += kThreads) s += part[(int64_t)b * G + g];
  return block_sum(s, red);
}

// The start and every replacement of the residual by the true one: the column
// takes rz and relres of the residual the tile kernel (MODE 1) just wrote.
// start != 0: every column, iteration count and beta reset; otherwise the
// columns flagged for replacement, which then get beta from the new rz.
template <typename T>
__global__ void __launch_bounds__(kThreads) replace_kernel(const T* prz, const double* prr, int G, double bnorm,
                                                           double tol, int maxit, int start, int defer,
                                                           Col<T>* st) {
  __shared__ T red[kThreads / 32];
  __shared__ double redd[kThreads / 32];
  const int b = blockIdx.x;
  if (!start && !st[b].upd) return;
  const T rz = column_sum(prz, b, G, red);
  const double rr = column_sum(prr, b, G, redd);
  if (threadIdx.x == 0) {
    Col<T> c = st[b];
    const double prev = c.rmax;
    c.upd = 0;
    c.relres = sqrt(rr) / bnorm;
    c.rmax = c.relres;
    if (start) {
      c.alpha = zero<T>();
      c.iters = 0;
      c.nrel = 0;
      c.nstag = 0;
      c.status = 0;
      c.active = 1;
    } else {
      c.nrel += 1;
      c.nstag = c.relres > 0.5 * prev ? c.nstag + 1 : 0;
    }
    if (!(c.relres == c.relres) || (!defer && !finitev(rz))) {
      c.status = 2;
      c.active = 0;
    } else if (c.relres <= tol) {
      c.status = 1;
      c.active = 0;
    } else if (c.nstag >= 4) {  // the true residual stopped falling: attainable accuracy reached
      c.status = 4;
      c.active = 0;
    } else if (c.iters >= maxit) {
      c.status = 3;
      c.active = 0;
    } else if (defer) {
      // rz and beta come after the preconditioner (rz_kernel)
    } else if (start) {
      c.beta = zero<T>();
    } else if (absq(c.rz) == 0.0) {
      c.status = 2;
      c.active = 0;
    } else {
      c.beta = divv(rz, c.rz);
    }
    if (!defer) c.rz = rz;
    st[b] = c;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) alpha_kernel(const T* ppq, int G, Col<T>* st) {
  __shared__ T red[kThreads / 32];
  const int b = blockIdx.x;
  if (!st[b].active) return;
  const T pq = column_sum(ppq, b, G, red);
  if (threadIdx.x == 0) {
    if (absq(pq) == 0.0 || !finitev(pq)) {
      st[b].status = 2;
      st[b].active = 0;
    } else {
      st[b].alpha = divv(st[b].rz, pq);
    }
  }
}

// After the update: the iterated residual's norm.  A column whose residual
// reached the tolerance, or (float32 iterates) fell below delta times the
// residual at its last replacement, is flagged for replacement by the true
// residual, which decides convergence and beta; the others take beta here.
template <typename T>
__global__ void __launch_bounds__(kThreads) beta_kernel(const T* prz, const double* prr, int G,
                                                        double bnorm, double tol, double delta, int maxit,
                                                        int defer, Col<T>* st) {
  __shared__ T red[kThreads / 32];
  __shared__ double redd[kThreads / 32];
  const int b = blockIdx.x;
  if (!st[b].active) return;
  const T rz = column_sum(prz, b, G, red);
  const double rr = column_sum(prr, b, G, redd);
  if (threadIdx.x == 0) {
    Col<T> c = st[b];
    c.iters += 1;
    c.relres = sqrt(rr) / bnorm;
    if (!(c.relres == c.relres) || (!defer && !finitev(rz))) {
      c.status = 2;
      c.active = 0;
    } else if (c.relres <= tol || c.relres < delta * c.rmax || c.iters >= maxit) {
      c.upd = 1;  // rz and beta come from the true residual
    } else if (defer) {
      // rz and beta come after the preconditioner (rz_kernel)
    } else if (absq(c.rz) == 0.0) {
      c.status = 2;
      c.active = 0;
    } else {
      c.beta = divv(rz, c.rz);
      c.rz = rz;
    }
    st[b] = c;
  }
}

// Elementwise kernels over the quad layout: grid (quads, row chunks), one row of
// a quad per thread and step.  Columns that are inactive (or padding) are
// left untouched.
template <typename T>
__device__ inline int quad_flags(const Col<T>* st, int q, int B, int which) {
  int m = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int b = 4 * q + j;
    if (b < B && (which == 0 ? st[b].active : st[b].upd)) m |= 1 << j;
  }
  return m;
}

// X += alpha P, R -= alpha Q (arithmetic in TL); partials (in T) of the new
// r^T D^{-1} r and ||r||^2 per column.
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) update_kernel(int64_t n, int B, TL* X, TL* R, const TL* P, const TL* Q,
                                                          const TL* invD, const Col<T>* st, T* prz,
                                                          double* prr, int64_t rows_per_cta) {
  __shared__ T red[kThreads / 32][4];
  __shared__ double redd[kThreads / 32][4];
  const int q = blockIdx.x, G = gridDim.y;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  TL alpha[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) alpha[j] = (on >> j) & 1 ? cvt<TL>(st[4 * q + j].alpha) : zero<TL>();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  // per-thread sums in the storage arithmetic (a few dozen terms), widened per warp
  TL rz[4];
  decltype(absq(rz[0])) rr[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    rz[j] = zero<TL>();
    rr[j] = 0;
  }
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    Quad<TL> x = ldq<TL>(X + o), r = ldq<TL>(R + o);
    const Quad<TL> p = ldq<TL>(P + o), qq = ldq<TL>(Q + o), d = ldq<TL>(invD + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((on >> j) & 1)) continue;
      x.v[j] += alpha[j] * p.v[j];
      r.v[j] -= alpha[j] * qq.v[j];
      rz[j] += r.v[j] * (d.v[j] * r.v[j]);
      rr[j] += absq(r.v[j]);
    }
    stq<TL>(X + o, x);
    stq<TL>(R + o, r);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const TL a = warp_sum(rz[j]);
    const auto c = warp_sum(rr[j]);
    if (lane == 0) {
      red[w][j] = cvt<T>(a);
      redd[w][j] = (double)c;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 && ((on >> threadIdx.x) & 1)) {
    const int j = threadIdx.x;
    T a = zero<T>();
    double c = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      a += red[k][j];
      c += redd[k][j];
    }
    prz[(int64_t)(4 * q + j) * G + blockIdx.y] = a;
    prr[(int64_t)(4 * q + j) * G + blockIdx.y] = c;
  }
}

// x (float64, column-major) += x_lo (quad layout); x_lo = 0, for the columns
// flagged for replacement (all != 0: every column)
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) fold_kernel(int64_t n, int B, T* X, TL* Xl, const Col<T>* st, int all,
                                                        int64_t rows_per_cta) {
  const int q = blockIdx.x;
  int on = quad_flags(st, q, B, 1);
  if (all)
    for (int j = 0; j < 4; ++j) on |= (4 * q + j < B) << j;
  if (!on) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    Quad<TL> xl = ldq<TL>(Xl + o);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((on >> j) & 1) {
        X[(int64_t)(4 * q + j) * n + i] += cvt<T>(xl.v[j]);
        xl.v[j] = zero<TL>();
      }
    stq<TL>(Xl + o, xl);
  }
}

// P = D^{-1} R + beta P
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) direction_kernel(int64_t n, int B, const TL* R, const TL* invD, TL* P,
                                                             const Col<T>* st, int64_t rows_per_cta) {
  const int q = blockIdx.x;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  TL beta[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) beta[j] = (on >> j) & 1 ? cvt<TL>(st[4 * q + j].beta) : zero<TL>();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    const Quad<TL> r = ldq<TL>(R + o), d = ldq<TL>(invD + o);
    Quad<TL> p = ldq<TL>(P + o);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((on >> j) & 1) p.v[j] = d.v[j] * r.v[j] + beta[j] * p.v[j];
    stq<TL>(P + o, p);
  }
}

// ------------------------------------------------------------------ BiCGStab
// For nonsymmetric A(p) (BiCGStab, van der Vorst 1992) with the diagonal as right
// preconditioner, float64 / complex128 iterates in the quad layout.  Per iteration:
//   p = r + beta (p - omega v), p^ = D^-1 p, v = A p^, alpha = rho / <r_hat, v>,
//   s = r - alpha v, s^ = D^-1 s, t = A s^, omega = <t, s> / <t, t>,
//   x += alpha p^ + omega s^, r = s - omega t, rho' = <r_hat, r>, beta = (rho'/rho)(alpha/omega),
// with <a, b> = sum conj(a) b.  When the iterated residual reaches the tolerance
// the true residual decides; if it is still above, the iteration restarts from it
// (r_hat = r, p = r), which is also how it starts.

template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_dir_kernel(int64_t n, int B, const T* R, T* Rh, T* P, const T* V,
                                                            const T* invD, T* Ph, const Col<T>* st,
                                                            int64_t rows_per_cta) {
  const int q = blockIdx.x;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  T beta[4], omega[4];
  int rs = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool a = (on >> j) & 1;
    beta[j] = a ? st[4 * q + j].beta : zero<T>();
    omega[j] = a ? st[4 * q + j].omega : zero<T>();
    if (a && st[4 * q + j].restart) rs |= 1 << j;
  }
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    const Quad<T> r = ldq<T>(R + o), v = ldq<T>(V + o), d = ldq<T>(invD + o);
    Quad<T> p = ldq<T>(P + o), ph = ldq<T>(Ph + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((on >> j) & 1)) continue;
      p.v[j] = (rs >> j) & 1 ? r.v[j] : r.v[j] + beta[j] * (p.v[j] - omega[j] * v.v[j]);
      ph.v[j] = d.v[j] * p.v[j];
    }
    stq<T>(P + o, p);
    stq<T>(Ph + o, ph);
    if (rs) {
      Quad<T> rh = ldq<T>(Rh + o);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((rs >> j) & 1) rh.v[j] = r.v[j];
      stq<T>(Rh + o, rh);
    }
  }
}

// partials of <A, Bv> (and of <C, D> when C is given) per active column
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_dot_kernel(int64_t n, int B, const T* A, const T* Bv, const T* C,
                                                            const T* D, const Col<T>* st, T* part0, T* part1,
                                                            int64_t rows_per_cta) {
  __shared__ T red0[kThreads / 32][4];
  __shared__ T red1[kThreads / 32][4];
  const int q = blockIdx.x, G = gridDim.y;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  T s0[4], s1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) s0[j] = s1[j] = zero<T>();
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    const Quad<T> a = ldq<T>(A + o), b = ldq<T>(Bv + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) s0[j] += conjv(a.v[j]) * b.v[j];
    if (C) {
      const Quad<T> c = ldq<T>(C + o), dd = ldq<T>(D + o);
#pragma unroll
      for (int j = 0; j < 4; ++j) s1[j] += conjv(c.v[j]) * dd.v[j];
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T a = warp_sum(s0[j]);
    const T c = warp_sum(s1[j]);
    if (lane == 0) {
      red0[w][j] = a;
      red1[w][j] = c;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 && ((on >> threadIdx.x) & 1)) {
    const int j = threadIdx.x;
    T a = zero<T>(), c = zero<T>();
    for (int k = 0; k < kThreads / 32; ++k) {
      a += red0[k][j];
      c += red1[k][j];
    }
    part0[(int64_t)(4 * q + j) * G + blockIdx.y] = a;
    if (C) part1[(int64_t)(4 * q + j) * G + blockIdx.y] = c;
  }
}

// s = r - alpha v, s^ = D^-1 s
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_s_kernel(int64_t n, int B, const T* R, const T* V, const T* invD,
                                                          T* Sv, T* Sh, const Col<T>* st, int64_t rows_per_cta) {
  const int q = blockIdx.x;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  T alpha[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) alpha[j] = (on >> j) & 1 ? st[4 * q + j].alpha : zero<T>();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    const Quad<T> r = ldq<T>(R + o), v = ldq<T>(V + o), d = ldq<T>(invD + o);
    Quad<T> sv = ldq<T>(Sv + o), sh = ldq<T>(Sh + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((on >> j) & 1)) continue;
      sv.v[j] = r.v[j] - alpha[j] * v.v[j];
      sh.v[j] = d.v[j] * sv.v[j];
    }
    stq<T>(Sv + o, sv);
    stq<T>(Sh + o, sh);
  }
}

// x += alpha p^ + omega s^, r = s - omega t; partials of rho' = <r_hat, r> and |r|^2
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_xr_kernel(int64_t n, int B, T* X, const T* Ph, const T* Sh,
                                                           const T* Sv, const T* Tv, const T* Rh, T* R,
                                                           const Col<T>* st, T* prz, double* prr,
                                                           int64_t rows_per_cta) {
  __shared__ T red[kThreads / 32][4];
  __shared__ double redd[kThreads / 32][4];
  const int q = blockIdx.x, G = gridDim.y;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  T alpha[4], omega[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    alpha[j] = (on >> j) & 1 ? st[4 * q + j].alpha : zero<T>();
    omega[j] = (on >> j) & 1 ? st[4 * q + j].omega : zero<T>();
  }
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  T rho[4];
  double rr[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    rho[j] = zero<T>();
    rr[j] = 0.0;
  }
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    Quad<T> x = ldq<T>(X + o), r = ldq<T>(R + o);
    const Quad<T> ph = ldq<T>(Ph + o), sh = ldq<T>(Sh + o), sv = ldq<T>(Sv + o), tv = ldq<T>(Tv + o),
                  rh = ldq<T>(Rh + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((on >> j) & 1)) continue;
      x.v[j] += alpha[j] * ph.v[j] + omega[j] * sh.v[j];
      r.v[j] = sv.v[j] - omega[j] * tv.v[j];
      rho[j] += conjv(rh.v[j]) * r.v[j];
      rr[j] += absq(r.v[j]);
    }
    stq<T>(X + o, x);
    stq<T>(R + o, r);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T a = warp_sum(rho[j]);
    const double c = warp_sum(rr[j]);
    if (lane == 0) {
      red[w][j] = a;
      redd[w][j] = c;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 && ((on >> threadIdx.x) & 1)) {
    const int j = threadIdx.x;
    T a = zero<T>();
    double c = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      a += red[k][j];
      c += redd[k][j];
    }
    prz[(int64_t)(4 * q + j) * G + blockIdx.y] = a;
    prr[(int64_t)(4 * q + j) * G + blockIdx.y] = c;
  }
}

// alpha = rho / <r_hat, v>
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_alpha_kernel(const T* pd, int G, Col<T>* st) {
  __shared__ T red[kThreads / 32];
  const int b = blockIdx.x;
  if (!st[b].active) return;
  const T d = column_sum(pd, b, G, red);
  if (threadIdx.x == 0) {
    if (absq(d) == 0.0 || !finitev(d)) {
      st[b].status = 2;
      st[b].active = 0;
    } else {
      st[b].alpha = divv(st[b].rz, d);
    }
  }
}

// omega = <t, s> / <t, t> (omega = 0 when t = 0: then s = 0 and r is already s)
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_omega_kernel(const T* pts, const T* ptt, int G, Col<T>* st) {
  __shared__ T red[kThreads / 32];
  const int b = blockIdx.x;
  if (!st[b].active) return;
  const T ts = column_sum(pts, b, G, red);
  const T tt = column_sum(ptt, b, G, red);
  if (threadIdx.x == 0) {
    if (!finitev(ts) || !finitev(tt)) {
      st[b].status = 2;
      st[b].active = 0;
    } else {
      st[b].omega = absq(tt) == 0.0 ? zero<T>() : divv(ts, tt);
    }
  }
}

// after x and r: the iterated residual; tolerance or limit -> the true residual decides
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_beta_kernel(const T* prho, const double* prr, int G, double bnorm,
                                                             double tol, int maxit, Col<T>* st) {
  __shared__ T red[kThreads / 32];
  __shared__ double redd[kThreads / 32];
  const int b = blockIdx.x;
  if (!st[b].active) return;
  const T rho = column_sum(prho, b, G, red);
  const double rr = column_sum(prr, b, G, redd);
  if (threadIdx.x == 0) {
    Col<T> c = st[b];
    c.iters += 1;
    c.restart = 0;
    c.relres = sqrt(rr) / bnorm;
    if (!(c.relres == c.relres) || !finitev(rho)) {
      c.status = 2;
      c.active = 0;
    } else if (c.relres <= tol || c.iters >= maxit) {
      c.upd = 1;
    } else if (absq(c.rz) == 0.0 || absq(c.omega) == 0.0) {
      c.upd = 1;  // breakdown of the recurrences: restart from the true residual
    } else {
      c.beta = divv(rho, c.rz) * divv(c.alpha, c.omega);
      c.rz = rho;
    }
    st[b] = c;
  }
}

// the true residual (written to R by the residual kernel) decides; otherwise restart
// from it: r_hat = r, p = r, rho = <r, r>
template <typename T>
__global__ void __launch_bounds__(kThreads) bicg_replace_kernel(const double* prr, int G, double bnorm, double tol,
                                                                int maxit, int start, Col<T>* st) {
  __shared__ double redd[kThreads / 32];
  const int b = blockIdx.x;
  if (!start && !st[b].upd) return;
  const double rr = column_sum(prr, b, G, redd);
  if (threadIdx.x == 0) {
    Col<T> c = st[b];
    const double prev = c.rmax;
    c.upd = 0;
    c.relres = sqrt(rr) / bnorm;
    c.rmax = c.relres;
    if (start) {
      c.iters = 0;
      c.nrel = 0;
      c.nstag = 0;
      c.status = 0;
      c.active = 1;
    } else {
      c.nrel += 1;
      c.nstag = c.relres > 0.5 * prev ? c.nstag + 1 : 0;
    }
    if (!(c.relres == c.relres)) {
      c.status = 2;
      c.active = 0;
    } else if (c.relres <= tol) {
      c.status = 1;
      c.active = 0;
    } else if (c.nstag >= 4) {
      c.status = 4;
      c.active = 0;
    } else if (c.iters >= maxit) {
      c.status = 3;
      c.active = 0;
    } else {
      c.restart = 1;
      c.rz = from_re<T>(rr);
      c.beta = zero<T>();
      c.omega = zero<T>();
      c.alpha = zero<T>();
    }
    st[b] = c;
  }
}

// ------------------------------------------------- fast Poisson preconditioner
// M_b = alpha_b L + beta_b I with L the unit-spacing Dirichlet Laplacian of an
// nx x ny x nz grid (sum over the axes of tridiag(-1, 2, -1)), i = ix + nx (iy + ny iz).
// The discrete sine transform (DST-I) diagonalises L: with S_N[j][k] =
// sin(pi (j+1)(k+1) / (N+1)), S_N S_N = (N+1)/2 I and S_N T_N S_N = (N+1)/2 diag(mu),
// mu_j = 2 - 2 cos(pi (j+1) / (N+1)).  So M_b^-1 r = c S (S r ./ (alpha_b (mu_x + mu_y + mu_z)
// + beta_b)) with c = prod 2/(N+1) and S the tensor product of the axes' S_N.  The
// transforms are dense matrix products along each axis (library GEMMs, float32
// accuracy); the kernels here build the matrices and eigenvalues, move data
// between the quad layout and planar float32 columns, and scale.

__global__ void dst_matrix_kernel(int N, float* S, float* mu) {
  const int64_t NN = (int64_t)N * N;
  const double pi = 3.14159265358979323846;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < NN;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx % N, k = idx / N;
    const int64_t a = ((j + 1) * (k + 1)) % (2 * (int64_t)(N + 1));  // sin has period 2(N+1) in a
    S[idx] = (float)sin(pi * (double)a / (double)(N + 1));
    if (k == 0) mu[j] = (float)(2.0 - 2.0 * cos(pi * (double)(j + 1) / (double)(N + 1)));
  }
}

// planar float32 columns: plane 0 (real parts) then plane 1 (imaginary parts), column b
// of plane p at U + (p * B + b) * n
template <typename TL> __host__ __device__ constexpr bool is_cplx() {
  return std::is_same<TL, zf>::value || std::is_same<TL, zd>::value;
}
template <typename TL> __device__ inline float re_f(TL v);
template <> __device__ inline float re_f<float>(float v) { return v; }
template <> __device__ inline float re_f<zf>(zf v) { return v.re; }
template <> __device__ inline float re_f<double>(double v) { return (float)v; }
template <> __device__ inline float re_f<zd>(zd v) { return (float)v.re; }
template <typename TL> __device__ inline float im_f(TL v);
template <> __device__ inline float im_f<float>(float) { return 0.0f; }
template <> __device__ inline float im_f<zf>(zf v) { return v.im; }
template <> __device__ inline float im_f<double>(double) { return 0.0f; }
template <> __device__ inline float im_f<zd>(zd v) { return (float)v.im; }
template <typename TL> __device__ inline TL mk_f(float re, float im);
template <> __device__ inline float mk_f<float>(float re, float) { return re; }
template <> __device__ inline zf mk_f<zf>(float re, float im) { return mkzf(re, im); }
template <> __device__ inline double mk_f<double>(float re, float) { return (double)re; }
template <> __device__ inline zd mk_f<zd>(float re, float im) { return mkz((double)re, (double)im); }

template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) unpack_kernel(int64_t n, int B, const TL* R, float* U, const Col<T>* st,
                                                          int64_t rows_per_cta) {
  const int q = blockIdx.x;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  const bool cplx = is_cplx<TL>();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const Quad<TL> r = ldq<TL>(R + ((int64_t)q * n + i) * 4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((on >> j) & 1)) continue;
      const int b = 4 * q + j;
      U[(int64_t)b * n + i] = re_f<TL>(r.v[j]);
      if (cplx) U[((int64_t)B + b) * n + i] = im_f<TL>(r.v[j]);
    }
  }
}

// U_b(i) /= alpha_b (mu_x[ix] + mu_y[iy] + mu_z[iz]) + beta_b, times c; coef is B x 4
// (alpha re, im, beta re, im) on the device
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) poisson_scale_kernel(int64_t nx, int64_t ny, int64_t nz, int B,
                                                                 float* U, const float* mux, const float* muy,
                                                                 const float* muz, const double* coef, double c,
                                                                 const Col<T>* st) {
  const int b = blockIdx.y;
  if (!st[b].active) return;
  const bool cplx = is_cplx<TL>();
  const int64_t n = nx * ny * nz;
  const double ar = coef[4 * b], ai = coef[4 * b + 1], br = coef[4 * b + 2], bi = coef[4 * b + 3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const double lam = (double)mux[ix] + (double)muy[iy] + (double)muz[iz];
    const double dr = ar * lam + br, di = ai * lam + bi;
    const double den = dr * dr + di * di;
    float* ur = U + (int64_t)b * n + i;
    if (cplx) {
      float* ui = U + ((int64_t)B + b) * n + i;
      const double xr = *ur, xi = *ui;
      *ur = (float)(c * (xr * dr + xi * di) / den);
      *ui = (float)(c * (xi * dr - xr * di) / den);
    } else {
      *ur = (float)(c * (double)*ur * dr / den);
    }
  }
}

// Z (quad layout) = the planar result; partials of r^T z per column (bilinear)
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) pack_rz_kernel(int64_t n, int B, const float* U, const TL* R, TL* Z,
                                                           const Col<T>* st, T* prz, int64_t rows_per_cta) {
  __shared__ T red[kThreads / 32][4];
  const int q = blockIdx.x, G = gridDim.y;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  const bool cplx = is_cplx<TL>();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  TL rz[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) rz[j] = zero<TL>();
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    const Quad<TL> r = ldq<TL>(R + o);
    Quad<TL> z = ldq<TL>(Z + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((on >> j) & 1)) continue;
      const int b = 4 * q + j;
      z.v[j] = mk_f<TL>(U[(int64_t)b * n + i], cplx ? U[((int64_t)B + b) * n + i] : 0.0f);
      rz[j] += r.v[j] * z.v[j];
    }
    stq<TL>(Z + o, z);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const TL a = warp_sum(rz[j]);
    if (lane == 0) red[w][j] = cvt<T>(a);
  }
  __syncthreads();
  if (threadIdx.x < 4 && ((on >> threadIdx.x) & 1)) {
    const int j = threadIdx.x;
    T a = zero<T>();
    for (int k = 0; k < kThreads / 32; ++k) a += red[k][j];
    prz[(int64_t)(4 * q + j) * G + blockIdx.y] = a;
  }
}

// beta from the preconditioned residual: rz = r^T M^-1 r (start: beta = 0)
template <typename T>
__global__ void __launch_bounds__(kThreads) rz_kernel(const T* prz, int G, int start, Col<T>* st) {
  __shared__ T red[kThreads / 32];
  const int b = blockIdx.x;
  if (!st[b].active) return;
  const T rz = column_sum(prz, b, G, red);
  if (threadIdx.x == 0) {
    Col<T> c = st[b];
    if (!finitev(rz) || (!start && absq(c.rz) == 0.0)) {
      c.status = 2;
      c.active = 0;
    } else {
      c.beta = start ? zero<T>() : divv(rz, c.rz);
      c.rz = rz;
    }
    st[b] = c;
  }
}

// P = Z + beta P
template <typename T, typename TL>
__global__ void __launch_bounds__(kThreads) direction_z_kernel(int64_t n, int B, const TL* Z, TL* P,
                                                               const Col<T>* st, int64_t rows_per_cta) {
  const int q = blockIdx.x;
  const int on = quad_flags(st, q, B, 0);
  if (!on) return;
  TL beta[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) beta[j] = (on >> j) & 1 ? cvt<TL>(st[4 * q + j].beta) : zero<TL>();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const int64_t o = ((int64_t)q * n + i) * 4;
    const Quad<TL> z = ldq<TL>(Z + o);
    Quad<TL> p = ldq<TL>(P + o);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((on >> j) & 1) p.v[j] = z.v[j] + beta[j] * p.v[j];
    stq<TL>(P + o, p);
  }
}

__global__ void __launch_bounds__(kThreads) norm_partial_kernel(const double* x, int64_t count, double* out) {
  __shared__ double redd[kThreads / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads)
    s += x[i] * x[i];
  s = block_sum(s, redd);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// ------------------------------------------------------------------ TSQR
//
// A panel is h x r, column-major in shared memory (entry (i, j) at A[j*h + i]).
// Level 0 panel p holds rows p*h .. p*h + h - 1 of X (zeros past n).  A panel
// at level l >= 1 stacks the R factors of g consecutive panels of level l - 1
// (zeros past the last one).  The kernel leaves, per panel: R (r x r,
// column-major, zeros below the diagonal), the reflectors' vectors (unit
// leading entry implied, zeros above it) and their tau.

template <typename T>
__global__ void __launch_bounds__(kThreads) tsqr_panel_kernel(int level0, const T* src, int64_t n,
                                                              int64_t ldsrc, int64_t nprev, int g,
                                                              int r, int h, T* V, int64_t ldv,
                                                              T* tau, T* Rout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);
  __shared__ T s_scale, s_tau, s_beta;
  const int64_t p = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < h * r; idx += kThreads) {
    const int j = idx / h, i = idx % h;
    T v = zero<T>();
    if (level0) {
      const int64_t row = p * h + i;
      if (row < n) v = src[(int64_t)j * ldsrc + row];
    } else {
      const int64_t blk = p * g + i / r;
      if (blk < nprev) v = src[blk * r * r + (int64_t)j * r + (i % r)];
    }
    A[idx] = v;
  }
  __syncthreads();
  const int steps = r < h ? r : h;
  for (int j = 0; j < steps; ++j) {
    T* a = A + (int64_t)j * h;
    if (warp == 0) {
      double s2 = 0.0;
      for (int i = j + 1 + lane; i < h; i += 32) s2 += absq(a[i]);
      s2 = warp_sum(s2);
      if (lane == 0) {
        const T alpha = a[j];
        const double ai = absq(alpha) - re_of(alpha) * re_of(alpha);  // |Im alpha|^2
        if (s2 == 0.0 && ai == 0.0) {
          s_tau = zero<T>();
          s_beta = alpha;
          s_scale = zero<T>();
        } else {
          const double nrm = sqrt(absq(alpha) + s2);
          const double beta = re_of(alpha) >= 0.0 ? -nrm : nrm;
          // tau = (beta - alpha) / beta, scale = 1 / (alpha - beta)
          s_tau = rscale(1.0 / beta, from_re<T>(beta) - alpha);
          s_beta = from_re<T>(beta);
          s_scale = divv(from_re<T>(1.0), alpha - from_re<T>(beta));
        }
      }
    }
    __syncthreads();
    const T t = s_tau, sc = s_scale;
    if (absq(t) != 0.0)
      for (int i = j + 1 + threadIdx.x; i < h; i += kThreads) a[i] = sc * a[i];
    __syncthreads();
    if (absq(t) != 0.0) {
      const T ct = conjv(t);
      for (int c = j + 1 + warp; c < r; c += kThreads / 32) {
        T* ac = A + (int64_t)c * h;
        T w = zero<T>();
        for (int i = j + lane; i < h; i += 32) w += (i == j ? ac[i] : conjv(a[i]) * ac[i]);
        w = warp_sum(w);
        const T f = ct * w;
        for (int i = j + lane; i < h; i += 32) ac[i] -= (i == j ? f : f * a[i]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tau[p * r + j] = t;
      a[j] = s_beta;
    }
    __syncthreads();
  }
  for (int j = steps; threadIdx.x == 0 && j < r; ++j) tau[p * r + j] = zero<T>();
  // R, then the reflectors (the strict lower part; rows past the data are zero anyway)
  for (int idx = threadIdx.x; idx < r * r; idx += kThreads) {
    const int j = idx / r, i = idx % r;
    Rout[p * r * r + idx] = (i <= j && i < h) ? A[(int64_t)j * h + i] : zero<T>();
  }
  for (int idx = threadIdx.x; idx < h * r; idx += kThreads) {
    const int j = idx / h, i = idx % h;
    const T v = i > j ? A[idx] : zero<T>();
    if (level0) {
      const int64_t row = p * h + i;
      if (row < n) V[(int64_t)j * ldv + row] = v;
    } else {
      V[p * (int64_t)h * r + idx] = v;
    }
  }
}

// Q formation at one level: panel p maps its r x r block C_p to
// H_1 ... H_r [C_p; 0] (h x r).  One warp per column of C; the column lives
// in registers (row i = lane + 32 k).  Level 0 writes rows of Q; higher
// levels write the r x r blocks of their children.
template <typename T, int KM>  // KM >= ceil(h / 32): register chunks of the column, no idle ones
__global__ void __launch_bounds__(kThreads) tsqr_apply_kernel(int level0, const T* V, int64_t ldv,
                                                              const T* tau, int r, int h, int g,
                                                              const T* Cin, T* out, int64_t ldout,
                                                              int64_t n, int64_t nchild) {
  const int64_t p = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.y * (kThreads / 32) + warp;
  if (c >= r) return;
  const int kc = (h + 31) / 32;
  int64_t vrows = h;  // rows of this panel that exist
  if (level0 && p * h + h > n) vrows = n - p * h;
  T w[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const int i = lane + 32 * k;
    w[k] = (k < kc && i < r) ? Cin[p * r * r + (int64_t)c * r + i] : zero<T>();
  }
  for (int j = r - 1; j >= 0; --j) {
    const T t = tau[p * r + j];
    if (absq(t) == 0.0) continue;
    const T* vj = level0 ? V + (int64_t)j * ldv + p * h : V + p * (int64_t)h * r + (int64_t)j * h;
    T vv[KM];
    T dot = zero<T>();
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int i = lane + 32 * k;
      vv[k] = zero<T>();
      if (k < kc && i >= j && i < vrows) {
        vv[k] = i == j ? from_re<T>(1.0) : vj[i];
        dot += conjv(vv[k]) * w[k];
      }
    }
    dot = warp_sum(dot);
    const T f = t * dot;
#pragma unroll
    for (int k = 0; k < KM; ++k) w[k] -= f * vv[k];
  }
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const int i = lane + 32 * k;
    if (k >= kc || i >= h) continue;
    if (level0) {
      const int64_t row = p * h + i;
      if (row < n) out[(int64_t)c * ldout + row] = w[k];
    } else {
      const int64_t blk = p * g + i / r;
      if (blk < nchild) out[blk * r * r + (int64_t)c * r + (i % r)] = w[k];
    }
  }
}

}  // namespace off

// ------------------------------------------------------------------ host

namespace {

using off::Col;
using off::kThreads;

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

sas_status fail_off(sas_status code, const std::string& msg) {
  set_error(msg);
  return code;
}

sas_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
}

// theta_k(p) on the host, the same rules as the online stage.
void theta_host(int rule, int K, const double* p, std::vector<std::complex<double>>& th) {
  th.assign(K, 0.0);
  if (rule == SAS_THETA_PENCIL) {
    th[0] = -1.0;
    th[1] = std::complex<double>(0.0, p[0]);
  } else if (rule == SAS_THETA_DELAY) {
    th[0] = std::complex<double>(0.0, p[0]);
    th[1] = -1.0;
    th[2] = -std::exp(std::complex<double>(0.0, p[0] * p[1]));
  } else {
    th[0] = 1.0;
    for (int k = 1; k < K; ++k) th[k] = p[k - 1];
  }
}

struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { cudaFree(p); }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
  template <typename U> U* as() const { return reinterpret_cast<U*>(p); }
};

// the merged product exists for float32 iterates only
template <typename T, typename TL>
void launch_product_merged(const off::Merged& mg, int K, int64_t n, int B, const TL* theta, const TL* P, TL* Q,
                           const Col<T>* st, T* part, int Gt, size_t smem, cudaStream_t s) {
  if constexpr (sizeof(TL) < sizeof(T))
    off::product_merged_kernel<T, TL><<<Gt, kThreads, smem, s>>>(mg, K, n, B, theta, P, Q, st, part);
}

// The fast Poisson preconditioner's state: DST matrices and eigenvalues per axis, planar
// work buffers, the per-column coefficients and the status word of the transform kernels.
struct PoissonPre {
  int ndim = 0;
  int64_t N[3] = {1, 1, 1};
  DevBuf S[3], mu[3], U, W, coef, status;
};

// One axis of the separable transform, out = in transformed along axis a, for C planar
// columns (x fastest, then y, then z, then the column): float32-accurate tensor-core
// products (three-term bfloat16 splits of both operands, float32 accumulation).
cudaError_t dst_axis(PoissonPre& pp, int a, int64_t C, const float* in, float* out, cudaStream_t s) {
  const int64_t nx = pp.N[0], ny = pp.N[1], nz = pp.N[2], n = nx * ny * nz, nxy = nx * ny;
  const float* Sa = pp.S[a].as<float>();
  int* status = pp.status.as<int>();
  if (a == 0) {  // out[l nx + i] = sum_x in[l nx + x] S_x[i + x nx] over the n / nx * C lines l
    const int64_t L = n / nx * C;
    if (L > (int64_t)65535 * 128) return cudaErrorInvalidValue;
    return gemm_split_tc(s, 3, nullptr, 0, status, (int)L, (int)nx, (int)nx, in, kMlpF32, nx, 1, 0, Sa,
                         kMlpF32, nx, 1, 0, out, nx, 0, 1, 0, nullptr, nullptr);
  }
  if (a == 1)  // per x-y slab b: out_b[y' nx + x] = sum_y S_y[y + y' ny] in_b[y nx + x]
    return gemm_split_tc(s, 3, nullptr, 0, status, (int)ny, (int)nx, (int)ny, Sa, kMlpF32, ny, 1, 0, in,
                         kMlpF32, nx, 1, nxy, out, nx, nxy, (int)(nz * C), 0, nullptr, nullptr);
  // per column c: out_c[z' nxy + xy] = sum_z S_z[z + z' nz] in_c[z nxy + xy]
  return gemm_split_tc(s, 3, nullptr, 0, status, (int)nz, (int)nxy, (int)nz, Sa, kMlpF32, nz, 1, 0, in,
                       kMlpF32, nxy, 1, n, out, nxy, n, (int)C, 0, nullptr, nullptr);
}

template <typename T, typename TL>
sas_status krylov_t(const sas_affine_desc* d, const double* params, int32_t B, T* X, bool warm,
                    bool mixed, bool bicg, double tol, int32_t maxit, const sas_krylov_precond* pc,
                    int32_t* iters_out, double* relres_out) {
  const bool poisson = pc && pc->kind == SAS_PRECOND_POISSON;
  const int64_t n = d->n;
  const int K = d->K;
  const int dp = d->theta_rule == SAS_THETA_PENCIL ? 1 : d->theta_rule == SAS_THETA_DELAY ? 2 : K - 1;
  const int sms = num_sms();
  // vector kernels: about 16 CTAs per SM over the whole batch, rows per CTA a multiple of the block
  int64_t rpc = (n * (int64_t)B + (int64_t)sms * 16 - 1) / ((int64_t)sms * 16);
  rpc = std::max<int64_t>(kThreads, (rpc + kThreads - 1) / kThreads * kThreads);
  const int G = (int)((n + rpc - 1) / rpc);

  const int Gt = (int)((n + off::kTileRows - 1) / off::kTileRows);  // tiles of the product kernel
  const int Gp = std::max(G, Gt);
  const int B4 = (B + 3) / 4;  // quads of columns
  const dim3 qgrid(B4, G);
  const size_t tile_smem = (size_t)B * 4 * sizeof(T) + (size_t)B * 4 * sizeof(double) + (size_t)B * sizeof(int);
  const double delta = mixed ? 0.1 : 0.0;  // replacement once the float32 residual fell 10x

  off::Ops ops;
  for (int k = 0; k < K; ++k) {
    ops.rp[k] = d->rowptr[k];
    ops.ci[k] = d->colind[k];
    ops.va[k] = d->values[k];
    ops.va32[k] = nullptr;
  }
  std::vector<T> th_h((size_t)B * K);
  std::vector<std::complex<double>> th;
  for (int b = 0; b < B; ++b) {
    theta_host(d->theta_rule, K, params + (size_t)b * dp, th);
    for (int k = 0; k < K; ++k) {
      if constexpr (sizeof(T) == 16) {
        th_h[(size_t)b * K + k] = mkz(th[k].real(), th[k].imag());
      } else {
        th_h[(size_t)b * K + k] = th[k].real();
      }
    }
  }
  // theta in the iterates' arithmetic, laid out [quad][k][4] (zero for padding columns)
  std::vector<TL> thl_h((size_t)B4 * K * 4, TL{});
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < K; ++k) {
      const T v = th_h[(size_t)b * K + k];
      TL w;
      if constexpr (sizeof(TL) == sizeof(T)) w = v;
      else if constexpr (sizeof(T) == 16) w = mkzf((float)v.re, (float)v.im);
      else w = (float)v;
      thl_h[((size_t)(b / 4) * K + k) * 4 + (b % 4)] = w;
    }
  DevBuf theta, theta_lo, D, invD, R, P, Q, Xl, prz, ppq, prr, st, bad, nb;
  DevBuf va32[SAS_MAX_TERMS];
  const size_t vec = (size_t)n * B4 * 4 * sizeof(TL);
  cudaError_t e = theta.alloc(th_h.size() * sizeof(T));
  if (e == cudaSuccess) e = theta_lo.alloc(thl_h.size() * sizeof(TL));
  if (e == cudaSuccess) e = D.alloc((size_t)K * n * sizeof(double));
  if (e == cudaSuccess) e = invD.alloc(vec);
  if (e == cudaSuccess) e = R.alloc(vec);
  if (e == cudaSuccess) e = P.alloc(vec);
  if (e == cudaSuccess) e = Q.alloc(vec);
  if (e == cudaSuccess) e = Xl.alloc(vec);
  if (e == cudaSuccess) e = prz.alloc((size_t)B * Gp * sizeof(T));
  if (e == cudaSuccess) e = ppq.alloc((size_t)B * Gt * sizeof(T));
  if (e == cudaSuccess) e = prr.alloc((size_t)B * Gp * sizeof(double));
  if (e == cudaSuccess) e = st.alloc((size_t)B * sizeof(Col<T>));
  if (e == cudaSuccess) e = bad.alloc(sizeof(int));
  if (e == cudaSuccess) e = nb.alloc((size_t)sms * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "krylov: allocation");
  using V = typename std::conditional<sizeof(TL) == sizeof(T), double, float>::type;
  auto* k_lo = off::product_kernel<T, TL, V>;
  auto* k_res = off::residual_kernel<T, TL>;
  e = cudaFuncSetAttribute(k_lo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: shared memory");
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: stream");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{s};
  if (mixed)
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
      int64_t nnz = 0;
      e = cudaMemcpy(&nnz, d->rowptr[k] + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = va32[k].alloc((size_t)std::max<int64_t>(nnz, 1) * sizeof(float));
      if (e == cudaSuccess) {
        off::to_float_kernel<<<sms * 4, kThreads, 0, s>>>(d->values[k], nnz, va32[k].as<float>());
        ops.va32[k] = va32[k].as<float>();
      }
    }
  if (e != cudaSuccess) return cuda_fail(e, "krylov: float copies of the blocks");
  // float32 iterates: merge the blocks into one pattern when they overlap enough that
  // gathering each x entry once for all blocks saves work
  DevBuf mcnt, mbad, mrp, mci, mva;
  off::Merged mg{nullptr, nullptr, nullptr};
  if (mixed && K > 1) {
    e = mcnt.alloc((size_t)n * sizeof(int));
    if (e == cudaSuccess) e = mbad.alloc(sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(mbad.p, 0, sizeof(int), s);
    if (e == cudaSuccess) {
      off::merge_count_kernel<<<sms * 4, kThreads, 0, s>>>(ops, K, n, mcnt.as<int>(), mbad.as<int>());
      e = cudaGetLastError();
    }
    std::vector<int> cnt_h((size_t)n);
    int bad_m = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt_h.data(), mcnt.p, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_m, mbad.p, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "krylov: merged pattern");
    int64_t nnz_sum = 0;
    for (int k = 0; k < K; ++k) {
      int64_t v = 0;
      e = cudaMemcpy(&v, d->rowptr[k] + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "krylov: block sizes");
      nnz_sum += v;
    }
    std::vector<int64_t> rp_h((size_t)n + 1);
    rp_h[0] = 0;
    for (int64_t i = 0; i < n; ++i) rp_h[(size_t)i + 1] = rp_h[(size_t)i] + cnt_h[(size_t)i];
    const int64_t nnz_m = rp_h[(size_t)n];
    if (!bad_m && nnz_m > 0 && 2 * nnz_sum >= 3 * nnz_m) {
      e = mrp.alloc(rp_h.size() * sizeof(int64_t));
      if (e == cudaSuccess) e = mci.alloc((size_t)nnz_m * sizeof(int32_t));
      if (e == cudaSuccess) e = mva.alloc((size_t)nnz_m * K * sizeof(float));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(mrp.p, rp_h.data(), rp_h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        off::merge_fill_kernel<<<sms * 4, kThreads, 0, s>>>(ops, K, n, mrp.as<int64_t>(), mci.as<int32_t>(),
                                                            mva.as<float>());
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // rp_h leaves scope
      if (e != cudaSuccess) return cuda_fail(e, "krylov: merged pattern");
      mg = off::Merged{mrp.as<int64_t>(), mci.as<int32_t>(), mva.as<float>()};
    }
  }
  const size_t merged_smem = (size_t)B * 4 * sizeof(T) + (size_t)B * sizeof(int);
  e = cudaMemcpyAsync(theta.p, th_h.data(), th_h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(theta_lo.p, thl_h.data(), thl_h.size() * sizeof(TL), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad.p, 0, sizeof(int), s);
  if (e == cudaSuccess && !warm) e = cudaMemsetAsync(X, 0, (size_t)n * B * sizeof(T), s);
  for (DevBuf* v : {&Xl, &P, &R, &Q, &invD})  // the padding columns stay zero
    if (e == cudaSuccess) e = cudaMemsetAsync(v->p, 0, vec, s);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: setup copies");
  off::diag_kernel<<<sms * 4, kThreads, 0, s>>>(ops, K, n, D.as<double>());
  off::inv_diag_kernel<T, TL><<<dim3(sms * 2, B), kThreads, 0, s>>>(D.as<double>(), K, n, theta.as<T>(),
                                                                    invD.as<TL>(), bad.as<int>());
  // ||b|| (b viewed as 2n doubles when complex)
  const int64_t bcount = n * (int64_t)(sizeof(T) / sizeof(double));
  off::norm_partial_kernel<<<sms, kThreads, 0, s>>>((const double*)d->b, bcount, nb.as<double>());
  // r = b - A x for every column
  k_res<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta.as<T>(), X, R.as<TL>(), (const T*)d->b,
                                        invD.as<TL>(), st.as<Col<T>>(), off::kSelAll, prz.as<T>(), prr.as<double>());
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "krylov: start launches");
  int bad_h = 0;
  std::vector<double> nb_h((size_t)sms);
  e = cudaMemcpyAsync(&bad_h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nb_h.data(), nb.p, nb_h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: start");
  if (bad_h && !poisson)
    return fail_off(SAS_EINVAL, "krylov: A(p) has a zero (or non-finite) diagonal entry; "
                                "the Jacobi preconditioner needs a non-zero diagonal");
  double bn2 = 0.0;
  for (double v : nb_h) bn2 += v;
  const double bnorm = std::sqrt(bn2);
  if (!(bnorm > 0.0)) return fail_off(SAS_EINVAL, "krylov: b = 0");

  // fast Poisson preconditioner: z = M^-1 r for every active column, written to Q (free between
  // the update and the next product), with the partial sums of r^T z
  PoissonPre pp;
  const int64_t Cpl = (int64_t)B * (off::is_cplx<T>() ? 2 : 1);  // planar float32 columns
  if (poisson) {
    pp.ndim = pc->ndim;
    for (int a = 0; a < 3; ++a) pp.N[a] = a < pc->ndim ? pc->dims[a] : 1;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
      const int64_t Na = pp.N[a];
      e = pp.S[a].alloc((size_t)Na * Na * sizeof(float));
      if (e == cudaSuccess) e = pp.mu[a].alloc((size_t)Na * sizeof(float));
      if (e == cudaSuccess && a < pp.ndim)
        off::dst_matrix_kernel<<<sms * 2, kThreads, 0, s>>>((int)Na, pp.S[a].as<float>(), pp.mu[a].as<float>());
      else if (e == cudaSuccess)
        e = cudaMemsetAsync(pp.mu[a].p, 0, sizeof(float), s);  // an absent axis adds nothing to L
    }
    if (e == cudaSuccess) e = pp.U.alloc((size_t)Cpl * n * sizeof(float));
    if (e == cudaSuccess) e = pp.W.alloc((size_t)Cpl * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(pp.U.p, 0, (size_t)Cpl * n * sizeof(float), s);
    if (e == cudaSuccess) e = pp.coef.alloc((size_t)B * 4 * sizeof(double));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pp.coef.p, pc->coef, (size_t)B * 4 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = pp.status.alloc(sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(pp.status.p, 0, sizeof(int), s);
    if (e == cudaSuccess) e = gemm_f32_tc_prepare();  // before the iteration is captured
    if (e != cudaSuccess) return cuda_fail(e, "krylov: preconditioner buffers");
  }
  double pc_scale = 1.0;
  for (int a = 0; a < pp.ndim; ++a) pc_scale *= 2.0 / (double)(pp.N[a] + 1);
  auto precondition = [&]() -> bool {
    off::unpack_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, R.as<TL>(), pp.U.as<float>(), st.as<Col<T>>(), rpc);
    float* cur = pp.U.as<float>();
    float* oth = pp.W.as<float>();
    for (int pass = 0; pass < 2; ++pass) {
      for (int a = 0; a < pp.ndim; ++a) {
        if (dst_axis(pp, a, Cpl, cur, oth, s) != cudaSuccess) return false;
        std::swap(cur, oth);
      }
      if (pass == 0)
        off::poisson_scale_kernel<T, TL><<<dim3(sms * 2, B), kThreads, 0, s>>>(
            pp.N[0], pp.N[1], pp.N[2], B, cur, pp.mu[0].as<float>(), pp.mu[1].as<float>(), pp.mu[2].as<float>(),
            pp.coef.as<double>(), pc_scale, st.as<Col<T>>());
    }
    off::pack_rz_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, cur, R.as<TL>(), Q.as<TL>(), st.as<Col<T>>(),
                                                          prz.as<T>(), rpc);
    return true;
  };

  const int defer = poisson ? 1 : 0;
  // BiCGStab's extra vectors (float64 iterates only): r_hat, p^, s, s^, t; v lives in Q
  DevBuf Rh, Ph, Sv, Sh, Tv, pz2;
  if (bicg) {
    for (DevBuf* v : {&Rh, &Ph, &Sv, &Sh, &Tv}) {
      if (e == cudaSuccess) e = v->alloc(vec);
      if (e == cudaSuccess) e = cudaMemsetAsync(v->p, 0, vec, s);
    }
    if (e == cudaSuccess) e = pz2.alloc((size_t)B * Gp * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "krylov: BiCGStab buffers");
  }
  if (bicg) {
    off::bicg_replace_kernel<T><<<B, kThreads, 0, s>>>(prr.as<double>(), Gt, bnorm, tol, maxit, 1, st.as<Col<T>>());
  } else {
    off::replace_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), prr.as<double>(), Gt, bnorm, tol, maxit, 1, defer,
                                                  st.as<Col<T>>());
  }
  if (bicg) {
    // the first iteration starts from r (restart flag set by bicg_replace_kernel)
  } else if (poisson) {
    if (!precondition()) return fail_off(SAS_ECUDA, "krylov: preconditioner GEMM failed");
    off::rz_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), G, 1, st.as<Col<T>>());
    off::direction_z_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, Q.as<TL>(), P.as<TL>(), st.as<Col<T>>(), rpc);
  } else {
    off::direction_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, R.as<TL>(), invD.as<TL>(), P.as<TL>(),
                                                            st.as<Col<T>>(), rpc);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "krylov: first direction");

  // the iteration, captured once as a graph of `chunk` steps and replayed
  const int chunk = 16;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: capture");
  for (int it = 0; it < chunk && bicg; ++it) {
    if constexpr (sizeof(TL) == sizeof(T)) {
      T* V = reinterpret_cast<T*>(Q.p);
      off::bicg_dir_kernel<T><<<qgrid, kThreads, 0, s>>>(n, B, (const T*)R.p, Rh.as<T>(), (T*)P.p, V,
                                                         (const T*)invD.p, Ph.as<T>(), st.as<Col<T>>(), rpc);
      k_lo<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta_lo.as<TL>(), (const TL*)Ph.p, Q.as<TL>(),
                                           st.as<Col<T>>(), ppq.as<T>());
      off::bicg_dot_kernel<T><<<qgrid, kThreads, 0, s>>>(n, B, Rh.as<T>(), V, nullptr, nullptr, st.as<Col<T>>(),
                                                         prz.as<T>(), nullptr, rpc);
      off::bicg_alpha_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), G, st.as<Col<T>>());
      off::bicg_s_kernel<T><<<qgrid, kThreads, 0, s>>>(n, B, (const T*)R.p, V, (const T*)invD.p, Sv.as<T>(),
                                                       Sh.as<T>(), st.as<Col<T>>(), rpc);
      k_lo<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta_lo.as<TL>(), (const TL*)Sh.p, (TL*)Tv.p,
                                           st.as<Col<T>>(), ppq.as<T>());
      off::bicg_dot_kernel<T><<<qgrid, kThreads, 0, s>>>(n, B, Tv.as<T>(), Sv.as<T>(), Tv.as<T>(), Tv.as<T>(),
                                                         st.as<Col<T>>(), prz.as<T>(), pz2.as<T>(), rpc);
      off::bicg_omega_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), pz2.as<T>(), G, st.as<Col<T>>());
      off::bicg_xr_kernel<T><<<qgrid, kThreads, 0, s>>>(n, B, (T*)Xl.p, Ph.as<T>(), Sh.as<T>(), Sv.as<T>(),
                                                        Tv.as<T>(), Rh.as<T>(), (T*)R.p, st.as<Col<T>>(),
                                                        prz.as<T>(), prr.as<double>(), rpc);
      off::bicg_beta_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), prr.as<double>(), G, bnorm, tol, maxit,
                                                      st.as<Col<T>>());
      off::fold_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, X, Xl.as<TL>(), st.as<Col<T>>(), 0, rpc);
      k_res<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta.as<T>(), X, R.as<TL>(), (const T*)d->b,
                                            invD.as<TL>(), st.as<Col<T>>(), off::kSelUpd, prz.as<T>(),
                                            prr.as<double>());
      off::bicg_replace_kernel<T><<<B, kThreads, 0, s>>>(prr.as<double>(), Gt, bnorm, tol, maxit, 0,
                                                         st.as<Col<T>>());
    }
  }
  for (int it = 0; it < chunk && !bicg; ++it) {
    if (mg.rp)
      launch_product_merged<T, TL>(mg, K, n, B, theta_lo.as<TL>(), P.as<TL>(), Q.as<TL>(), st.as<Col<T>>(),
                                   ppq.as<T>(), Gt, merged_smem, s);
    else
      k_lo<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta_lo.as<TL>(), P.as<TL>(), Q.as<TL>(),
                                           st.as<Col<T>>(), ppq.as<T>());
    off::alpha_kernel<T><<<B, kThreads, 0, s>>>(ppq.as<T>(), Gt, st.as<Col<T>>());
    off::update_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, Xl.as<TL>(), R.as<TL>(), P.as<TL>(), Q.as<TL>(),
                                                         invD.as<TL>(), st.as<Col<T>>(), prz.as<T>(),
                                                         prr.as<double>(), rpc);
    off::beta_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), prr.as<double>(), G, bnorm, tol, delta, maxit, defer,
                                               st.as<Col<T>>());
    off::fold_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, X, Xl.as<TL>(), st.as<Col<T>>(), 0, rpc);
    k_res<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta.as<T>(), X, R.as<TL>(), (const T*)d->b,
                                          invD.as<TL>(), st.as<Col<T>>(), off::kSelUpd, prz.as<T>(),
                                          prr.as<double>());
    off::replace_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), prr.as<double>(), Gt, bnorm, tol, maxit, 0, defer,
                                                  st.as<Col<T>>());
    if (poisson) {
      if (!precondition()) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        return fail_off(SAS_ECUDA, "krylov: preconditioner GEMM failed in capture");
      }
      off::rz_kernel<T><<<B, kThreads, 0, s>>>(prz.as<T>(), G, 0, st.as<Col<T>>());
      off::direction_z_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, Q.as<TL>(), P.as<TL>(), st.as<Col<T>>(),
                                                                rpc);
    } else {
      off::direction_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, R.as<TL>(), invD.as<TL>(), P.as<TL>(),
                                                              st.as<Col<T>>(), rpc);
    }
  }
  e = cudaStreamEndCapture(s, &graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e, "krylov: graph");
  }
  std::vector<Col<T>> st_h((size_t)B);
  const int64_t max_chunks = ((int64_t)std::max(maxit, 0) + chunk - 1) / chunk + 1;
  for (int64_t ch = 0; ch < max_chunks && e == cudaSuccess; ++ch) {
    e = cudaMemcpyAsync(st_h.data(), st.p, st_h.size() * sizeof(Col<T>), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    bool any = false;
    for (const auto& c : st_h) any = any || c.active;
    if (!any) break;
    e = cudaGraphLaunch(exec, s);
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: iteration");
  e = cudaMemcpyAsync(st_h.data(), st.p, st_h.size() * sizeof(Col<T>), cudaMemcpyDeviceToHost, s);
  // columns that stopped on a breakdown or the iteration limit may hold corrections not yet folded
  off::fold_kernel<T, TL><<<qgrid, kThreads, 0, s>>>(n, B, X, Xl.as<TL>(), st.as<Col<T>>(), 1, rpc);
  // true residual of the returned iterates
  k_res<<<Gt, kThreads, tile_smem, s>>>(ops, K, n, B, theta.as<T>(), X, Q.as<TL>(), (const T*)d->b,
                                        invD.as<TL>(), st.as<Col<T>>(), off::kSelAll, nullptr, prr.as<double>());
  std::vector<double> prr_h((size_t)B * Gt);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(prr_h.data(), prr.p, prr_h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  int tstat = 0;
  if (e == cudaSuccess && poisson)
    e = cudaMemcpyAsync(&tstat, pp.status.p, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "krylov: final residual");
  if (tstat != 0) return fail_off(SAS_ETIMEOUT, "krylov: a preconditioner transform timed out");
  int failed = 0, broke = 0, stalled = 0;
  for (int b = 0; b < B; ++b) {
    double rr = 0.0;
    for (int g = 0; g < Gt; ++g) rr += prr_h[(size_t)b * Gt + g];
    if (iters_out) iters_out[b] = st_h[b].iters;
    if (relres_out) relres_out[b] = std::sqrt(rr) / bnorm;
    if (st_h[b].status != 1) ++failed;
    if (st_h[b].status == 2) ++broke;
    if (st_h[b].status == 4) ++stalled;
  }
  if (failed)
    return fail_off(SAS_ENOCONV, "krylov: " + std::to_string(failed) + " of " + std::to_string(B) +
                                     " columns did not reach the tolerance (" + std::to_string(broke) +
                                     " broke down, " + std::to_string(stalled) +
                                     " stagnated above it); X holds the last iterates");
  return SAS_OK;
}

// panel height for TSQR: a multiple g*r of r with g >= 2, h <= 512, the panel within ~100 KB
// of shared memory where that allows g >= 2, else the largest that fits the opt-in limit.
int tsqr_height(int r, size_t elt, int& g) {
  const size_t soft = 100 * 1024, hard = 227 * 1024 - 1024;
  g = std::max(2, (int)std::min<size_t>(512 / r, soft / ((size_t)r * r * elt)));
  while (g > 2 && (size_t)g * r * r * elt > soft) --g;
  if ((size_t)g * r * r * elt > hard || g * r > 512) return 0;
  return g * r;
}

template <typename T>
sas_status tsqr_t(const T* X, int64_t n, int r, int64_t ldx, T* Qout, int64_t ldq, T* R_host) {
  int g = 0;
  const int h = tsqr_height(r, sizeof(T), g);
  if (h == 0) return fail_off(SAS_ENOTSUP, "tsqr: r too large for a panel in shared memory");
  const size_t smem = (size_t)h * r * sizeof(T);
  // level sizes
  std::vector<int64_t> P{(n + h - 1) / h};
  while (P.back() > 1) P.push_back((P.back() + g - 1) / g);
  const int L = (int)P.size();
  DevBuf V0;
  std::vector<DevBuf> V(L), tau(L), Rb(L), Cb(L);
  cudaError_t e = V0.alloc((size_t)n * r * sizeof(T));
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    if (l > 0) e = V[l].alloc((size_t)P[l] * h * r * sizeof(T));
    if (e == cudaSuccess) e = tau[l].alloc((size_t)P[l] * r * sizeof(T));
    if (e == cudaSuccess) e = Rb[l].alloc((size_t)P[l] * r * r * sizeof(T));
    if (e == cudaSuccess) e = Cb[l].alloc((size_t)P[l] * r * r * sizeof(T));
  }
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: allocation");
  e = cudaFuncSetAttribute(off::tsqr_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: shared memory");
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: stream");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{s};
  for (int l = 0; l < L; ++l) {
    const bool lv0 = l == 0;
    off::tsqr_panel_kernel<T><<<(unsigned)P[l], kThreads, smem, s>>>(
        lv0 ? 1 : 0, lv0 ? X : Rb[l - 1].as<T>(), n, ldx, lv0 ? 0 : P[l - 1], g, r, h,
        lv0 ? V0.as<T>() : V[l].as<T>(), n, tau[l].as<T>(), Rb[l].as<T>());
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: factor launches");
  // top R and the column signs
  std::vector<T> Rt((size_t)r * r);
  e = cudaMemcpyAsync(Rt.data(), Rb[L - 1].p, Rt.size() * sizeof(T), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: top R");
  std::vector<T> Dg((size_t)r * r, zero<T>());
  for (int j = 0; j < r; ++j) {
    double dj;
    if constexpr (sizeof(T) == 16) dj = Rt[(size_t)j * r + j].re;
    else dj = Rt[(size_t)j * r + j];
    const double sg = dj < 0.0 ? -1.0 : 1.0;
    if constexpr (sizeof(T) == 16) Dg[(size_t)j * r + j] = mkz(sg, 0.0);
    else Dg[(size_t)j * r + j] = sg;
    if (R_host)
      for (int c = 0; c < r; ++c) {  // row j of D R
        const T v = Rt[(size_t)c * r + j];
        R_host[(size_t)c * r + j] = c >= j ? rscale(sg, v) : zero<T>();
      }
  }
  e = cudaMemcpyAsync(Cb[L - 1].p, Dg.data(), Dg.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: signs");
  const dim3 cols_grid(1, (r + kThreads / 32 - 1) / (kThreads / 32));
  for (int l = L - 1; l >= 0; --l) {
    const bool lv0 = l == 0;
    const int kc = (h + 31) / 32;
    const dim3 ag((unsigned)P[l], cols_grid.y);
    const T* Vl = lv0 ? V0.as<T>() : V[l].as<T>();
    T* outl = lv0 ? Qout : Cb[l - 1].as<T>();
    const int64_t nch = lv0 ? 0 : P[l - 1];
#define SAS_TSQR_APPLY(KMV) off::tsqr_apply_kernel<T, KMV><<<ag, kThreads, 0, s>>>( \
        lv0 ? 1 : 0, Vl, n, tau[l].as<T>(), r, h, g, Cb[l].as<T>(), outl, ldq, n, nch)
    if (kc <= 2) SAS_TSQR_APPLY(2);
    else if (kc <= 4) SAS_TSQR_APPLY(4);
    else if (kc <= 6) SAS_TSQR_APPLY(6);
    else if (kc <= 8) SAS_TSQR_APPLY(8);
    else if (kc <= 12) SAS_TSQR_APPLY(12);
    else SAS_TSQR_APPLY(16);
#undef SAS_TSQR_APPLY
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "tsqr: Q formation");
  return SAS_OK;
}

}  // namespace
}  // namespace sas

using namespace sas;

sas_status subapsnap_krylov_affine_ex(const sas_affine_desc* d, const double* params, int32_t B, void* X,
                                      int32_t flags, double tol, int32_t maxit, const sas_krylov_precond* pc,
                                      int32_t* iters_out, double* relres_out) {
  const bool warm = (flags & SAS_KRYLOV_WARM) != 0, mixed = (flags & SAS_KRYLOV_MIXED) != 0;
  const bool bicg = (flags & SAS_KRYLOV_BICGSTAB) != 0;
  if (!d || !params || !X) return fail_off(SAS_EINVAL, "NULL argument");
  if (B < 1 || B > 256) return fail_off(SAS_EINVAL, "need 1 <= B <= 256");
  if (d->n < 1) return fail_off(SAS_EINVAL, "need n >= 1");
  if (d->K < 1 || d->K > SAS_MAX_TERMS) return fail_off(SAS_EINVAL, "K must be in [1, 8]");
  if (d->dtype != SAS_REAL64 && d->dtype != SAS_COMPLEX128) return fail_off(SAS_EINVAL, "bad dtype");
  if (d->theta_rule == SAS_THETA_PENCIL && (d->K != 2 || d->dtype != SAS_COMPLEX128))
    return fail_off(SAS_EINVAL, "pencil rule needs K = 2 and complex data");
  if (d->theta_rule == SAS_THETA_DELAY && (d->K != 3 || d->dtype != SAS_COMPLEX128))
    return fail_off(SAS_EINVAL, "delay rule needs K = 3 and complex data");
  if (d->theta_rule != SAS_THETA_LINEAR && d->theta_rule != SAS_THETA_PENCIL &&
      d->theta_rule != SAS_THETA_DELAY)
    return fail_off(SAS_EINVAL, "bad theta rule");
  if (!(tol >= 0.0)) return fail_off(SAS_EINVAL, "tol must be >= 0");
  if (flags & ~(SAS_KRYLOV_WARM | SAS_KRYLOV_MIXED | SAS_KRYLOV_BICGSTAB))
    return fail_off(SAS_EINVAL, "unknown flag bits");
  if (bicg && (mixed || (pc && pc->kind != SAS_PRECOND_JACOBI)))
    return fail_off(SAS_ENOTSUP, "BiCGStab runs float64 iterates with the diagonal preconditioner");
  if (pc) {
    if (pc->kind != SAS_PRECOND_JACOBI && pc->kind != SAS_PRECOND_POISSON)
      return fail_off(SAS_EINVAL, "unknown preconditioner");
    if (pc->kind == SAS_PRECOND_POISSON) {
      if (pc->ndim < 1 || pc->ndim > 3) return fail_off(SAS_EINVAL, "Poisson preconditioner: ndim must be 1, 2 or 3");
      int64_t prod = 1;
      for (int a = 0; a < pc->ndim; ++a) {
        if (pc->dims[a] < 1 || pc->dims[a] > 8192)
          return fail_off(SAS_EINVAL, "Poisson preconditioner: every axis needs 1 <= N <= 8192");
        prod *= pc->dims[a];
      }
      if (prod != d->n) return fail_off(SAS_EINVAL, "Poisson preconditioner: the grid does not have n points");
      if (!pc->coef) return fail_off(SAS_EINVAL, "Poisson preconditioner: coef is NULL");
      for (int b = 0; b < B; ++b) {
        const double* c = pc->coef + 4 * b;
        if (!std::isfinite(c[0]) || !std::isfinite(c[1]) || !std::isfinite(c[2]) || !std::isfinite(c[3]))
          return fail_off(SAS_EINVAL, "Poisson preconditioner: coefficients must be finite");
        if (d->dtype == SAS_REAL64 && (c[1] != 0.0 || c[3] != 0.0))
          return fail_off(SAS_EINVAL, "Poisson preconditioner: real data needs real alpha and beta");
      }
    }
  }
  if (!on_device(X) || !on_device(d->b)) return fail_off(SAS_EINVAL, "X and b must be device pointers");
  for (int k = 0; k < d->K; ++k)
    if (!on_device(d->rowptr[k]) || !on_device(d->colind[k]) || !on_device(d->values[k]))
      return fail_off(SAS_EINVAL, "CSR arrays must be device pointers");
  if (d->dtype == SAS_COMPLEX128)
    return mixed ? krylov_t<zd, zf>(d, params, B, (zd*)X, warm, true, false, tol, maxit, pc, iters_out, relres_out)
                 : krylov_t<zd, zd>(d, params, B, (zd*)X, warm, false, bicg, tol, maxit, pc, iters_out,
                                    relres_out);
  return mixed ? krylov_t<double, float>(d, params, B, (double*)X, warm, true, false, tol, maxit, pc, iters_out,
                                         relres_out)
               : krylov_t<double, double>(d, params, B, (double*)X, warm, false, bicg, tol, maxit, pc, iters_out,
                                          relres_out);
}

sas_status subapsnap_krylov_affine(const sas_affine_desc* d, const double* params, int32_t B, void* X,
                                   int32_t flags, double tol, int32_t maxit, int32_t* iters_out,
                                   double* relres_out) {
  return subapsnap_krylov_affine_ex(d, params, B, X, flags, tol, maxit, nullptr, iters_out, relres_out);
}

sas_status subapsnap_tsqr(const void* X, int64_t n, int32_t r, int64_t ldx, int32_t dtype, void* Q,
                          int64_t ldq, void* R_out) {
  if (!X || !Q) return fail_off(SAS_EINVAL, "NULL argument");
  if (r < 1 || n < r) return fail_off(SAS_EINVAL, "need 1 <= r <= n");
  if (ldx < n || ldq < n) return fail_off(SAS_EINVAL, "leading dimensions must be >= n");
  if (dtype != SAS_REAL64 && dtype != SAS_COMPLEX128) return fail_off(SAS_EINVAL, "bad dtype");
  if (!on_device(X) || !on_device(Q)) return fail_off(SAS_EINVAL, "X and Q must be device pointers");
  if (dtype == SAS_COMPLEX128)
    return tsqr_t<zd>((const zd*)X, n, r, ldx, (zd*)Q, ldq, (zd*)R_out);
  return tsqr_t<double>((const double*)X, n, r, ldx, (double*)Q, ldq, (double*)R_out);
}
