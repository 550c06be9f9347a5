// Batched subsampled least squares of the SubApSnap online stage.
//
// For every parameter p of a batch: assemble M(p) = sum_k theta_k(p) G_k
// (G_k = (A_k)_{J,:} S precomputed; Sec. 3.1 "Computing S A(p*) X") and
// solve min_y ||M y - b_J|| (Alg. 1 step 4) by Householder QR, then back
// substitution.  The residual norm comes for free from the trailing part of
// Q^H b_J; the QoI (c^T S) y (Sec. 5.2.2) is formed in the epilogue.
//
// Plain form: float64 / complex128 throughout, one CTA per parameter.  When
// s x (r+1) does not fit in shared memory, rows are streamed in blocks of t:
// the first block is factorised in place, every later block is folded into
// the r x r triangle by the Householder update of the stacked [R; P] (the
// row-blocked, sequential form of TSQR).  The result is the same QR up to
// rounding.
//
// Mixed form (not in the paper): float32 assembly and Householder QR with the
// reflectors kept, then iterative refinement y += R^{-1} Q^H (b_J - M y) where
// the residual is formed in float64 from the float64 blocks.
#include "sas_internal.cuh"

namespace sas {

template <typename T> __device__ inline T theta_k(int rule, int k, const double* p);
template <> __device__ inline double theta_k<double>(int rule, int k, const double* p) {
  (void)rule;
  return k == 0 ? 1.0 : p[k - 1];
}
template <> __device__ inline zd theta_k<zd>(int rule, int k, const double* p) {
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

template <int NT>
__device__ inline double block_sum(double v, double* red) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) tot += red[w];
  __syncthreads();
  return tot;
}

// One Householder step on the stacked column [piv_k; tail_k(0..len-1)], applied
// to columns k+1..ncol-1 (the last column is the right-hand side).  Column j's
// pivot-row entry sits at piv[j*ldp], its tail at tail + j*ldt.  The reflector is
// H = I - tau v v^H with v = x - beta e_1, beta = -phase(alpha) ||x||, so that
// H x = beta e_1 and H = H^H; on return piv[k*ldp] holds beta (= R_kk).
//
// Thread map: G consecutive lanes share a column; lane g of the group takes the
// rows g, g + G, ... of the tail, and the G partial dot products are combined
// with log2(G) shuffles inside the group.  The NT/G groups take columns
// k+1+slot, k+1+slot+NT/G, ...  One barrier per step: nrm2[k & 1] must hold
// ||tail_k||^2 on entry (the caller's pre-pass for k = 0); the group that owns
// column k+1 writes ||tail_{k+1}[next_off..len)||^2 to nrm2[(k+1) & 1].
template <typename T, typename R, int NT, int G>
__device__ inline void householder_step(int k, int ncol, T* piv, int ldp, T* tail, int ldt, int len,
                                        int next_off, R* nrm2, T* v0_out, R* tau_out) {
  constexpr int NSLOT = NT / G;
  const int tid = threadIdx.x, g = tid % G, slot = tid / G;
  const unsigned gmask = ((1u << G) - 1u) << ((tid & 31) & ~(G - 1));
  const T* tk = tail + (size_t)k * ldt;
  const R tail2 = nrm2[k & 1];
  const T alpha = piv[(size_t)k * ldp];
  const R a2 = absq(alpha);
  const R nrm = sqrt(a2 + tail2);
  const R aa = sqrt(a2);
  const T beta = rscale(-nrm, phase(alpha));
  const T v0 = alpha - beta;
  const R tau = nrm > R(0) ? R(1) / (nrm * (nrm + aa)) : R(0);
  for (int j = k + 1 + slot; j < ncol; j += NSLOT) {
    T* tj = tail + (size_t)j * ldt;
    T w = g == 0 ? conjv(v0) * piv[(size_t)j * ldp] : zero<T>();
    for (int i = g; i < len; i += G) w += conjv(tk[i]) * tj[i];
#pragma unroll
    for (int o = 1; o < G; o <<= 1) w += shfl_xor_m(gmask, w, o);
    const T tw = rscale(tau, w);
    if (g == 0) piv[(size_t)j * ldp] -= tw * v0;
    for (int i = g; i < len; i += G) tj[i] -= tw * tk[i];
    if (j == k + 1) {
      __syncwarp(gmask);
      R part = R(0);
      for (int i = next_off + g; i < len; i += G) part += absq(tj[i]);
#pragma unroll
      for (int o = 1; o < G; o <<= 1) part += shfl_xor_m(gmask, part, o);
      if (g == 0) nrm2[(k + 1) & 1] = part;
    }
  }
  __syncthreads();
  if (tid == 0) {
    piv[(size_t)k * ldp] = beta;
    if (v0_out) v0_out[k] = v0;
    if (tau_out) tau_out[k] = tau;
  }
}

// Leading dimension of a shared-memory panel with `rows` rows of elements of
// `es` bytes: the smallest ld >= rows with ld = 4 (mod 128 / es), so that the
// column groups of a warp (4 lanes each, 8 groups) spread over the banks with
// no more wavefronts than the access size needs; at most 128/es - 1 rows of
// padding.
__host__ __device__ inline int panel_ld(int rows, int es) {
  const int mod = 128 / es;
  return rows + ((4 - rows % mod) % mod + mod) % mod;
}

// ||col[0..len)||^2 by warp 0 into *slot (the caller synchronises afterwards).
template <typename T, typename R>
__device__ inline void tail_norm_warp0(const T* col, int len, R* slot) {
  if ((threadIdx.x >> 5) != 0) return;
  const int lane = threadIdx.x & 31;
  R part = R(0);
  for (int i = lane; i < len; i += 32) part += absq(col[i]);
  part = warp_sum(part);
  if (lane == 0) *slot = part;
}

// Back substitution R y = z by one warp: R upper triangular r x r (ld ldr), z
// in registers distributed as z[lane + 32 c].  Writes y to ys[0..r).  Returns
// min/max |R_ii| through dmin/dmax (lane 0).
template <typename T, typename R>
__device__ inline void backsolve_warp(const T* Rm, int ldr, int r, T* zr /*[4]*/, T* ys, R& dmin,
                                      R& dmax) {
  const int lane = threadIdx.x & 31;
  dmin = R(INFINITY);
  dmax = R(0);
  for (int i = r - 1; i >= 0; --i) {
    const int owner = i & 31, slot = i >> 5;
    const T rii = Rm[i + (size_t)i * ldr];
    T zi = zero<T>();
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c == slot) zi = zr[c];
    zi = shfl_idx(zi, owner);
    const T yi = divv(zi, rii);
    if (lane == 0) ys[i] = yi;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = lane + 32 * c;
      if (j < i) zr[c] -= Rm[j + (size_t)i * ldr] * yi;
    }
    const R ad = sqrt(absq(rii));
    dmin = ad < dmin ? ad : dmin;
    dmax = ad > dmax ? ad : dmax;
  }
  __syncwarp();
}

// ------------------------------------------------------------------ plain
template <typename T>
struct LsPlainArgs {
  const T* Mg;  // dense M per parameter (m x s x r, ld s), or null: assemble from G
  const T* G;
  const T* bJ;
  const T* wq;
  const double* params;
  int64_t m;
  int s, r, K, dp, rule, t, ldt;
  double bJ_norm;
  T* yout;
  T* qoi;
  uint32_t* flags;
  double* rho;
};

// One parameter q of the plain solve (shared by the grid-stride and the
// persistent multi-problem kernels).
template <typename T, int NT, int G>
__device__ __forceinline__ void ls_plain_body(const LsPlainArgs<T>& a, int64_t q,
                                              unsigned char* smem_raw, double* nrm2) {

  const int s = a.s, r = a.r, t = a.t, ldt = a.ldt, K = a.K;
  const bool single = t >= s;
  const int ldr = single ? ldt : r;
  T* P = reinterpret_cast<T*>(smem_raw);
  T* Rm = single ? P : P + (size_t)ldt * (r + 1);
  T* th = P + (size_t)ldt * (r + 1) + (single ? 0 : (size_t)r * (r + 1));
  T* ys = th + kMaxDp;
  double* red = reinterpret_cast<double*>(ys + kMaxR);
  const int tid = threadIdx.x, warp = tid >> 5;


    if (tid < K) th[tid] = theta_k<T>(a.rule, tid, a.params + q * a.dp);
    __syncthreads();
    double res2 = 0.0;
    for (int row0 = 0; row0 < s; row0 += t) {
      const int tb = min(t, s - row0);
      for (int idx = tid; idx < tb * (r + 1); idx += NT) {
        const int i = idx % tb, j = idx / tb;
        T v;
        if (j < r) {
          if (a.Mg) {
            v = a.Mg[(size_t)q * s * r + (size_t)j * s + row0 + i];
          } else {
            v = zero<T>();
            const T* g = a.G + (size_t)j * s + row0 + i;
            for (int k = 0; k < K; ++k) v += th[k] * g[(size_t)k * s * r];
          }
        } else {
          v = a.bJ[row0 + i];
        }
        P[i + (size_t)j * ldt] = v;
      }
      __syncthreads();
      if (row0 == 0) {
        tail_norm_warp0<T, double>(P + 1, tb - 1, &nrm2[0]);
        __syncthreads();
        for (int k = 0; k < r; ++k)
          householder_step<T, double, NT, G>(k, r + 1, P + k, ldt, P + k + 1, ldt, tb - k - 1, 1,
                                             nrm2, (T*)nullptr, (double*)nullptr);
        __syncthreads();
        double part = 0.0;
        for (int i = r + tid; i < tb; i += NT) part += absq(P[i + (size_t)r * ldt]);
        res2 += block_sum<NT>(part, red);
        if (!single) {
          for (int idx = tid; idx < r * (r + 1); idx += NT) {
            const int i = idx % r, j = idx / r;
            Rm[i + (size_t)j * r] = P[i + (size_t)j * ldt];
          }
        }
      } else {
        tail_norm_warp0<T, double>(P, tb, &nrm2[0]);
        __syncthreads();
        for (int k = 0; k < r; ++k)
          householder_step<T, double, NT, G>(k, r + 1, Rm + k, r, P, ldt, tb, 0, nrm2,
                                             (T*)nullptr, (double*)nullptr);
        __syncthreads();
        double part = 0.0;
        for (int i = tid; i < tb; i += NT) part += absq(P[i + (size_t)r * ldt]);
        res2 += block_sum<NT>(part, red);
      }
      __syncthreads();
    }
    if (warp == 0) {
      T zr[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = (tid & 31) + 32 * c;
        zr[c] = i < r ? Rm[i + (size_t)r * ldr] : zero<T>();
      }
      double dmin, dmax;
      backsolve_warp<T, double>(Rm, ldr, r, zr, ys, dmin, dmax);
      const int lane = tid & 31;
      bool fin = true;
      T h = zero<T>();
      for (int i = lane; i < r; i += 32) {
        const T yi = ys[i];
        fin = fin && finitev(yi);
        if (a.yout) a.yout[q * r + i] = yi;
        if (a.qoi) h += a.wq[i] * yi;
      }
      fin = __all_sync(0xffffffffu, fin);
      if (a.qoi) {
        h = warp_sum(h);
        if (lane == 0) a.qoi[q] = h;
      }
      if (lane == 0) {
        if (a.rho) a.rho[q] = sqrt(res2) / a.bJ_norm;
        if (a.flags) {
          uint32_t f = 0;
          if (!(dmin > 1e-13 * dmax)) f |= SAS_FLAG_ILLCOND;
          if (!fin) f |= SAS_FLAG_NONFINITE;
          a.flags[q] = f;
        }
      }
    }
    __syncthreads();
  }

template <typename T, int NT, int G>
__global__ void __launch_bounds__(NT, 512 / NT) ls_plain_affine_kernel(LsPlainArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double nrm2[2];
  for (int64_t q = blockIdx.x; q < a.m; q += gridDim.x) ls_plain_body<T, NT, G>(a, q, smem_raw, nrm2);
}

constexpr int kLsThreads = 256;  // largest CTA of any variant (sizes the reduction scratch)
constexpr size_t kSmemLimit = 227 * 1024 - 1024;

// Launch shapes of the least-squares kernels: threads per CTA and lanes per
// column group of the Householder step; the mixed kernel also chooses whether
// to keep M in float64 shared memory (when it fits).  The autotuner times
// them per context.
struct LsShape {
  int nt, g;
};
static const LsShape kLsShapes[] = {{256, 4}, {128, 4}, {256, 8}, {128, 2}, {256, 2}};
constexpr int kNumLsShapes = sizeof(kLsShapes) / sizeof(kLsShapes[0]);

// Blocked Householder variants of the mixed kernel (real only): threads,
// lanes per column group, registers per lane for a trailing column (s <= G E).
struct LsBlockedShape {
  // pw: 0 panel factorised by the CTA; 1 by warp 0 alone (warp-synchronous); 2 by
  // warp 0 with the panel in registers, and the refinement corrections too (s <= 128)
  int nt, g, e, pw;
};
static const LsBlockedShape kLsBlocked[] = {{128, 4, 32, 0}, {128, 8, 16, 0}, {256, 8, 32, 0},
                                            {128, 8, 32, 0}, {128, 8, 16, 1}, {128, 4, 32, 1},
                                            {256, 8, 32, 1}, {128, 8, 16, 1}, {128, 8, 16, 2}};
constexpr int kLsRegRows = 128;  // largest s of the register-panel variant (4 rows per lane)
constexpr int kNumLsBlocked = sizeof(kLsBlocked) / sizeof(kLsBlocked[0]);
constexpr int kLsPanel = 8;  // columns per panel of the blocked variants
constexpr int kFirstBlocked = 3 * kNumLsShapes + 2;

// plain: the smem shapes, then one register-resident variant; mixed: the smem
// shapes with the float64 M in shared memory, without it, two register-resident
// variants, the smem shapes with the float64 M in a global slot per CTA, then
// the blocked variants (M in a global slot)
int ls_num_variants(bool mixed) {
  return mixed ? kFirstBlocked + kNumLsBlocked : kNumLsShapes + 1;
}

// Mixed variant index -> shape index; -1 for the register-resident variants,
// -2 for the blocked ones.
static int mixed_shape(int v) {
  if (v < 2 * kNumLsShapes) return v % kNumLsShapes;
  if (v < 2 * kNumLsShapes + 2) return -1;
  if (v < kFirstBlocked) return v - (2 * kNumLsShapes + 2);
  return -2;
}
// Where the float64 M lives: 1 shared memory, 0 recomputed, 2 a global slot.
static int mixed_keep_kind(int v) {
  if (v < kNumLsShapes) return 1;
  if (v < 2 * kNumLsShapes + 2) return 0;
  return 2;
}

size_t ls_plain_smem_bytes(const sas_ctx* c, int* rows_per_block) {
  const size_t es = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  const size_t extra = (size_t)(kMaxDp + kMaxR) * es + (kLsThreads / 32) * 8;
  const int ies = (int)es;
  const size_t single = (size_t)panel_ld(c->s, ies) * (c->r + 1) * es + extra;
  if (single <= kSmemLimit) {
    *rows_per_block = c->s;
    return single;
  }
  const size_t rbuf = (size_t)c->r * (c->r + 1) * es;
  if (rbuf + extra >= kSmemLimit) return 0;
  int t = (int)((kSmemLimit - rbuf - extra) / ((c->r + 1) * es));
  if (t > c->s) t = c->s;
  while (t >= c->r && (size_t)panel_ld(t, ies) * (c->r + 1) * es + rbuf + extra > kSmemLimit) --t;
  if (t < c->r) return 0;
  *rows_per_block = t;
  return (size_t)panel_ld(t, ies) * (c->r + 1) * es + rbuf + extra;
}

template <typename T>
static size_t fill_plain_args(const sas_ctx* c, const double* params, int64_t m, void* yout,
                              void* qoi, uint32_t* flags, double* rho, const void* Mg,
                              LsPlainArgs<T>& a) {
  int t = 0;
  const size_t smem = ls_plain_smem_bytes(c, &t);
  if (smem == 0) return 0;
  a.Mg = (const T*)Mg;
  a.G = (const T*)c->G;
  a.bJ = (const T*)c->bJ;
  a.wq = (const T*)c->wq;
  a.params = params;
  a.m = m;
  a.s = c->s;
  a.r = c->r;
  a.K = c->K;
  a.dp = c->dp;
  a.rule = c->theta_rule;
  a.t = t;
  a.ldt = panel_ld(t, (int)sizeof(T));
  a.bJ_norm = c->bJ_norm;
  a.yout = (T*)yout;
  a.qoi = (T*)qoi;
  a.flags = flags;
  a.rho = rho;
  return smem;
}

template <typename T>
static cudaError_t launch_plain_t(const sas_ctx* c, const double* params, int64_t m, void* yout,
                                  void* qoi, uint32_t* flags, double* rho, cudaStream_t st,
                                  const void* Mg) {
  LsPlainArgs<T> a;
  const size_t smem = fill_plain_args<T>(c, params, m, yout, qoi, flags, rho, Mg, a);
  if (smem == 0) return cudaErrorInvalidConfiguration;
  if (c->ls_variant_plain >= kNumLsShapes) {
    if constexpr (sizeof(T) == 8) return launch_plain_reg(c, a, m, st);
    return cudaErrorInvalidConfiguration;
  }
  const int v = c->ls_variant_plain % kNumLsShapes;
  void (*kern)(LsPlainArgs<T>) = nullptr;
  switch (v) {
    case 0: kern = ls_plain_affine_kernel<T, 256, 4>; break;
    case 1: kern = ls_plain_affine_kernel<T, 128, 4>; break;
    case 2: kern = ls_plain_affine_kernel<T, 256, 8>; break;
    case 3: kern = ls_plain_affine_kernel<T, 128, 2>; break;
    default: kern = ls_plain_affine_kernel<T, 256, 2>; break;
  }
  const int nt = kLsShapes[v].nt;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (grid > m) grid = m;
  kern<<<(unsigned)grid, nt, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ls_plain(const sas_ctx* c, const double* params, int64_t m, void* yout,
                            void* qoi, uint32_t* flags, double* rho, cudaStream_t st,
                            const void* Mg) {
  if (m == 0) return cudaSuccess;
  if (c->dtype == SAS_COMPLEX128)
    return launch_plain_t<zd>(c, params, m, yout, qoi, flags, rho, st, Mg);
  return launch_plain_t<double>(c, params, m, yout, qoi, flags, rho, st, Mg);
}

// ------------------------------------------------------------------ mixed
template <typename TH, typename TL>
struct LsMixedArgs {
  const TH* Mg;     // dense M per parameter (m x s x r, ld s), or null: assemble from G
  const TH* G;      // float64 blocks
  const TL* G32;    // float32 blocks (used when M64 is not kept)
  const TH* bJ;
  const TL* bJ32;
  const TH* wq;
  const double* params;
  int64_t m;
  int s, r, K, dp, rule, ldt, rpad, max_refine;
  int keep64;       // M in float64: 0 recomputed per residual, 1 shared memory, 2 global slot
  TH* M64g;         // keep64 == 2: nslots slots of s x r, one per CTA (L2-resident)
  int nslots;
  double bJ_norm, tol;
  TH* yout;
  TH* qoi;
  float* ysplit;    // real only: [2][m][rpad] tf32 hi / lo parts of y (or null)
  uint32_t* flags;
  double* rho;
};

__device__ inline float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// Mixed-precision solve of one parameter per CTA iteration.
//  1. theta(p); M assembled once in float64 (kept in shared memory when it
//     fits, keep64) and rounded to float32 for the factorisation;
//  2. float32 Householder QR with the reflectors kept below the diagonal;
//  3. y = R^{-1} [Q^H b_J]_{0:r};
//  4. refinement: res = b_J - M y in float64, delta = R^{-1} [Q^H res]_{0:r} in
//     float32, y += delta, until ||delta|| <= tol ||y|| or a step no longer
//     halves the correction; the last residual evaluated belongs to the
//     returned y, so rho is exact in float64.
// One parameter q of the mixed solve (shared by the grid-stride and the
// persistent multi-problem kernels).
// Blocked form of the Householder sweep (real float32 panel): after the
// reflectors of panel columns [c0, pe) are formed, each trailing column j in
// [pe, ncol) is loaded once into registers (rows c0 + g + G e of lane g of its
// column group), all panel reflectors are applied there in order, and it is
// stored back.  Vb holds the panel's reflectors as full columns of length s
// (zero above the diagonal, v0 on it); tau their scales.  The same products as
// the column-by-column sweep, with one shared-memory pass over the trailing
// matrix per panel instead of one per reflector.
// Panel factorisation by warp 0 alone (real float32): reflectors of columns
// [c0, pe), each applied to the rest of the panel, with warp shuffles and no
// CTA barrier; the same reflector formulas as householder_step.
__device__ inline void panel_warp0(float* P, int ldt, int s, int c0, int pe, float* v0s,
                                   float* taus) {
  const int lane = threadIdx.x & 31;
  for (int k = c0; k < pe; ++k) {
    const float* pk = P + (size_t)k * ldt;
    float t2 = 0.f;
    for (int i = k + 1 + lane; i < s; i += 32) t2 = fmaf(pk[i], pk[i], t2);
    t2 = warp_sum(t2);
    const float alpha = pk[k];
    const float nrm = sqrtf(alpha * alpha + t2);
    const float beta = -nrm * phase(alpha);
    const float v0 = alpha - beta;
    const float tau = nrm > 0.f ? 1.f / (nrm * (nrm + fabsf(alpha))) : 0.f;
    for (int j = k + 1; j < pe; ++j) {
      float* pj = P + (size_t)j * ldt;
      float w = lane == 0 ? v0 * pj[k] : 0.f;
      for (int i = k + 1 + lane; i < s; i += 32) w = fmaf(pk[i], pj[i], w);
      w = warp_sum(w);
      const float tw = tau * w;
      if (lane == 0) pj[k] -= tw * v0;
      for (int i = k + 1 + lane; i < s; i += 32) pj[i] = fmaf(-tw, pk[i], pj[i]);
      __syncwarp();
    }
    if (lane == 0) {
      P[k + (size_t)k * ldt] = beta;
      v0s[k] = v0;
      taus[k] = tau;
    }
    __syncwarp();
  }
}

// Sum over the warp, every lane receiving it (xor butterfly).
__device__ inline float butterfly_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Element (i & 3) of a lane's four rows, taken from lane i >> 2.
__device__ inline float row_of(const float (&x)[4], int i) {
  float v = x[0];
  v = (i & 3) == 1 ? x[1] : v;
  v = (i & 3) == 2 ? x[2] : v;
  v = (i & 3) == 3 ? x[3] : v;
  return __shfl_sync(0xffffffffu, v, i >> 2);
}

// Rows 4 lane .. 4 lane + 3 of column c of P (16 bytes: the panel and its leading
// dimension are 16-byte aligned), rows >= s as zeros.
__device__ inline void load_rows4(const float* P, int ldt, int s, int c, float (&x)[4]) {
  const int i0 = 4 * (threadIdx.x & 31);
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i0 < s) q = *reinterpret_cast<const float4*>(P + (size_t)c * ldt + i0);
  x[0] = q.x;
  x[1] = i0 + 1 < s ? q.y : 0.f;
  x[2] = i0 + 2 < s ? q.z : 0.f;
  x[3] = i0 + 3 < s ? q.w : 0.f;
}

// Panel factorisation by one warp with the panel in registers (s <= 128): lane l
// holds rows 4l .. 4l+3 of the panel's nb <= BW columns, loaded and stored with one
// 16-byte access per column.  Each reflector costs a few multiply-adds per column
// and one butterfly for all of the panel's remaining columns together; the
// reflector formulas are those of householder_step.
template <int BW>
__device__ inline void panel_regs(float* P, int ldt, int s, int c0, int nb, float* v0s,
                                  float* taus) {
  const int lane = threadIdx.x & 31, i0 = 4 * lane;
  float col[BW][4];
#pragma unroll
  for (int a = 0; a < BW; ++a) {
    if (a < nb) {
      load_rows4(P, ldt, s, c0 + a, col[a]);
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) col[a][t] = 0.f;
    }
  }
#pragma unroll
  for (int a = 0; a < BW; ++a) {
    if (a < nb) {
      const int k = c0 + a;
      float t2 = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float x = i0 + t > k ? col[a][t] : 0.f;
        t2 = fmaf(x, x, t2);
      }
      t2 = butterfly_sum(t2);
      const float alpha = row_of(col[a], k);
      const float nrm = sqrtf(alpha * alpha + t2);
      const float beta = -nrm * phase(alpha);
      const float v0 = alpha - beta;
      const float tau = nrm > 0.f ? 1.f / (nrm * (nrm + fabsf(alpha))) : 0.f;
      float vv[4];  // this lane's rows of the reflector (v0 at row k, zero above)
#pragma unroll
      for (int t = 0; t < 4; ++t) vv[t] = i0 + t > k ? col[a][t] : (i0 + t == k ? v0 : 0.f);
      float w[BW];
#pragma unroll
      for (int j = 0; j < BW; ++j) {
        w[j] = 0.f;
        if (j > a && j < nb) {
#pragma unroll
          for (int t = 0; t < 4; ++t) w[j] = fmaf(vv[t], col[j][t], w[j]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = a + 1; j < BW; ++j)
          if (j < nb) w[j] += __shfl_xor_sync(0xffffffffu, w[j], o);
      }
#pragma unroll
      for (int j = a + 1; j < BW; ++j) {
        if (j < nb) {
          const float tw = tau * w[j];
#pragma unroll
          for (int t = 0; t < 4; ++t) col[j][t] = fmaf(-tw, vv[t], col[j][t]);
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (i0 + t == k) col[a][t] = beta;
      if (lane == 0) {
        v0s[k] = v0;
        taus[k] = tau;
      }
    }
  }
  if (i0 < s) {
#pragma unroll
    for (int a = 0; a < BW; ++a)
      if (a < nb)
        *reinterpret_cast<float4*>(P + (size_t)(c0 + a) * ldt + i0) =
            make_float4(col[a][0], col[a][1], col[a][2], col[a][3]);
  }
  __syncwarp();
}

// One refinement correction by one warp with the vector in registers (s <= 128;
// lane l holds rows 4l .. 4l+3): x = Q^T res (float32) one reflector at a time, each a
// 16-byte load of its column, four multiply-adds, a butterfly and four more; then
// R delta = x_{0:r} by back substitution with the reciprocal diagonal rinv.  Writes
// delta to dl[0..r).
__device__ inline void correction_regs(const float* P, int ldt, int s, int r, const double* res,
                                       const float* v0, const float* tau, const float* rinv,
                                       float* dl) {
  const int lane = threadIdx.x & 31, i0 = 4 * lane;
  float x[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) x[t] = i0 + t < s ? (float)res[i0 + t] : 0.f;
#pragma unroll 2
  for (int k = 0; k < r; ++k) {
    float vv[4];
    load_rows4(P, ldt, s, k, vv);
    const float vk0 = v0[k], tk = tau[k];
#pragma unroll
    for (int t = 0; t < 4; ++t) vv[t] = i0 + t > k ? vv[t] : (i0 + t == k ? vk0 : 0.f);
    float w = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) w = fmaf(vv[t], x[t], w);
    const float tw = tk * butterfly_sum(w);
#pragma unroll
    for (int t = 0; t < 4; ++t) x[t] = fmaf(-tw, vv[t], x[t]);
  }
  for (int i = r - 1; i >= 0; --i) {
    const float yi = row_of(x, i) * rinv[i];
    if (lane == 0) dl[i] = yi;
    float rc[4];
    load_rows4(P, ldt, s, i, rc);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (i0 + t < i) x[t] = fmaf(-rc[t], yi, x[t]);
  }
  __syncwarp();
}

template <int NT, int G, int E>
__device__ inline void blocked_trailing_update(float* P, int ldt, int s, int c0, int pe, int ncol,
                                               const float* Vb, const float* tau) {
  constexpr int NSLOT = NT / G;
  const int tid = threadIdx.x, g = tid % G, slot = tid / G;
  const unsigned gmask = ((1u << G) - 1u) << ((tid & 31) & ~(G - 1));
  for (int j = pe + slot; j < ncol; j += NSLOT) {
    float* pj = P + (size_t)j * ldt;
    float av[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = c0 + g + G * e;
      av[e] = i < s ? pj[i] : 0.f;
    }
    for (int k = c0; k < pe; ++k) {
      const float* v = Vb + (size_t)(k - c0) * s;
      float vv[E];
      float w = 0.f;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int i = c0 + g + G * e;
        vv[e] = i < s ? v[i] : 0.f;
        w = fmaf(vv[e], av[e], w);
      }
#pragma unroll
      for (int o = 1; o < G; o <<= 1) w += __shfl_xor_sync(gmask, w, o);
      const float tw = tau[k] * w;
#pragma unroll
      for (int e = 0; e < E; ++e) av[e] = fmaf(-tw, vv[e], av[e]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = c0 + g + G * e;
      if (i < s) pj[i] = av[e];
    }
  }
}

template <typename TH, typename TL, int NT, int G, int BW = 0, int E = 0, int PW = 0>
__device__ __forceinline__ void ls_mixed_body(const LsMixedArgs<TH, TL>& a, int64_t q,
                                              unsigned char* smem_raw, double* ctl) {

  const int s = a.s, r = a.r, ldt = a.ldt, K = a.K;
  TH* th = reinterpret_cast<TH*>(smem_raw);      // kMaxDp
  TH* y = th + kMaxDp;                           // kMaxR
  TH* res = y + kMaxR;                           // kMaxS (float64 residual)
  double* red = reinterpret_cast<double*>(res + kMaxS);  // NT/32
  TL* th32 = reinterpret_cast<TL*>(red + NT / 32);
  TL* v0 = th32 + kMaxDp;                        // kMaxR
  TL* dl = v0 + kMaxR;                           // kMaxR (correction)
  float* tau = reinterpret_cast<float*>(dl + kMaxR);  // kMaxR
  float* nrm2 = tau + kMaxR;                     // 2 (+2 padding)
  TL* P = reinterpret_cast<TL*>(nrm2 + 4);       // ldt x (r+1)
  // the register-panel variant moves rows of P four at a time in 16-byte accesses
  static_assert(PW != 2 || ((kMaxDp + kMaxR + kMaxS + NT / 32) * sizeof(TH) +
                            (kMaxDp + 3 * kMaxR + 4) * sizeof(TL)) % 16 == 0,
                "P must start on a 16-byte boundary");
  // float64 M: in shared memory (keep64 1), in this CTA's global slot (keep64 2)
  // or not kept (recomputed from the blocks for every residual)
  const bool gslot = a.keep64 == 2 && (int)blockIdx.x < a.nslots;
  const bool keep = a.keep64 == 1 || gslot;
  // blocked form: the panel's reflectors as full columns, BW x s, after P
  float* Vb = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(P + (size_t)ldt * (r + 1)) + 15) & ~(uintptr_t)15);
  TH* M64 = gslot ? a.M64g + (size_t)blockIdx.x * s * r
                  : reinterpret_cast<TH*>(
                        (reinterpret_cast<uintptr_t>(Vb + (size_t)BW * s) + 15) &
                        ~(uintptr_t)15);  // s x r
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;


    if (tid < K) {
      th[tid] = theta_k<TH>(a.rule, tid, a.params + q * a.dp);
      th32[tid] = to_lo(th[tid]);
    }
    __syncthreads();
    if (keep) {
      for (int idx = tid; idx < s * r; idx += NT) {
        const int i = idx % s, j = idx / s;
        TH v = zero<TH>();
        if (a.Mg) {
          v = a.Mg[(size_t)q * s * r + idx];
        } else {
          const TH* g = a.G + idx;
          for (int k = 0; k < K; ++k) v += th[k] * g[(size_t)k * s * r];
        }
        M64[idx] = v;
        P[i + (size_t)j * ldt] = to_lo(v);
      }
      for (int i = tid; i < s; i += NT) P[i + (size_t)r * ldt] = a.bJ32[i];
    } else {
      for (int idx = tid; idx < s * (r + 1); idx += NT) {
        const int i = idx % s, j = idx / s;
        TL v;
        if (j < r) {
          if (a.Mg) {
            v = to_lo(a.Mg[(size_t)q * s * r + idx]);
          } else {
            v = zero<TL>();
            const TL* g = a.G32 + (size_t)j * s + i;
            for (int k = 0; k < K; ++k) v += th32[k] * g[(size_t)k * s * r];
          }
        } else {
          v = a.bJ32[i];
        }
        P[i + (size_t)j * ldt] = v;
      }
    }
    __syncthreads();
    tail_norm_warp0<TL, float>(P + 1, s - 1, &nrm2[0]);
    __syncthreads();
    if constexpr (BW > 0) {
      // panels of BW columns: reflectors within the panel, then one register pass
      // over every trailing column (the right-hand side included)
      for (int c0 = 0; c0 < r; c0 += BW) {
        const int pe = c0 + BW < r ? c0 + BW : r;
        if constexpr (PW == 2) {
          if (warp == 0) panel_regs<BW>(P, ldt, s, c0, pe - c0, v0, tau);
        } else if constexpr (PW) {
          if (warp == 0) panel_warp0(P, ldt, s, c0, pe, v0, tau);
        } else {
          for (int k = c0; k < pe; ++k)
            householder_step<TL, float, NT, G>(k, pe, P + k, ldt, P + k + 1, ldt, s - k - 1, 1, nrm2,
                                               v0, tau);
        }
        __syncthreads();
        for (int idx = tid; idx < (pe - c0) * s; idx += NT) {
          const int kk = idx / s, i = idx % s, k = c0 + kk;
          Vb[idx] = i < k ? 0.f : (i == k ? v0[k] : P[i + (size_t)k * ldt]);
        }
        __syncthreads();
        blocked_trailing_update<NT, G, E>(P, ldt, s, c0, pe, r + 1, Vb, tau);
        __syncthreads();
        if (!PW && pe < r) {
          tail_norm_warp0<TL, float>(P + (size_t)pe * ldt + pe + 1, s - pe - 1, &nrm2[pe & 1]);
          __syncthreads();
        }
      }
    } else {
      for (int k = 0; k < r; ++k)
        householder_step<TL, float, NT, G>(k, r + 1, P + k, ldt, P + k + 1, ldt, s - k - 1, 1, nrm2,
                                           v0, tau);
      __syncthreads();
    }
    // y0 = R^{-1} z
    float dmin = 0.f, dmax = 0.f;
    if (warp == 0) {
      TL zr[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = lane + 32 * c;
        zr[c] = i < r ? P[i + (size_t)r * ldt] : zero<TL>();
      }
      backsolve_warp<TL, float>(P, ldt, r, zr, dl, dmin, dmax);
      for (int i = lane; i < r; i += 32) y[i] = to_hi(dl[i]);
      if constexpr (PW == 2)
        for (int i = lane; i < r; i += 32) Vb[i] = 1.f / P[i + (size_t)i * ldt];
    }
    __syncthreads();
    double rn2 = 0.0;
    bool converged = false;
    double last_rel = 1.0;
    if (tid == 0) ctl[1] = 1.0;
    __syncthreads();
    for (int it = 0;; ++it) {
      // float64 residual of the subsampled system: res = b_J - M y.  Once the last
      // correction delta is below 1e-7 |y|, r(y) = r(y - delta) - M delta with M delta
      // in float32: its rounding, ~u32 |M| |delta| <= 6e-15 |M| |y|, is at the level
      // of the float64 product, and the float64 pipe is spared.
      const bool update = (keep || a.Mg) && it > 0 && last_rel <= 1e-7;
      double part = 0.0;
      for (int i = tid; i < s; i += NT) {
        if (update) {
          const TH* mrow = keep ? M64 + i : a.Mg + (size_t)q * s * r + i;
          TL accl[4] = {zero<TL>(), zero<TL>(), zero<TL>(), zero<TL>()};
          int j = 0;
          for (; j + 4 <= r; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) accl[u] += to_lo(mrow[(size_t)(j + u) * s]) * dl[j + u];
          }
          for (; j < r; ++j) accl[0] += to_lo(mrow[(size_t)j * s]) * dl[j];
          const TH ri = res[i] - to_hi((accl[0] + accl[1]) + (accl[2] + accl[3]));
          res[i] = ri;
          part += absq(ri);
          continue;
        }
        TH acc = zero<TH>();
        if (keep || a.Mg) {
          // four independent partial sums: the row product is a latency chain otherwise
          const TH* mrow = keep ? M64 + i : a.Mg + (size_t)q * s * r + i;
          TH acc4[4] = {zero<TH>(), zero<TH>(), zero<TH>(), zero<TH>()};
          int j = 0;
          for (; j + 4 <= r; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc4[u] += mrow[(size_t)(j + u) * s] * y[j + u];
          }
          for (; j < r; ++j) acc4[0] += mrow[(size_t)j * s] * y[j];
          acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
        } else {
          for (int k = 0; k < K; ++k) {
            const TH* g = a.G + (size_t)k * s * r + i;
            TH mk = zero<TH>();
            for (int j = 0; j < r; ++j) mk += g[(size_t)j * s] * y[j];
            acc += th[k] * mk;
          }
        }
        const TH ri = a.bJ[i] - acc;
        res[i] = ri;
        part += absq(ri);
      }
      rn2 = block_sum<NT>(part, red);
      if (converged || it >= a.max_refine) break;
      // correction: delta = R^{-1} [Q^H res]_{0:r} in float32 (warp 0)
      if (warp == 0) {
        if constexpr (PW == 2) {
          correction_regs(P, ldt, s, r, res, v0, tau, Vb, dl);
        } else {
          for (int i = lane; i < s; i += 32) P[i + (size_t)r * ldt] = to_lo(res[i]);
          __syncwarp();
          for (int k = 0; k < r; ++k) {
            const TL* vk = P + (size_t)k * ldt;  // tail entries below the diagonal
            TL w = lane == 0 ? conjv(v0[k]) * P[k + (size_t)r * ldt] : zero<TL>();
            for (int i = k + 1 + lane; i < s; i += 32) w += conjv(vk[i]) * P[i + (size_t)r * ldt];
            w = warp_sum(w);
            const TL tw = rscale(tau[k], w);
            __syncwarp();
            if (lane == 0) P[k + (size_t)r * ldt] -= tw * v0[k];
            for (int i = k + 1 + lane; i < s; i += 32) P[i + (size_t)r * ldt] -= tw * vk[i];
            __syncwarp();
          }
          TL zr[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = lane + 32 * c;
            zr[c] = i < r ? P[i + (size_t)r * ldt] : zero<TL>();
          }
          float d0, d1;
          backsolve_warp<TL, float>(P, ldt, r, zr, dl, d0, d1);
        }
        double dn = 0.0, yn = 0.0;
        for (int i = lane; i < r; i += 32) {
          const TH di = to_hi(dl[i]);
          y[i] += di;
          dn += absq(di);
          yn += absq(y[i]);
        }
        dn = warp_sum(dn);
        yn = warp_sum(yn);
        if (lane == 0) {
          // stop at the tolerance, or once a correction no longer halves: the
          // iteration has reached the accuracy the float32 factor allows
          const double rel = sqrt(dn / yn);
          ctl[0] = (rel <= a.tol || rel > 0.5 * ctl[1]) ? 1.0 : 0.0;
          ctl[1] = rel;
        }
      }
      __syncthreads();
      converged = ctl[0] != 0.0;
      last_rel = ctl[1];
      __syncthreads();
    }
    if (warp == 0) {
      bool fin = true;
      TH h = zero<TH>();
      for (int i = lane; i < r; i += 32) {
        const TH yi = y[i];
        fin = fin && finitev(yi);
        if (a.yout) a.yout[q * r + i] = yi;
        if (a.qoi) h += a.wq[i] * yi;
      }
      fin = __all_sync(0xffffffffu, fin);
      if (a.qoi) {
        h = warp_sum(h);
        if (lane == 0) a.qoi[q] = h;
      }
      if (lane == 0) {
        if (a.rho) a.rho[q] = sqrt(rn2) / a.bJ_norm;
        if (a.flags) {
          uint32_t f = 0;
          if (!(dmin > 1e-6f * dmax)) f |= SAS_FLAG_ILLCOND;
          if (!fin) f |= SAS_FLAG_NONFINITE;
          if (!(last_rel <= 1e-8)) f |= SAS_FLAG_REFINE_STALL;
          a.flags[q] = f;
        }
      }
    }
    if (a.ysplit) {
      // tf32 split of y for the tensor-core reconstruction; zero padding to rpad
      for (int i = tid; i < a.rpad; i += NT) {
        float hi = 0.f, lo = 0.f;
        if (i < r) {
          const float yf = (float)(*reinterpret_cast<const double*>(&y[i]));
          hi = tf32_round(yf);
          lo = yf - hi;
        }
        a.ysplit[(size_t)q * a.rpad + i] = hi;
        a.ysplit[(size_t)a.m * a.rpad + (size_t)q * a.rpad + i] = lo;
      }
    }
    __syncthreads();
  }

template <typename TH, typename TL, int NT, int G>
__global__ void __launch_bounds__(NT, 512 / NT) ls_mixed_affine_kernel(LsMixedArgs<TH, TL> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double ctl[2];  // refinement control: stop flag, last relative correction
  for (int64_t q = blockIdx.x; q < a.m; q += gridDim.x) ls_mixed_body<TH, TL, NT, G>(a, q, smem_raw, ctl);
}

static size_t mixed_base_bytes(const sas_ctx* c) {
  const bool cplx = c->dtype == SAS_COMPLEX128;
  const size_t eh = cplx ? 16 : 8, el = cplx ? 8 : 4;
  size_t b = (size_t)(kMaxDp + kMaxR + kMaxS) * eh + (kLsThreads / 32) * 8;
  b += (size_t)(kMaxDp + 2 * kMaxR) * el + (size_t)kMaxR * 4 + 4 * 4;
  b += (size_t)panel_ld(c->s, (int)el) * (c->r + 1) * el;
  return (b + 15) / 16 * 16 + 16;
}

static bool mixed_keep64(const sas_ctx* c) {
  const size_t eh = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  // keep M in float64 shared memory when the variant asks for it, it fits and
  // leaves room for two CTAs per SM
  if (mixed_keep_kind(c->ls_variant_mixed) != 1) return false;
  return mixed_base_bytes(c) + (size_t)c->s * c->r * eh <= kSmemLimit / 2;
}

size_t ls_mixed_smem_bytes(const sas_ctx* c) {
  const size_t eh = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  const size_t vb = mixed_shape(c->ls_variant_mixed) == -2 ? (size_t)kLsPanel * c->s * 4 + 16 : 0;
  return mixed_base_bytes(c) + vb + (mixed_keep64(c) ? (size_t)c->s * c->r * eh : 0);
}

// Global float64-M slots of a mixed context: one per CTA that can be resident
// (bounded by the shared memory each CTA needs at least).
int64_t ls_mixed_slots(const sas_ctx* c) {
  const size_t base = mixed_base_bytes(c) + 1024;
  int64_t per_sm = (int64_t)(228 * 1024) / (int64_t)base;
  if (per_sm > 16) per_sm = 16;
  if (per_sm < 1) per_sm = 1;
  return per_sm * c->num_sms;
}

template <typename TH, typename TL>
static size_t fill_mixed_args(const sas_ctx* c, const double* params, int64_t m, void* yout,
                              void* qoi, float* ysplit, uint32_t* flags, double* rho,
                              const void* Mg, LsMixedArgs<TH, TL>& a) {
  const size_t smem = ls_mixed_smem_bytes(c);
  if (smem > kSmemLimit) return 0;
  a.Mg = (const TH*)Mg;
  a.G = (const TH*)c->G;
  a.G32 = (const TL*)c->G32;
  a.bJ = (const TH*)c->bJ;
  a.bJ32 = (const TL*)c->bJ32;
  a.wq = (const TH*)c->wq;
  a.params = params;
  a.m = m;
  a.s = c->s;
  a.r = c->r;
  a.K = c->K;
  a.dp = c->dp;
  a.rule = c->theta_rule;
  a.ldt = panel_ld(c->s, (int)sizeof(TL));
  a.rpad = (c->r + 31) / 32 * 32;
  a.max_refine = c->max_refine;
  a.keep64 = mixed_keep64(c) ? 1 : 0;
  a.M64g = nullptr;
  a.nslots = 0;
  if (mixed_keep_kind(c->ls_variant_mixed) == 2 && c->ls_slots) {
    a.keep64 = 2;
    a.M64g = (TH*)c->ls_slots;
    a.nslots = (int)c->ls_slots_n;
  }
  a.tol = c->refine_tol;
  a.bJ_norm = c->bJ_norm;
  a.yout = (TH*)yout;
  a.qoi = (TH*)qoi;
  a.ysplit = ysplit;
  a.flags = flags;
  a.rho = rho;
  return smem;
}

template <int NT, int G, int E, int PW, int MINB>
__global__ void __launch_bounds__(NT, MINB) ls_mixed_blocked_kernel(LsMixedArgs<double, float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double ctl[2];
  for (int64_t q = blockIdx.x; q < a.m; q += gridDim.x)
    ls_mixed_body<double, float, NT, G, kLsPanel, E, PW>(a, q, smem_raw, ctl);
}

static cudaError_t launch_mixed_blocked(const sas_ctx* c, const LsMixedArgs<double, float>& a,
                                        int64_t m, size_t smem, int b, cudaStream_t st) {
  if (b < 0 || b >= kNumLsBlocked) return cudaErrorInvalidConfiguration;
  const LsBlockedShape sh = kLsBlocked[b];
  if (c->s > sh.g * sh.e) return cudaErrorInvalidConfiguration;  // a trailing column must fit
  if (sh.pw == 2 && c->s > kLsRegRows) return cudaErrorInvalidConfiguration;
  void (*kern)(LsMixedArgs<double, float>) = nullptr;
  switch (b) {
    case 0: kern = ls_mixed_blocked_kernel<128, 4, 32, 0, 4>; break;
    case 1: kern = ls_mixed_blocked_kernel<128, 8, 16, 0, 4>; break;
    case 2: kern = ls_mixed_blocked_kernel<256, 8, 32, 0, 2>; break;
    case 3: kern = ls_mixed_blocked_kernel<128, 8, 32, 0, 4>; break;
    case 4: kern = ls_mixed_blocked_kernel<128, 8, 16, 1, 4>; break;
    case 5: kern = ls_mixed_blocked_kernel<128, 4, 32, 1, 4>; break;
    case 6: kern = ls_mixed_blocked_kernel<256, 8, 32, 1, 2>; break;
    case 7: kern = ls_mixed_blocked_kernel<128, 8, 16, 1, 5>; break;  // 5 CTAs per SM
    default: kern = ls_mixed_blocked_kernel<128, 8, 16, 2, 4>; break;  // panel in registers
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sh.nt, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (grid > m) grid = m;
  kern<<<(unsigned)grid, sh.nt, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename TH, typename TL>
static cudaError_t launch_mixed_t(const sas_ctx* c, const double* params, int64_t m, void* yout,
                                  void* qoi, float* ysplit, uint32_t* flags, double* rho,
                                  cudaStream_t st, const void* Mg) {
  LsMixedArgs<TH, TL> a;
  const size_t smem = fill_mixed_args<TH, TL>(c, params, m, yout, qoi, ysplit, flags, rho, Mg, a);
  if (smem == 0) return cudaErrorInvalidConfiguration;
  const int v = mixed_shape(c->ls_variant_mixed);
  if (v == -2) {
    if constexpr (sizeof(TH) == 8)
      return launch_mixed_blocked(c, a, m, smem, c->ls_variant_mixed - kFirstBlocked, st);
    return cudaErrorInvalidConfiguration;
  }
  if (v < 0) {
    if constexpr (sizeof(TH) == 8)
      return launch_mixed_reg(c, a, m, c->ls_variant_mixed - 2 * kNumLsShapes, st);
    return cudaErrorInvalidConfiguration;
  }
  void (*kern)(LsMixedArgs<TH, TL>) = nullptr;
  switch (v) {
    case 0: kern = ls_mixed_affine_kernel<TH, TL, 256, 4>; break;
    case 1: kern = ls_mixed_affine_kernel<TH, TL, 128, 4>; break;
    case 2: kern = ls_mixed_affine_kernel<TH, TL, 256, 8>; break;
    case 3: kern = ls_mixed_affine_kernel<TH, TL, 128, 2>; break;
    default: kern = ls_mixed_affine_kernel<TH, TL, 256, 2>; break;
  }
  const int nt = kLsShapes[v].nt;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (grid > m) grid = m;
  kern<<<(unsigned)grid, nt, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ls_mixed(const sas_ctx* c, const double* params, int64_t m, void* yout,
                            void* qoi, float* ysplit, uint32_t* flags, double* rho,
                            cudaStream_t st, const void* Mg) {
  if (m == 0) return cudaSuccess;
  if (c->dtype == SAS_COMPLEX128)
    return launch_mixed_t<zd, zf>(c, params, m, yout, qoi, nullptr, flags, rho, st, Mg);
  return launch_mixed_t<double, float>(c, params, m, yout, qoi, ysplit, flags, rho, st, Mg);
}

// --------------------------------------------- register-resident variants
// Householder with static column ownership: the G lanes of slot q own the
// columns j = q, q + NSLOT, ... (up to CPS of them) for the whole
// factorisation, lane g the rows g, g + G, ... (up to RPT) of each, in
// registers.  Step k: the owner of column k writes that column (rows >= k) to
// V[:, k] in shared memory, computes the reflector from it, replaces V[k, k]
// by v0 and writes R's column k; after one barrier every slot applies
// H_k = I - tau v v^H to its own columns from V[:, k].  V[:, k] is never
// overwritten, so one barrier per step suffices, and V is the stored Q of
// the mixed refinement.
template <typename TF, typename RF, int NT, int G, int RPT, int CPS>
__device__ inline void reg_householder(TF (&m)[CPS][RPT], int s, int r, TF* V, int ldv, RF* taus,
                                       TF* Rs, int ldr, TF* zs, RF* res2) {
  constexpr int NSLOT = NT / G;
  const int tid = threadIdx.x, g = tid % G, slot = tid / G;
  const unsigned gmask = ((1u << G) - 1u) << ((tid & 31) & ~(G - 1));
  for (int k = 0; k < r; ++k) {
    const int owner = k % NSLOT, ck = k / NSLOT;
    if (slot == owner) {
      RF part = RF(0);
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int i = g + G * u;
        const TF val = ck == 0 ? m[0][u] : m[CPS > 1 ? 1 : 0][u];
        if (i >= k && i < s) V[i + (size_t)k * ldv] = val;
        if (i > k && i < s) part += absq(val);
        if (i < k) Rs[i + (size_t)k * ldr] = val;  // rows above k are final
      }
#pragma unroll
      for (int o = 1; o < G; o <<= 1) part += shfl_xor_m(gmask, part, o);
      __syncwarp(gmask);
      const TF alpha = V[k + (size_t)k * ldv];
      const RF a2 = absq(alpha);
      const RF nrm = sqrt(a2 + part);
      const RF aa = sqrt(a2);
      const TF beta = rscale(-nrm, phase(alpha));
      __syncwarp(gmask);
      if (g == 0) {
        V[k + (size_t)k * ldv] = alpha - beta;  // v0
        taus[k] = nrm > RF(0) ? RF(1) / (nrm * (nrm + aa)) : RF(0);
        Rs[k + (size_t)k * ldr] = beta;
      }
    }
    __syncthreads();
    const RF tau = taus[k];
#pragma unroll
    for (int c = 0; c < CPS; ++c) {
      const int j = slot + c * NSLOT;
      if (j > k && j <= r) {
        TF w = zero<TF>();
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
          const int i = g + G * u;
          if (i >= k && i < s) w += conjv(V[i + (size_t)k * ldv]) * m[c][u];
        }
#pragma unroll
        for (int o = 1; o < G; o <<= 1) w += shfl_xor_m(gmask, w, o);
        const TF tw = rscale(tau, w);
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
          const int i = g + G * u;
          if (i >= k && i < s) m[c][u] -= tw * V[i + (size_t)k * ldv];
        }
      }
    }
  }
  // right-hand side column r: z = rows 0..r-1, residual = rows r..s-1
  {
    const int owner = r % NSLOT, cr = r / NSLOT;
    if (slot == owner) {
      RF part = RF(0);
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int i = g + G * u;
        const TF val = cr == 0 ? m[0][u] : m[CPS > 1 ? 1 : 0][u];
        if (i < r) zs[i] = val;
        else if (i < s) part += absq(val);
      }
#pragma unroll
      for (int o = 1; o < G; o <<= 1) part += shfl_xor_m(gmask, part, o);
      if (g == 0) *res2 = part;
    }
  }
  __syncthreads();
}

template <int NT, int G, int RPT, int CPS>
struct RegShape {
  static constexpr int nt = NT, g = G, rpt = RPT, cps = CPS;
  static bool fits(int s, int r) { return s <= G * RPT && r + 1 <= (NT / G) * CPS; }
};

// Plain float64, register-resident: same outputs as ls_plain_body.
template <int NT, int G, int RPT, int CPS>
__global__ void __launch_bounds__(NT, 1) ls_plain_reg_kernel(LsPlainArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NSLOT = NT / G;
  const int s = a.s, r = a.r, K = a.K;
  const int ldv = s | 1;  // odd stride: the 32 lanes of a column read distinct banks
  double* V = reinterpret_cast<double*>(smem_raw);          // ldv x r
  double* Rs = V + (size_t)ldv * r;                         // r x r (ld r)
  double* zs = Rs + (size_t)r * r;                          // r
  double* taus = zs + kMaxR;                                // r
  double* th = taus + kMaxR;                                // K
  double* ys = th + kMaxDp;                                 // r
  __shared__ double res2;
  const int tid = threadIdx.x, g = tid % G, slot = tid / G, warp = tid >> 5;
  for (int64_t q = blockIdx.x; q < a.m; q += gridDim.x) {
    if (tid < K) th[tid] = theta_k<double>(a.rule, tid, a.params + q * a.dp);
    __syncthreads();
    double m[CPS][RPT];
#pragma unroll
    for (int c = 0; c < CPS; ++c) {
      const int j = slot + c * NSLOT;
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int i = g + G * u;
        double v = 0.0;
        if (i < s && j < r) {
          if (a.Mg) {
            v = a.Mg[(size_t)q * s * r + (size_t)j * s + i];
          } else {
            const double* gp = a.G + (size_t)j * s + i;
            for (int k = 0; k < K; ++k) v += th[k] * gp[(size_t)k * s * r];
          }
        } else if (i < s && j == r) {
          v = a.bJ[i];
        }
        m[c][u] = v;
      }
    }
    reg_householder<double, double, NT, G, RPT, CPS>(m, s, r, V, ldv, taus, Rs, r, zs, &res2);
    if (warp == 0) {
      double zr[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = (tid & 31) + 32 * c;
        zr[c] = i < r ? zs[i] : 0.0;
      }
      double dmin, dmax;
      backsolve_warp<double, double>(Rs, r, r, zr, ys, dmin, dmax);
      const int lane = tid & 31;
      bool fin = true;
      double h = 0.0;
      for (int i = lane; i < r; i += 32) {
        const double yi = ys[i];
        fin = fin && isfinite(yi);
        if (a.yout) a.yout[q * r + i] = yi;
        if (a.qoi) h += a.wq[i] * yi;
      }
      fin = __all_sync(0xffffffffu, fin);
      if (a.qoi) {
        h = warp_sum(h);
        if (lane == 0) a.qoi[q] = h;
      }
      if (lane == 0) {
        if (a.rho) a.rho[q] = sqrt(res2) / a.bJ_norm;
        if (a.flags) {
          uint32_t f = 0;
          if (!(dmin > 1e-13 * dmax)) f |= SAS_FLAG_ILLCOND;
          if (!fin) f |= SAS_FLAG_NONFINITE;
          a.flags[q] = f;
        }
      }
    }
    __syncthreads();
  }
}

static size_t plain_reg_smem(int s, int r) {
  return sizeof(double) * ((size_t)(s | 1) * r + (size_t)r * r + 3 * kMaxR + kMaxDp) + 64;
}

// Mixed, register-resident: float32 factorisation in registers, V and R in
// shared memory, refinement exactly as ls_mixed_body.
template <int NT, int G, int RPT, int CPS>
__global__ void __launch_bounds__(NT, 1) ls_mixed_reg_kernel(LsMixedArgs<double, float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NSLOT = NT / G;
  const int s = a.s, r = a.r, K = a.K;
  const int ldv = s | 1;
  double* th = reinterpret_cast<double*>(smem_raw);   // kMaxDp
  double* y = th + kMaxDp;                            // kMaxR
  double* res = y + kMaxR;                            // kMaxS
  double* red = res + kMaxS;                          // 8
  float* V = reinterpret_cast<float*>(red + 8);       // ldv x r
  float* Rs = V + (size_t)ldv * r;                    // r x r
  float* zs = Rs + (size_t)r * r;                     // kMaxS (also the correction rhs)
  float* taus = zs + kMaxS;                           // kMaxR
  float* dl = taus + kMaxR;                           // kMaxR
  float* th32 = dl + kMaxR;                           // kMaxDp
  __shared__ float res2f;
  __shared__ double ctl[2];
  const int tid = threadIdx.x, g = tid % G, slot = tid / G, lane = tid & 31, warp = tid >> 5;
  for (int64_t q = blockIdx.x; q < a.m; q += gridDim.x) {
    if (tid < K) {
      th[tid] = theta_k<double>(a.rule, tid, a.params + q * a.dp);
      th32[tid] = (float)th[tid];
    }
    __syncthreads();
    float m[CPS][RPT];
#pragma unroll
    for (int c = 0; c < CPS; ++c) {
      const int j = slot + c * NSLOT;
#pragma unroll
      for (int u = 0; u < RPT; ++u) {
        const int i = g + G * u;
        float v = 0.f;
        if (i < s && j < r) {
          if (a.Mg) {
            v = (float)a.Mg[(size_t)q * s * r + (size_t)j * s + i];
          } else {
            const float* gp = a.G32 + (size_t)j * s + i;
            for (int k = 0; k < K; ++k) v += th32[k] * gp[(size_t)k * s * r];
          }
        } else if (i < s && j == r) {
          v = a.bJ32[i];
        }
        m[c][u] = v;
      }
    }
    reg_householder<float, float, NT, G, RPT, CPS>(m, s, r, V, ldv, taus, Rs, r, zs, &res2f);
    float dmin = 0.f, dmax = 0.f;
    if (warp == 0) {
      float zr[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = lane + 32 * c;
        zr[c] = i < r ? zs[i] : 0.f;
      }
      backsolve_warp<float, float>(Rs, r, r, zr, dl, dmin, dmax);
      for (int i = lane; i < r; i += 32) y[i] = (double)dl[i];
    }
    __syncthreads();
    double rn2 = 0.0;
    bool converged = false;
    double last_rel = 1.0;
    if (tid == 0) ctl[1] = 1.0;
    __syncthreads();
    for (int it = 0;; ++it) {
      double part = 0.0;
      for (int i = tid; i < s; i += NT) {
        double acc = 0.0;
        if (a.Mg) {
          const double* mrow = a.Mg + (size_t)q * s * r + i;
          for (int j = 0; j < r; ++j) acc += mrow[(size_t)j * s] * y[j];
        } else {
          for (int k = 0; k < K; ++k) {
            const double* gp = a.G + (size_t)k * s * r + i;
            double mk = 0.0;
            for (int j = 0; j < r; ++j) mk += gp[(size_t)j * s] * y[j];
            acc += th[k] * mk;
          }
        }
        const double ri = a.bJ[i] - acc;
        res[i] = ri;
        part += ri * ri;
      }
      rn2 = block_sum<NT>(part, red);
      if (converged || it >= a.max_refine) break;
      if (warp == 0) {
        for (int i = lane; i < s; i += 32) zs[i] = (float)res[i];
        __syncwarp();
        for (int k = 0; k < r; ++k) {
          const float* vk = V + (size_t)k * ldv;  // rows k..s-1 (v0 at row k)
          float w = 0.f;
          for (int i = k + lane; i < s; i += 32) w += vk[i] * zs[i];
          w = warp_sum(w);
          const float tw = taus[k] * w;
          __syncwarp();
          for (int i = k + lane; i < s; i += 32) zs[i] -= tw * vk[i];
          __syncwarp();
        }
        float zr[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = lane + 32 * c;
          zr[c] = i < r ? zs[i] : 0.f;
        }
        float d0, d1;
        backsolve_warp<float, float>(Rs, r, r, zr, dl, d0, d1);
        double dn = 0.0, yn = 0.0;
        for (int i = lane; i < r; i += 32) {
          const double di = (double)dl[i];
          y[i] += di;
          dn += di * di;
          yn += y[i] * y[i];
        }
        dn = warp_sum(dn);
        yn = warp_sum(yn);
        if (lane == 0) {
          const double rel = sqrt(dn / yn);
          ctl[0] = (rel <= a.tol || rel > 0.5 * ctl[1]) ? 1.0 : 0.0;
          ctl[1] = rel;
        }
      }
      __syncthreads();
      converged = ctl[0] != 0.0;
      last_rel = ctl[1];
      __syncthreads();
    }
    if (warp == 0) {
      bool fin = true;
      double h = 0.0;
      for (int i = lane; i < r; i += 32) {
        const double yi = y[i];
        fin = fin && isfinite(yi);
        if (a.yout) a.yout[q * r + i] = yi;
        if (a.qoi) h += a.wq[i] * yi;
      }
      fin = __all_sync(0xffffffffu, fin);
      if (a.qoi) {
        h = warp_sum(h);
        if (lane == 0) a.qoi[q] = h;
      }
      if (lane == 0) {
        if (a.rho) a.rho[q] = sqrt(rn2) / a.bJ_norm;
        if (a.flags) {
          uint32_t f = 0;
          if (!(dmin > 1e-6f * dmax)) f |= SAS_FLAG_ILLCOND;
          if (!fin) f |= SAS_FLAG_NONFINITE;
          if (!(last_rel <= 1e-8)) f |= SAS_FLAG_REFINE_STALL;
          a.flags[q] = f;
        }
      }
    }
    if (a.ysplit) {
      for (int i = tid; i < a.rpad; i += NT) {
        float hi = 0.f, lo = 0.f;
        if (i < r) {
          const float yf = (float)y[i];
          hi = tf32_round(yf);
          lo = yf - hi;
        }
        a.ysplit[(size_t)q * a.rpad + i] = hi;
        a.ysplit[(size_t)a.m * a.rpad + (size_t)q * a.rpad + i] = lo;
      }
    }
    __syncthreads();
  }
}

static size_t mixed_reg_smem(int s, int r) {
  return sizeof(double) * (kMaxDp + kMaxR + kMaxS + 8) +
         sizeof(float) * ((size_t)(s | 1) * r + (size_t)r * r + kMaxS + 2 * kMaxR + kMaxDp) + 64;
}

template <typename K, typename A>
static cudaError_t launch_persistent(K kern, int nt, size_t smem, const sas_ctx* c, int64_t m, A a,
                                     cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)c->num_sms * per_sm;
  if (grid > m) grid = m;
  kern<<<(unsigned)grid, nt, smem, st>>>(a);
  return cudaGetLastError();
}

// Register variants: plain (256 threads, 8 lanes per column, 16 rows, 2 columns);
// mixed (128 x 4 x 32 x 2) and (256 x 4 x 32 x 1).
static cudaError_t launch_plain_reg(const sas_ctx* c, const LsPlainArgs<double>& a, int64_t m,
                                    cudaStream_t st) {
  using Sh = RegShape<256, 8, 16, 2>;
  if (!Sh::fits(c->s, c->r)) return cudaErrorInvalidConfiguration;
  return launch_persistent(ls_plain_reg_kernel<256, 8, 16, 2>, Sh::nt, plain_reg_smem(c->s, c->r),
                           c, m, a, st);
}

static cudaError_t launch_mixed_reg(const sas_ctx* c, const LsMixedArgs<double, float>& a, int64_t m,
                                    int which, cudaStream_t st) {
  const size_t smem = mixed_reg_smem(c->s, c->r);
  if (which == 0) {
    using Sh = RegShape<128, 4, 32, 2>;
    if (!Sh::fits(c->s, c->r)) return cudaErrorInvalidConfiguration;
    return launch_persistent(ls_mixed_reg_kernel<128, 4, 32, 2>, Sh::nt, smem, c, m, a, st);
  }
  using Sh = RegShape<256, 4, 32, 1>;
  if (!Sh::fits(c->s, c->r)) return cudaErrorInvalidConfiguration;
  return launch_persistent(ls_mixed_reg_kernel<256, 4, 32, 1>, Sh::nt, smem, c, m, a, st);
}

// ------------------------------------------ persistent multi-problem launch
// One launch drains a task list spanning several contexts whose (s, r, K)
// differ: task t belongs to problem p with offs[p] <= t < offs[p+1]; CTAs take
// tasks from a global counter, so uneven problems balance across the SMs.  The
// per-task work is the same body the single-problem kernels run.
template <typename T, int NT, int G>
__global__ void __launch_bounds__(NT, 512 / NT) ls_plain_multi_kernel(const LsPlainArgs<T>* probs,
                                                                      const int64_t* offs, int nprob,
                                                                      unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double nrm2[2];
  __shared__ long long task;
  const int64_t total = offs[nprob];
  while (true) {
    if (threadIdx.x == 0) task = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t t = task;
    if (t >= total) break;
    int p = 0;
    while (offs[p + 1] <= t) ++p;
    ls_plain_body<T, NT, G>(probs[p], t - offs[p], smem_raw, nrm2);
    __syncthreads();
  }
}

template <typename TH, typename TL, int NT, int G>
__global__ void __launch_bounds__(NT, 512 / NT) ls_mixed_multi_kernel(
    const LsMixedArgs<TH, TL>* probs, const int64_t* offs, int nprob, unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double ctl[2];
  __shared__ long long task;
  const int64_t total = offs[nprob];
  while (true) {
    if (threadIdx.x == 0) task = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t t = task;
    if (t >= total) break;
    int p = 0;
    while (offs[p + 1] <= t) ++p;
    ls_mixed_body<TH, TL, NT, G>(probs[p], t - offs[p], smem_raw, ctl);
    __syncthreads();
  }
}

template <typename A>
static cudaError_t upload(const std::vector<A>& h, void** d) {
  cudaError_t e = cudaMalloc(d, sizeof(A) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), sizeof(A) * h.size(), cudaMemcpyHostToDevice);
  return e;
}

template <typename T>
static cudaError_t plan_plain(MultiPlan* pl, sas_ctx* const* ctxs, int n, const double* const* params,
                              const int64_t* m, int32_t out_kind, void* const* outs,
                              uint32_t* const* flags, double* const* rho) {
  std::vector<LsPlainArgs<T>> a(n);
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    const size_t sm = fill_plain_args<T>(ctxs[i], params[i], m[i], out_kind == SAS_OUT_Y ? outs[i] : nullptr,
                                         out_kind == SAS_OUT_QOI ? outs[i] : nullptr,
                                         flags ? flags[i] : nullptr, rho ? rho[i] : nullptr, nullptr, a[i]);
    if (sm == 0) return cudaErrorInvalidConfiguration;
    smem = sm > smem ? sm : smem;
  }
  const int v = ctxs[0]->ls_variant_plain % kNumLsShapes;
  void (*k)(const LsPlainArgs<T>*, const int64_t*, int, unsigned long long*) = nullptr;
  switch (v) {
    case 0: k = ls_plain_multi_kernel<T, 256, 4>; break;
    case 1: k = ls_plain_multi_kernel<T, 128, 4>; break;
    case 2: k = ls_plain_multi_kernel<T, 256, 8>; break;
    case 3: k = ls_plain_multi_kernel<T, 128, 2>; break;
    default: k = ls_plain_multi_kernel<T, 256, 2>; break;
  }
  pl->kernel = (const void*)k;
  pl->nt = kLsShapes[v].nt;
  pl->smem = smem;
  return upload(a, &pl->d_probs);
}

template <typename TH, typename TL>
static cudaError_t plan_mixed(MultiPlan* pl, sas_ctx* const* ctxs, int n, const double* const* params,
                              const int64_t* m, int32_t out_kind, void* const* outs,
                              uint32_t* const* flags, double* const* rho) {
  std::vector<LsMixedArgs<TH, TL>> a(n);
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    const size_t sm = fill_mixed_args<TH, TL>(ctxs[i], params[i], m[i],
                                              out_kind == SAS_OUT_Y ? outs[i] : nullptr,
                                              out_kind == SAS_OUT_QOI ? outs[i] : nullptr, nullptr,
                                              flags ? flags[i] : nullptr, rho ? rho[i] : nullptr,
                                              nullptr, a[i]);
    if (sm == 0) return cudaErrorInvalidConfiguration;
    smem = sm > smem ? sm : smem;
  }
  int v = mixed_shape(ctxs[0]->ls_variant_mixed);
  if (v < 0) v = ctxs[0]->ls_variant_mixed - 2 * kNumLsShapes;  // register variants: nearest shape
  void (*k)(const LsMixedArgs<TH, TL>*, const int64_t*, int, unsigned long long*) = nullptr;
  switch (v) {
    case 0: k = ls_mixed_multi_kernel<TH, TL, 256, 4>; break;
    case 1: k = ls_mixed_multi_kernel<TH, TL, 128, 4>; break;
    case 2: k = ls_mixed_multi_kernel<TH, TL, 256, 8>; break;
    case 3: k = ls_mixed_multi_kernel<TH, TL, 128, 2>; break;
    default: k = ls_mixed_multi_kernel<TH, TL, 256, 2>; break;
  }
  pl->kernel = (const void*)k;
  pl->nt = kLsShapes[v].nt;
  pl->smem = smem;
  return upload(a, &pl->d_probs);
}

cudaError_t multi_plan_build(MultiPlan* pl, sas_ctx* const* ctxs, int n, const double* const* params,
                             const int64_t* m, int32_t out_kind, void* const* outs,
                             uint32_t* const* flags, double* const* rho) {
  const bool mixed = ctxs[0]->mode == SAS_MODE_MIXED;
  const bool cplx = ctxs[0]->dtype == SAS_COMPLEX128;
  cudaError_t e;
  if (mixed)
    e = cplx ? plan_mixed<zd, zf>(pl, ctxs, n, params, m, out_kind, outs, flags, rho)
             : plan_mixed<double, float>(pl, ctxs, n, params, m, out_kind, outs, flags, rho);
  else
    e = cplx ? plan_plain<zd>(pl, ctxs, n, params, m, out_kind, outs, flags, rho)
             : plan_plain<double>(pl, ctxs, n, params, m, out_kind, outs, flags, rho);
  if (e != cudaSuccess) return e;
  std::vector<int64_t> offs(n + 1, 0);
  for (int i = 0; i < n; ++i) offs[i + 1] = offs[i] + m[i];
  pl->total = offs[n];
  e = upload(offs, (void**)&pl->d_offs);
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->d_counter, sizeof(unsigned long long));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pl->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl->kernel, pl->nt, pl->smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctxs[0]->num_sms * per_sm;
  if (grid > pl->total) grid = pl->total;
  pl->grid = (int)grid;
  pl->nprob = n;
  return cudaSuccess;
}

cudaError_t multi_plan_enqueue(MultiPlan* pl, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(pl->d_counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || pl->total == 0) return e;
  void* args[] = {(void*)&pl->d_probs, (void*)&pl->d_offs, (void*)&pl->nprob, (void*)&pl->d_counter};
  return cudaLaunchKernel(pl->kernel, dim3(pl->grid), dim3(pl->nt), args, pl->smem, st);
}

// ------------------------------------------------- subsampled residual
template <typename T, int NT>
__global__ void __launch_bounds__(NT) residual_affine_kernel(const T* G, const T* bJ,
                                                             const double* params, int64_t m,
                                                             int s, int r, int K, int dp, int rule,
                                                             const T* Y, double bJ_norm,
                                                             double* rho, const T* Mg) {
  __shared__ T th[kMaxDp];
  __shared__ T y[kMaxR];
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x;
  for (int64_t q = blockIdx.x; q < m; q += gridDim.x) {
    if (tid < K) th[tid] = theta_k<T>(rule, tid, params + q * dp);
    for (int i = tid; i < r; i += NT) y[i] = Y[q * r + i];
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < s; i += NT) {
      T acc = zero<T>();
      if (Mg) {
        const T* mrow = Mg + (size_t)q * s * r + i;
        for (int j = 0; j < r; ++j) acc += mrow[(size_t)j * s] * y[j];
      } else {
        for (int k = 0; k < K; ++k) {
          const T* g = G + (size_t)k * s * r + i;
          T mk = zero<T>();
          for (int j = 0; j < r; ++j) mk += g[(size_t)j * s] * y[j];
          acc += th[k] * mk;
        }
      }
      part += absq(bJ[i] - acc);
    }
    const double tot = block_sum<NT>(part, red);
    if (tid == 0) rho[q] = sqrt(tot) / bJ_norm;
    __syncthreads();
  }
}

cudaError_t launch_residual(const sas_ctx* c, const double* params, int64_t m, const void* Y,
                            double* rho, cudaStream_t st, const void* Mg) {
  if (m == 0) return cudaSuccess;
  int64_t grid = m < (int64_t)c->num_sms * 8 ? m : (int64_t)c->num_sms * 8;
  if (c->dtype == SAS_COMPLEX128)
    residual_affine_kernel<zd, 256><<<(unsigned)grid, 256, 0, st>>>(
        (const zd*)c->G, (const zd*)c->bJ, params, m, c->s, c->r, c->K, c->dp, c->theta_rule,
        (const zd*)Y, c->bJ_norm, rho, (const zd*)Mg);
  else
    residual_affine_kernel<double, 256><<<(unsigned)grid, 256, 0, st>>>(
        (const double*)c->G, (const double*)c->bJ, params, m, c->s, c->r, c->K, c->dp,
        c->theta_rule, (const double*)Y, c->bJ_norm, rho, (const double*)Mg);
  return cudaGetLastError();
}

}  // namespace sas
