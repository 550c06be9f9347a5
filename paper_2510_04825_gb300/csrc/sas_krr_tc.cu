// Gaussian-kernel rows on the tensor cores (sm_103a, tcgen05) for the mixed
// form of kernel ridge regression (Sec. 5.3):
//     M_q = K_{sigma_q}(X_J, X) S + lambda_q S_J,
//     K_sigma(x, x') = exp(-|x - x'|^2 / (2 sigma^2)),
// for a batch of parameters q = (sigma_q, lambda_q).  The s x N kernel block
// is never stored: its entries are formed in shared memory, 128 rows of J x 32
// points at a time, and fed straight to tcgen05.mma as the A operand, while S
// streams through as the B operand (only the rows at J are evaluated, the
// point of Sec. 3.1).
//
// Arithmetic.  Entries: direct coordinate differences of float32 hi/lo pairs
// (the difference of two nearby points keeps float32 relative accuracy), the
// squared distance in float32 and exp as ex2.approx of the scaled distance.
// Each entry E and each S value is split into a tf32 high part and a float32
// remainder, and E S is accumulated as E_hi S_hi + E_hi S_lo + E_lo S_hi
// (kind::tf32, float32 accumulation in TMEM): ~2^-21 per product, with the
// float32 exponent range (entries far below 2^-14, common at small sigma, stay
// normal numbers, which an f16 split would flush).  The TMEM accumulator is
// folded into a float64 sum in M every seg_chunks x 32 points (a context
// option), so the float32 rounding of the accumulator grows with the segment
// length, not with the number of points N.
//
// Structure (one persistent CTA per SM, 14 warps):
//   warp 0      TMA producer: per 32-point chunk the S_hi and S_lo boxes (nb
//               rows x 32 points, K-major, 128-byte swizzle) and the chunk's
//               coordinates (bulk copy) into a 2-stage ring;
//   warp 1      MMA issuer (one thread): per chunk and parameter 3 products x
//               4 K-steps of M = 128, N = nb, K = 8 into TMEM;
//   warps 2-5   fold: at each segment end, tcgen05.ld of the accumulators
//               (lane quarter = warp % 4) and a float64 read-add-write into M;
//               the last segment also adds lambda S_J;
//   warps 6-13  generators: E for the chunk (4 rows of J x 4 points per
//               thread: the rows' coordinates stay in registers as packed row
//               pairs, each point's coordinates are read once per chunk;
//               distances shared by the pair of parameters, two rows per f32x2
//               instruction), tf32 split, written in the swizzled K-major
//               operand layout.
// Work unit: one 128-row tile of J and a pair of parameters, reduced over all
// points; the two accumulators of the pair are double-buffered in TMEM (2 x 2
// x nb <= 512 columns) so that the fold of one segment overlaps the MMAs of
// the next.  Every mbarrier wait is bounded (2 s): on expiry the kernel
// records SAS_ETIMEOUT, stops, drains its copies and MMAs, frees TMEM and
// returns.
#include <cstring>

#include "sas_internal.cuh"
#include "sas_tc_common.cuh"

namespace sas {

namespace krrtc {

using namespace tc;

constexpr int kGenWarps = 8;
constexpr int kFirstGenWarp = 6;
constexpr int kThreads = 32 * (kFirstGenWarp + kGenWarps);  // 448
constexpr int kRows = 128;       // rows of J per tile (MMA M)
constexpr int kChunk = 32;       // points per K box (128 B of tf32)
constexpr int kQ = 2;            // parameters per work unit
constexpr int kABox = kRows * 128;  // one E operand (hi or lo): 16 KB
constexpr uint32_t kTmemCols = 512;

struct Params {
  const float* xj;       // s x 2dp: hi then lo coordinates of the rows of J (zero padded)
  const float* xc;       // per 32-point chunk: hi [dp][32] then lo [dp][32] (zero padded)
  const double* params;  // m x 2: (sigma, lambda)
  const double* SJ;      // s x r (ld s)
  double* M;             // m x (s x r), column-major per parameter (ld s)
  int nchunks;           // npad / 32
  int dp;                // coordinate stride: d rounded up to a multiple of 4
  int r, s, nb;          // nb: MMA N, r rounded up to a multiple of 16
  int64_t m;
  int njt;               // ceil(s / 128)
  int seg_chunks;        // 32-point chunks per TMEM segment before the float64 fold
  int num_units;         // njt * ceil(m / 2)
  uint32_t idesc;
  uint32_t bbox;         // bytes of one S box: nb x 128
  uint32_t cbytes;       // bytes of one chunk's coordinates: 32 x 2dp x 4
  uint32_t stage_bytes;
  int* status;
};

__device__ inline float tf32_hi(float x) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// Packed pairs of float32 (low half = first element) and the f32x2 arithmetic
// of sm_100-family SMs: two lanes of float32 per instruction.
typedef unsigned long long f2;
__device__ inline f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ inline void f2_unpack(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ inline f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ inline f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ inline f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ inline f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ inline float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int DP4>
__global__ void __maxnreg__(128)  // 448 threads x 128 registers per CTA, one CTA per SM
    krr_tc_kernel(const __grid_constant__ CUtensorMap tmShi,
                  const __grid_constant__ CUtensorMap tmSlo, Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  // stage layout: E operands [q][hi, lo] (kQ x 2 x 16 KB), S boxes [hi, lo], coordinates
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * (size_t)p.stage_bytes);
  // bars: full[2], gen[2], empty[2], accfull[2], accempty[2]
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(&bars[0]), gen0 = smem_u32(&bars[2]);
  const uint32_t empty0 = smem_u32(&bars[4]), accfull0 = smem_u32(&bars[6]);
  const uint32_t accempty0 = smem_u32(&bars[8]);
  const int nseg = (p.nchunks + p.seg_chunks - 1) / p.seg_chunks;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < 2; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(gen0 + 8 * s, kGenWarps);
      mbar_init(empty0 + 8 * s, 1);
      mbar_init(accfull0 + 8 * s, 1);
      mbar_init(accempty0 + 8 * s, 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t eoff = (uint32_t)kQ * 2 * kABox;  // S boxes follow the E operands
  const uint32_t coff = eoff + 2 * p.bbox;          // coordinates follow the S boxes

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int it = 0;
      int issued[2] = {-1, -1};
      bool stop = false;
      for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
        for (int c = 0; c < p.nchunks; ++c, ++it) {
          const int st = it & 1;
          if (!mbar_wait(empty0 + 8 * st, ((uint32_t)(it >> 1) & 1u) ^ 1u, &abort_flag, p.status)) {
            stop = true;
            break;
          }
          uint8_t* sb = base + (size_t)st * p.stage_bytes;
          mbar_expect_tx(full0 + 8 * st, 2 * p.bbox + p.cbytes);
          tma_load_2d(smem_u32(sb + eoff), &tmShi, c * kChunk, 0, full0 + 8 * st);
          tma_load_2d(smem_u32(sb + eoff + p.bbox), &tmSlo, c * kChunk, 0, full0 + 8 * st);
          bulk_load(smem_u32(sb + coff), p.xc + (size_t)c * kChunk * 2 * p.dp, p.cbytes,
                    full0 + 8 * st);
          issued[st] = it;
        }
      }
      if (abort_flag) {
        for (int s = 0; s < 2; ++s)
          if (issued[s] >= 0) mbar_drain(full0 + 8 * s, (uint32_t)(issued[s] >> 1) & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, seg = 0, last = -1;
      bool stop = false;
      for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
        for (int c = 0; c < p.nchunks; ++c, ++it) {
          const int st = it & 1;
          const uint32_t ph = (uint32_t)(it >> 1) & 1u;
          const int cin = c % p.seg_chunks;
          const int buf = seg & 1;
          if (cin == 0 &&
              !mbar_wait(accempty0 + 8 * buf, ((uint32_t)(seg >> 1) & 1u) ^ 1u, &abort_flag,
                         p.status)) {
            stop = true;
            break;
          }
          if (!mbar_wait(full0 + 8 * st, ph, &abort_flag, p.status) ||
              !mbar_wait(gen0 + 8 * st, ph, &abort_flag, p.status)) {
            stop = true;
            break;
          }
          fence_after();
          const uint8_t* sb = base + (size_t)st * p.stage_bytes;
          const uint32_t bhi = smem_u32(sb + eoff), blo = bhi + p.bbox;
          for (int q = 0; q < kQ; ++q) {
            const uint32_t d = tmem + (uint32_t)(buf * kQ * p.nb + q * p.nb);
            const uint32_t ehi = smem_u32(sb + (size_t)(q * 2) * kABox), elo = ehi + kABox;
            const uint32_t Aop[3] = {ehi, ehi, elo};  // E_hi S_hi + E_hi S_lo + E_lo S_hi
            const uint32_t Bop[3] = {bhi, blo, bhi};
            for (int prod = 0; prod < 3; ++prod) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t acc = (cin == 0 && prod == 0 && ks == 0) ? 0u : 1u;
                mma_tf32(d, smem_desc(Aop[prod] + ks * 32), smem_desc(Bop[prod] + ks * 32), p.idesc,
                         acc);
              }
            }
          }
          mma_commit(empty0 + 8 * st);
          last = it;
          if (cin == p.seg_chunks - 1 || c == p.nchunks - 1) {
            mma_commit(accfull0 + 8 * buf);
            ++seg;
          }
        }
      }
      if (last >= 0) mbar_drain(empty0 + 8 * (last & 1), (uint32_t)(last >> 1) & 1u);
    }
  } else if (warp < kFirstGenWarp) {
    // ---------------- fold: warps 2..5, lane quarter qr = warp % 4
    const int qr = warp & 3;
    int seg = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
      const int jt = u % p.njt, qg = u / p.njt;
      const int row = jt * kRows + qr * 32 + lane;
      for (int g = 0; g < nseg; ++g, ++seg) {
        const int buf = seg & 1;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(accfull0 + 8 * buf, (uint32_t)(seg >> 1) & 1u,
                                                          &abort_flag, p.status));
        if (!ok) {
          stop = true;
          break;
        }
        fence_after();
        for (int q = 0; q < kQ; ++q) {
          const int64_t qi = (int64_t)qg * kQ + q;
          const bool live = qi < p.m && row < p.s;
          const double lambda = (live && g == nseg - 1) ? p.params[qi * 2 + 1] : 0.0;
          double* Mq = p.M + qi * (int64_t)p.s * p.r;
          for (int cb = 0; cb < p.nb / 16; ++cb) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(qr * 32) << 16) + (uint32_t)(buf * kQ * p.nb + q * p.nb + cb * 16),
                      v);
            if (live) {
              // all sixteen loads before any store, so that they are in flight together
              double prev[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int col = cb * 16 + e;
                prev[e] = 0.0;
                if (col < p.r) {
                  if (g > 0) prev[e] = Mq[(int64_t)col * p.s + row];
                  if (g == nseg - 1) prev[e] += lambda * p.SJ[(int64_t)col * p.s + row];
                }
              }
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int col = cb * 16 + e;
                if (col < p.r) Mq[(int64_t)col * p.s + row] = prev[e] + (double)v[e];
              }
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(accempty0 + 8 * buf);
      }
    }
  } else {
    // ---------------- generators: rows 4 rg .. 4 rg + 3 of the J tile, points 4 pg .. 4 pg + 3
    // of each chunk; warp w holds row groups 4w .. 4w + 3 (lane = 8 rgl + pg)
    const int gt = threadIdx.x - kFirstGenWarp * 32;
    const int rg = (gt >> 5) * 4 + ((gt & 31) >> 3), pg = gt & 7;
    constexpr int DP = 4 * DP4;
    int it = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
      const int jt = u % p.njt, qg = u / p.njt;
      const int row0 = jt * kRows + 4 * rg;
      bool valid[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) valid[a] = row0 + a < p.s;
      // rows' coordinates as packed pairs: xh[rp][t] = (x_{row 2rp}[t], x_{row 2rp+1}[t])
      f2 xh[2][DP], xl[2][DP];
#pragma unroll
      for (int rp = 0; rp < 2; ++rp) {
#pragma unroll
        for (int t = 0; t < DP; ++t) {
          float h[2], l[2];
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const int a = 2 * rp + b;
            h[b] = valid[a] ? p.xj[(size_t)(row0 + a) * 2 * p.dp + t] : 0.f;
            l[b] = valid[a] ? p.xj[(size_t)(row0 + a) * 2 * p.dp + p.dp + t] : 0.f;
          }
          xh[rp][t] = f2_pack(h[0], h[1]);
          xl[rp][t] = f2_pack(l[0], l[1]);
        }
      }
      f2 cq[kQ];
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        int64_t qi = (int64_t)qg * kQ + q;
        if (qi >= p.m) qi = p.m - 1;  // a lone last parameter: its twin's output is dropped
        const double sg = p.params[qi * 2];
        const float c = (float)(-1.4426950408889634 / (2.0 * sg * sg));  // -log2(e) / (2 sigma^2)
        cq[q] = f2_pack(c, c);
      }
      for (int c = 0; c < p.nchunks; ++c, ++it) {
        const int st = it & 1;
        const bool ok =
            __all_sync(0xffffffffu, mbar_wait(full0 + 8 * st, (uint32_t)(it >> 1) & 1u, &abort_flag,
                                              p.status));
        if (!ok) {
          stop = true;
          break;
        }
        uint8_t* sb = base + (size_t)st * p.stage_bytes;
        // chunk coordinates, dimension-major: hi [t][32 points], then lo [t][32 points]
        const float* C = reinterpret_cast<const float*>(sb + coff) + pg * 4;
        f2 acc[2][4];  // acc[rp][e]: squared distances of rows (2rp, 2rp+1) to point e
#pragma unroll
        for (int rp = 0; rp < 2; ++rp)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[rp][e] = 0ull;
#pragma unroll
        for (int t = 0; t < DP; ++t) {
          const float4 ch = *reinterpret_cast<const float4*>(C + t * 32);
          const float4 cl = *reinterpret_cast<const float4*>(C + (DP + t) * 32);
          const float chv[4] = {ch.x, ch.y, ch.z, ch.w}, clv[4] = {cl.x, cl.y, cl.z, cl.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const f2 CH = f2_pack(chv[e], chv[e]), CL = f2_pack(clv[e], clv[e]);
#pragma unroll
            for (int rp = 0; rp < 2; ++rp) {
              const f2 df = f2_add(f2_sub(xh[rp][t], CH), f2_sub(xl[rp][t], CL));
              acc[rp][e] = f2_fma(df, df, acc[rp][e]);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          uint8_t* ehi = sb + (size_t)(q * 2) * kABox;
          uint8_t* elo = ehi + kABox;
          float ev[4][4];  // ev[row a][point e]
#pragma unroll
          for (int rp = 0; rp < 2; ++rp)
#pragma unroll
            for (int e = 0; e < 4; ++e) f2_unpack(f2_mul(acc[rp][e], cq[q]), ev[2 * rp][e], ev[2 * rp + 1][e]);
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = 4 * rg + a;
            float hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x = valid[a] ? ex2_approx(ev[a][e]) : 0.f;
              hi[e] = tf32_hi(x);
              lo[e] = x - hi[e];
            }
            // swizzled K-major: 8-row groups of 1024 B, 16-byte chunk pg XOR (row % 8)
            const uint32_t off =
                (uint32_t)(i >> 3) * 1024u + (uint32_t)(i & 7) * 128u + (uint32_t)((pg ^ (i & 7)) * 16);
            *reinterpret_cast<float4*>(ehi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4*>(elo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(gen0 + 8 * st);
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// K-major B operand map: rows = columns of S (nb), 32 points (128 B) per box row.
static bool make_s_map(CUtensorMap* map, const float* base, int64_t npad, int nb) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)nb};
  cuuint64_t strides[1] = {(cuuint64_t)npad * sizeof(float)};
  cuuint32_t box[2] = {32, (cuuint32_t)nb};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Setup copies: S^T split into tf32 hi / float32 lo (nb x npad, zero padded),
// coordinates of every point (per 32-point chunk, dimension-major) and of the
// rows of J (row-major) as float32 hi / lo pairs.
__global__ void krr_tc_copies_kernel(const double* S, int64_t ldS, int64_t n, int r, int nb,
                                     int64_t npad, const double* X, const double* XJ, int d, int dp,
                                     int s, float* sthi, float* stlo, float* xc, float* xj) {
  const int64_t total_s = (int64_t)nb * npad;
  const int64_t total_x = npad * dp;
  const int64_t total_j = (int64_t)s * dp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total_s; idx += stride) {
    const int l = (int)(idx / npad);
    const int64_t k = idx % npad;
    float h = 0.f, lo = 0.f;
    if (l < r && k < n) {
      const float x = (float)S[k + (int64_t)l * ldS];
      h = tf32_hi(x);
      lo = x - h;
    }
    sthi[idx] = h;
    stlo[idx] = lo;
  }
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total_x; idx += stride) {
    const int64_t k = idx / dp;
    const int t = (int)(idx % dp);
    const double x = (k < n && t < d) ? X[k * d + t] : 0.0;
    const float h = (float)x;
    // chunk c = k / 32 holds hi [t][32] then lo [t][32]
    const int64_t cbase = (k / 32) * 64 * dp;
    xc[cbase + (int64_t)t * 32 + (k % 32)] = h;
    xc[cbase + (int64_t)(dp + t) * 32 + (k % 32)] = (float)(x - (double)h);
  }
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total_j; idx += stride) {
    const int64_t j = idx / dp;
    const int t = (int)(idx % dp);
    const double x = t < d ? XJ[j * d + t] : 0.0;
    const float h = (float)x;
    xj[j * 2 * dp + t] = h;
    xj[j * 2 * dp + dp + t] = (float)(x - (double)h);
  }
}

}  // namespace krrtc

int krr_tc_nb(int r) { return (r + 15) / 16 * 16; }
int64_t krr_tc_npad(int64_t n) { return (n + krrtc::kChunk - 1) / krrtc::kChunk * krrtc::kChunk; }
int krr_tc_dp(int d) { return (d + 3) / 4 * 4; }

static uint32_t krr_tc_stage_bytes(int nb, int dp) {
  const uint32_t cbytes = (uint32_t)(krrtc::kChunk * 2 * dp * sizeof(float));
  return (uint32_t)(krrtc::kQ * 2 * krrtc::kABox) + 2u * (uint32_t)nb * 128u +
         (cbytes + 1023u) / 1024u * 1024u;
}

size_t krr_tc_smem_bytes(int r, int d) {
  return 1024 + 2 * (size_t)krr_tc_stage_bytes(krr_tc_nb(r), krr_tc_dp(d)) + 10 * sizeof(uint64_t);
}

bool krr_tc_supported(const sas_ctx* c) {
  return c->family == 1 && c->StHi != nullptr && tc::encode_fn() != nullptr && c->r <= 128 &&
         c->d <= 16;
}

cudaError_t launch_krr_tc_copies(const sas_ctx* c, cudaStream_t st) {
  krrtc::krr_tc_copies_kernel<<<c->num_sms * 8, 256, 0, st>>>(
      (const double*)c->S, c->ldS, c->n, c->r, krr_tc_nb(c->r), krr_tc_npad(c->n), c->X, c->XJ, c->d,
      krr_tc_dp(c->d), c->s, c->StHi, c->StLo, c->Xc32, c->XJ32);
  return cudaGetLastError();
}

cudaError_t launch_krr_assemble_tc(const sas_ctx* c, const double* params, int64_t m, double* M,
                                   cudaStream_t st) {
  using namespace krrtc;
  if (m == 0) return cudaSuccess;
  const int nb = krr_tc_nb(c->r), dp = krr_tc_dp(c->d);
  const int64_t npad = krr_tc_npad(c->n);
  if (npad / kChunk > 2147483647 || m > 2147483647) return cudaErrorInvalidValue;
  Params p;
  p.xj = c->XJ32;
  p.xc = c->Xc32;
  p.params = params;
  p.SJ = c->SJ;
  p.M = M;
  p.nchunks = (int)(npad / kChunk);
  p.dp = dp;
  p.r = c->r;
  p.s = c->s;
  p.nb = nb;
  p.m = m;
  p.njt = (c->s + kRows - 1) / kRows;
  p.seg_chunks = c->krr_seg_points / kChunk;
  if (p.seg_chunks < 1) p.seg_chunks = 1;
  const int64_t units = (int64_t)p.njt * ((m + kQ - 1) / kQ);
  if (units > 2147483647) return cudaErrorInvalidValue;
  p.num_units = (int)units;
  p.idesc = tc::tf32_idesc(kRows, nb);
  p.bbox = (uint32_t)nb * 128u;
  p.cbytes = (uint32_t)(kChunk * 2 * dp * sizeof(float));
  p.stage_bytes = krr_tc_stage_bytes(nb, dp);
  p.status = c->dev_status;
  CUtensorMap mhi, mlo;
  if (!make_s_map(&mhi, c->StHi, npad, nb) || !make_s_map(&mlo, c->StLo, npad, nb))
    return cudaErrorInvalidValue;
  const size_t smem = krr_tc_smem_bytes(c->r, c->d);
  const int grid = (int)(units < c->num_sms ? units : c->num_sms);
  cudaError_t e;
#define SAS_KRR_TC(DP4)                                                                          \
  e = cudaFuncSetAttribute(krr_tc_kernel<DP4>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                           (int)smem);                                                           \
  if (e != cudaSuccess) return e;                                                                \
  krr_tc_kernel<DP4><<<grid, kThreads, smem, st>>>(mhi, mlo, p);
  switch (dp / 4) {
    case 1: SAS_KRR_TC(1) break;
    case 2: SAS_KRR_TC(2) break;
    case 3: SAS_KRR_TC(3) break;
    case 4: SAS_KRR_TC(4) break;
    default: return cudaErrorInvalidValue;
  }
#undef SAS_KRR_TC
  return cudaGetLastError();
}

}  // namespace sas
