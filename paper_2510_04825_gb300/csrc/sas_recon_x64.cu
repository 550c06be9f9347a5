// Float64-accurate reconstruction x_hat = S y on the tensor cores (mixed form, sm_103a).
//
// x_hat is the output of the online stage (Alg. 1 step 4, "output S y").  Its
// true residual ||A(p) x_hat - b|| / ||b|| is what the paper reports (Sec. 5.2.2,
// Table 3; Sec. 5.2.3, Table 4), and for a discretised PDE that residual sees
// every rounding of x_hat amplified by up to ||A||: a float32 x_hat is not
// residual-equivalent to a float64 one.  This kernel therefore returns x_hat in
// float64 with an error far below float64 rounding of the product, while doing
// the n r m multiply-adds on the f16 tensor cores.
//
// Method: fixed-point digit splitting of both operands, the error-free product
// splitting of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication", 2012)
// in a fixed-point form with one exponent per row of S and per column of y:
//   S[i,k] = 2^{e_i} sum_{a<5} sigma_a[i,k] 2^{-9(a+1)},  |sigma_0| <= 512,
//            |sigma_a| <= 256 (a >= 1), e_i from max_k |S[i,k]|;
//   y[k,j] = 2^{f_j} sum_{b<5} tau_b[k,j] 2^{-9(b+1)},   f_j from ||y_j||_1, so
//            that sum_k |tau_0[k,j]| <= 512 + 32.
// Digits are integers, exact in f16, and the product of two is exact in the f32
// accumulator.  Products of level L = a + b share one accumulator.  With K <= 64
// every partial sum of a level stays below 2^24 for L <= 2:
//   |P_0| <= 512 (512 + 32)                              < 2^19
//   |P_1| <= 512*256*64 + 256 (512 + 32)                 < 2^24
//   |P_2| <= 512*256*64 + 256*256*64 + 256 (512 + 32)    < 2^24
// so P_0, P_1, P_2 come out of TMEM exactly.  Levels 3 and 4 share a fourth
// accumulator T = P_3 + 2^-9 P_4 (the tensor core's scale-input-d), whose
// rounding is a few units of 2^-45.  Pairs with a + b >= 5 are dropped; each is
// below 2^-45 of the scale 2^{e_i + f_j}.  The result
//   x[i,j] = 2^{e_i + f_j - 45} (P_0 2^27 + P_1 2^18 + P_2 2^9 + rint(T))
// is formed as an exact int64 (below 2^46) and converted to float64 once.
//
// Structure (one persistent CTA per SM, 18 warps; tiles of 128 rows x 128 parameters):
//   warp 0     TMA producer: per work unit the five S digit tiles of 128 rows
//              (80 KB, resident for the unit), then for every parameter tile its
//              five y digit tiles (16 KB each, L2-resident) into an 8-slot ring;
//   warp 1     MMA issuer: the whole warp runs the loop (descriptors stay
//              warp-uniform) and the elected lane issues tcgen05.mma (kind::f16,
//              M = N = 128, K = 16): per tile 15 digit products x 4 K-steps into 4
//              TMEM accumulators of 128 columns (all 512), in the order L0, L1,
//              tail (L4, then L3 on the scaled sum), L2;
//   warps 2-17 epilogue, 4 per TMEM lane quarter, 32 columns each.  They drain
//              P_0 and P_1 (into a = P_0 2^9 + P_1) as each completes and release
//              it at once, so that the next tile's first 12 MMAs run while they
//              assemble this tile; then, 16 columns at a time, rint(T) and P_2
//              (both released once the second half is loaded, for the next
//              tile's remaining 48 MMAs); they convert (alternating the int64 ->
//              float64 conversion, which runs on the float64 pipe, and an
//              integer-only normalisation, so that both work side by side), scale
//              and store 8 bytes per lane (one coalesced 256-byte warp store per
//              parameter).  18 warps put 5 on some SM sub-partitions, which caps
//              registers at 96 per thread.
// A shared-memory operand pair of f16 at N = 128 reads 8 KB per 64-clock MMA,
// the SM's shared-memory bandwidth: 128-parameter tiles keep the MMA at its
// full rate, narrower ones would not.
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// records SAS_ETIMEOUT, stops issuing work, waits (bounded) for its copies and
// MMAs in flight, frees its TMEM and returns.
#include <cuda_fp16.h>

#include <cstring>

#include "sas_internal.cuh"
#include "sas_tc_common.cuh"

namespace sas {
namespace x64 {

using namespace tc;

constexpr int kBM = 128;                  // rows of S per tile (MMA M)
constexpr int kBN = 128;                  // parameters per tile (MMA N)
constexpr int kDigits = 5;                // 9-bit digits per operand
constexpr int kSlots = 8;                 // y digit ring
constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kATileBytes = kBM * 128;  // one S digit tile: 128 rows x 64 f16 (128-byte rows)
constexpr uint32_t kBTileBytes = kBN * 128;  // one y digit tile: 128 rows x 64 f16
constexpr uint32_t kTmemCols = 512;          // 4 accumulators x 128 columns
constexpr uint32_t kIdesc = f16_idesc(kBM, kBN);
constexpr int kNumBars = 2 + 2 * kSlots + 8;

struct Params {
  double* out;        // m x n, row j at out + j n
  int64_t n, m;
  const int* erow;    // e_i, n entries
  const int* ecol;    // f_j, m entries
  int s_plane;        // rows of one S digit plane (n rounded up to 128)
  int y_plane;        // rows of one y digit plane (m rounded up to 128)
  int num_mtiles, num_ntiles, ngroups, ntpg, num_units;
  int* status;
};

__device__ inline void unit_range(const Params& p, int u, int& mt, int& nt0, int& nt1) {
  mt = u / p.ngroups;
  const int g = u % p.ngroups;
  nt0 = g * p.ntpg;
  nt1 = nt0 + p.ntpg < p.num_ntiles ? nt0 + p.ntpg : p.num_ntiles;
}

__device__ inline int cvt_rni(float x) {
  int r;
  asm("cvt.rni.s32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// One entry of the fast path: V = a 2^18 + rint(P_2) 2^9 + t as an exact int64,
// converted once to float64, with the scale 2^E applied as an integer add of
// add = E 2^20 to the high word (V = 0 keeps its all-zero bits).
__device__ __forceinline__ double assemble(int a, float p2, int t, int add) {
  double x;
  asm("{\n"
      " .reg .s32 i2, lo, hi;\n"
      " .reg .s64 t64, v;\n"
      " .reg .f64 d;\n"
      " .reg .pred pz;\n"
      " cvt.rni.s32.f32 i2, %2;\n"
      " cvt.s64.s32 t64, %3;\n"
      " mad.wide.s32 v, i2, 512, t64;\n"
      " mad.wide.s32 v, %1, 262144, v;\n"
      " cvt.rn.f64.s64 d, v;\n"
      " mov.b64 {lo, hi}, d;\n"
      " setp.ne.s32 pz, hi, 0;\n"
      " @pz add.s32 hi, hi, %4;\n"
      " mov.b64 %0, {lo, hi};\n"
      "}\n"
      : "=d"(x)
      : "r"(a), "f"(p2), "r"(t), "r"(add));
  return x;
}

// The same entry converted with integer operations only (no int64 -> float64
// conversion unit): sign and magnitude of V, leading-zero count, the mantissa shifted
// to bit 52 and the exponent 1086 - lz + E built in the high word.  The fast path
// alternates this with assemble() so that the slow conversion unit and the integer
// pipes work side by side.
__device__ __forceinline__ double assemble_int(int a, float p2, int t, int add) {
  const int i2 = cvt_rni(p2);
  const long long v = (long long)a * 262144ll + (long long)i2 * 512ll + (long long)t;
  const long long s = v >> 63;
  unsigned long long u = (unsigned long long)((v ^ s) - s);
  const int lz = __clzll((long long)u);
  u <<= (lz - 11);  // leading bit at 52 (|V| < 2^47, so lz >= 17)
  unsigned h = ((unsigned)(u >> 32) & 0xFFFFFu) | ((unsigned)(1086 - lz) << 20);
  h += (unsigned)add;
  h |= (unsigned)s & 0x80000000u;
  if (lz == 64) h = 0;  // V = 0
  return __hiloint2double((int)h, (int)(unsigned)u);
}

__global__ void __launch_bounds__(kThreads, 1)
    reconstruct_x64_kernel(const __grid_constant__ CUtensorMap tmS,
                           const __grid_constant__ CUtensorMap tmY, Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* A0 = base;                                    // sigma_0..4 of the unit's row tile
  uint8_t* B0 = A0 + (size_t)kDigits * kATileBytes;      // ring of y digit tiles
  uint64_t* bars = reinterpret_cast<uint64_t*>(B0 + (size_t)kSlots * kBTileBytes);
  // bars: afull, aempty, bfull[kSlots], bempty[kSlots], tfull[4], tempty[4]
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ __align__(16) int colexp[kEpiWarps][32];  // per epilogue warp: (f_j - 45) 2^20

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t afull = smem_u32(&bars[0]), aempty = smem_u32(&bars[1]);
  const uint32_t bfull0 = smem_u32(&bars[2]), bempty0 = smem_u32(&bars[2 + kSlots]);
  const uint32_t tfull0 = smem_u32(&bars[2 + 2 * kSlots]);
  const uint32_t tempty0 = smem_u32(&bars[2 + 2 * kSlots + 4]);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(afull, 1);
    mbar_init(aempty, 1);
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(bfull0 + 8 * s, 1);
      mbar_init(bempty0 + 8 * s, 1);
    }
    for (int a = 0; a < 4; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, kEpiWarps);
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

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int g = 0, at = 0, a_issued = -1;
      bool stop = false;
      for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
        int mt, nt0, nt1;
        unit_range(p, u, mt, nt0, nt1);
        for (int k = 0; k < nt1 - nt0 && !stop; ++k) {
          const int nt = nt0 + k;
          for (int b = 0; b < kDigits; ++b) {
            const int s = g % kSlots;
            if (!mbar_wait_idle(bempty0 + 8 * s, ((uint32_t)(g / kSlots) & 1u) ^ 1u, &abort_flag,
                           p.status)) {
              stop = true;
              break;
            }
            mbar_expect_tx(bfull0 + 8 * s, kBTileBytes);
            tma_load_2d(smem_u32(B0 + (size_t)s * kBTileBytes), &tmY, 0,
                        b * p.y_plane + nt * kBN, bfull0 + 8 * s);
            ++g;
            if (k == 0 && b == 0) {
              // the S digit tiles free when the last MMA of the previous unit completes
              if (!mbar_wait_idle(aempty, ((uint32_t)at & 1u) ^ 1u, &abort_flag, p.status)) {
                stop = true;
                break;
              }
              mbar_expect_tx(afull, kDigits * kATileBytes);
              for (int a = 0; a < kDigits; ++a)
                tma_load_2d(smem_u32(A0 + (size_t)a * kATileBytes), &tmS, 0,
                            a * p.s_plane + mt * kBM, afull);
              a_issued = at++;
            }
          }
        }
      }
      if (abort_flag) {
        // the last copy issued to slot s had ring index gl = the largest gl < g with gl % kSlots == s
        for (int s = 0; s < kSlots && s < g; ++s) {
          const int gl = g - 1 - (g - 1 - s) % kSlots;
          mbar_drain(bfull0 + 8 * s, (uint32_t)(gl / kSlots) & 1u);
        }
        if (a_issued >= 0) mbar_drain(afull, (uint32_t)a_issued & 1u);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: the whole warp runs the loop, so that descriptors and
    // counters are warp-uniform; the elected lane issues the MMAs and their commits.
    // Per tile the levels go in the order L0, L1, tail (L4 then L3), L2: the epilogue
    // drains the first two as they complete, so that while it assembles the tile the
    // next tile's first 12 MMAs already run, and the tail and L2 half-way through.
    const bool leader = elect_one();
    int t = 0, ua = 0;
    uint32_t last_bar = 0, last_par = 0;
    bool any = false, stop = false;
    const uint32_t a_base = smem_u32(A0), b_base = smem_u32(B0);
    uint64_t ad[kDigits];  // descriptors of the resident S digit tiles
#pragma unroll
    for (int a = 0; a < kDigits; ++a) ad[a] = smem_desc(a_base + (uint32_t)a * kATileBytes);
    auto wait_all = [&](uint32_t bar, uint32_t par) -> bool {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_idle(bar, par, &abort_flag, p.status));
      fence_after();
      return ok;
    };
    for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
      int mt, nt0, nt1;
      unit_range(p, u, mt, nt0, nt1);
      if (nt0 >= nt1) continue;
      if (!wait_all(afull, (uint32_t)ua & 1u)) break;
      for (int k = 0; k < nt1 - nt0; ++k) {
        const int gb = kDigits * t;  // ring index of this tile's tau_0
        const uint32_t free_par = ((uint32_t)t & 1u) ^ 1u;  // accumulators drained for tile t - 1
        // descriptors of this tile's y digits; a K step of 16 f16 advances the start
        // address field (16-byte units) by 2
        uint64_t bd[kDigits];
        uint32_t bfull_b[kDigits], bpar[kDigits];
#pragma unroll
        for (int b = 0; b < kDigits; ++b) {
          const int gg = gb + b, sl = gg % kSlots;
          bd[b] = smem_desc(b_base + (uint32_t)sl * kBTileBytes);
          bfull_b[b] = bfull0 + 8 * sl;
          bpar[b] = (uint32_t)(gg / kSlots) & 1u;
        }
        // one digit product sigma_a tau_b (K = 64 in four steps of 16) into accumulator acc
        auto prod = [&](int acc, int a, int b, bool first) {
          const uint32_t d = tmem + (uint32_t)(acc * kBN);
          if (first)
            mma_f16_c<false>(d, ad[a], bd[b], kIdesc);
          else
            mma_f16_c<true>(d, ad[a], bd[b], kIdesc);
#pragma unroll
          for (int ks = 1; ks < 4; ++ks) mma_f16_c<true>(d, ad[a] + 2 * ks, bd[b] + 2 * ks, kIdesc);
        };
        auto prod_scaled = [&](int acc, int a, int b) {
          const uint32_t d = tmem + (uint32_t)(acc * kBN);
          mma_f16_scale9(d, ad[a], bd[b], kIdesc);
#pragma unroll
          for (int ks = 1; ks < 4; ++ks) mma_f16_c<true>(d, ad[a] + 2 * ks, bd[b] + 2 * ks, kIdesc);
        };
        // levels 0 and 1
        if (!wait_all(bfull_b[0], bpar[0]) || !wait_all(bfull_b[1], bpar[1]) ||
            !wait_all(tempty0, free_par) || !wait_all(tempty0 + 8, free_par)) {
          stop = true;
          break;
        }
        if (leader) {
          prod(0, 0, 0, true);
          mma_commit(tfull0);
          prod(1, 0, 1, true);
          prod(1, 1, 0, false);
          mma_commit(tfull0 + 8);
        }
        __syncwarp();
        // the tail, T = P_3 + 2^-9 P_4: level 4 first, then level 3 on the scaled sum
        if (!wait_all(tempty0 + 24, free_par) || !wait_all(bfull_b[2], bpar[2])) {
          stop = true;
          break;
        }
        if (leader) {
          prod(3, 4, 0, true);
          prod(3, 3, 1, false);
          prod(3, 2, 2, false);
        }
        __syncwarp();
        if (!wait_all(bfull_b[3], bpar[3]) || !wait_all(bfull_b[4], bpar[4])) {
          stop = true;
          break;
        }
        if (leader) {
          prod(3, 1, 3, false);
          prod(3, 0, 4, false);
          prod_scaled(3, 3, 0);
          prod(3, 2, 1, false);
          prod(3, 1, 2, false);
          prod(3, 0, 3, false);
          mma_commit(tfull0 + 24);
        }
        __syncwarp();
        // level 2 last
        if (!wait_all(tempty0 + 16, free_par)) {
          stop = true;
          break;
        }
        if (leader) {
          prod(2, 0, 2, true);
          prod(2, 1, 1, false);
          prod(2, 2, 0, false);
          mma_commit(tfull0 + 16);
#pragma unroll
          for (int b = 0; b < kDigits; ++b) mma_commit(bfull_b[b] + 8 * kSlots);  // bempty of the slot
          if (k == nt1 - nt0 - 1) mma_commit(aempty);
        }
        __syncwarp();
        last_bar = tfull0 + 16;
        last_par = (uint32_t)t & 1u;
        any = true;
        ++t;
      }
      ++ua;
    }
    if (any && leader) mbar_drain(last_bar, last_par);
  } else {
    // ---------------- epilogue: warps 2 .. 17; lane quarter q = warp % 4 (the TMEM lanes
    // this warp may read), column block cb of 32 of the tile's 128 parameters
    const int q = warp & 3, cb = (warp - 2) >> 2;
    int t = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
      int mt, nt0, nt1;
      unit_range(p, u, mt, nt0, nt1);
      const int64_t row = (int64_t)mt * kBM + q * 32 + lane;
      const bool row_ok = row < p.n;
      const int erow = row_ok ? p.erow[row] : 0;
      const bool rows_full = __all_sync(0xffffffffu, row_ok);  // the fast path stores unguarded
      const int emin = __reduce_min_sync(0xffffffffu, erow);
      const int emax = __reduce_max_sync(0xffffffffu, erow);
      const int ehi = erow * (1 << 20);  // e_i in the exponent field of the high word
      for (int k = 0; k < nt1 - nt0; ++k, ++t) {
        const int64_t j0 = (int64_t)(nt0 + k) * kBN + cb * 32;
        const int fcol = j0 + lane < p.m ? p.ecol[j0 + lane] : 0;
        // fast path (warp-uniform): all 32 columns present and every E = e_i + f_j - 45 such
        // that V 2^E with 1 <= |V| < 2^46 stays a normal float64; then the scaling is one
        // integer add to the high word.  Otherwise every entry takes the checked path.
        const int fmin = __reduce_min_sync(0xffffffffu, fcol);
        const int fmax = __reduce_max_sync(0xffffffffu, fcol);
        const bool fast = rows_full && j0 + 32 <= p.m && emin + fmin - 45 >= -1022 &&
                          emax + fmax - 45 <= 977;
        // (f_j - 45) in the exponent field, column c's at colexp[.][c]: read back as
        // broadcast 16-byte loads (one per 4 entries) instead of a shuffle per entry
        int* fsh = colexp[warp - 2];
        __syncwarp();  // the previous tile's reads are done
        fsh[lane] = (fcol - 45) * (1 << 20);
        __syncwarp();
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * 32);
        const uint32_t par = (uint32_t)t & 1u;
        int acol[32];
        float v[32];
        auto wait_acc = [&](int acc) -> bool {
          const bool ok = __all_sync(0xffffffffu, mbar_wait_idle(tfull0 + 8 * acc, par, &abort_flag,
                                                                p.status));
          fence_after();
          return ok;
        };
        auto release = [&](int acc) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
        };
        // P_0 and P_1 -> a = P_0 2^9 + P_1 (|a| < 2^28); each accumulator is released as soon
        // as it is read, for the next tile's first 12 MMAs
        if (!wait_acc(0)) { stop = true; break; }
        tmem_ld32(ta, v);
        release(0);
#pragma unroll
        for (int c = 0; c < 32; ++c) acol[c] = cvt_rni(v[c]);
        if (!wait_acc(1)) { stop = true; break; }
        tmem_ld32(ta + kBN, v);
        release(1);
#pragma unroll
        for (int c = 0; c < 32; ++c) acol[c] = acol[c] * 512 + cvt_rni(v[c]);
        // then kSub columns at a time: rint(T) and P_2, and x = 2^{e_i + f_j - 45} (a 2^18 +
        // P_2 2^9 + rint(T)); the tail and P_2 accumulators are released once the last
        // sub-block is loaded (kSub live tail values instead of 32 relieve the register cap)
        if (!wait_acc(3) || !wait_acc(2)) { stop = true; break; }
        double* orow = p.out + j0 * p.n + row;
        constexpr int kSub = 8;
#pragma unroll
        for (int h = 0; h < 32 / kSub; ++h) {
          int itail[kSub];
          float w[kSub];
          tmem_ld8(ta + 3 * kBN + kSub * h, w);
#pragma unroll
          for (int c = 0; c < kSub; ++c) itail[c] = cvt_rni(w[c]);
          tmem_ld8(ta + 2 * kBN + kSub * h, w);
          if (h == 32 / kSub - 1) {
            release(3);
            release(2);
          }
          if (fast) {
            double* o = orow + (int64_t)(kSub * h) * p.n;
            const int64_t ns = p.n;
            int fc[kSub];
#pragma unroll
            for (int c = 0; c < kSub; c += 4)
              *reinterpret_cast<int4*>(fc + c) = *reinterpret_cast<const int4*>(fsh + kSub * h + c);
#pragma unroll
            for (int c = 0; c < kSub; ++c) {
              const int add = ehi + fc[c];
              const double x = (c & 1) ? assemble(acol[kSub * h + c], w[c], itail[c], add)
                                       : assemble_int(acol[kSub * h + c], w[c], itail[c], add);
              __stcs(o + c * ns, x);
            }
          } else {
            // checked: V 2^E tested against the float64 range (below it the entry is
            // flushed to zero, above it it overflows to +-inf), ragged columns skipped
#pragma unroll
            for (int c = 0; c < kSub; ++c) {
              const int cc = kSub * h + c;
              const int E = erow + __shfl_sync(0xffffffffu, fcol, cc) - 45;
              const double d = assemble(acol[cc], w[c], itail[c], 0);
              int hi = __double2hiint(d), lo = __double2loint(d);
              const int ex = ((hi >> 20) & 0x7ff) + E;
              if (hi == 0 || ex <= 0) {
                hi = 0;
                lo = 0;
              } else if (ex >= 2047) {
                hi = (hi & (int)0x80000000) | 0x7ff00000;
                lo = 0;
              } else {
                hi += E * (1 << 20);
              }
              if (row_ok && j0 + cc < p.m) __stcs(orow + (int64_t)cc * p.n, __hiloint2double(hi, lo));
            }
          }
        }
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

constexpr size_t kSmemBytes = 1024 + (size_t)kDigits * kATileBytes + (size_t)kSlots * kBTileBytes +
                               (size_t)kNumBars * sizeof(uint64_t);

// Digit planes of an operand: `plane` rows of 64 f16 per digit, plane a at
// D + a*plane*64.  One warp per row of 64 values v (zero beyond r): exponent
// e = ilogb(scale) + 1 with scale = max |v| (rows of S) or sum |v| (columns of
// y), then 5 rounded base-512 digits of v 2^-e.  Every step is exact in float64.
__device__ inline void split_row(double v0, double v1, bool l1, int lane, int64_t plane, int64_t i,
                                 __half* D, int* eout) {
  double sc = l1 ? fabs(v0) + fabs(v1) : fmax(fabs(v0), fabs(v1));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, sc, o);
    sc = l1 ? sc + w : fmax(sc, w);
  }
  const int e = sc > 0.0 ? ilogb(sc) + 1 : 0;
  v0 = ldexp(v0, 9 - e);
  v1 = ldexp(v1, 9 - e);
#pragma unroll
  for (int a = 0; a < kDigits; ++a) {
    const double d0 = rint(v0), d1 = rint(v1);
    __half* row = D + ((int64_t)a * plane + i) * 64;
    row[lane] = __double2half(d0);
    row[lane + 32] = __double2half(d1);
    v0 = (v0 - d0) * 512.0;
    v1 = (v1 - d1) * 512.0;
  }
  if (eout && lane == 0) *eout = e;
}

// S (n x r, column-major, ld ldS) -> digit planes of max-scaled rows and e_i.
// Blocks of 256 threads stage 64 rows x 64 columns in shared memory so that the
// reads of S are coalesced along its columns.
__global__ void __launch_bounds__(256) split_basis_kernel(const double* __restrict__ S, int64_t ldS,
                                                          int64_t n, int r, int64_t plane,
                                                          __half* D, int* erow) {
  __shared__ double tile[64][65];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t i0 = (int64_t)blockIdx.x * 64; i0 < plane; i0 += (int64_t)gridDim.x * 64) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
      const int k = idx >> 6, rr = idx & 63;
      const int64_t i = i0 + rr;
      tile[rr][k] = (k < r && i < n) ? S[i + (int64_t)k * ldS] : 0.0;
    }
    __syncthreads();
    for (int rr = w; rr < 64; rr += 8) {
      const int64_t i = i0 + rr;
      split_row(tile[rr][lane], tile[rr][lane + 32], false, lane, plane, i, D,
                i < n ? erow + i : nullptr);
    }
  }
}

// y (m x r, row j at Y + j r) -> digit planes of L1-scaled columns and f_j; the
// rows from m to plane are zero.
__global__ void split_coeff_kernel(const double* __restrict__ Y, int64_t m, int r, int64_t plane,
                                   __half* D, int* ecol) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < plane;
       j += warps) {
    const double v0 = (j < m && lane < r) ? Y[j * r + lane] : 0.0;
    const double v1 = (j < m && lane + 32 < r) ? Y[j * r + lane + 32] : 0.0;
    split_row(v0, v1, true, lane, plane, j, D, j < m ? ecol + j : nullptr);
  }
}

static bool make_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {64, (cuuint64_t)rows};
  cuuint64_t strides[1] = {64 * sizeof(__half)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace x64

int64_t x64_plane_rows(int64_t rows) { return (rows + x64::kBM - 1) / x64::kBM * x64::kBM; }

size_t x64_coeff_bytes(int64_t m) {
  return (size_t)x64::kDigits * x64_plane_rows(m) * 64 * sizeof(__half) + (size_t)m * sizeof(int) + 256;
}

bool reconstruct_x64_supported(const sas_ctx* c) {
  return c->dtype == SAS_REAL64 && c->r <= 64 && c->Sx64 != nullptr && tc::encode_fn() != nullptr;
}

cudaError_t setup_x64_basis(sas_ctx* c, cudaStream_t st) {
  if (c->dtype != SAS_REAL64 || c->r > 64) return cudaSuccess;
  const int64_t plane = x64_plane_rows(c->n);
  if ((int64_t)x64::kDigits * plane > 2147483647) return cudaSuccess;  // TMA row coordinate range
  cudaError_t e = cudaMalloc(&c->Sx64, (size_t)x64::kDigits * plane * 64 * sizeof(__half));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->Sx64_exp, (size_t)c->n * sizeof(int));
  if (e != cudaSuccess) return e;
  const int64_t blocks = (plane + 63) / 64;
  x64::split_basis_kernel<<<(unsigned)(blocks < 8 * c->num_sms ? blocks : 8 * c->num_sms), 256, 0,
                            st>>>((const double*)c->S, c->ldS, c->n, c->r, plane,
                                  (__half*)c->Sx64, c->Sx64_exp);
  return cudaGetLastError();
}

// x_hat (m x n float64, row j at out + j n) = S Y^T from the float64 coefficients
// Y (m x r).  scratch holds x64_coeff_bytes(m) bytes of device memory.
cudaError_t launch_reconstruct_x64(const sas_ctx* c, const double* Y, int64_t m, double* out,
                                   void* scratch, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  if (!reconstruct_x64_supported(c) || !scratch) return cudaErrorInvalidValue;
  const int64_t yplane = x64_plane_rows(m);
  if ((int64_t)x64::kDigits * yplane > 2147483647) return cudaErrorInvalidValue;
  __half* Yd = reinterpret_cast<__half*>(scratch);
  int* ecol = reinterpret_cast<int*>(Yd + (size_t)x64::kDigits * yplane * 64);
  {
    const int64_t warps = yplane;
    const int64_t blocks = (warps + 7) / 8;
    x64::split_coeff_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(
        Y, m, c->r, yplane, Yd, ecol);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(x64::reconstruct_x64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)x64::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  CUtensorMap mS, mY;
  const int64_t splane = x64_plane_rows(c->n);
  if (!x64::make_map(&mS, c->Sx64, x64::kDigits * splane, x64::kBM) ||
      !x64::make_map(&mY, Yd, x64::kDigits * yplane, x64::kBN))
    return cudaErrorInvalidValue;
  x64::Params p;
  p.out = out;
  p.n = c->n;
  p.m = m;
  p.erow = c->Sx64_exp;
  p.ecol = ecol;
  p.s_plane = (int)splane;
  p.y_plane = (int)yplane;
  reconstruct_tc_split(c->n, m, c->num_sms, x64::kBN, &p.num_mtiles, &p.num_ntiles, &p.ngroups,
                       &p.ntpg);
  const int64_t units = (int64_t)p.num_mtiles * p.ngroups;
  if (units > 2147483647) return cudaErrorInvalidValue;
  p.num_units = (int)units;
  p.status = c->dev_status;
  const int grid = (int)(units < c->num_sms ? units : c->num_sms);
  x64::reconstruct_x64_kernel<<<grid, x64::kThreads, x64::kSmemBytes, st>>>(mS, mY, p);
  return cudaGetLastError();
}

}  // namespace sas
