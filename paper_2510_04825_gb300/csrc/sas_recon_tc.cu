// Tensor-core reconstruction x_hat = S y for the mixed form (sm_103a, tcgen05).
//
// out[j*n + i] = sum_k S[i,k] y[j,k] in float32, computed as
//     S_hi y_hi + S_hi y_lo + S_lo y_hi
// where S = S_hi + S_lo and y = y_hi + y_lo are tf32 splits (S_hi, y_hi
// rounded to tf32; the low parts are the float32 remainders, truncated to
// tf32 by the tensor core).  The dropped S_lo y_lo term and the truncation of
// the low parts leave ~2^-21 relative error per product: float32-class
// accuracy at tf32 tensor-core rates.  The kernel is bound by HBM: it writes
// 4 n bytes per parameter and reads the split S (8 n rpad bytes) once per
// launch, however many parameters the launch has.
//
// Structure (one persistent CTA per SM; 2 + EW warps):
//   warp 0    TMA producer: for each work unit the S tile (S_hi, S_lo of 128
//             rows), then the unit's y tiles (y_hi, y_lo of BN parameters,
//             L2-resident) into a ring of stages;
//   warp 1    one thread issues tcgen05.mma (M = 128, N = BN) into TMEM
//             accumulator slots of BN columns;
//   epilogue  EW = 4 warps (one per TMEM lane quarter) or 8 (two per quarter,
//             alternate column halves): tcgen05.ld 32 lanes x 32 columns at a
//             time, then either direct coalesced streaming stores (lane = row,
//             one 128-byte warp store per parameter; the default) or, with
//             SAS_OPT_RECON_STORE = 0 and 4 warps, staging in shared memory and
//             TMA bulk-tensor stores.
// The default launch (SAS_OPT_RECON_KERNEL 0 or 3) is kind::tf32 with BN = 128,
// 2 stages, 4 accumulator slots, 4 epilogue warps and direct stores; option 2
// takes 64-parameter tiles, 4 rotates the order of the parameter tiles, 5 is
// the f16 variant and 6 the 8-warp epilogue.
// A work unit is one 128-row tile of S and a range of BN-parameter tiles; the
// S tile stays resident while the unit's y tiles stream past it.  With at
// least as many row tiles as SMs a unit covers every parameter tile, so S is
// read from HBM once; with fewer (small n) the parameter tiles are split into
// ranges so that every SM has work.  K = rpad (32 or 64) in boxes of 32 floats
// (128 B rows, 128-byte swizzle).
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// records SAS_ETIMEOUT in the status word, stops issuing work, waits (bounded)
// for its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda_fp16.h>

#include <cstring>

#include "sas_internal.cuh"
#include "sas_tc_common.cuh"

namespace sas {

namespace tc {

// 2 warps (TMA, MMA) + EW epilogue warps: EW = 4 (one per TMEM lane quarter)
// or 8 (two per quarter, each taking half of a tile's columns; direct stores)
template <int EW>
constexpr int threads_for() { return 64 + 32 * EW; }
constexpr int kBM = 128;              // rows of S per tile (MMA M)
constexpr int kABox = 128 * 128;      // A box: 128 rows x 32 floats (128-byte rows)

// Parameter-tile width BN (MMA N), operand type and the depths that keep the
// shared-memory and TMEM budgets:
//   tf32 (three split products into one accumulator): 64 x 4 stages or
//     128 x 2 stages, 4 accumulator slots of BN columns;
//   f16 (S_hi y_hi into one accumulator, S_hi y_lo + S_lo y_hi into a second,
//     the low parts carrying a 2^11 scale): 128 x 4 stages, 2 slots of 2 BN
//     columns.  Operand rows are 128 B in both: 32 tf32 or 64 f16 values.
template <int BN, bool F16>
struct Shape {
  static constexpr int kBBox = BN * 128;  // B box: BN rows x 128 B
  static constexpr int kBStages = F16 ? 4 : (BN == 64 ? 4 : 2);
  static constexpr int kAcc = F16 ? 2 : 4;
  static constexpr int kSlotCols = F16 ? 2 * BN : BN;
  static constexpr uint32_t kTmemCols = kAcc * kSlotCols;
  static constexpr uint32_t kIdesc = F16 ? f16_idesc(kBM, BN) : tf32_idesc(kBM, BN);
};

struct Params {
  float* out;
  int64_t n;
  int64_t m;
  int kboxes;      // rpad / 32 (1 or 2)
  int num_mtiles;  // ceil(n / kBM)
  int num_ntiles;  // ceil(m / BN)
  int ngroups;     // parameter tiles of one row tile are split into ngroups ranges
  int ntpg;        // parameter tiles per range
  int num_units;   // num_mtiles * ngroups
  int rotate;      // 1: each unit starts its parameter tiles at a unit-dependent offset
  const float* yscale;  // f16 form: per-parameter power-of-two scale of the product (m)
  int tma_store;   // 1: epilogue through shared memory and TMA stores
  int* status;
};

constexpr int kStageFloats = 32 * 32;  // one epilogue staging tile: 32 parameters x 32 rows

// Work unit u: row tile u / ngroups, parameter tiles [g ntpg, min((g+1) ntpg, num_ntiles))
// with g = u % ngroups.  All three roles walk the same units in the same order.
// With rotate, unit u visits its len tiles starting at offset (u * 37) % len, so
// that CTAs running at the same time write different parameters' rows.
__device__ inline void unit_range(const Params& p, int u, int& mt, int& nt0, int& nt1) {
  mt = u / p.ngroups;
  const int g = u % p.ngroups;
  nt0 = g * p.ntpg;
  nt1 = nt0 + p.ntpg < p.num_ntiles ? nt0 + p.ntpg : p.num_ntiles;
}
__device__ inline int unit_tile(const Params& p, int u, int nt0, int nt1, int k) {
  const int len = nt1 - nt0;
  if (!p.rotate) return nt0 + k;
  const int off = (int)(((long long)u * 37) % len);
  const int t = k + off;
  return nt0 + (t >= len ? t - len : t);
}

template <int BN, bool F16, int EW>
__global__ void __launch_bounds__(threads_for<EW>(), 1)
    reconstruct_tc_kernel(const __grid_constant__ CUtensorMap tmAhi,
                          const __grid_constant__ CUtensorMap tmAlo,
                          const __grid_constant__ CUtensorMap tmBhi,
                          const __grid_constant__ CUtensorMap tmBlo,
                          const __grid_constant__ CUtensorMap tmOut, Params p) {
  constexpr int kBN = BN;
  constexpr int kBBox = Shape<BN, F16>::kBBox;
  constexpr int kBStages = Shape<BN, F16>::kBStages;
  constexpr int kAcc = Shape<BN, F16>::kAcc;
  constexpr int kSlotCols = Shape<BN, F16>::kSlotCols;
  constexpr uint32_t kTmemCols = Shape<BN, F16>::kTmemCols;
  constexpr uint32_t kIdesc = Shape<BN, F16>::kIdesc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const int kb = p.kboxes;
  const uint32_t aop = (uint32_t)kb * kABox;  // one S tile (hi or lo)
  const uint32_t bop = (uint32_t)kb * kBBox;  // one y tile (hi or lo)
  uint8_t* A0 = base;                                 // S tile: hi at A0, lo after it
  uint8_t* B0 = A0 + (size_t)2 * aop;                 // stage s: hi at B0 + 2 s bop, lo after it
  float* stage = reinterpret_cast<float*>(B0 + (size_t)kBStages * 2 * bop);  // 4 warps x 2
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + 8 * kStageFloats);
  // bars: afull, aempty, bfull[kBStages], bempty[kBStages], tfull[kAcc], tempty[kAcc]
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t afull = smem_u32(&bars[0]), aempty = smem_u32(&bars[1]);
  const uint32_t bfull0 = smem_u32(&bars[2]), bempty0 = smem_u32(&bars[2 + kBStages]);
  const uint32_t tfull0 = smem_u32(&bars[2 + 2 * kBStages]);
  const uint32_t tempty0 = smem_u32(&bars[2 + 2 * kBStages + kAcc]);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(afull, 1);
    mbar_init(aempty, 1);
    for (int s = 0; s < kBStages; ++s) {
      mbar_init(bfull0 + 8 * s, 1);
      mbar_init(bempty0 + 8 * s, 1);
    }
    for (int a = 0; a < kAcc; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, EW);
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
      // ---------------- TMA producer: per unit, the S tile once, then its y tiles
      int bt = 0, at = 0;
      int b_issued[4] = {-1, -1, -1, -1}, a_issued = -1;
      bool stop = false;
      for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
        int mt, nt0, nt1;
        unit_range(p, u, mt, nt0, nt1);
        for (int k = 0; k < nt1 - nt0; ++k) {
          const int nt = unit_tile(p, u, nt0, nt1, k);
          const int s = bt & (kBStages - 1);
          if (!mbar_wait(bempty0 + 8 * s, ((uint32_t)(bt / kBStages) & 1u) ^ 1u, &abort_flag,
                         p.status)) {
            stop = true;
            break;
          }
          uint8_t* Bhi = B0 + (size_t)s * 2 * bop;
          mbar_expect_tx(bfull0 + 8 * s, 2 * bop);
          for (int kx = 0; kx < kb; ++kx) {
            tma_load_2d(smem_u32(Bhi + kx * kBBox), &tmBhi, kx * 32, nt * kBN, bfull0 + 8 * s);
            tma_load_2d(smem_u32(Bhi + bop + kx * kBBox), &tmBlo, kx * 32, nt * kBN,
                        bfull0 + 8 * s);
          }
          b_issued[s] = bt++;
          if (k == 0) {
            // the S tile frees when the last MMA of the previous unit completes; the
            // accumulators queued ahead of the epilogue cover the reload
            if (!mbar_wait(aempty, ((uint32_t)at & 1u) ^ 1u, &abort_flag, p.status)) {
              stop = true;
              break;
            }
            mbar_expect_tx(afull, 2 * aop);
            for (int kx = 0; kx < kb; ++kx) {
              tma_load_2d(smem_u32(A0 + kx * kABox), &tmAhi, kx * 32, mt * kBM, afull);
              tma_load_2d(smem_u32(A0 + aop + kx * kABox), &tmAlo, kx * 32, mt * kBM, afull);
            }
            a_issued = at++;
          }
        }
      }
      if (abort_flag) {
        // drain: wait for the copies in flight of every stage
        for (int s = 0; s < kBStages; ++s)
          if (b_issued[s] >= 0)
            mbar_drain(bfull0 + 8 * s, (uint32_t)(b_issued[s] / kBStages) & 1u);
        if (a_issued >= 0) mbar_drain(afull, (uint32_t)a_issued & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int t = 0, ua = 0, last = -1;
      bool stop = false;
      for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
        int mt, nt0, nt1;
        unit_range(p, u, mt, nt0, nt1);
        if (nt0 >= nt1) continue;
        if (!mbar_wait(afull, (uint32_t)ua & 1u, &abort_flag, p.status)) break;
        const uint8_t* Ahi = A0;
        for (int k = 0; k < nt1 - nt0; ++k) {
          const int s = t & (kBStages - 1), acc = t & (kAcc - 1);
          if (!mbar_wait(bfull0 + 8 * s, (uint32_t)(t / kBStages) & 1u, &abort_flag, p.status) ||
              !mbar_wait(tempty0 + 8 * acc, ((uint32_t)(t / kAcc) & 1u) ^ 1u, &abort_flag,
                         p.status)) {
            stop = true;
            break;
          }
          fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * kSlotCols);
          const uint8_t* Bhi = B0 + (size_t)s * 2 * bop;
          if constexpr (F16) {
            // D1 = S_hi y_hi; D2 = S_hi y_lo' + S_lo' y_hi (K = 64 f16 in 4 steps of 16)
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Ahi + aop);
            const uint32_t bh = smem_u32(Bhi), bl = smem_u32(Bhi + bop);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_f16(d, smem_desc(ah + ks * 32), smem_desc(bh + ks * 32), kIdesc, ks > 0 ? 1u : 0u);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_f16(d + kBN, smem_desc(ah + ks * 32), smem_desc(bl + ks * 32), kIdesc,
                      ks > 0 ? 1u : 0u);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_f16(d + kBN, smem_desc(al + ks * 32), smem_desc(bh + ks * 32), kIdesc, 1u);
          } else {
            const uint8_t* Aop[3] = {Ahi + aop, Ahi, Ahi};  // S_lo y_hi + S_hi y_lo + S_hi y_hi
            const uint8_t* Bop[3] = {Bhi, Bhi + bop, Bhi};
            uint32_t accum = 0;
            for (int prod = 0; prod < 3; ++prod) {
              for (int ks = 0; ks < kb * 4; ++ks) {
                const uint32_t ka = (uint32_t)(ks >> 2) * kABox + (uint32_t)(ks & 3) * 32u;
                const uint32_t kbo = (uint32_t)(ks >> 2) * kBBox + (uint32_t)(ks & 3) * 32u;
                mma_tf32(d, smem_desc(smem_u32(Aop[prod]) + ka),
                         smem_desc(smem_u32(Bop[prod]) + kbo), kIdesc, accum);
                accum = 1;
              }
            }
          }
          mma_commit(bempty0 + 8 * s);
          if (k == nt1 - nt0 - 1) mma_commit(aempty);
          mma_commit(tfull0 + 8 * acc);
          last = t++;
        }
        ++ua;
      }
      if (last >= 0) mbar_drain(tfull0 + 8 * (last & (kAcc - 1)), (uint32_t)(last / kAcc) & 1u);
    }
  } else {
    // ---------------- epilogue: warps 2 .. 2 + EW - 1, lane quarter q = warp % 4; with
    // EW = 8 the two warps of a quarter take alternate halves of each tile's columns
    const int q = warp & 3;
    constexpr int kBoxes = kBN / 32, kMine = EW == 8 ? kBoxes / 2 : kBoxes;
    const int cb0 = EW == 8 ? ((warp - 2) >> 2) * kMine : 0;
    int issued = 0;  // TMA stores issued by this warp: selects the staging buffer
    int t = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
      int mt, nt0, nt1;
      unit_range(p, u, mt, nt0, nt1);
      const int64_t xs = (int64_t)mt * kBM + q * 32;
      for (int k = 0; k < nt1 - nt0; ++k, ++t) {
        const int nt = unit_tile(p, u, nt0, nt1, k);
        const int acc = t & (kAcc - 1);
        const bool ok = __all_sync(
            0xffffffffu, mbar_wait(tfull0 + 8 * acc, (uint32_t)(t / kAcc) & 1u, &abort_flag, p.status));
        if (!ok) {
          stop = true;
          break;
        }
        fence_after();
        for (int cb = cb0; cb < cb0 + kMine; ++cb) {
          float v[32];
          const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kSlotCols + cb * 32);
          tmem_ld32(ta, v);
          const int64_t ys = (int64_t)nt * kBN + cb * 32;
          if constexpr (F16) {
            // x = scale_j (D1 + 2^-11 D2); lane c of the warp holds column c's scale
            float v2[32];
            tmem_ld32(ta + kBN, v2);
            const float sc = ys + lane < p.m ? p.yscale[ys + lane] : 0.f;
#pragma unroll
            for (int c = 0; c < 32; ++c)
              v[c] = fmaf(v2[c], 0x1p-11f, v[c]) * __shfl_sync(0xffffffffu, sc, c);
          }
          if (p.tma_store) {
            // stage [32 parameters][32 rows] and hand it to the TMA engine; a box
            // wholly past the end is skipped and touches no staging buffer, so
            // that "at most one store pending" always means the other buffer
            if (xs < p.n && ys < p.m) {
              float* sb = stage + (q * 2 + (issued & 1)) * kStageFloats;
              ++issued;
              if (lane == 0) bulk_wait_read1();
              __syncwarp();
#pragma unroll
              for (int c = 0; c < 32; ++c) sb[c * 32 + lane] = v[c];
              fence_async_smem();
              __syncwarp();
              if (lane == 0) {
                tma_store_2d(&tmOut, smem_u32(sb), (int)xs, (int)ys);
                bulk_commit();
              }
            }
          } else if (xs + lane < p.n && ys < p.m) {
            // coalesced streaming stores: lane = row, one 128-byte warp store per parameter
            float* o = p.out + ys * p.n + xs + lane;
            if (ys + 32 <= p.m) {
#pragma unroll
              for (int c = 0; c < 32; ++c) __stcs(o + (int64_t)c * p.n, v[c]);
            } else {
#pragma unroll
              for (int c = 0; c < 32; ++c)
                if (ys + c < p.m) __stcs(o + (int64_t)c * p.n, v[c]);
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
      }
    }
    if (p.tma_store && lane == 0) bulk_wait_all();
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

// Row-major rows x rpad float32 matrix, box box_rows x 32 floats, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const void* base, int64_t rows, int cols, int box_rows,
                     bool f16) {
  // rows x cols row-major, 128-byte rows (32 float32 or 64 f16 values per box row)
  auto fn = encode_fn();
  if (!fn) return false;
  const size_t es = f16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * es};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
static bool make_out_map(CUtensorMap* map, float* base, int64_t n, int64_t m) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float)};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing
// arrives on; the wait must give up after limit_ns, record SAS_ETIMEOUT in
// *status and return.
__global__ void wait_selftest_kernel(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, status, limit_ns);
  if (threadIdx.x == 0 && ok) atomicExch(status, -1);  // a phase completed that nothing drove
}

}  // namespace tc

cudaError_t launch_wait_selftest(int* status, double seconds, cudaStream_t st) {
  tc::wait_selftest_kernel<<<1, 32, 0, st>>>(status, (unsigned long long)(seconds * 1e9));
  return cudaGetLastError();
}

template <int BN, bool F16>
static size_t tc_smem_bytes(int rpad) {
  using Sh = tc::Shape<BN, F16>;
  const size_t kb = F16 ? 1 : (size_t)(rpad / 32);
  return 1024 + 2 * kb * tc::kABox + (size_t)Sh::kBStages * 2 * kb * Sh::kBBox +
         8 * tc::kStageFloats * sizeof(float) + (2 + 2 * Sh::kBStages + 2 * Sh::kAcc) * sizeof(uint64_t);
}

size_t reconstruct_tc_smem_bytes(int rpad) {
  const size_t a = tc_smem_bytes<64, false>(rpad), b = tc_smem_bytes<128, false>(rpad);
  const size_t c = tc_smem_bytes<128, true>(rpad);
  const size_t ab = a > b ? a : b;
  return ab > c ? ab : c;
}

bool reconstruct_tc_supported(const sas_ctx* c) {
  const int rpad = (c->r + 31) / 32 * 32;
  return c->dtype == SAS_REAL64 && rpad <= 64 && tc::encode_fn() != nullptr;
}

// Work split: one unit = one 128-row tile of S and a range of BN-parameter
// tiles.  When there are fewer row tiles than SMs, the parameter tiles of a
// row tile are split into ranges so that every SM has work; otherwise each
// unit covers all parameter tiles and S is read from HBM exactly once.
void reconstruct_tc_split(int64_t n, int64_t m, int num_sms, int bn, int* num_mtiles,
                          int* num_ntiles, int* ngroups, int* ntpg) {
  const int64_t mt = (n + tc::kBM - 1) / tc::kBM;
  const int64_t nt = (m + bn - 1) / bn;
  int64_t ng = 1;
  if (mt < num_sms) {
    ng = (num_sms + mt - 1) / mt;
    if (ng > nt) ng = nt;
  }
  const int64_t per = (nt + ng - 1) / ng;
  ng = (nt + per - 1) / per;  // no empty range
  *num_mtiles = (int)mt;
  *num_ntiles = (int)nt;
  *ngroups = (int)ng;
  *ntpg = (int)per;
}

namespace tc {

// f16 form: y (float32 = tf32 hi + lo of the split) -> per-parameter scale
// 2^e (|y| 2^-e < 1), f16 high part and 2^11-scaled f16 remainder, zero padded
// to 64; the product scale 2^(e - shift) goes to ysc.  One warp per parameter.
__global__ void split_y16_kernel(const float* ys, int64_t m, int rpad, int r, int shift,
                                 __half* y16, float* ysc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < m; q += warps) {
    float v[2];
    float amax = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      v[h] = k < r ? ys[q * rpad + k] + ys[m * rpad + q * rpad + k] : 0.f;
      amax = fmaxf(amax, fabsf(v[h]));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const int e = amax > 0.f ? ilogbf(amax) + 1 : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      const float yp = ldexpf(v[h], -e);
      const __half hi = __float2half_rn(yp);
      const __half lo = __float2half_rn((yp - __half2float(hi)) * 2048.f);
      y16[q * 64 + k] = hi;
      y16[m * 64 + q * 64 + k] = lo;
    }
    if (lane == 0) ysc[q] = ldexpf(1.f, e - shift);
  }
}

}  // namespace tc

template <int BN, bool F16, int EW>
static cudaError_t launch_tc(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                             bool rotate, cudaStream_t st) {
  if (m > 2147483647 - BN || c->n > 2147483647 - tc::kBM) return cudaErrorInvalidValue;
  const int rpad = (c->r + 31) / 32 * 32;
  const size_t smem = tc_smem_bytes<BN, F16>(rpad);
  cudaError_t e = cudaFuncSetAttribute(tc::reconstruct_tc_kernel<BN, F16, EW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  const float* ysc = nullptr;
  if constexpr (F16) {
    if (!c->S16hi || !c->ysplit16 || c->ysplit16_bytes < (size_t)m * (2 * 64 * 2 + 4))
      return cudaErrorInvalidValue;
    __half* y16 = reinterpret_cast<__half*>(c->ysplit16);
    float* sc = reinterpret_cast<float*>(y16 + (size_t)2 * m * 64);
    tc::split_y16_kernel<<<(unsigned)((m + 7) / 8 < 4096 ? (m + 7) / 8 : 4096), 256, 0, st>>>(
        ysplit, m, rpad, c->r, c->s16_shift, y16, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ysc = sc;
    if (!tc::make_map(&mAhi, c->S16hi, c->n, 64, tc::kBM, true) ||
        !tc::make_map(&mAlo, c->S16lo, c->n, 64, tc::kBM, true) ||
        !tc::make_map(&mBhi, y16, m, 64, BN, true) ||
        !tc::make_map(&mBlo, y16 + (size_t)m * 64, m, 64, BN, true))
      return cudaErrorInvalidValue;
  } else {
    if (!tc::make_map(&mAhi, c->Shi, c->n, rpad, tc::kBM, false) ||
        !tc::make_map(&mAlo, c->Slo, c->n, rpad, tc::kBM, false) ||
        !tc::make_map(&mBhi, ysplit, m, rpad, BN, false) ||
        !tc::make_map(&mBlo, ysplit + (size_t)m * rpad, m, rpad, BN, false))
      return cudaErrorInvalidValue;
  }
  // TMA stores need 16-byte aligned rows: n a multiple of 4 and an aligned base
  CUtensorMap mOut;
  // staging buffers exist for 4 epilogue warps: 8 warps store directly
  const bool tma_store = EW == 4 && c->recon_store == 0 && (c->n % 4 == 0) &&
                         ((reinterpret_cast<uintptr_t>(out) & 15) == 0) &&
                         tc::make_out_map(&mOut, out, c->n, m);
  if (!tma_store) std::memset(&mOut, 0, sizeof(mOut));
  tc::Params p;
  p.tma_store = tma_store ? 1 : 0;
  p.out = out;
  p.n = c->n;
  p.m = m;
  p.kboxes = F16 ? 1 : rpad / 32;
  reconstruct_tc_split(c->n, m, c->num_sms, BN, &p.num_mtiles, &p.num_ntiles, &p.ngroups, &p.ntpg);
  const int64_t units = (int64_t)p.num_mtiles * p.ngroups;
  if (units > 2147483647) return cudaErrorInvalidValue;
  p.num_units = (int)units;
  p.rotate = rotate ? 1 : 0;
  p.yscale = ysc;
  p.status = c->dev_status;
  const int grid = (int)(units < c->num_sms ? units : c->num_sms);
  tc::reconstruct_tc_kernel<BN, F16, EW><<<grid, tc::threads_for<EW>(), smem, st>>>(
      mAhi, mAlo, mBhi, mBlo, mOut, p);
  return cudaGetLastError();
}

namespace tc {

// f16 split of S: 2^shift S with max |2^shift S| in [1, 2), the f16 high part
// and the 2^11-scaled f16 remainder, rows of 64 (zero padded).
__global__ void maxabs_kernel(const double* S, int64_t ldS, int64_t n, int r, unsigned int* out) {
  float m = 0.f;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * r;
       idx += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, (float)fabs(S[(idx % n) + (idx / n) * ldS]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as ints
}

__global__ void split_basis16_kernel(const double* S, int64_t ldS, int64_t n, int r, int shift,
                                     __half* hi, __half* lo) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * 64;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / 64;
    const int k = (int)(idx % 64);
    __half h = __float2half_rn(0.f), l = __float2half_rn(0.f);
    if (k < r) {
      const double x = ldexp(S[i + (int64_t)k * ldS], shift);
      h = __double2half(x);
      l = __double2half((x - (double)__half2float(h)) * 2048.0);
    }
    hi[idx] = h;
    lo[idx] = l;
  }
}

}  // namespace tc

cudaError_t setup_f16_basis(sas_ctx* c, cudaStream_t st) {
  if (c->dtype != SAS_REAL64 || c->r > 64) return cudaSuccess;
  unsigned int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    tc::maxabs_kernel<<<c->num_sms * 4, 256, 0, st>>>((const double*)c->S, c->ldS, c->n, c->r, d);
    e = cudaGetLastError();
  }
  unsigned int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return e;
  float amax;
  std::memcpy(&amax, &bits, sizeof(amax));
  c->s16_shift = amax > 0.f ? -ilogbf(amax) : 0;
  e = cudaMalloc(&c->S16hi, (size_t)c->n * 64 * sizeof(__half));
  if (e == cudaSuccess) e = cudaMalloc(&c->S16lo, (size_t)c->n * 64 * sizeof(__half));
  if (e != cudaSuccess) return e;
  tc::split_basis16_kernel<<<c->num_sms * 8, 256, 0, st>>>((const double*)c->S, c->ldS, c->n, c->r,
                                                           c->s16_shift, (__half*)c->S16hi,
                                                           (__half*)c->S16lo);
  return cudaGetLastError();
}

// recon_kernel: 2 = tf32, 64-parameter tiles; 3 and 0 (automatic) = tf32,
// 128-parameter tiles; 4 = as 3 in a rotated tile order; 5 = f16 splits,
// 128-parameter tiles; 6 = as 3 with 8 epilogue warps (direct stores).
cudaError_t launch_reconstruct_tc(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                                  cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  switch (c->recon_kernel) {
    case 2: return launch_tc<64, false, 4>(c, ysplit, m, out, false, st);
    case 4: return launch_tc<128, false, 4>(c, ysplit, m, out, true, st);
    case 5: return launch_tc<128, true, 4>(c, ysplit, m, out, false, st);
    case 6: return launch_tc<128, false, 8>(c, ysplit, m, out, false, st);
    default: return launch_tc<128, false, 4>(c, ysplit, m, out, false, st);
  }
}

}  // namespace sas
