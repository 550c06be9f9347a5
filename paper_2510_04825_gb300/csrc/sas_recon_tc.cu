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
// Structure (one persistent CTA per SM, 6 warps):
//   warp 0    TMA producer: for each work unit the S tile (S_hi, S_lo of 128
//             rows) into a 2-stage buffer, then the unit's y tiles (y_hi, y_lo
//             of 64 parameters, L2-resident) into a 2-stage ring;
//   warp 1    one thread issues tcgen05.mma (kind::tf32, M=128, N=64, K=8)
//             into 4 TMEM accumulators of 64 columns;
//   warps 2-5 epilogue: tcgen05.ld 32 lanes x 32 columns at a time, staged in
//             shared memory and written by TMA bulk-tensor stores; each warp
//             owns its TMEM lane quarter.
// A work unit is one 128-row tile of S and a range of 64-parameter tiles; the
// S tile stays resident while the unit's y tiles stream past it.  With at
// least as many row tiles as SMs a unit covers every parameter tile, so S is
// read from HBM once; with fewer (small n) the parameter tiles are split into
// ranges so that every SM has work.  K = rpad (32 or 64) in boxes of 32 floats
// (128 B rows, 128-byte swizzle).
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the kernel
// records SAS_ETIMEOUT in the status word, stops issuing work, waits (bounded)
// for its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "sas_internal.cuh"

namespace sas {

namespace tc {

constexpr int kThreads = 192;
constexpr int kBM = 128;              // rows of S per tile (MMA M)
constexpr int kBN = 64;               // parameters per tile (MMA N)
constexpr int kABox = 128 * 128;      // A box: 128 rows x 32 floats (128-byte rows)
constexpr int kBBox = kBN * 128;      // B box: 64 rows x 32 floats
constexpr int kAStages = 2;
constexpr int kBStages = 2;
constexpr int kAcc = 4;               // TMEM accumulators of kBN columns
constexpr uint32_t kTmemCols = kAcc * kBN;
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ inline uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ inline bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false on timeout or abort.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                 int* status, unsigned long long limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status, (int)SAS_ETIMEOUT);
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag (used to drain work in flight).
__device__ inline void mbar_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(bar, parity)) {
    if (globaltimer() - t0 > kWaitNs) return;
  }
}

__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ inline void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                   uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ inline void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(src)
      : "memory");
}
__device__ inline void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ inline void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ inline void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ inline void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 B, 8-row groups 1024 B apart.
__device__ inline uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ inline void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ inline void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ inline void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ inline void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct Params {
  float* out;
  int64_t n;
  int64_t m;
  int kboxes;      // rpad / 32 (1 or 2)
  int num_mtiles;  // ceil(n / kBM)
  int num_ntiles;  // ceil(m / kBN)
  int ngroups;     // parameter tiles of one row tile are split into ngroups ranges
  int ntpg;        // parameter tiles per range
  int num_units;   // num_mtiles * ngroups
  int tma_store;   // 1: epilogue through shared memory and TMA stores
  int* status;
};

constexpr int kStageFloats = 32 * 32;  // one epilogue staging tile: 32 parameters x 32 rows

// Work unit u: row tile u / ngroups, parameter tiles [g ntpg, min((g+1) ntpg, num_ntiles))
// with g = u % ngroups.  All three roles walk the same units in the same order.
__device__ inline void unit_range(const Params& p, int u, int& mt, int& nt0, int& nt1) {
  mt = u / p.ngroups;
  const int g = u % p.ngroups;
  nt0 = g * p.ntpg;
  nt1 = nt0 + p.ntpg < p.num_ntiles ? nt0 + p.ntpg : p.num_ntiles;
}

__global__ void __launch_bounds__(kThreads, 1)
    reconstruct_tc_kernel(const __grid_constant__ CUtensorMap tmAhi,
                          const __grid_constant__ CUtensorMap tmAlo,
                          const __grid_constant__ CUtensorMap tmBhi,
                          const __grid_constant__ CUtensorMap tmBlo,
                          const __grid_constant__ CUtensorMap tmOut, Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const int kb = p.kboxes;
  const uint32_t aop = (uint32_t)kb * kABox;  // one S tile (hi or lo)
  const uint32_t bop = (uint32_t)kb * kBBox;  // one y tile (hi or lo)
  uint8_t* A0 = base;                                 // stage s: hi at A0 + 2 s aop, lo after it
  uint8_t* B0 = A0 + (size_t)kAStages * 2 * aop;      // stage s: hi at B0 + 2 s bop, lo after it
  float* stage = reinterpret_cast<float*>(B0 + (size_t)kBStages * 2 * bop);  // 4 warps x 2
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + 8 * kStageFloats);
  // bars: afull[2], aempty[2], bfull[2], bempty[2], tfull[4], tempty[4]
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t afull0 = smem_u32(&bars[0]), aempty0 = smem_u32(&bars[2]);
  const uint32_t bfull0 = smem_u32(&bars[4]), bempty0 = smem_u32(&bars[6]);
  const uint32_t tfull0 = smem_u32(&bars[8]), tempty0 = smem_u32(&bars[12]);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < 2; ++s) {
      mbar_init(afull0 + 8 * s, 1);
      mbar_init(aempty0 + 8 * s, 1);
      mbar_init(bfull0 + 8 * s, 1);
      mbar_init(bempty0 + 8 * s, 1);
    }
    for (int a = 0; a < kAcc; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 4);
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
      int b_issued[kBStages] = {-1, -1}, a_issued[kAStages] = {-1, -1};
      bool stop = false;
      for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
        int mt, nt0, nt1;
        unit_range(p, u, mt, nt0, nt1);
        for (int nt = nt0; nt < nt1; ++nt) {
          const int s = bt & 1;
          if (!mbar_wait(bempty0 + 8 * s, ((uint32_t)(bt >> 1) & 1u) ^ 1u, &abort_flag, p.status)) {
            stop = true;
            break;
          }
          uint8_t* Bhi = B0 + (size_t)s * 2 * bop;
          mbar_expect_tx(bfull0 + 8 * s, 2 * bop);
          for (int k = 0; k < kb; ++k) {
            tma_load_2d(smem_u32(Bhi + k * kBBox), &tmBhi, k * 32, nt * kBN, bfull0 + 8 * s);
            tma_load_2d(smem_u32(Bhi + bop + k * kBBox), &tmBlo, k * 32, nt * kBN, bfull0 + 8 * s);
          }
          b_issued[s] = bt++;
          if (nt == nt0) {
            // the S tile: its stage frees when the last MMA of the unit two back completes
            const int sa = at & 1;
            if (!mbar_wait(aempty0 + 8 * sa, ((uint32_t)(at >> 1) & 1u) ^ 1u, &abort_flag,
                           p.status)) {
              stop = true;
              break;
            }
            uint8_t* Ahi = A0 + (size_t)sa * 2 * aop;
            mbar_expect_tx(afull0 + 8 * sa, 2 * aop);
            for (int k = 0; k < kb; ++k) {
              tma_load_2d(smem_u32(Ahi + k * kABox), &tmAhi, k * 32, mt * kBM, afull0 + 8 * sa);
              tma_load_2d(smem_u32(Ahi + aop + k * kABox), &tmAlo, k * 32, mt * kBM,
                          afull0 + 8 * sa);
            }
            a_issued[sa] = at++;
          }
        }
      }
      if (abort_flag) {
        // drain: wait for the copies in flight of every stage
        for (int s = 0; s < kBStages; ++s)
          if (b_issued[s] >= 0) mbar_drain(bfull0 + 8 * s, (uint32_t)(b_issued[s] >> 1) & 1u);
        for (int s = 0; s < kAStages; ++s)
          if (a_issued[s] >= 0) mbar_drain(afull0 + 8 * s, (uint32_t)(a_issued[s] >> 1) & 1u);
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
        const int sa = ua & 1;
        if (!mbar_wait(afull0 + 8 * sa, (uint32_t)(ua >> 1) & 1u, &abort_flag, p.status)) break;
        const uint8_t* Ahi = A0 + (size_t)sa * 2 * aop;
        for (int nt = nt0; nt < nt1; ++nt) {
          const int s = t & 1, acc = t & (kAcc - 1);
          if (!mbar_wait(bfull0 + 8 * s, (uint32_t)(t >> 1) & 1u, &abort_flag, p.status) ||
              !mbar_wait(tempty0 + 8 * acc, ((uint32_t)(t >> 2) & 1u) ^ 1u, &abort_flag,
                         p.status)) {
            stop = true;
            break;
          }
          fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * kBN);
          const uint8_t* Bhi = B0 + (size_t)s * 2 * bop;
          const uint8_t* Aop[3] = {Ahi + aop, Ahi, Ahi};  // S_lo y_hi + S_hi y_lo + S_hi y_hi
          const uint8_t* Bop[3] = {Bhi, Bhi + bop, Bhi};
          uint32_t accum = 0;
          for (int prod = 0; prod < 3; ++prod) {
            for (int ks = 0; ks < kb * 4; ++ks) {
              const uint32_t ka = (uint32_t)(ks >> 2) * kABox + (uint32_t)(ks & 3) * 32u;
              const uint32_t kbo = (uint32_t)(ks >> 2) * kBBox + (uint32_t)(ks & 3) * 32u;
              mma_tf32(d, smem_desc(smem_u32(Aop[prod]) + ka), smem_desc(smem_u32(Bop[prod]) + kbo),
                       accum);
              accum = 1;
            }
          }
          mma_commit(bempty0 + 8 * s);
          if (nt == nt1 - 1) mma_commit(aempty0 + 8 * sa);
          mma_commit(tfull0 + 8 * acc);
          last = t++;
        }
        ++ua;
      }
      if (last >= 0) mbar_drain(tfull0 + 8 * (last & (kAcc - 1)), (uint32_t)(last >> 2) & 1u);
    }
  } else {
    // ---------------- epilogue: warps 2..5, lane quarter q = warp % 4
    const int q = warp & 3;
    int issued = 0;  // TMA stores issued by this warp: selects the staging buffer
    int t = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < p.num_units && !stop; u += gridDim.x) {
      int mt, nt0, nt1;
      unit_range(p, u, mt, nt0, nt1);
      const int64_t xs = (int64_t)mt * kBM + q * 32;
      for (int nt = nt0; nt < nt1; ++nt, ++t) {
        const int acc = t & (kAcc - 1);
        const bool ok = __all_sync(
            0xffffffffu, mbar_wait(tfull0 + 8 * acc, (uint32_t)(t >> 2) & 1u, &abort_flag, p.status));
        if (!ok) {
          stop = true;
          break;
        }
        fence_after();
        for (int cb = 0; cb < kBN / 32; ++cb) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + cb * 32), v);
          const int64_t ys = (int64_t)nt * kBN + cb * 32;
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
          } else if (xs + lane < p.n) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int64_t j = ys + c;
              if (j < p.m) __stcs(p.out + j * p.n + xs + lane, v[c]);
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

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// Row-major rows x rpad float32 matrix, box box_rows x 32 floats, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const float* base, int64_t rows, int rpad, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)rpad * sizeof(float)};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Output m x n float32 (row j = x_hat_j), box 32 rows (i) x 32 parameters (j), no swizzle.
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

size_t reconstruct_tc_smem_bytes(int rpad) {
  const size_t kb = (size_t)(rpad / 32);
  return 1024 + (size_t)tc::kAStages * 2 * kb * tc::kABox + (size_t)tc::kBStages * 2 * kb * tc::kBBox +
         8 * tc::kStageFloats * sizeof(float) + (4 * 2 + 2 * tc::kAcc) * sizeof(uint64_t);
}

bool reconstruct_tc_supported(const sas_ctx* c) {
  const int rpad = (c->r + 31) / 32 * 32;
  return c->dtype == SAS_REAL64 && rpad <= 64 && tc::encode_fn() != nullptr;
}

// Work split: one unit = one 128-row tile of S and a range of 64-parameter
// tiles.  When there are fewer row tiles than SMs, the parameter tiles of a
// row tile are split into ranges so that every SM has work; otherwise each
// unit covers all parameter tiles and S is read from HBM exactly once.
void reconstruct_tc_split(int64_t n, int64_t m, int num_sms, int* num_mtiles, int* num_ntiles,
                          int* ngroups, int* ntpg) {
  const int64_t mt = (n + tc::kBM - 1) / tc::kBM;
  const int64_t nt = (m + tc::kBN - 1) / tc::kBN;
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

cudaError_t launch_reconstruct_tc(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                                  cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  if (m > 2147483647 - tc::kBN || c->n > 2147483647 - tc::kBM) return cudaErrorInvalidValue;
  const int rpad = (c->r + 31) / 32 * 32;
  const size_t smem = reconstruct_tc_smem_bytes(rpad);
  cudaError_t e = cudaFuncSetAttribute(tc::reconstruct_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  if (!tc::make_map(&mAhi, c->Shi, c->n, rpad, tc::kBM) ||
      !tc::make_map(&mAlo, c->Slo, c->n, rpad, tc::kBM) ||
      !tc::make_map(&mBhi, ysplit, m, rpad, tc::kBN) ||
      !tc::make_map(&mBlo, ysplit + (size_t)m * rpad, m, rpad, tc::kBN))
    return cudaErrorInvalidValue;
  // TMA stores need 16-byte aligned rows: n a multiple of 4 and an aligned base
  CUtensorMap mOut;
  const bool tma_store = (c->n % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0) &&
                         tc::make_out_map(&mOut, out, c->n, m);
  if (!tma_store) std::memset(&mOut, 0, sizeof(mOut));
  tc::Params p;
  p.tma_store = tma_store ? 1 : 0;
  p.out = out;
  p.n = c->n;
  p.m = m;
  p.kboxes = rpad / 32;
  reconstruct_tc_split(c->n, m, c->num_sms, &p.num_mtiles, &p.num_ntiles, &p.ngroups, &p.ntpg);
  const int64_t units = (int64_t)p.num_mtiles * p.ngroups;
  if (units > 2147483647) return cudaErrorInvalidValue;
  p.num_units = (int)units;
  p.status = c->dev_status;
  const int grid = (int)(units < c->num_sms ? units : c->num_sms);
  tc::reconstruct_tc_kernel<<<grid, tc::kThreads, smem, st>>>(mAhi, mAlo, mBhi, mBlo, mOut, p);
  return cudaGetLastError();
}

}  // namespace sas
