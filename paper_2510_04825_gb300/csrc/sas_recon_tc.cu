// Tensor-core reconstruction x_hat = S y for the mixed form (sm_103a, tcgen05).
//
// out[j*n + i] = sum_k S[i,k] y[j,k] in float32, computed as
//     S_hi y_hi + S_hi y_lo + S_lo y_hi
// where S = S_hi + S_lo and y = y_hi + y_lo are tf32 splits (S_hi, y_hi
// rounded to tf32; the low parts are the float32 remainders, truncated to
// tf32 by the tensor core).  The dropped S_lo y_lo term and the truncation of
// the low parts leave ~2^-21 relative error per product: float32-class
// accuracy at tf32 tensor-core rates.  The kernel is bound by HBM (it writes
// 4 n bytes per parameter and reads S once per 128-parameter tile pair).
//
// Structure (one persistent CTA per SM, 6 warps):
//   warp 0    TMA producer: B tiles (y_hi, y_lo of this CTA's 128 parameters)
//             once, then A tiles (S_hi, S_lo rows) into a 2-stage ring;
//   warp 1    one thread issues tcgen05.mma (kind::tf32, M=128, N=128, K=8)
//             into a double-buffered TMEM accumulator (2 x 128 columns);
//   warps 2-5 epilogue: tcgen05.ld 32 lanes x 32 columns at a time and
//             streaming stores; each warp owns its TMEM lane quarter.
// Tiles: M = 128 rows of S, N = 128 parameters, K = rpad (32 or 64) in boxes
// of 32 floats (128 B rows, 128-byte swizzle).  CTA c handles parameter tile
// c % ntiles and row tiles c / ntiles, c / ntiles + G / ntiles, ... so that
// the CTAs sharing a row tile run at the same time and the second read of it
// comes from L2.
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
constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kBoxBytes = 128 * 128;  // 128 rows x 32 floats
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 256;
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
  int num_mtiles;
  int num_ntiles;
  int tma_store;   // 1: epilogue through shared memory and TMA stores
  int* status;
};

constexpr int kStageFloats = 32 * 32;  // one epilogue staging tile: 32 parameters x 32 rows

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
  const uint32_t opbytes = (uint32_t)kb * kBoxBytes;  // one operand tile (hi or lo)
  uint8_t* Bhi = base;
  uint8_t* Blo = Bhi + opbytes;
  uint8_t* Abase = Blo + opbytes;  // stage s: hi at Abase + s*2*opbytes, lo right after
  float* stage = reinterpret_cast<float*>(Abase + (size_t)kStages * 2 * opbytes);  // 4 warps x 2
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + 8 * kStageFloats);
  // bars: full[2], empty[2], tfull[2], tempty[2], bbar
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[2]);
  const uint32_t tfull0 = smem_u32(&bars[4]), tempty0 = smem_u32(&bars[6]);
  const uint32_t bbar = smem_u32(&bars[8]);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
      mbar_init(tfull0 + 8 * s, 1);
      mbar_init(tempty0 + 8 * s, 4);
    }
    mbar_init(bbar, 1);
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

  const int ntile = blockIdx.x % p.num_ntiles;
  const int first = blockIdx.x / p.num_ntiles;
  const int step = gridDim.x / p.num_ntiles;
  const int iters = first < p.num_mtiles ? (p.num_mtiles - first + step - 1) / step : 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      mbar_expect_tx(bbar, 2 * opbytes);
      for (int k = 0; k < kb; ++k) {
        tma_load_2d(smem_u32(Bhi + k * kBoxBytes), &tmBhi, k * 32, ntile * kBN, bbar);
        tma_load_2d(smem_u32(Blo + k * kBoxBytes), &tmBlo, k * 32, ntile * kBN, bbar);
      }
      int issued[kStages] = {-1, -1};
      for (int it = 0; it < iters; ++it) {
        const int s = it & 1;
        const uint32_t ph = (uint32_t)(it >> 1) & 1u;
        if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, &abort_flag, p.status)) break;
        const int mt = first + it * step;
        uint8_t* Ahi = Abase + (size_t)s * 2 * opbytes;
        uint8_t* Alo = Ahi + opbytes;
        mbar_expect_tx(full0 + 8 * s, 2 * opbytes);
        for (int k = 0; k < kb; ++k) {
          tma_load_2d(smem_u32(Ahi + k * kBoxBytes), &tmAhi, k * 32, mt * kBM, full0 + 8 * s);
          tma_load_2d(smem_u32(Alo + k * kBoxBytes), &tmAlo, k * 32, mt * kBM, full0 + 8 * s);
        }
        issued[s] = it;
      }
      if (abort_flag) {
        // drain: wait for the copies in flight of every stage and for B
        for (int s = 0; s < kStages; ++s)
          if (issued[s] >= 0) mbar_drain(full0 + 8 * s, (uint32_t)(issued[s] >> 1) & 1u);
        mbar_drain(bbar, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int last = -1;
      if (mbar_wait(bbar, 0, &abort_flag, p.status)) {
        for (int it = 0; it < iters; ++it) {
          const int s = it & 1, acc = it & 1;
          const uint32_t ph = (uint32_t)(it >> 1) & 1u;
          if (!mbar_wait(full0 + 8 * s, ph, &abort_flag, p.status)) break;
          if (!mbar_wait(tempty0 + 8 * acc, ph ^ 1u, &abort_flag, p.status)) break;
          fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * kBN);
          const uint8_t* Ahi = Abase + (size_t)s * 2 * opbytes;
          const uint8_t* Alo = Ahi + opbytes;
          const uint8_t* Aop[3] = {Alo, Ahi, Ahi};
          const uint8_t* Bop[3] = {Bhi, Blo, Bhi};
          uint32_t accum = 0;
          for (int prod = 0; prod < 3; ++prod) {
            for (int ks = 0; ks < kb * 4; ++ks) {
              const uint32_t off = (uint32_t)(ks >> 2) * kBoxBytes + (uint32_t)(ks & 3) * 32u;
              mma_tf32(d, smem_desc(smem_u32(Aop[prod]) + off), smem_desc(smem_u32(Bop[prod]) + off),
                       accum);
              accum = 1;
            }
          }
          mma_commit(empty0 + 8 * s);
          mma_commit(tfull0 + 8 * acc);
          last = it;
        }
      }
      if (last >= 0) mbar_drain(tfull0 + 8 * (last & 1), (uint32_t)(last >> 1) & 1u);
    }
  } else {
    // ---------------- epilogue: warps 2..5, lane quarter q = warp % 4
    const int q = warp & 3;
    int issued = 0;  // TMA stores issued by this warp: selects the staging buffer
    for (int it = 0; it < iters; ++it) {
      const int acc = it & 1;
      const uint32_t ph = (uint32_t)(it >> 1) & 1u;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * acc, ph, &abort_flag, p.status));
      if (!ok) break;
      fence_after();
      const int mt = first + it * step;
      const int64_t i = (int64_t)mt * kBM + q * 32 + lane;
      const int64_t j0 = (int64_t)ntile * kBN;
      for (int cb = 0; cb < kBN / 32; ++cb) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + cb * 32), v);
        if (p.tma_store) {
          // stage [32 parameters][32 rows] and hand it to the TMA engine; a box
          // wholly past the end is skipped and touches no staging buffer, so
          // that "at most one store pending" always means the other buffer
          const int64_t xs = (int64_t)mt * kBM + q * 32, ys = j0 + cb * 32;
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
        } else if (i < p.n) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int64_t j = j0 + cb * 32 + c;
            if (j < p.m) __stcs(p.out + j * p.n + i, v[c]);
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
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

// Row-major rows x rpad float32 matrix, box 128 rows x 32 floats, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const float* base, int64_t rows, int rpad) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)rpad * sizeof(float)};
  cuuint32_t box[2] = {32, 128};
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
  const size_t op = (size_t)(rpad / 32) * tc::kBoxBytes;
  return 1024 + 2 * op + (size_t)tc::kStages * 2 * op + 8 * tc::kStageFloats * sizeof(float) +
         9 * sizeof(uint64_t);
}

bool reconstruct_tc_supported(const sas_ctx* c) {
  const int rpad = (c->r + 31) / 32 * 32;
  return c->dtype == SAS_REAL64 && rpad <= 64 && tc::encode_fn() != nullptr;
}

cudaError_t launch_reconstruct_tc(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                                  cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  const int rpad = (c->r + 31) / 32 * 32;
  const int num_ntiles_all = (int)((m + tc::kBN - 1) / tc::kBN);
  const size_t smem = reconstruct_tc_smem_bytes(rpad);
  cudaError_t e = cudaFuncSetAttribute(tc::reconstruct_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // parameter tiles are processed in groups of at most num_sms tiles per launch
  const int group = c->num_sms;
  for (int nt0 = 0; nt0 < num_ntiles_all; nt0 += group) {
    const int nts = num_ntiles_all - nt0 < group ? num_ntiles_all - nt0 : group;
    const int64_t j0 = (int64_t)nt0 * tc::kBN;
    const int64_t mm = m - j0 < (int64_t)nts * tc::kBN ? m - j0 : (int64_t)nts * tc::kBN;
    CUtensorMap mAhi, mAlo, mBhi, mBlo;
    if (!tc::make_map(&mAhi, c->Shi, c->n, rpad) || !tc::make_map(&mAlo, c->Slo, c->n, rpad) ||
        !tc::make_map(&mBhi, ysplit + j0 * rpad, mm, rpad) ||
        !tc::make_map(&mBlo, ysplit + (size_t)m * rpad + j0 * rpad, mm, rpad))
      return cudaErrorInvalidValue;
    // TMA stores need 16-byte aligned rows: n a multiple of 4 and an aligned base
    CUtensorMap mOut;
    const bool tma_store = (c->n % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0) &&
                           tc::make_out_map(&mOut, out + j0 * c->n, c->n, mm);
    if (!tma_store) std::memset(&mOut, 0, sizeof(mOut));
    tc::Params p;
    p.tma_store = tma_store ? 1 : 0;
    p.out = out + j0 * c->n;
    p.n = c->n;
    p.m = mm;
    p.kboxes = rpad / 32;
    p.num_mtiles = (int)((c->n + tc::kBM - 1) / tc::kBM);
    p.num_ntiles = nts;
    p.status = c->dev_status;
    int grid = (c->num_sms / nts) * nts;
    if (grid < nts) grid = nts;
    const int max_grid = p.num_mtiles * nts;
    if (grid > max_grid) grid = max_grid;
    tc::reconstruct_tc_kernel<<<grid, tc::kThreads, smem, st>>>(mAhi, mAlo, mBhi, mBlo, mOut, p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sas
