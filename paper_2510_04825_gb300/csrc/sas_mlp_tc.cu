// Tensor-core GEMM with bfloat16-split operands (sm_103a, tcgen05): the learned surrogate's
// products and the fast Poisson preconditioner's sine transforms.
//
// C[i, j] = sum_k A(i, k) B(k, j), with A(i, k) = A[i lai + k lak] and B(k, j) = B[k lbk +
// j lbj] (any strides, so transposed operands need no copies), optionally over a batch
// (A, B, C advanced by bsa, bsb, bsc per batch entry).  Operands are bfloat16 or float32; the
// MMA is tcgen05 kind::f16 with bfloat16 A and B and float32 accumulation in TMEM:
//   * a bfloat16 operand enters as it is;
//   * a float32 operand v is split into NS bfloat16 terms t_0 = bf16(v), t_1 = bf16(v - t_0),
//     ... (each remainder is exact in float32), and the product takes every pair of terms
//     (t_a, u_b) with a + b < max(terms of A, terms of B).  NS = 2 (the surrogate) leaves
//     ~2^-17 relative error per product; NS = 3 represents a float32 value exactly (3 x 8
//     significant bits) and drops only pairs of order 2^-24: float32-accurate products (the
//     preconditioner).
// Epilogues: 0 = store C; 1 = Z = C + bias and H = gelu(Z) (exact erf form); 2 = C + bias;
// 3 = gelu(C + bias) only (inference, where Z is not needed).
//
// Structure: one CTA (256 threads for two-term splits, 512 for three-term ones) per 128 x BN
// tile of C (BN = 16 .. 256) and K range (split-K for the surrogate's weight gradients, whose K
// is the batch) or batch entry: K in blocks of 64 (128-byte K-major rows, 128-byte swizzle),
// two shared-memory stages.  All threads load, split and store a K block; one elected thread
// issues its MMAs (K = 16 each) and commits them to the stage's mbarrier, which the threads
// wait on before they overwrite that stage.  The warps drain TMEM: warp w reads lane quarter
// w % 4 and every (threads / 128)-th 16-column chunk from chunk w / 4.  A split-K launch writes
// float32 partial tiles that a second kernel sums in a fixed order.  Every wait is bounded (2 s
// of %globaltimer); on expiry the kernel records SAS_ETIMEOUT, stops, waits (bounded) for its
// MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "sas_internal.cuh"
#include "sas_tc_common.cuh"

namespace sas {
namespace mlptc {

using namespace tc;

// threads per CTA: 256 for two-term kernels (two CTAs per SM), 512 for three-term ones (one CTA
// per SM by shared memory: twice the warps to hide the staging latency)
__host__ __device__ constexpr int threads_for(int ns) { return ns == 3 ? 512 : 256; }
constexpr int kBM = 128;
constexpr int kKB = 64;  // K per block: 64 bfloat16 = one 128-byte swizzled row

// kind::f16 instruction descriptor with bfloat16 A and B (K-major), float32 D.
__host__ __device__ constexpr uint32_t bf16_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <typename T> __device__ inline float ldv(const T* p, int64_t i);
template <> __device__ inline float ldv<float>(const float* p, int64_t i) { return p[i]; }
template <> __device__ inline float ldv<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

__device__ inline float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

struct GemmArgs {
  int M, N, K;
  int kb_per;  // K blocks per split (blockIdx.z when nbatch == 1)
  int nbatch;  // > 1: blockIdx.z is the batch entry
  const void* A;
  int64_t lai, lak, bsa;
  const void* B;
  int64_t lbk, lbj, bsb;
  float* C;  // output, or the partial tiles [split][M][N] of a split-K launch
  int64_t ldc, bsc;
  int epi;
  const float* bias;
  float* H;
  int* status;
  int a_vec, b_vec;  // 1: rows K-contiguous, 2: K-strided with rows contiguous (float32 only)
};

// Byte offset of element (row, k) of a K-major bfloat16 tile with 128-byte rows and the
// 128-byte swizzle (16-byte units XOR-ed with row % 8).
__device__ inline uint32_t swz(int row, int k) {
  return (uint32_t)row * 128u + ((((uint32_t)k >> 3) ^ (uint32_t)(row & 7)) << 4) + (((uint32_t)k & 7u) << 1);
}

// The NT bfloat16 terms of a pair of values (t_0 = bf16(v), t_1 = bf16(v - t_0), ...).
template <int NT>
__device__ inline void split_pair(float v0, float v1, __nv_bfloat162* t) {
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    t[i] = __floats2bfloat162_rn(v0, v1);
    if (i + 1 < NT) {
      const float2 f = __bfloat1622float2(t[i]);
      v0 -= f.x;
      v1 -= f.y;
    }
  }
}

__device__ inline uint32_t bits(__nv_bfloat162 h) { return *reinterpret_cast<const uint32_t*>(&h); }

// Operand tile: rows x 64 (K block at k0) as NT bfloat16 term tiles (term i at tile + i *
// tstride) in the swizzled K-major layout.  Each thread takes a (row, k, k + 1) pair; the
// pair index runs along the operand's unit-stride direction so that loads coalesce.
template <typename T, int NT, int ROWS, int NTH>
__device__ inline void stage_tile(const T* src, int64_t lrow, int64_t lk, int row0, int nrows,
                                  int k0, int K, uint8_t* tile, uint32_t tstride) {
  const bool k_fast = lk == 1;
  for (int idx = threadIdx.x; idx < ROWS * 32; idx += NTH) {
    const int r = k_fast ? idx >> 5 : idx % ROWS;
    const int kp = k_fast ? idx & 31 : idx / ROWS;
    const int k = k0 + 2 * kp;
    float v0 = 0.f, v1 = 0.f;
    if (r < nrows) {
      const T* p = src + (int64_t)(row0 + r) * lrow;
      if (k < K) v0 = ldv<T>(p, (int64_t)k * lk);
      if (k + 1 < K) v1 = ldv<T>(p, (int64_t)(k + 1) * lk);
    }
    const uint32_t o = swz(r, 2 * kp);
    __nv_bfloat162 t[NT];
    split_pair<NT>(v0, v1, t);
#pragma unroll
    for (int i = 0; i < NT; ++i) *reinterpret_cast<__nv_bfloat162*>(tile + i * tstride + o) = t[i];
  }
}

// As stage_tile for operands whose rows are K-contiguous with 16-byte aligned starts: each
// thread takes 16-byte chunks (4 float32 or 8 bfloat16 of one row), issues all of its loads
// before it converts and stores any of them, and writes whole swizzle units (bfloat16) or
// 8-byte halves of them (float32 terms).  Chunks past K or past the valid rows are filled
// element by element (zeros outside).
template <typename T, int NT, int ROWS, int NTH>
__device__ inline void stage_tile_vec(const T* src, int64_t lrow, int row0, int nrows, int k0, int K,
                                      uint8_t* tile, uint32_t tstride) {
  constexpr int kPer = 16 / sizeof(T);          // elements per 16-byte chunk
  constexpr int kChunks = kKB / kPer;           // chunks per row
  constexpr int kIters = ROWS * kChunks / NTH;
  static_assert(ROWS * kChunks % NTH == 0 || ROWS * kChunks < NTH, "tile and block");
  constexpr int kBatch = kIters < 8 ? (kIters < 1 ? 1 : kIters) : 8;
#pragma unroll 1
  for (int it0 = 0; it0 < (kIters < 1 ? 1 : kIters); it0 += kBatch) {
    uint4 v[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int idx = threadIdx.x + (it0 + b) * NTH;
      const int r = idx / kChunks, c = idx % kChunks;
      const int k = k0 + c * kPer;
      v[b] = make_uint4(0u, 0u, 0u, 0u);
      if (idx >= ROWS * kChunks || r >= nrows) continue;
      const T* p = src + (int64_t)(row0 + r) * lrow + k;
      if (k + kPer <= K) {
        v[b] = __ldg(reinterpret_cast<const uint4*>(p));
      } else {
        T tmp[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) tmp[e] = k + e < K ? p[e] : T(0.f);
        v[b] = *reinterpret_cast<const uint4*>(tmp);
      }
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int idx = threadIdx.x + (it0 + b) * NTH;
      if (idx >= ROWS * kChunks) continue;
      const int r = idx / kChunks, c = idx % kChunks;
      if (sizeof(T) == 2) {  // 8 bfloat16: one swizzle unit
        *reinterpret_cast<uint4*>(tile + swz(r, 8 * c)) = v[b];
      } else {  // 4 float32 -> NT terms of 4 bfloat16 (8 bytes each)
        __nv_bfloat162 t01[NT], t23[NT];
        split_pair<NT>(__uint_as_float(v[b].x), __uint_as_float(v[b].y), t01);
        split_pair<NT>(__uint_as_float(v[b].z), __uint_as_float(v[b].w), t23);
        const uint32_t o = swz(r, 4 * c);
#pragma unroll
        for (int i = 0; i < NT; ++i)
          *reinterpret_cast<uint2*>(tile + i * tstride + o) = make_uint2(bits(t01[i]), bits(t23[i]));
      }
    }
  }
}

// Float32 operand tile whose rows are contiguous and whose K index is strided (lk a multiple
// of 4, 16-byte aligned rows of the tile): each unit of work is a 4 x 4 block (four rows, four
// consecutive k) read as four 16-byte loads (one per k), transposed in registers and written
// as 8-byte row pieces of every term.  Lanes of a warp cover 8 K-quads x 4 row-quads, so that
// each load instruction reads 64 contiguous bytes at each of 8 k and the 8-byte stores spread
// over the banks.  Blocks that cross the valid rows or K are filled element by element.
template <int NT, int ROWS, int NTH>
__device__ inline void stage_tile_vec_t(const float* src, int64_t lk, int row0, int nrows, int k0,
                                        int K, uint8_t* tile, uint32_t tstride) {
  constexpr int kRQ = ROWS / 4;                 // row-quads
  constexpr int kRQhi = kRQ >= 4 ? kRQ / 4 : 1;  // row-quad groups of 4 per warp
  constexpr int kUnits = 16 * kRQ;              // 16 K-quads per K block
  constexpr int kIters = (kUnits + NTH - 1) / NTH;
#pragma unroll 1
  for (int it = 0; it < kIters; ++it) {
    const int idx = threadIdx.x + it * NTH;
    if (idx >= kUnits) break;
    const int kq_lo = idx & 7, rq_lo = kRQ >= 4 ? (idx >> 3) & 3 : (idx >> 3) % kRQ;
    const int rest = kRQ >= 4 ? idx >> 5 : (idx >> 3) / kRQ;
    const int rq = (rest % kRQhi) * 4 + rq_lo, kq = (rest / kRQhi) * 8 + kq_lo;
    const int r = 4 * rq, kl = 4 * kq, k = k0 + kl;
    float x[4][4];  // x[kk][e]: element (row r + e, k + kk)
    if (r + 4 <= nrows && k + 4 <= K) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(src + (int64_t)(k + kk) * lk + row0 + r));
        x[kk][0] = f.x;
        x[kk][1] = f.y;
        x[kk][2] = f.z;
        x[kk][3] = f.w;
      }
    } else {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          x[kk][e] = (r + e < nrows && k + kk < K) ? src[(int64_t)(k + kk) * lk + row0 + r + e] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat162 t01[NT], t23[NT];
      split_pair<NT>(x[0][e], x[1][e], t01);
      split_pair<NT>(x[2][e], x[3][e], t23);
      const uint32_t o = swz(r + e, kl);
#pragma unroll
      for (int i = 0; i < NT; ++i)
        *reinterpret_cast<uint2*>(tile + i * tstride + o) = make_uint2(bits(t01[i]), bits(t23[i]));
    }
  }
}

// Register-prefetched staging of a float32 operand in the vector modes (1: rows
// K-contiguous, 2: K strided with rows contiguous), split in two halves so that the next K
// block's loads are in flight while this block's MMAs run: load_vec reads this thread's
// chunks (zeros outside the valid rows and K) into kPF 16-byte registers, store_vec splits
// them into the NT term tiles.  Work units as in stage_tile_vec (mode 1: 4 floats of a row)
// and stage_tile_vec_t (mode 2: a 4 x 4 block).
constexpr int kPF = 8;
template <int ROWS, int NTH>
__device__ inline void load_vec(int mode, const float* src, int64_t lrow, int64_t lk, int row0, int nrows,
                                int k0, int K, uint4 (&rg)[kPF]) {
  if (mode == 1) {
    constexpr int kUnits = ROWS * 16, kIt = kUnits / NTH > 0 ? kUnits / NTH : 1;
    static_assert(kIt <= kPF, "prefetch registers");
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
      const int idx = threadIdx.x + i * NTH;
      const int r = idx >> 4, k = k0 + 4 * (idx & 15);
      rg[i] = make_uint4(0u, 0u, 0u, 0u);
      if (idx >= kUnits || r >= nrows) continue;
      const float* p = src + (int64_t)(row0 + r) * lrow + k;
      if (k + 4 <= K) {
        rg[i] = __ldg(reinterpret_cast<const uint4*>(p));
      } else {
        float t[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) t[e] = k + e < K ? p[e] : 0.f;
        rg[i] = make_uint4(__float_as_uint(t[0]), __float_as_uint(t[1]), __float_as_uint(t[2]),
                           __float_as_uint(t[3]));
      }
    }
  } else {
    constexpr int kRQ = ROWS / 4, kRQhi = kRQ / 4, kUnits = 16 * kRQ;
    constexpr int kIt = (kUnits + NTH - 1) / NTH;
    static_assert(4 * kIt <= kPF && kRQ >= 4, "prefetch registers");
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
      const int idx = threadIdx.x + i * NTH;
      const int rest = idx >> 5;
      const int r = 4 * ((rest % kRQhi) * 4 + ((idx >> 3) & 3));
      const int k = k0 + 4 * ((rest / kRQhi) * 8 + (idx & 7));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        uint4& q = rg[4 * i + kk];
        q = make_uint4(0u, 0u, 0u, 0u);
        if (idx >= kUnits || k + kk >= K) continue;
        const float* p = src + (int64_t)(k + kk) * lk + row0 + r;
        if (r + 4 <= nrows) {
          q = __ldg(reinterpret_cast<const uint4*>(p));
        } else {
          float t[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) t[e] = r + e < nrows ? p[e] : 0.f;
          q = make_uint4(__float_as_uint(t[0]), __float_as_uint(t[1]), __float_as_uint(t[2]),
                         __float_as_uint(t[3]));
        }
      }
    }
  }
}

template <int NT, int ROWS, int NTH>
__device__ inline void store_vec(int mode, const uint4 (&rg)[kPF], uint8_t* tile, uint32_t tstride) {
  if (mode == 1) {
    constexpr int kUnits = ROWS * 16, kIt = kUnits / NTH > 0 ? kUnits / NTH : 1;
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
      const int idx = threadIdx.x + i * NTH;
      if (idx >= kUnits) continue;
      __nv_bfloat162 t01[NT], t23[NT];
      split_pair<NT>(__uint_as_float(rg[i].x), __uint_as_float(rg[i].y), t01);
      split_pair<NT>(__uint_as_float(rg[i].z), __uint_as_float(rg[i].w), t23);
      const uint32_t o = swz(idx >> 4, 4 * (idx & 15));
#pragma unroll
      for (int j = 0; j < NT; ++j)
        *reinterpret_cast<uint2*>(tile + j * tstride + o) = make_uint2(bits(t01[j]), bits(t23[j]));
    }
  } else {
    constexpr int kRQ = ROWS / 4, kRQhi = kRQ / 4, kUnits = 16 * kRQ;
    constexpr int kIt = (kUnits + NTH - 1) / NTH;
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
      const int idx = threadIdx.x + i * NTH;
      if (idx >= kUnits) continue;
      const int rest = idx >> 5;
      const int r = 4 * ((rest % kRQhi) * 4 + ((idx >> 3) & 3));
      const int kl = 4 * ((rest / kRQhi) * 8 + (idx & 7));
      const float* x = reinterpret_cast<const float*>(&rg[4 * i]);  // x[4 kk + e]
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 t01[NT], t23[NT];
        split_pair<NT>(x[0 + e], x[4 + e], t01);
        split_pair<NT>(x[8 + e], x[12 + e], t23);
        const uint32_t o = swz(r + e, kl);
#pragma unroll
        for (int j = 0; j < NT; ++j)
          *reinterpret_cast<uint2*>(tile + j * tstride + o) = make_uint2(bits(t01[j]), bits(t23[j]));
      }
    }
  }
}

template <typename T, int NT, int ROWS, int NTH>
__device__ inline void stage(int mode, const T* src, int64_t lrow, int64_t lk, int row0, int nrows,
                             int k0, int K, uint8_t* tile, uint32_t tstride) {
  if (mode == 1) {
    stage_tile_vec<T, NT, ROWS, NTH>(src, lrow, row0, nrows, k0, K, tile, tstride);
  } else if (mode == 2) {
    if constexpr (std::is_same<T, float>::value)
      stage_tile_vec_t<NT, ROWS, NTH>(src, lk, row0, nrows, k0, K, tile, tstride);
  } else {
    stage_tile<T, NT, ROWS, NTH>(src, lrow, lk, row0, nrows, k0, K, tile, tstride);
  }
}

template <typename TA, typename TB, int BN, int NS>
struct Shape {
  static constexpr int kNA = std::is_same<TA, float>::value ? NS : 1;  // terms of A
  static constexpr int kNB = std::is_same<TB, float>::value ? NS : 1;  // terms of B
  static constexpr int kMaxT = kNA > kNB ? kNA : kNB;
  static constexpr uint32_t kATile = kBM * 128, kBTile = BN * 128;
  static constexpr uint32_t kStage = kATile * kNA + kBTile * kNB;
  static constexpr int kSmem = 2 * (int)kStage + 1024;
};

// Three-term kernels run one CTA per SM (shared memory), so they can spend registers on
// prefetching the next K block; two-term kernels keep two CTAs per SM instead.
template <typename TA, typename TB, int BN, int NS>
__global__ void __launch_bounds__(threads_for(NS), NS == 3 ? 1 : 2) gemm_bf16_kernel(GemmArgs g) {
  using S = Shape<TA, TB, BN, NS>;
  constexpr int NTH = threads_for(NS);
  constexpr bool kPrefetch = NS == 3 && std::is_same<TA, float>::value && std::is_same<TB, float>::value;
  constexpr uint32_t kIdesc = bf16_idesc(kBM, BN);
  constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N for M = 128");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[3];  // stage 0, stage 1, all MMAs done
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const uint32_t bar0 = smem_u32(&bars[0]), barf = smem_u32(&bars[2]);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    mbar_init(barf, 1);
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
  const bool batched = g.nbatch > 1;
  const int64_t bz = batched ? blockIdx.z : 0;
  const TA* Ab = static_cast<const TA*>(g.A) + bz * g.bsa;
  const TB* Bb = static_cast<const TB*>(g.B) + bz * g.bsb;
  const int nkb_all = (g.K + kKB - 1) / kKB;
  const int kb0 = batched ? 0 : blockIdx.z * g.kb_per;
  const int kb1 = batched ? nkb_all : min(nkb_all, kb0 + g.kb_per);
  const int mv = min(g.M - m0, kBM);
  const int nv = min(g.N - n0, BN);
  bool ok = true;
  int issued = 0;  // K blocks whose MMAs were committed
  // prefetch: both operands in a vector mode; the next block's chunks are loaded into
  // registers before this block's MMAs are issued
  const bool pf = kPrefetch && g.a_vec != 0 && g.b_vec != 0;
  uint4 ra[kPF], rb[kPF];
  if constexpr (kPrefetch) {
    if (pf && kb0 < kb1) {
      load_vec<kBM, NTH>(g.a_vec, reinterpret_cast<const float*>(Ab), g.lai, g.lak, m0, mv, kb0 * kKB, g.K, ra);
      load_vec<BN, NTH>(g.b_vec, reinterpret_cast<const float*>(Bb), g.lbj, g.lbk, n0, nv, kb0 * kKB, g.K, rb);
    }
  }
  for (int kb = kb0; kb < kb1; ++kb, ++issued) {
    const int s = issued & 1;
    uint8_t* at = base + (size_t)s * S::kStage;
    uint8_t* bt = at + S::kATile * S::kNA;
    if (issued >= 2) {  // the MMAs that read this stage two blocks ago are done
      const bool mine = mbar_wait(bar0 + 8 * s, (uint32_t)((issued >> 1) - 1) & 1u, &abort_flag, g.status);
      ok = __syncthreads_and(mine) != 0;
      if (!ok) break;
      fence_after();
    }
    bool staged = false;
    if constexpr (kPrefetch) {
      if (pf) {
        store_vec<S::kNA, kBM, NTH>(g.a_vec, ra, at, S::kATile);
        store_vec<S::kNB, BN, NTH>(g.b_vec, rb, bt, S::kBTile);
        if (kb + 1 < kb1) {
          load_vec<kBM, NTH>(g.a_vec, reinterpret_cast<const float*>(Ab), g.lai, g.lak, m0, mv, (kb + 1) * kKB,
                             g.K, ra);
          load_vec<BN, NTH>(g.b_vec, reinterpret_cast<const float*>(Bb), g.lbj, g.lbk, n0, nv, (kb + 1) * kKB,
                            g.K, rb);
        }
        staged = true;
      }
    }
    if (!staged) {
      stage<TA, S::kNA, kBM, NTH>(g.a_vec, Ab, g.lai, g.lak, m0, mv, kb * kKB, g.K, at, S::kATile);
      stage<TB, S::kNB, BN, NTH>(g.b_vec, Bb, g.lbj, g.lbk, n0, nv, kb * kKB, g.K, bt, S::kBTile);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
      const uint32_t a0 = smem_u32(at), b0 = smem_u32(bt);
#pragma unroll
      for (int ks = 0; ks < kKB / 16; ++ks) {
        bool first = issued == 0 && ks == 0;
#pragma unroll
        for (int ia = 0; ia < S::kNA; ++ia)
#pragma unroll
          for (int ib = 0; ib < S::kNB; ++ib)
            if (ia + ib < S::kMaxT) {
              mma_f16(tmem, smem_desc(a0 + ia * S::kATile + ks * 32), smem_desc(b0 + ib * S::kBTile + ks * 32),
                      kIdesc, first ? 0u : 1u);
              first = false;
            }
      }
      mma_commit(bar0 + 8 * s);
      if (kb == kb1 - 1) mma_commit(barf);
    }
  }
  bool done = false;
  if (ok && issued > 0) {
    const bool mine = mbar_wait(barf, 0, &abort_flag, g.status);
    done = __syncthreads_and(mine) != 0;
  }
  if (done) {
    fence_after();
    // warp w reads TMEM lane quarter w % 4 and the 16-column chunks part, part + parts, ...
    constexpr int kParts = NTH / 128, kChunks16 = BN / 16;
    const int q = warp & 3, part = warp >> 2;
    const int row = q * 32 + (threadIdx.x & 31);
    const bool split = !batched && gridDim.z > 1;
    float* C = split ? g.C + (int64_t)blockIdx.z * g.M * g.N : g.C + bz * g.bsc;
    const int64_t ldc = split ? g.N : g.ldc;
    const int epi = split ? 0 : g.epi;
    const bool vec = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) &&
                     (epi != 1 || (reinterpret_cast<uintptr_t>(g.H) & 15) == 0);
#pragma unroll 1
    for (int ch = part; ch < kChunks16; ch += kParts) {
      const int c0 = ch * 16;
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
      if (row >= mv || c0 >= nv) continue;
      const int64_t at = (int64_t)(m0 + row) * ldc + n0 + c0;
      const int cols = min(16, nv - c0);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (epi >= 1 && c < cols) v[c] += g.bias[n0 + c0 + c];
      if (epi == 3) {
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = gelu_f(v[c]);
      }
      if (vec && cols == 16) {
#pragma unroll
        for (int c = 0; c < 16; c += 4)
          *reinterpret_cast<float4*>(C + at + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        if (epi == 1) {
#pragma unroll
          for (int c = 0; c < 16; c += 4)
            *reinterpret_cast<float4*>(g.H + at + c) =
                make_float4(gelu_f(v[c]), gelu_f(v[c + 1]), gelu_f(v[c + 2]), gelu_f(v[c + 3]));
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          if (c >= cols) break;
          C[at + c] = v[c];
          if (epi == 1) g.H[at + c] = gelu_f(v[c]);
        }
      }
    }
  } else if (threadIdx.x == 0 && issued > 0) {
    // stopped early: wait (bounded) for the MMAs in flight before the TMEM is freed
    mbar_drain(bar0 + 8 * ((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1));
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
}

// C[i ldc + j] = sum over splits of the partial tiles (fixed order).
__global__ void splitk_sum_kernel(const float* part, int splits, int M, int N, float* C, int64_t ldc) {
  const int64_t count = (int64_t)M * N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[z * count + t];
    C[(t / N) * ldc + t % N] = s;
  }
}

}  // namespace mlptc

namespace {

template <typename TA, typename TB, int BN, int NS>
cudaError_t set_smem_attr() {
  static bool done = false;  // per instantiation; the attribute is a property of the function
  if (done) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(mlptc::gemm_bf16_kernel<TA, TB, BN, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             mlptc::Shape<TA, TB, BN, NS>::kSmem);
  if (e == cudaSuccess) done = true;
  return e;
}

template <typename TA, typename TB, int BN, int NS>
cudaError_t launch_bn(cudaStream_t st, dim3 grid, const mlptc::GemmArgs& g) {
  cudaError_t e = set_smem_attr<TA, TB, BN, NS>();
  if (e != cudaSuccess) return e;
  mlptc::gemm_bf16_kernel<TA, TB, BN, NS>
      <<<grid, mlptc::threads_for(NS), mlptc::Shape<TA, TB, BN, NS>::kSmem, st>>>(g);
  return cudaGetLastError();
}

template <typename TA, typename TB, int NS>
cudaError_t launch_typed(cudaStream_t st, int bn, dim3 grid, const mlptc::GemmArgs& g) {
  switch (bn) {
    case 16: return launch_bn<TA, TB, 16, NS>(st, grid, g);
    case 32: return launch_bn<TA, TB, 32, NS>(st, grid, g);
    case 64: return launch_bn<TA, TB, 64, NS>(st, grid, g);
    case 128: return launch_bn<TA, TB, 128, NS>(st, grid, g);
    default:
      if constexpr (NS == 2) return launch_bn<TA, TB, 256, NS>(st, grid, g);
      return cudaErrorInvalidValue;
  }
}

// Staging mode of an operand whose element (row, k) sits at row * lrow + k * lk (+ batch * bs):
// 1 = rows K-contiguous, 2 = K strided with rows contiguous (float32 only), 0 = element-wise.
int stage_mode(const void* p, size_t es, int64_t lrow, int64_t lk, int64_t bs) {
  const int64_t per = 16 / (int64_t)es;
  if ((reinterpret_cast<uintptr_t>(p) & 15) != 0 || bs % per != 0) return 0;
  if (lk == 1 && lrow % per == 0) return 1;
  if (es == 4 && lrow == 1 && lk % per == 0) return 2;
  return 0;
}

}  // namespace

// C = A B (epilogue) on the tensor cores with NS-term splits of float32 operands (2 or 3), over
// nbatch batch entries; see the file comment.  ta: kMlpF32; tb: kMlpBF16 or kMlpF32 (NS = 3:
// kMlpF32 only).  Epilogue 0 of one batch entry with part != NULL may split K over CTAs (at
// most part_cap floats of partial tiles); other launches never split.
cudaError_t gemm_split_tc(cudaStream_t st, int ns, float* part, int64_t part_cap, int* status, int M,
                          int N, int K, const void* A, int ta, int64_t lai, int64_t lak, int64_t bsa,
                          const void* B, int tb, int64_t lbk, int64_t lbj, int64_t bsb, float* C,
                          int64_t ldc, int64_t bsc, int nbatch, int epi, const float* bias, float* H) {
  if (M <= 0 || N <= 0 || K <= 0 || nbatch < 1 || nbatch > 65535 || ta != kMlpF32 ||
      (tb != kMlpF32 && tb != kMlpBF16) || (ns != 2 && ns != 3) || (ns == 3 && tb != kMlpF32))
    return cudaErrorInvalidValue;
  const int mt = (M + mlptc::kBM - 1) / mlptc::kBM;
  // N tile: the smallest MMA width that covers N, but 128-wide tiles when there are enough
  // CTAs to fill the SMs twice over (two CTAs per SM overlap their loads and MMAs), and at
  // most 128 for three-term operands (shared memory)
  int bn = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  if (bn == 256 && ((int64_t)M * nbatch >= 2 * 152 * mlptc::kBM || ns == 3)) bn = 128;
  const int nt = (N + bn - 1) / bn;
  const int nkb = (K + mlptc::kKB - 1) / mlptc::kKB;
  int splits = 1;
  if (nbatch == 1 && epi == 0 && part && nkb > 1) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    splits = std::max(1, std::min(nkb, sms / (mt * nt)));
    splits = (int)std::min<int64_t>(splits, std::min<int64_t>(32, part_cap / ((int64_t)M * N)));
    splits = std::max(splits, 1);
  }
  const int kb_per = (nkb + splits - 1) / splits;
  splits = (nkb + kb_per - 1) / kb_per;  // every split has at least one K block
  const size_t eb = tb == kMlpBF16 ? 2 : 4;
  mlptc::GemmArgs g{M, N, K, kb_per, nbatch, A, lai, lak, bsa, B, lbk, lbj, bsb,
                    splits > 1 ? part : C, ldc, bsc, epi, bias, H, status,
                    stage_mode(A, 4, lai, lak, bsa), stage_mode(B, eb, lbj, lbk, bsb)};
  const dim3 grid(nt, mt, nbatch > 1 ? nbatch : splits);
  cudaError_t e;
  if (ns == 3)
    e = launch_typed<float, float, 3>(st, bn, grid, g);
  else
    e = tb == kMlpBF16 ? launch_typed<float, __nv_bfloat16, 2>(st, bn, grid, g)
                       : launch_typed<float, float, 2>(st, bn, grid, g);
  if (e == cudaSuccess && splits > 1) {
    const int64_t count = (int64_t)M * N;
    const int blocks = (int)std::min<int64_t>(1024, (count + 255) / 256);
    mlptc::splitk_sum_kernel<<<blocks, 256, 0, st>>>(part, splits, M, N, C, ldc);
    e = cudaGetLastError();
  }
  return e;
}

// The surrogate's products: two-term splits, no batch.
cudaError_t mlp_gemm_tc(cudaStream_t st, float* part, int64_t part_cap, int* status, int M, int N,
                        int K, const void* A, int ta, int64_t lai, int64_t lak, const void* B, int tb,
                        int64_t lbk, int64_t lbj, float* C, int64_t ldc, int epi, const float* bias,
                        float* H) {
  return gemm_split_tc(st, 2, part, part_cap, status, M, N, K, A, ta, lai, lak, 0, B, tb, lbk, lbj, 0,
                       C, ldc, 0, 1, epi, bias, H);
}

// Set the shared-memory limit of the float32-accurate (three-term) kernels once, outside any
// stream capture.
cudaError_t gemm_f32_tc_prepare() {
  cudaError_t e = set_smem_attr<float, float, 16, 3>();
  if (e == cudaSuccess) e = set_smem_attr<float, float, 32, 3>();
  if (e == cudaSuccess) e = set_smem_attr<float, float, 64, 3>();
  if (e == cudaSuccess) e = set_smem_attr<float, float, 128, 3>();
  return e;
}

}  // namespace sas
