// Tensor-core GEMM of the learned surrogate's training and inference (sm_103a, tcgen05).
//
// C[i, j] = sum_k A(i, k) B(k, j) for the network's forward products, input gradients and
// weight gradients, with A(i, k) = A[i lai + k lak] and B(k, j) = B[k lbk + j lbj] (any
// strides, so transposed operands need no copies).  Operands are bfloat16 weights or float32
// activations, gradients and (optionally) float32 weights; the MMA is tcgen05 kind::f16 with
// bfloat16 A and B and float32 accumulation in TMEM:
//   * a bfloat16 operand enters as it is;
//   * a float32 operand v is split into hi = bf16(v) and lo = bf16(v - hi) (v - hi is exact
//     in float32), |v - hi - lo| <= 2^-18 |v|, and the product takes the terms hi x hi,
//     hi x lo and lo x hi, so that each product carries ~2^-17 relative error: float32-class
//     results from bfloat16 tensor cores.
// Epilogues: 0 = store C; 1 = Z = C + bias and H = gelu(Z) (exact erf form); 2 = C + bias;
// 3 = gelu(C + bias) only (inference, where Z is not needed).
//
// Structure: one CTA of 256 threads per 128 x BN tile of C (BN = 16 .. 256) and K range
// (split-K for the weight gradients, whose K is the batch): K in blocks of 64 (128-byte
// K-major rows, 128-byte swizzle), two shared-memory stages.  All threads load, split and
// store a K block; one elected thread issues its MMAs (K = 16 each) and commits them to the
// stage's mbarrier, which the threads wait on before they overwrite that stage.  Eight
// warps drain TMEM (warp w reads lane quarter w % 4 and half w / 4 of the columns).  A
// split-K launch writes float32 partial tiles that a second kernel sums in a fixed order.
// Every wait is bounded (2 s of %globaltimer); on expiry the kernel records SAS_ETIMEOUT,
// stops, waits (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <type_traits>

#include "sas_internal.cuh"
#include "sas_tc_common.cuh"

namespace sas {
namespace mlptc {

using namespace tc;

constexpr int kThreads = 256;
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
  int kb_per;  // K blocks per split (blockIdx.z)
  const void* A;
  int64_t lai, lak;
  const void* B;
  int64_t lbk, lbj;
  float* C;  // output, or the partial tiles [split][M][N] of a split-K launch
  int64_t ldc;
  int epi;
  const float* bias;
  float* H;
  int* status;
  int a_vec, b_vec;  // operand rows are K-contiguous and 16-byte aligned: vector staging
};

// Operand tile: rows x 64 (K block at k0) as bfloat16 hi (and lo) in the swizzled K-major
// layout.  Each thread takes a (row, k, k + 1) pair and stores it as one bfloat16x2; the
// pair index runs along the operand's unit-stride direction so that loads coalesce.
template <typename T, bool SPLIT, int ROWS>
__device__ inline void stage_tile(const T* src, int64_t lrow, int64_t lk, int row0, int nrows,
                                  int k0, int K, uint8_t* hi, uint8_t* lo) {
  const bool k_fast = lk == 1;
  for (int idx = threadIdx.x; idx < ROWS * 32; idx += kThreads) {
    const int r = k_fast ? idx >> 5 : idx % ROWS;
    const int kp = k_fast ? idx & 31 : idx / ROWS;
    const int k = k0 + 2 * kp;
    float v0 = 0.f, v1 = 0.f;
    if (r < nrows) {
      const T* p = src + (int64_t)(row0 + r) * lrow;
      if (k < K) v0 = ldv<T>(p, (int64_t)k * lk);
      if (k + 1 < K) v1 = ldv<T>(p, (int64_t)(k + 1) * lk);
    }
    const uint32_t o = (uint32_t)r * 128u + ((((uint32_t)kp >> 2) ^ (uint32_t)(r & 7)) << 4) +
                       (((uint32_t)kp & 3u) << 2);
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    *reinterpret_cast<__nv_bfloat162*>(hi + o) = h;
    if (SPLIT) {
      const float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(lo + o) = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    }
  }
}

// As stage_tile for operands whose rows are K-contiguous with 16-byte aligned starts: each
// thread takes 16-byte chunks (4 float32 or 8 bfloat16 of one row), issues all of its loads
// before it converts and stores any of them, and writes whole swizzle units.  Chunks past K
// or past the valid rows are filled element by element (zeros outside).
template <typename T, bool SPLIT, int ROWS>
__device__ inline void stage_tile_vec(const T* src, int64_t lrow, int row0, int nrows, int k0, int K,
                                      uint8_t* hi, uint8_t* lo) {
  constexpr int kPer = 16 / sizeof(T);          // elements per 16-byte chunk
  constexpr int kChunks = kKB / kPer;           // chunks per row
  constexpr int kIters = ROWS * kChunks / kThreads;
  static_assert(ROWS * kChunks % kThreads == 0 || ROWS * kChunks < kThreads, "tile and block");
  constexpr int kBatch = kIters < 8 ? (kIters < 1 ? 1 : kIters) : 8;
#pragma unroll 1
  for (int it0 = 0; it0 < (kIters < 1 ? 1 : kIters); it0 += kBatch) {
    uint4 v[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int idx = threadIdx.x + (it0 + b) * kThreads;
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
      const int idx = threadIdx.x + (it0 + b) * kThreads;
      if (idx >= ROWS * kChunks) continue;
      const int r = idx / kChunks, c = idx % kChunks;
      if (sizeof(T) == 2) {  // 8 bfloat16: one swizzle unit
        *reinterpret_cast<uint4*>(hi + (uint32_t)r * 128u + (((uint32_t)c ^ (uint32_t)(r & 7)) << 4)) = v[b];
      } else {  // 4 float32 -> 4 bfloat16 (8 bytes) of hi and of lo
        const float f0 = __uint_as_float(v[b].x), f1 = __uint_as_float(v[b].y);
        const float f2 = __uint_as_float(v[b].z), f3 = __uint_as_float(v[b].w);
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(f0, f1), h23 = __floats2bfloat162_rn(f2, f3);
        const uint32_t o = (uint32_t)r * 128u + ((((uint32_t)c >> 1) ^ (uint32_t)(r & 7)) << 4) +
                           (((uint32_t)c & 1u) << 3);
        uint2 hv;
        hv.x = *reinterpret_cast<const uint32_t*>(&h01);
        hv.y = *reinterpret_cast<const uint32_t*>(&h23);
        *reinterpret_cast<uint2*>(hi + o) = hv;
        if (SPLIT) {
          const float2 a = __bfloat1622float2(h01), b2 = __bfloat1622float2(h23);
          const __nv_bfloat162 l01 = __floats2bfloat162_rn(f0 - a.x, f1 - a.y);
          const __nv_bfloat162 l23 = __floats2bfloat162_rn(f2 - b2.x, f3 - b2.y);
          uint2 lv;
          lv.x = *reinterpret_cast<const uint32_t*>(&l01);
          lv.y = *reinterpret_cast<const uint32_t*>(&l23);
          *reinterpret_cast<uint2*>(lo + o) = lv;
        }
      }
    }
  }
}

template <typename TA, typename TB, int BN>
__global__ void __launch_bounds__(kThreads, 2) gemm_bf16_kernel(GemmArgs g) {
  constexpr bool SA = std::is_same<TA, float>::value;  // split into hi / lo
  constexpr bool SB = std::is_same<TB, float>::value;
  constexpr uint32_t kATile = kBM * 128, kBTile = BN * 128;
  constexpr uint32_t kStage = kATile * (SA ? 2 : 1) + kBTile * (SB ? 2 : 1);
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
  const int nkb_all = (g.K + kKB - 1) / kKB;
  const int kb0 = blockIdx.z * g.kb_per;
  const int kb1 = min(nkb_all, kb0 + g.kb_per);
  const int mv = min(g.M - m0, kBM);
  const int nv = min(g.N - n0, BN);
  bool ok = true;
  int issued = 0;  // K blocks whose MMAs were committed
  for (int kb = kb0; kb < kb1; ++kb, ++issued) {
    const int s = issued & 1;
    uint8_t* ahi = base + (size_t)s * kStage;
    uint8_t* alo = ahi + kATile;
    uint8_t* bhi = ahi + kATile * (SA ? 2 : 1);
    uint8_t* blo = bhi + kBTile;
    if (issued >= 2) {  // the MMAs that read this stage two blocks ago are done
      const bool mine = mbar_wait(bar0 + 8 * s, (uint32_t)((issued >> 1) - 1) & 1u, &abort_flag, g.status);
      ok = __syncthreads_and(mine) != 0;
      if (!ok) break;
      fence_after();
    }
    if (g.a_vec)
      stage_tile_vec<TA, SA, kBM>(static_cast<const TA*>(g.A), g.lai, m0, mv, kb * kKB, g.K, ahi, alo);
    else
      stage_tile<TA, SA, kBM>(static_cast<const TA*>(g.A), g.lai, g.lak, m0, mv, kb * kKB, g.K, ahi, alo);
    if (g.b_vec)
      stage_tile_vec<TB, SB, BN>(static_cast<const TB*>(g.B), g.lbj, n0, nv, kb * kKB, g.K, bhi, blo);
    else
      stage_tile<TB, SB, BN>(static_cast<const TB*>(g.B), g.lbj, g.lbk, n0, nv, kb * kKB, g.K, bhi, blo);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
      const uint32_t ah = smem_u32(ahi), al = smem_u32(alo), bh = smem_u32(bhi), bl = smem_u32(blo);
#pragma unroll
      for (int ks = 0; ks < kKB / 16; ++ks) {
        const uint32_t acc = (issued > 0 || ks > 0) ? 1u : 0u;
        mma_f16(tmem, smem_desc(ah + ks * 32), smem_desc(bh + ks * 32), kIdesc, acc);
        if (SB) mma_f16(tmem, smem_desc(ah + ks * 32), smem_desc(bl + ks * 32), kIdesc, 1u);
        if (SA) mma_f16(tmem, smem_desc(al + ks * 32), smem_desc(bh + ks * 32), kIdesc, 1u);
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
    const int q = warp & 3, half = warp >> 2;
    const int row = q * 32 + (threadIdx.x & 31);
    constexpr int kHalf = BN / 2;
    const bool split = gridDim.z > 1;
    float* C = split ? g.C + (int64_t)blockIdx.z * g.M * g.N : g.C;
    const int64_t ldc = split ? g.N : g.ldc;
    const int epi = split ? 0 : g.epi;
    const bool vec = ((ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) &&
                     (epi != 1 || (reinterpret_cast<uintptr_t>(g.H) & 15) == 0);
#pragma unroll 1
    for (int c0 = half * kHalf; c0 < half * kHalf + kHalf; c0 += 16) {
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

template <typename TA, typename TB, int BN>
cudaError_t launch_bn(cudaStream_t st, dim3 grid, const mlptc::GemmArgs& g) {
  constexpr bool SA = std::is_same<TA, float>::value;
  constexpr bool SB = std::is_same<TB, float>::value;
  constexpr int kStage = mlptc::kBM * 128 * (SA ? 2 : 1) + BN * 128 * (SB ? 2 : 1);
  constexpr int kSmem = 2 * kStage + 1024;
  static bool attr = false;  // per instantiation; the attribute is a property of the function
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mlptc::gemm_bf16_kernel<TA, TB, BN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  mlptc::gemm_bf16_kernel<TA, TB, BN><<<grid, mlptc::kThreads, kSmem, st>>>(g);
  return cudaGetLastError();
}

template <typename TA, typename TB>
cudaError_t launch_typed(cudaStream_t st, int bn, dim3 grid, const mlptc::GemmArgs& g) {
  switch (bn) {
    case 16: return launch_bn<TA, TB, 16>(st, grid, g);
    case 32: return launch_bn<TA, TB, 32>(st, grid, g);
    case 64: return launch_bn<TA, TB, 64>(st, grid, g);
    case 128: return launch_bn<TA, TB, 128>(st, grid, g);
    default: return launch_bn<TA, TB, 256>(st, grid, g);
  }
}

}  // namespace

// C = A B (epilogue) on the tensor cores; see the file comment.  ta: operand type of A
// (kMlpF32 only), tb: kMlpBF16 or kMlpF32.  Epilogue 0 with part != NULL may split K over
// CTAs (at most part_cap floats of partial tiles); epilogues 1 and 2 never split.
cudaError_t mlp_gemm_tc(cudaStream_t st, float* part, int64_t part_cap, int* status, int M, int N,
                        int K, const void* A, int ta, int64_t lai, int64_t lak, const void* B, int tb,
                        int64_t lbk, int64_t lbj, float* C, int64_t ldc, int epi, const float* bias,
                        float* H) {
  if (M <= 0 || N <= 0 || K <= 0 || ta != kMlpF32 || (tb != kMlpF32 && tb != kMlpBF16))
    return cudaErrorInvalidValue;
  // N tile: the smallest MMA width that covers N, but 128-wide tiles when there are enough
  // row tiles to fill the SMs twice over (two CTAs per SM overlap their loads and MMAs)
  int bn = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  if (bn == 256 && (int64_t)M >= 2 * 152 * mlptc::kBM) bn = 128;
  const int mt = (M + mlptc::kBM - 1) / mlptc::kBM, nt = (N + bn - 1) / bn;
  const int nkb = (K + mlptc::kKB - 1) / mlptc::kKB;
  int splits = 1;
  if (epi == 0 && part && nkb > 1) {
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
  const int a_vec = lak == 1 && lai % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const int b_vec = lbk == 1 && (lbj * (int64_t)eb) % 16 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  mlptc::GemmArgs g{M, N, K, kb_per, A, lai, lak, B, lbk, lbj, splits > 1 ? part : C, ldc, epi,
                    bias, H, status, a_vec, b_vec};
  const dim3 grid(nt, mt, splits);
  cudaError_t e = tb == kMlpBF16 ? launch_typed<float, __nv_bfloat16>(st, bn, grid, g)
                                 : launch_typed<float, float>(st, bn, grid, g);
  if (e == cudaSuccess && splits > 1) {
    const int64_t count = (int64_t)M * N;
    const int blocks = (int)std::min<int64_t>(1024, (count + 255) / 256);
    mlptc::splitk_sum_kernel<<<blocks, 256, 0, st>>>(part, splits, M, N, C, ldc);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace sas
