// Internal declarations of the SubApSnap online-stage library (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "subapsnap.h"

namespace sas {

// ---------------------------------------------------------------- complex
struct __align__(16) zd {
  double re, im;
};

__host__ __device__ inline zd mkz(double a, double b) { zd z; z.re = a; z.im = b; return z; }
__host__ __device__ inline zd operator+(zd a, zd b) { return mkz(a.re + b.re, a.im + b.im); }
__host__ __device__ inline zd operator-(zd a, zd b) { return mkz(a.re - b.re, a.im - b.im); }
__host__ __device__ inline zd operator-(zd a) { return mkz(-a.re, -a.im); }
__host__ __device__ inline zd operator*(zd a, zd b) {
  return mkz(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
__host__ __device__ inline zd operator*(double a, zd b) { return mkz(a * b.re, a * b.im); }
__host__ __device__ inline zd& operator+=(zd& a, zd b) { a = a + b; return a; }
__host__ __device__ inline zd& operator-=(zd& a, zd b) { a = a - b; return a; }

struct __align__(8) zf {
  float re, im;
};
__host__ __device__ inline zf mkzf(float a, float b) { zf z; z.re = a; z.im = b; return z; }
__host__ __device__ inline zf operator+(zf a, zf b) { return mkzf(a.re + b.re, a.im + b.im); }
__host__ __device__ inline zf operator-(zf a, zf b) { return mkzf(a.re - b.re, a.im - b.im); }
__host__ __device__ inline zf operator-(zf a) { return mkzf(-a.re, -a.im); }
__host__ __device__ inline zf operator*(zf a, zf b) {
  return mkzf(fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re));
}
__host__ __device__ inline zf operator*(float a, zf b) { return mkzf(a * b.re, a * b.im); }
__host__ __device__ inline zf& operator+=(zf& a, zf b) { a = a + b; return a; }
__host__ __device__ inline zf& operator-=(zf& a, zf b) { a = a - b; return a; }

// Uniform helpers so that kernels can be templated on the scalar type.
__host__ __device__ inline double conjv(double x) { return x; }
__host__ __device__ inline float conjv(float x) { return x; }
__host__ __device__ inline zd conjv(zd x) { return mkz(x.re, -x.im); }
__host__ __device__ inline zf conjv(zf x) { return mkzf(x.re, -x.im); }
__host__ __device__ inline double absq(double x) { return x * x; }
__host__ __device__ inline float absq(float x) { return x * x; }
__host__ __device__ inline double absq(zd x) { return x.re * x.re + x.im * x.im; }
__host__ __device__ inline float absq(zf x) { return x.re * x.re + x.im * x.im; }
template <typename T> __host__ __device__ inline T zero();
template <> __host__ __device__ inline double zero<double>() { return 0.0; }
template <> __host__ __device__ inline float zero<float>() { return 0.0f; }
template <> __host__ __device__ inline zd zero<zd>() { return mkz(0.0, 0.0); }
template <> __host__ __device__ inline zf zero<zf>() { return mkzf(0.0f, 0.0f); }
// scale by a real number
__host__ __device__ inline double rscale(double a, double x) { return a * x; }
__host__ __device__ inline float rscale(float a, float x) { return a * x; }
__host__ __device__ inline zd rscale(double a, zd x) { return a * x; }
__host__ __device__ inline zf rscale(float a, zf x) { return a * x; }
// conversions between precisions
__host__ __device__ inline float to_lo(double x) { return (float)x; }
__host__ __device__ inline zf to_lo(zd x) { return mkzf((float)x.re, (float)x.im); }
__host__ __device__ inline double to_hi(float x) { return (double)x; }
__host__ __device__ inline zd to_hi(zf x) { return mkz((double)x.re, (double)x.im); }
// division a / b for b on the complex plane (Smith-free: b is a Householder diagonal)
__host__ __device__ inline double divv(double a, double b) { return a / b; }
__host__ __device__ inline float divv(float a, float b) { return a / b; }
__host__ __device__ inline zd divv(zd a, zd b) {
  double d = b.re * b.re + b.im * b.im;
  return mkz((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__host__ __device__ inline zf divv(zf a, zf b) {
  float d = b.re * b.re + b.im * b.im;
  return mkzf((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
// phase of a number: a/|a| (1 for 0)
__host__ __device__ inline double phase(double a) { return a < 0.0 ? -1.0 : 1.0; }
__host__ __device__ inline float phase(float a) { return a < 0.0f ? -1.0f : 1.0f; }
__host__ __device__ inline zd phase(zd a) {
  double m = sqrt(absq(a));
  return m > 0.0 ? mkz(a.re / m, a.im / m) : mkz(1.0, 0.0);
}
__host__ __device__ inline zf phase(zf a) {
  float m = sqrtf(absq(a));
  return m > 0.0f ? mkzf(a.re / m, a.im / m) : mkzf(1.0f, 0.0f);
}
__device__ inline bool finitev(double x) { return isfinite(x); }
__device__ inline bool finitev(zd x) { return isfinite(x.re) && isfinite(x.im); }

template <typename T> __device__ inline T shfl_down(T v, int o);
template <> __device__ inline double shfl_down<double>(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
template <> __device__ inline float shfl_down<float>(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
template <> __device__ inline zd shfl_down<zd>(zd v, int o) {
  return mkz(__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o));
}
template <> __device__ inline zf shfl_down<zf>(zf v, int o) {
  return mkzf(__shfl_down_sync(0xffffffffu, v.re, o), __shfl_down_sync(0xffffffffu, v.im, o));
}
template <typename T> __device__ inline T shfl_idx(T v, int l);
template <> __device__ inline double shfl_idx<double>(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
template <> __device__ inline float shfl_idx<float>(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
template <> __device__ inline zd shfl_idx<zd>(zd v, int l) {
  return mkz(__shfl_sync(0xffffffffu, v.re, l), __shfl_sync(0xffffffffu, v.im, l));
}
template <> __device__ inline zf shfl_idx<zf>(zf v, int l) {
  return mkzf(__shfl_sync(0xffffffffu, v.re, l), __shfl_sync(0xffffffffu, v.im, l));
}
template <typename T> __device__ inline T shfl_xor_m(unsigned mask, T v, int o);
template <> __device__ inline double shfl_xor_m<double>(unsigned mask, double v, int o) {
  return __shfl_xor_sync(mask, v, o);
}
template <> __device__ inline float shfl_xor_m<float>(unsigned mask, float v, int o) {
  return __shfl_xor_sync(mask, v, o);
}
template <> __device__ inline zd shfl_xor_m<zd>(unsigned mask, zd v, int o) {
  return mkz(__shfl_xor_sync(mask, v.re, o), __shfl_xor_sync(mask, v.im, o));
}
template <> __device__ inline zf shfl_xor_m<zf>(unsigned mask, zf v, int o) {
  return mkzf(__shfl_xor_sync(mask, v.re, o), __shfl_xor_sync(mask, v.im, o));
}
template <typename T> __device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_down(v, o);
  return shfl_idx(v, 0);
}

// ----------------------------------------------------------------- limits
constexpr int kMaxR = 128;
constexpr int kMaxS = 512;
constexpr int kMaxDp = SAS_MAX_TERMS;

enum Family { kAffine = 0, kKernel = 1 };

// Per-parameter coefficient rule, evaluated on the device.
struct ThetaRule {
  int rule;  // SAS_THETA_*
  int K;
  int dp;
};

}  // namespace sas

// ------------------------------------------------------------------ context
struct sas_ctx {
  int family;
  int64_t n;
  int r, s, K, dtype, theta_rule, mode, dp, qoi_kind;
  // caller-owned device data
  const void* S;
  int64_t ldS;
  const int64_t* rowptr[SAS_MAX_TERMS];
  const int32_t* colind[SAS_MAX_TERMS];
  const double* values[SAS_MAX_TERMS];
  const void* b_full;
  const double* X;
  int d;
  // owned device data
  int64_t* J_dev;      // s
  void* G;             // K blocks, each s x r column-major (ld s), dtype
  void* G32;           // mixed: float / complex-float copy of G
  void* bJ;            // s, dtype
  void* bJ32;          // mixed copy
  void* wq;            // r, dtype: c^T S (QoI)
  double* SJ;          // kernel family: s x r (ld s)
  double* XJ;          // kernel family: s x d
  float* Shi;          // mixed reconstruction: high tf32 part of S, n x r (ld n)
  float* Slo;          // low part
  void* S16hi;         // mixed reconstruction, f16 form: 2^shift S high part, n x 64 (f16)
  void* S16lo;         // 2^11-scaled remainder
  int s16_shift;       // power-of-two scale of S in the f16 split
  void* Sx64;          // mixed reconstruction, float64-accurate form: 5 planes of 9-bit
                       // digits of the max-scaled rows of S (f16, rows of 64, n rounded to 128)
  int* Sx64_exp;       // per-row exponent e_i of that split (n)
  float* StHi;         // mixed kernel family: S^T tf32 high part, nb x npad (tensor-core rows)
  float* StLo;         // low part
  float* Xc32;         // mixed kernel family: float32 hi/lo coordinates of every point
  float* XJ32;         // mixed kernel family: float32 hi/lo coordinates of the rows of J
  double bJ_norm;
  // scratch (grown on demand)
  double* Mbuf;        // kernel family: dense M for a sub-batch (mcap x s x r)
  int64_t Mbuf_cap;    // parameters Mbuf holds
  void* ybuf;          // m x r dtype
  size_t ybuf_bytes;
  float* ysplit;       // mixed: y split into tf32 hi/lo, 2 x m x r
  size_t ysplit_bytes;
  void* ysplit16;      // mixed, f16 reconstruction: y split into f16 hi/lo (2 x m x 64) + m scales
  size_t ysplit16_bytes;
  void* yx64;          // mixed, float64-accurate reconstruction: digit planes of y + exponents
  size_t yx64_bytes;
  void* hstage;        // host-buffer calls: device staging of params, small outputs, x_hat chunks
  size_t hstage_bytes;
  size_t host_chunk;   // bytes of one pageable x_hat chunk (0 = 1 GiB)
  int* dev_status;     // device status word
  int num_sms;
  int ls_blocks_per_sm;
  void* surrogate;     // learned surrogate network (sas_mlp.cu), or null
  // options
  int recon_kernel;    // 0 auto, 1 CUDA cores, 2-4 tensor cores tf32, 5 tensor cores f16
  int xhat_f32;        // mixed form: 1 = x_hat in float32 (tf32 x 3), 0 = float64-accurate
  int surr_f32_out;    // surrogate: 1 = output layer with float32 weights (hi + lo bfloat16)
  int kernel_shard;    // kernel family: 1 = this context holds one shard of the points
  double* surr_aP;     // surrogate anchors for the next training (device, surr_na x dp)
  double* surr_aY;     // and their coefficient vectors (device, surr_na x r)
  int64_t surr_na;
  int recon_store;     // tensor-core reconstruction epilogue: 0 TMA stores, 1 direct stores
  int krr_kernel;      // kernel rows of the mixed form: 0 auto, 1 CUDA cores, 2 tensor cores
  int krr_seg_points;  // tensor-core rows: points per TMEM segment before the float64 fold
  int ls_variant_plain;  // launch shape of the plain LS kernel (autotuned)
  int ls_variant_mixed;  // launch shape (+ where the float64 M lives) of the mixed LS kernel
  void* ls_slots;        // mixed affine: global float64-M slots, one per resident CTA
  int64_t ls_slots_n;
  int max_refine;
  double refine_tol;
  // tracing
  int tracing;
  struct TraceRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<TraceRec>* trace;     // pending records
  std::vector<cudaEvent_t>* event_pool;
};

namespace sas {

// Thread-local error text.
void set_error(const std::string& msg);

// Tracing helpers: begin records an event before a launch, end after it.
struct TraceScope {
  sas_ctx* c;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  TraceScope(sas_ctx* ctx, int k, cudaStream_t s);
  ~TraceScope();
};

// ------------------------------------------------------- kernel launchers
// setup
cudaError_t launch_gather_blocks(const sas_ctx* c, cudaStream_t st);
cudaError_t launch_gather_vectors(const sas_ctx* c, const double* cvec, cudaStream_t st);
cudaError_t launch_make_mixed_copies(const sas_ctx* c, cudaStream_t st);
cudaError_t setup_f16_basis(sas_ctx* c, cudaStream_t st);  // S16hi / S16lo / s16_shift
// rows of A(p_sel) S, row-major with row stride ldv (sas_select.cu)
cudaError_t operator_rows_affine(const sas_affine_desc* d, const double* p_sel, void* V, int ldv);
// leverage-score weights of the subsampled rows (sas_leverage.cu)
cudaError_t launch_weight_rows(sas_ctx* c, const double* w_host, cudaStream_t st);
// tensor-core kernel rows (sas_krr_tc.cu)
int krr_tc_nb(int r);
int64_t krr_tc_npad(int64_t n);
int krr_tc_dp(int d);
size_t krr_tc_smem_bytes(int r, int d);
bool krr_tc_supported(const sas_ctx* c);
cudaError_t launch_krr_tc_copies(const sas_ctx* c, cudaStream_t st);
cudaError_t launch_krr_assemble_tc(const sas_ctx* c, const double* params, int64_t m, double* M,
                                   cudaStream_t st);
// solve
cudaError_t launch_ls_plain(const sas_ctx* c, const double* params, int64_t m, void* yout,
                            void* qoi_out, uint32_t* flags, double* rho, cudaStream_t st,
                            const void* Mg = nullptr);
cudaError_t launch_ls_mixed(const sas_ctx* c, const double* params, int64_t m, void* yout,
                            void* qoi_out, float* ysplit, uint32_t* flags, double* rho,
                            cudaStream_t st, const void* Mg = nullptr);
size_t ls_plain_smem_bytes(const sas_ctx* c, int* rows_per_block);
int64_t ls_mixed_slots(const sas_ctx* c);
int ls_num_variants(bool mixed);
size_t ls_mixed_smem_bytes(const sas_ctx* c);
cudaError_t launch_reconstruct_f64(const sas_ctx* c, const void* Y, int64_t m, void* out,
                                   cudaStream_t st);
cudaError_t launch_reconstruct_mixed(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                                     cudaStream_t st);
cudaError_t launch_reconstruct_tc(const sas_ctx* c, const float* ysplit, int64_t m, float* out,
                                  cudaStream_t st);
bool reconstruct_tc_supported(const sas_ctx* c);
void reconstruct_tc_split(int64_t n, int64_t m, int num_sms, int bn, int* num_mtiles,
                          int* num_ntiles, int* ngroups, int* ntpg);
// fixed device array of subapsnap_solve_batch_xhat_noalloc: address lookup at set-up
cudaError_t noalloc_prepare();
// float64-accurate tensor-core reconstruction (sas_recon_x64.cu)
cudaError_t setup_x64_basis(sas_ctx* c, cudaStream_t st);
bool reconstruct_x64_supported(const sas_ctx* c);
int64_t x64_plane_rows(int64_t rows);
size_t x64_coeff_bytes(int64_t m);
cudaError_t launch_reconstruct_x64(const sas_ctx* c, const double* Y, int64_t m, double* out,
                                   void* scratch, cudaStream_t st);
cudaError_t launch_wait_selftest(int* status, double seconds, cudaStream_t st);
cudaError_t launch_split_y(const double* Y, int64_t m, int r, int rpad, float* ysplit,
                           cudaStream_t st);
cudaError_t launch_residual(const sas_ctx* c, const double* params, int64_t m, const void* Y,
                            double* rho, cudaStream_t st, const void* Mg = nullptr);
cudaError_t launch_krr_assemble(const sas_ctx* c, const double* params, int64_t m, double* M,
                                bool f32, cudaStream_t st);
cudaError_t launch_gather_kernel_rows(const sas_ctx* c, cudaStream_t st);
cudaError_t launch_true_residual(const sas_ctx* c, const double* params, int64_t m, const void* X,
                                 double* rho, cudaStream_t st);
// surrogate
sas_status surrogate_create(sas_ctx* c, uint64_t seed);
void destroy_surrogate(sas_ctx* c);
sas_status surrogate_train(sas_ctx* c, const double* P, const double* Y, int64_t ntrain, int epochs,
                           int batch, double lr, uint64_t seed, double* loss_out, cudaStream_t st);
cudaError_t surrogate_predict(sas_ctx* c, const double* params, int64_t m, double* Yhat,
                              cudaStream_t st);
sas_status surrogate_grad(sas_ctx* c, const double* X, const double* Yn, int64_t B, double* loss,
                          float* grads_host, cudaStream_t st);
sas_status surrogate_io(sas_ctx* c, int get, float* theta, double* norm);
int64_t surrogate_nparam(const sas_ctx* c);
bool surrogate_ready(const sas_ctx* c);
sas_status surrogate_solve(sas_ctx* c, const double* params, int64_t m, int32_t out_kind, void* out,
                           uint32_t* flags, double* rho_out, double tol, int64_t* accepted,
                           cudaStream_t st);
sas_status surrogate_set_anchors(sas_ctx* c, const double* P, const double* Y, int64_t n);
// kernel-ridge snapshots by multishift CG (sas_krr_snap.cu)
sas_status krr_snapshots(const sas_kernel_desc* d, const double* sigma, int32_t ns, const double* lambda,
                         int32_t nl, double tol, int32_t maxit, double* Xout, int64_t ldx, int32_t* iters_out,
                         double* relres_out, cudaStream_t st);
// tensor-core GEMM with bfloat16-split operands (sas_mlp_tc.cu): operand types of A and B
enum { kMlpF32 = 0, kMlpBF16 = 1 };
cudaError_t mlp_gemm_tc(cudaStream_t st, float* part, int64_t part_cap, int* status, int M, int N,
                        int K, const void* A, int ta, int64_t lai, int64_t lak, const void* B, int tb,
                        int64_t lbk, int64_t lbj, float* C, int64_t ldc, int epi, const float* bias,
                        float* H);
// the same kernel with ns-term splits (2 or 3: float32-accurate) and a batch of nbatch entries
cudaError_t gemm_split_tc(cudaStream_t st, int ns, float* part, int64_t part_cap, int* status, int M,
                          int N, int K, const void* A, int ta, int64_t lai, int64_t lak, int64_t bsa,
                          const void* B, int tb, int64_t lbk, int64_t lbj, int64_t bsb, float* C,
                          int64_t ldc, int64_t bsc, int nbatch, int epi, const float* bias, float* H);
cudaError_t gemm_f32_tc_prepare();
// persistent multi-problem launch
struct MultiPlan {
  const void* kernel = nullptr;
  void* d_probs = nullptr;
  int64_t* d_offs = nullptr;
  unsigned long long* d_counter = nullptr;
  int nprob = 0, nt = 0, grid = 0;
  size_t smem = 0;
  int64_t total = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;  // stream the graph was captured on
};
cudaError_t multi_plan_build(MultiPlan* pl, sas_ctx* const* ctxs, int n, const double* const* params,
                             const int64_t* m, int32_t out_kind, void* const* outs,
                             uint32_t* const* flags, double* const* rho);
cudaError_t multi_plan_enqueue(MultiPlan* pl, cudaStream_t st);
// selection
sas_status select_rows_affine(const sas_affine_desc* d, const double* p_sel, int64_t* J_out,
                              double* gap_out);
sas_status select_rows_kernel(const sas_kernel_desc* d, const double* p_sel, int64_t* J_out,
                              double* gap_out);

}  // namespace sas
