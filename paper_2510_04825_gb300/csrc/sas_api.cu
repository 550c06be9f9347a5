// C ABI of the SubApSnap online-stage library: argument checks, context
// set-up and the dispatch of every entry point to its kernels.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <new>
#include <string>
#include <unordered_set>
#include <vector>

#include <cmath>

#include "sas_internal.cuh"

namespace sas {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

static cudaEvent_t pool_get(sas_ctx* c) {
  if (!c->event_pool) c->event_pool = new std::vector<cudaEvent_t>();
  if (!c->event_pool->empty()) {
    cudaEvent_t e = c->event_pool->back();
    c->event_pool->pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

TraceScope::TraceScope(sas_ctx* ctx, int k, cudaStream_t s) : c(ctx), cls(k), st(s) {
  if (c && c->tracing) {
    a = pool_get(c);
    cudaEventRecord(a, st);
  }
}

TraceScope::~TraceScope() {
  if (a) {
    cudaEvent_t b = pool_get(c);
    cudaEventRecord(b, st);
    if (!c->trace) c->trace = new std::vector<sas_ctx::TraceRec>();
    c->trace->push_back({cls, a, b});
  }
}

static sas_status fail(sas_status code, const std::string& msg) {
  set_error(msg);
  return code;
}

static sas_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static sas_status check_J(const int64_t* J, int s, int64_t n) {
  if (!J) return fail(SAS_EINVAL, "J is NULL");
  std::unordered_set<int64_t> seen;
  seen.reserve((size_t)s * 2);
  for (int i = 0; i < s; ++i) {
    if (J[i] < 0 || J[i] >= n)
      return fail(SAS_EINVAL, "J[" + std::to_string(i) + "] = " + std::to_string(J[i]) + " is out of range");
    if (!seen.insert(J[i]).second)
      return fail(SAS_EINVAL, "J holds the index " + std::to_string(J[i]) + " twice");
  }
  return SAS_OK;
}

static void free_ctx(sas_ctx* c) {
  if (!c) return;
  cudaFree(c->J_dev);
  cudaFree(c->G);
  cudaFree(c->G32);
  cudaFree(c->bJ);
  cudaFree(c->bJ32);
  cudaFree(c->wq);
  cudaFree(c->SJ);
  cudaFree(c->XJ);
  cudaFree(c->Shi);
  cudaFree(c->Slo);
  cudaFree(c->ls_slots);
  cudaFree(c->S16hi);
  cudaFree(c->S16lo);
  cudaFree(c->ysplit16);
  cudaFree(c->Sx64);
  cudaFree(c->Sx64_exp);
  cudaFree(c->yx64);
  cudaFree(c->StHi);
  cudaFree(c->StLo);
  cudaFree(c->Xc32);
  cudaFree(c->XJ32);
  cudaFree(c->ybuf);
  cudaFree(c->ysplit);
  cudaFree(c->Mbuf);
  cudaFree(c->hstage);
  cudaFree(c->dev_status);
  cudaFree(c->surr_aP);
  cudaFree(c->surr_aY);
  destroy_surrogate(c);
  if (c->trace) {
    for (auto& t : *c->trace) {
      cudaEventDestroy(t.a);
      cudaEventDestroy(t.b);
    }
    delete c->trace;
  }
  if (c->event_pool) {
    for (auto e : *c->event_pool) cudaEventDestroy(e);
    delete c->event_pool;
  }
  delete c;
}

static sas_status check_affine_desc(const sas_affine_desc* d, bool need_J) {
  if (!d) return fail(SAS_EINVAL, "descriptor is NULL");
  if (d->n < 1) return fail(SAS_EINVAL, "n must be positive");
  if (d->r < 1 || d->r > kMaxR) return fail(SAS_EINVAL, "r must be in [1, 128]");
  if (d->s < d->r || d->s > kMaxS || (int64_t)d->s > d->n)
    return fail(SAS_EINVAL, "need r <= s <= min(n, 512)");
  if (d->K < 1 || d->K > SAS_MAX_TERMS) return fail(SAS_EINVAL, "K must be in [1, 8]");
  if (d->dtype != SAS_REAL64 && d->dtype != SAS_COMPLEX128) return fail(SAS_EINVAL, "bad dtype");
  if (d->theta_rule == SAS_THETA_PENCIL) {
    if (d->dtype != SAS_COMPLEX128 || d->K != 2)
      return fail(SAS_EINVAL, "the pencil rule needs complex128 and K = 2");
  } else if (d->theta_rule == SAS_THETA_DELAY) {
    if (d->dtype != SAS_COMPLEX128 || d->K != 3)
      return fail(SAS_EINVAL, "the delay rule needs complex128 and K = 3");
  } else if (d->theta_rule != SAS_THETA_LINEAR) {
    return fail(SAS_EINVAL, "bad theta rule");
  }
  if (d->w)
    for (int i = 0; i < d->s; ++i)
      if (!(d->w[i] > 0.0) || !std::isfinite(d->w[i]))
        return fail(SAS_EINVAL, "row weights must be positive and finite");
  if (d->mode != SAS_MODE_PLAIN && d->mode != SAS_MODE_MIXED) return fail(SAS_EINVAL, "bad mode");
  if (d->ldS < d->n) return fail(SAS_EINVAL, "ldS < n");
  if (!is_device_ptr(d->S)) return fail(SAS_EINVAL, "S must be a device pointer");
  for (int k = 0; k < d->K; ++k) {
    if (!is_device_ptr(d->rowptr[k]) || !is_device_ptr(d->colind[k]) || !is_device_ptr(d->values[k]))
      return fail(SAS_EINVAL, "CSR arrays of term " + std::to_string(k) + " must be device pointers");
  }
  if (need_J) {
    if (!is_device_ptr(d->b)) return fail(SAS_EINVAL, "b must be a device pointer");
    sas_status st = check_J(d->J, d->s, d->n);
    if (st != SAS_OK) return st;
    if (d->qoi_kind == SAS_QOI_TRANSPOSE && !is_device_ptr(d->c))
      return fail(SAS_EINVAL, "c must be a device pointer for SAS_QOI_TRANSPOSE");
    if (d->qoi_kind != SAS_QOI_NONE && d->qoi_kind != SAS_QOI_TRANSPOSE && d->qoi_kind != SAS_QOI_MEAN)
      return fail(SAS_EINVAL, "bad qoi kind");
  }
  return SAS_OK;
}

template <typename T>
static cudaError_t dmalloc(T** p, size_t bytes) {
  return cudaMalloc((void**)p, bytes);
}

static sas_status ensure_scratch(sas_ctx* c, int64_t m, bool mixed, cudaStream_t st) {
  const size_t es = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  const size_t need = (size_t)m * c->r * es;
  if (need > c->ybuf_bytes) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "solve_batch");
    cudaFree(c->ybuf);
    c->ybuf = nullptr;
    c->ybuf_bytes = 0;
    e = cudaMalloc(&c->ybuf, need);
    if (e != cudaSuccess) return cuda_fail(e, "solve_batch scratch");
    c->ybuf_bytes = need;
  }
  if (mixed && !c->xhat_f32) {
    // float64-accurate x_hat: digit planes of y and their exponents
    const size_t need4 = reconstruct_x64_supported(c) ? x64_coeff_bytes(m) : 0;
    if (need4 > c->yx64_bytes) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "solve_batch");
      cudaFree(c->yx64);
      c->yx64 = nullptr;
      c->yx64_bytes = 0;
      e = cudaMalloc(&c->yx64, need4);
      if (e != cudaSuccess) return cuda_fail(e, "solve_batch scratch");
      c->yx64_bytes = need4;
    }
  }
  if (mixed && c->xhat_f32) {
    const int rpad = (c->r + 31) / 32 * 32;
    const size_t need2 = (size_t)2 * m * rpad * sizeof(float);
    if (need2 > c->ysplit_bytes) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "solve_batch");
      cudaFree(c->ysplit);
      c->ysplit = nullptr;
      c->ysplit_bytes = 0;
      e = cudaMalloc((void**)&c->ysplit, need2);
      if (e != cudaSuccess) return cuda_fail(e, "solve_batch scratch");
      c->ysplit_bytes = need2;
    }
    // f16 form of the reconstruction: hi and lo (2 x m x 64 f16) and m float scales
    const size_t need3 = (size_t)m * (2 * 64 * 2 + 4);
    if (c->S16hi && need3 > c->ysplit16_bytes) {
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "solve_batch");
      cudaFree(c->ysplit16);
      c->ysplit16 = nullptr;
      c->ysplit16_bytes = 0;
      e = cudaMalloc(&c->ysplit16, need3);
      if (e != cudaSuccess) return cuda_fail(e, "solve_batch scratch");
      c->ysplit16_bytes = need3;
    }
  }
  return SAS_OK;
}

// x_hat of the mixed form from the float64 coefficients in c->ybuf: float64 from
// the digit products on the tensor cores (or the float64 CUDA-core product where
// the digit split does not apply: r > 64, or SAS_OPT_RECON_KERNEL = 1).
static cudaError_t reconstruct_mixed_f64(sas_ctx* c, int64_t m, double* out, cudaStream_t st) {
  if (c->recon_kernel != 1 && reconstruct_x64_supported(c))
    return launch_reconstruct_x64(c, (const double*)c->ybuf, m, out, c->yx64, st);
  return launch_reconstruct_f64(c, c->ybuf, m, out, st);
}

}  // namespace sas

using namespace sas;

extern "C" {

const char* subapsnap_version(void) { return "subapsnap-gb300 0.1 (sm_103a)"; }

sas_status subapsnap_selftest_wait(sas_ctx* c, double seconds, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (!(seconds > 0.0 && seconds <= 2.0)) return fail(SAS_EINVAL, "seconds must be in (0, 2]");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_wait_selftest(c->dev_status, seconds, st);
  if (e != cudaSuccess) return cuda_fail(e, "selftest_wait");
  return subapsnap_device_status(c, stream);
}

const char* subapsnap_last_error(void) { return g_last_error.c_str(); }

sas_status subapsnap_setup_affine(const sas_affine_desc* d, sas_ctx** out) {
  if (!out) return fail(SAS_EINVAL, "out is NULL");
  *out = nullptr;
  sas_status st = check_affine_desc(d, true);
  if (st != SAS_OK) return st;
  sas_ctx* c = new (std::nothrow) sas_ctx();
  if (!c) return fail(SAS_ENOMEM, "host allocation failed");
  std::memset((void*)c, 0, sizeof(sas_ctx));
  c->family = kAffine;
  c->n = d->n;
  c->r = d->r;
  c->s = d->s;
  c->K = d->K;
  c->dtype = d->dtype;
  c->theta_rule = d->theta_rule;
  c->mode = d->mode;
  c->dp = d->theta_rule == SAS_THETA_PENCIL ? 1 : d->theta_rule == SAS_THETA_DELAY ? 2 : d->K - 1;
  c->qoi_kind = d->qoi_kind;
  c->S = d->S;
  c->ldS = d->ldS;
  for (int k = 0; k < SAS_MAX_TERMS; ++k) {
    c->rowptr[k] = k < d->K ? d->rowptr[k] : nullptr;
    c->colind[k] = k < d->K ? d->colind[k] : nullptr;
    c->values[k] = k < d->K ? d->values[k] : nullptr;
  }
  c->b_full = d->b;
  c->recon_kernel = 0;
  c->recon_store = 1;
  c->max_refine = 4;
  c->refine_tol = 1e-13;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t es = d->dtype == SAS_COMPLEX128 ? 16 : 8;
  const size_t esl = es / 2;
  cudaError_t e = cudaSuccess;
  cudaStream_t sst = nullptr;
#define TRY(x)                                        \
  do {                                                \
    e = (x);                                          \
    if (e != cudaSuccess) {                           \
      st = cuda_fail(e, "setup_affine");              \
      if (sst) cudaStreamDestroy(sst);                \
      free_ctx(c);                                    \
      return st;                                      \
    }                                                 \
  } while (0)
  TRY(cudaStreamCreateWithFlags(&sst, cudaStreamNonBlocking));
  TRY(dmalloc(&c->J_dev, sizeof(int64_t) * d->s));
  TRY(cudaMemcpy(c->J_dev, d->J, sizeof(int64_t) * d->s, cudaMemcpyHostToDevice));
  TRY(cudaMalloc(&c->G, (size_t)d->K * d->s * d->r * es));
  TRY(cudaMalloc(&c->bJ, (size_t)d->s * es));
  TRY(cudaMalloc(&c->wq, (size_t)d->r * es));
  TRY(cudaMemset(c->wq, 0, (size_t)d->r * es));
  TRY(dmalloc(&c->dev_status, sizeof(int)));
  TRY(cudaMemset(c->dev_status, 0, sizeof(int)));
  TRY(launch_gather_blocks(c, sst));
  TRY(launch_gather_vectors(c, d->c, sst));
  TRY(noalloc_prepare());  // the fixed array of the no-allocation entry point
  if (d->w) TRY(launch_weight_rows(c, d->w, sst));  // weighted rows: W M(p), W b_J
  if (d->mode == SAS_MODE_MIXED) {
    TRY(cudaMalloc(&c->G32, (size_t)d->K * d->s * d->r * esl));
    TRY(cudaMalloc(&c->bJ32, (size_t)d->s * esl));
    if (d->dtype == SAS_REAL64) {
      const int rpad = (d->r + 31) / 32 * 32;
      TRY(dmalloc(&c->Shi, (size_t)d->n * rpad * sizeof(float)));
      TRY(dmalloc(&c->Slo, (size_t)d->n * rpad * sizeof(float)));
    }
    TRY(launch_make_mixed_copies(c, sst));
    TRY(setup_f16_basis(c, sst));
    TRY(setup_x64_basis(c, sst));
    // float64 M slots for the least-squares variants that keep M in global memory
    c->ls_slots_n = ls_mixed_slots(c);
    TRY(cudaMalloc(&c->ls_slots, (size_t)c->ls_slots_n * d->s * d->r * es));
  }
  TRY(cudaStreamSynchronize(sst));
  {
    std::vector<double> hb((size_t)d->s * (es / 8));
    TRY(cudaMemcpy(hb.data(), c->bJ, (size_t)d->s * es, cudaMemcpyDeviceToHost));
    double nrm2 = 0.0;
    for (double v : hb) nrm2 += v * v;
    c->bJ_norm = std::sqrt(nrm2);
    if (!(c->bJ_norm > 0.0)) {
      cudaStreamDestroy(sst);
      free_ctx(c);
      return fail(SAS_EINVAL, "b_J is zero: the subsampled system has no right-hand side");
    }
  }
  cudaStreamDestroy(sst);
#undef TRY
  *out = c;
  return SAS_OK;
}

// Kernel-family context.  ext == NULL: the rows at J are gathered from X, S and b.  ext != NULL
// (a point shard): X and S hold this shard's points only, and the rows X_J, S_J, b_J come from
// the caller (device arrays, copied).
static sas_status setup_kernel_impl(const sas_kernel_desc* d, const sas_kernel_shard_desc* ext,
                                    sas_ctx** out) {
  if (!out) return fail(SAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(SAS_EINVAL, "descriptor is NULL");
  if (d->n < 1) return fail(SAS_EINVAL, "n must be positive");
  if (d->d < 1 || d->d > 16) return fail(SAS_EINVAL, "d must be in [1, 16]");
  if (d->r < 1 || d->r > kMaxR) return fail(SAS_EINVAL, "r must be in [1, 128]");
  if (d->s < d->r || d->s > kMaxS || (!ext && (int64_t)d->s > d->n))
    return fail(SAS_EINVAL, "need r <= s <= min(n, 512)");
  if (d->mode != SAS_MODE_PLAIN && d->mode != SAS_MODE_MIXED) return fail(SAS_EINVAL, "bad mode");
  if (d->ldS < d->n) return fail(SAS_EINVAL, "ldS < n");
  if (!is_device_ptr(d->X) || !is_device_ptr(d->S))
    return fail(SAS_EINVAL, "X and S must be device pointers");
  sas_status st = SAS_OK;
  if (ext) {
    if (!is_device_ptr(ext->XJ) || !is_device_ptr(ext->SJ) || !is_device_ptr(ext->bJ))
      return fail(SAS_EINVAL, "XJ, SJ and bJ must be device pointers");
  } else {
    if (!is_device_ptr(d->b)) return fail(SAS_EINVAL, "b must be a device pointer");
    st = check_J(d->J, d->s, d->n);
    if (st != SAS_OK) return st;
  }
  sas_ctx* c = new (std::nothrow) sas_ctx();
  if (!c) return fail(SAS_ENOMEM, "host allocation failed");
  std::memset((void*)c, 0, sizeof(sas_ctx));
  c->family = kKernel;
  c->n = d->n;
  c->r = d->r;
  c->s = d->s;
  c->K = 0;
  c->d = d->d;
  c->dtype = SAS_REAL64;
  c->theta_rule = -1;
  c->mode = d->mode;
  c->dp = 2;
  c->qoi_kind = SAS_QOI_NONE;
  c->S = d->S;
  c->ldS = d->ldS;
  c->X = d->X;
  c->b_full = d->b;
  c->recon_kernel = 0;
  c->recon_store = 1;
  c->max_refine = 4;
  c->refine_tol = 1e-13;
  c->krr_seg_points = 1024;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  cudaStream_t sst = nullptr;
#define TRYK(x)                              \
  do {                                       \
    e = (x);                                 \
    if (e != cudaSuccess) {                  \
      st = cuda_fail(e, "setup_kernel");     \
      if (sst) cudaStreamDestroy(sst);       \
      free_ctx(c);                           \
      return st;                             \
    }                                        \
  } while (0)
  TRYK(cudaStreamCreateWithFlags(&sst, cudaStreamNonBlocking));
  TRYK(dmalloc(&c->XJ, sizeof(double) * d->s * d->d));
  TRYK(dmalloc(&c->SJ, sizeof(double) * d->s * d->r));
  TRYK(cudaMalloc(&c->bJ, sizeof(double) * d->s));
  TRYK(cudaMalloc(&c->wq, sizeof(double) * d->r));
  TRYK(cudaMemset(c->wq, 0, sizeof(double) * d->r));
  TRYK(dmalloc(&c->dev_status, sizeof(int)));
  TRYK(cudaMemset(c->dev_status, 0, sizeof(int)));
  if (ext) {
    c->kernel_shard = 1;
    TRYK(cudaMemcpy(c->XJ, ext->XJ, sizeof(double) * d->s * d->d, cudaMemcpyDeviceToDevice));
    TRYK(cudaMemcpy(c->SJ, ext->SJ, sizeof(double) * d->s * d->r, cudaMemcpyDeviceToDevice));
    TRYK(cudaMemcpy(c->bJ, ext->bJ, sizeof(double) * d->s, cudaMemcpyDeviceToDevice));
  } else {
    TRYK(dmalloc(&c->J_dev, sizeof(int64_t) * d->s));
    TRYK(cudaMemcpy(c->J_dev, d->J, sizeof(int64_t) * d->s, cudaMemcpyHostToDevice));
    TRYK(launch_gather_kernel_rows(c, sst));
  }
  if (d->mode == SAS_MODE_MIXED) {
    TRYK(cudaMalloc(&c->bJ32, sizeof(float) * d->s));
    const int rpad = (d->r + 31) / 32 * 32;
    TRYK(dmalloc(&c->Shi, (size_t)d->n * rpad * sizeof(float)));
    TRYK(dmalloc(&c->Slo, (size_t)d->n * rpad * sizeof(float)));
    TRYK(launch_make_mixed_copies(c, sst));
    TRYK(setup_f16_basis(c, sst));
    TRYK(setup_x64_basis(c, sst));
    // tensor-core kernel rows: S^T split, float32 hi/lo coordinates
    const int nb = krr_tc_nb(d->r), dp = krr_tc_dp(d->d);
    const int64_t npad = krr_tc_npad(d->n);
    TRYK(dmalloc(&c->StHi, (size_t)nb * npad * sizeof(float)));
    TRYK(dmalloc(&c->StLo, (size_t)nb * npad * sizeof(float)));
    TRYK(dmalloc(&c->Xc32, (size_t)npad * 2 * dp * sizeof(float)));
    TRYK(dmalloc(&c->XJ32, (size_t)d->s * 2 * dp * sizeof(float)));
    TRYK(launch_krr_tc_copies(c, sst));
  }
  TRYK(cudaStreamSynchronize(sst));
  {
    std::vector<double> hb((size_t)d->s);
    TRYK(cudaMemcpy(hb.data(), c->bJ, sizeof(double) * d->s, cudaMemcpyDeviceToHost));
    double nrm2 = 0.0;
    for (double v : hb) nrm2 += v * v;
    c->bJ_norm = std::sqrt(nrm2);
    if (!(c->bJ_norm > 0.0)) {
      cudaStreamDestroy(sst);
      free_ctx(c);
      return fail(SAS_EINVAL, "b_J is zero: the subsampled system has no right-hand side");
    }
  }
  cudaStreamDestroy(sst);
#undef TRYK
  *out = c;
  return SAS_OK;
}

sas_status subapsnap_setup_kernel(const sas_kernel_desc* d, sas_ctx** out) {
  return setup_kernel_impl(d, nullptr, out);
}

sas_status subapsnap_setup_kernel_shard(const sas_kernel_shard_desc* d, sas_ctx** out) {
  if (!d) {
    if (out) *out = nullptr;
    return fail(SAS_EINVAL, "descriptor is NULL");
  }
  return setup_kernel_impl(&d->base, d, out);
}

namespace sas {
// Dense-M scratch of the kernel family: room for `cap` parameters.
static sas_status ensure_mbuf(sas_ctx* c, int64_t cap, cudaStream_t st) {
  if (c->Mbuf_cap >= cap) return SAS_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel rows scratch");
  cudaFree(c->Mbuf);
  c->Mbuf = nullptr;
  c->Mbuf_cap = 0;
  e = cudaMalloc((void**)&c->Mbuf, sizeof(double) * (size_t)cap * c->s * c->r);
  if (e != cudaSuccess) return cuda_fail(e, "kernel rows scratch");
  c->Mbuf_cap = cap;
  return SAS_OK;
}
constexpr int64_t kKernelSubBatch = 512;
constexpr int64_t kKernelSubBatchTc = 2048;  // tensor-core rows: fewer, fuller waves

static sas_status solve_kernel_family(sas_ctx* c, const double* params, int64_t m, int32_t out_kind,
                                      void* out, uint32_t* flags, double* rho, cudaStream_t st) {
  const bool mixed = c->mode == SAS_MODE_MIXED;
  if (out_kind != SAS_OUT_Y && out_kind != SAS_OUT_XHAT)
    return fail(SAS_EINVAL, "the kernel family returns y or x_hat");
  const bool tc_rows = mixed && c->krr_kernel != 1 && krr_tc_supported(c);
  if (mixed && c->krr_kernel == 2 && !tc_rows)
    return fail(SAS_ENOTSUP, "tensor-core kernel rows are not available for this context");
  const int64_t sub = tc_rows ? kKernelSubBatchTc : kKernelSubBatch;
  const int64_t cap = m < sub ? m : sub;
  sas_status s2 = ensure_mbuf(c, cap, st);
  if (s2 != SAS_OK) return s2;
  if (out_kind == SAS_OUT_XHAT) {
    s2 = ensure_scratch(c, cap, mixed, st);
    if (s2 != SAS_OK) return s2;
  }
  cudaError_t e = cudaSuccess;
  for (int64_t b0 = 0; b0 < m && e == cudaSuccess; b0 += cap) {
    const int64_t mb = m - b0 < cap ? m - b0 : cap;
    const double* pb = params + b0 * 2;
    {
      TraceScope ts(c, SAS_KERNEL_ASSEMBLE, st);
      e = tc_rows ? launch_krr_assemble_tc(c, pb, mb, c->Mbuf, st)
                  : launch_krr_assemble(c, pb, mb, c->Mbuf, mixed, st);
    }
    if (e != cudaSuccess) break;
    void* yout = out_kind == SAS_OUT_Y ? (void*)((double*)out + b0 * c->r) : c->ybuf;
    uint32_t* fb = flags ? flags + b0 : nullptr;
    double* rb = rho ? rho + b0 : nullptr;
    {
      TraceScope ts(c, SAS_KERNEL_LS, st);
      e = mixed ? launch_ls_mixed(c, pb, mb, yout, nullptr,
                                  out_kind == SAS_OUT_XHAT && c->xhat_f32 ? c->ysplit : nullptr, fb,
                                  rb, st, c->Mbuf)
                : launch_ls_plain(c, pb, mb, yout, nullptr, fb, rb, st, c->Mbuf);
    }
    if (e != cudaSuccess || out_kind != SAS_OUT_XHAT) continue;
    {
      TraceScope ts(c, SAS_KERNEL_RECONSTRUCT, st);
      if (mixed && c->xhat_f32)
        e = launch_reconstruct_mixed(c, c->ysplit, mb, (float*)out + b0 * c->n, st);
      else if (mixed)
        e = reconstruct_mixed_f64(c, mb, (double*)out + b0 * c->n, st);
      else
        e = launch_reconstruct_f64(c, c->ybuf, mb, (double*)out + b0 * c->n, st);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "solve_batch");
  return SAS_OK;
}
}  // namespace sas

sas_status subapsnap_kernel_rows(sas_ctx* c, const double* params, int64_t m, double* M, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (c->family != kKernel) return fail(SAS_ENOTSUP, "kernel rows need a Gaussian-kernel context");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!params || !M) return fail(SAS_EINVAL, "params and M must be non-NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const bool mixed = c->mode == SAS_MODE_MIXED;
  const bool tc_rows = mixed && c->krr_kernel != 1 && krr_tc_supported(c);
  if (mixed && c->krr_kernel == 2 && !tc_rows)
    return fail(SAS_ENOTSUP, "tensor-core kernel rows are not available for this context");
  const int64_t sub = tc_rows ? kKernelSubBatchTc : kKernelSubBatch;
  cudaError_t e = cudaSuccess;
  for (int64_t b0 = 0; b0 < m && e == cudaSuccess; b0 += sub) {
    const int64_t mb = m - b0 < sub ? m - b0 : sub;
    double* Mb = M + b0 * (int64_t)c->s * c->r;
    TraceScope ts(c, SAS_KERNEL_ASSEMBLE, st);
    e = tc_rows ? launch_krr_assemble_tc(c, params + b0 * 2, mb, Mb, st)
                : launch_krr_assemble(c, params + b0 * 2, mb, Mb, mixed, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel_rows");
  return SAS_OK;
}

sas_status subapsnap_solve_batch_rows(sas_ctx* c, const double* params, int64_t m, const double* M,
                                      double* Y, uint32_t* flags, double* rho, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (c->family != kKernel) return fail(SAS_ENOTSUP, "solve from rows needs a Gaussian-kernel context");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!params || !M || !Y) return fail(SAS_EINVAL, "params, M and Y must be non-NULL");
  cudaStream_t st = (cudaStream_t)stream;
  TraceScope ts(c, SAS_KERNEL_LS, st);
  const cudaError_t e = c->mode == SAS_MODE_MIXED
                            ? launch_ls_mixed(c, params, m, Y, nullptr, nullptr, flags, rho, st, M)
                            : launch_ls_plain(c, params, m, Y, nullptr, flags, rho, st, M);
  if (e != cudaSuccess) return cuda_fail(e, "solve_batch_rows");
  return SAS_OK;
}

sas_status subapsnap_solve_batch(sas_ctx* c, const double* params, int64_t m, int32_t out_kind,
                                 void* out, uint32_t* flags, double* rho, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (c->kernel_shard)
    return fail(SAS_ENOTSUP, "a point-shard context forms partial rows only: sum them over the shards "
                             "and call subapsnap_solve_batch_rows");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!params || !out) return fail(SAS_EINVAL, "params and out must be non-NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  const bool mixed = c->mode == SAS_MODE_MIXED;
  if (c->family == kKernel) return solve_kernel_family(c, params, m, out_kind, out, flags, rho, st);
  if (c->family != kAffine) return fail(SAS_ENOTSUP, "family not supported");
  switch (out_kind) {
    case SAS_OUT_Y: {
      TraceScope ts(c, SAS_KERNEL_LS, st);
      e = mixed ? launch_ls_mixed(c, params, m, out, nullptr, nullptr, flags, rho, st)
                : launch_ls_plain(c, params, m, out, nullptr, flags, rho, st);
      break;
    }
    case SAS_OUT_QOI: {
      if (c->qoi_kind == SAS_QOI_NONE) return fail(SAS_EINVAL, "context was set up without a QoI");
      TraceScope ts(c, SAS_KERNEL_LS, st);
      e = mixed ? launch_ls_mixed(c, params, m, nullptr, out, nullptr, flags, rho, st)
                : launch_ls_plain(c, params, m, nullptr, out, flags, rho, st);
      break;
    }
    case SAS_OUT_XHAT: {
      if (c->dtype != SAS_REAL64) return fail(SAS_ENOTSUP, "x_hat output is real-only");
      sas_status s2 = ensure_scratch(c, m, mixed, st);
      if (s2 != SAS_OK) return s2;
      {
        TraceScope ts(c, SAS_KERNEL_LS, st);
        e = mixed ? launch_ls_mixed(c, params, m, c->ybuf, nullptr,
                                    c->xhat_f32 ? c->ysplit : nullptr, flags, rho, st)
                  : launch_ls_plain(c, params, m, c->ybuf, nullptr, flags, rho, st);
      }
      if (e == cudaSuccess) {
        TraceScope ts(c, SAS_KERNEL_RECONSTRUCT, st);
        if (mixed && c->xhat_f32)
          e = launch_reconstruct_mixed(c, c->ysplit, m, (float*)out, st);
        else if (mixed)
          e = reconstruct_mixed_f64(c, m, (double*)out, st);
        else
          e = launch_reconstruct_f64(c, c->ybuf, m, out, st);
      }
      break;
    }
    default:
      return fail(SAS_EINVAL, "bad out_kind");
  }
  if (e != cudaSuccess) return cuda_fail(e, "solve_batch");
  return SAS_OK;
}

namespace {
// device staging for host-buffer calls, grown on demand (256-byte aligned pieces)
cudaError_t host_stage(sas_ctx* c, size_t bytes, cudaStream_t st) {
  if (bytes <= c->hstage_bytes) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  cudaFree(c->hstage);
  c->hstage = nullptr;
  c->hstage_bytes = 0;
  e = cudaMalloc(&c->hstage, bytes);
  if (e == cudaSuccess) c->hstage_bytes = bytes;
  return e;
}
size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

sas_status subapsnap_solve_batch_host(sas_ctx* c, const double* params, int64_t m, int32_t out_kind,
                                      void* out, uint32_t* flags, double* rho, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!params || !out) return fail(SAS_EINVAL, "params and out must be non-NULL");
  if (is_device_ptr(params) || is_device_ptr(out) || (flags && is_device_ptr(flags)) ||
      (rho && is_device_ptr(rho)))
    return fail(SAS_EINVAL, "solve_batch_host takes host buffers (use subapsnap_solve_batch for device ones)");
  cudaStream_t st = (cudaStream_t)stream;
  const bool mixed = c->mode == SAS_MODE_MIXED;
  const size_t elt = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  size_t out_row;  // bytes of one parameter's output
  if (out_kind == SAS_OUT_Y) out_row = (size_t)c->r * elt;
  else if (out_kind == SAS_OUT_QOI) out_row = elt;
  else if (out_kind == SAS_OUT_XHAT) out_row = (size_t)c->n * (mixed && c->xhat_f32 ? 4 : 8);
  else return fail(SAS_EINVAL, "bad out_kind");
  // x_hat goes straight into the caller's memory when it is page-locked and mapped: the
  // reconstruction's stores then stream over the host link, which is what bounds this path
  void* out_mapped = nullptr;
  if (out_kind == SAS_OUT_XHAT) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost)
      out_mapped = at.devicePointer;
    cudaGetLastError();
  }
  // x_hat into pageable memory: chunks of at most 1 GiB through a device buffer
  int64_t chunk = m;
  if (out_kind == SAS_OUT_XHAT && !out_mapped)
    chunk = std::max<int64_t>(1, std::min<int64_t>(m, (int64_t)(c->host_chunk ? c->host_chunk : (size_t)1 << 30) /
                                                             (int64_t)out_row));
  const size_t pb = align256((size_t)m * c->dp * sizeof(double));
  const size_t fb = align256((size_t)m * sizeof(uint32_t));
  const size_t rb = align256((size_t)m * sizeof(double));
  const size_t ob = out_mapped ? 0 : align256((size_t)chunk * out_row);
  cudaError_t e = host_stage(c, pb + fb + rb + ob, st);
  if (e != cudaSuccess) return cuda_fail(e, "solve_batch_host: staging");
  char* base = (char*)c->hstage;
  double* p_d = (double*)base;
  uint32_t* f_d = flags ? (uint32_t*)(base + pb) : nullptr;
  double* r_d = rho ? (double*)(base + pb + fb) : nullptr;
  void* o_d = out_mapped ? nullptr : (void*)(base + pb + fb + rb);
  e = cudaMemcpyAsync(p_d, params, (size_t)m * c->dp * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && f_d) e = cudaMemsetAsync(f_d, 0, (size_t)m * sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "solve_batch_host: parameters");
  const int saved_store = c->recon_store;
  if (out_mapped) c->recon_store = 1;  // direct stores: no tensor map over host memory
  sas_status rc = SAS_OK;
  for (int64_t q0 = 0; q0 < m && rc == SAS_OK; q0 += chunk) {
    const int64_t mq = std::min<int64_t>(chunk, m - q0);
    void* dst = out_mapped ? (void*)((char*)out_mapped + (size_t)q0 * out_row) : o_d;
    rc = subapsnap_solve_batch(c, p_d + q0 * c->dp, mq, out_kind, dst, f_d ? f_d + q0 : nullptr,
                               r_d ? r_d + q0 : nullptr, stream);
    if (rc == SAS_OK && !out_mapped) {
      e = cudaMemcpyAsync((char*)out + (size_t)q0 * out_row, o_d, (size_t)mq * out_row,
                          cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "solve_batch_host: output copy");
    }
  }
  c->recon_store = saved_store;
  if (rc != SAS_OK) return rc;
  if (f_d) e = cudaMemcpyAsync(flags, f_d, (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && r_d) e = cudaMemcpyAsync(rho, r_d, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "solve_batch_host");
  return SAS_OK;
}

sas_status subapsnap_reconstruct(sas_ctx* c, const void* Y, int64_t m, void* out, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!Y || !out) return fail(SAS_EINVAL, "Y and out must be non-NULL");
  if (c->dtype != SAS_REAL64) return fail(SAS_ENOTSUP, "x_hat output is real-only");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (c->mode == SAS_MODE_MIXED && c->xhat_f32) {
    sas_status s2 = ensure_scratch(c, m, true, st);
    if (s2 != SAS_OK) return s2;
    const int rpad = (c->r + 31) / 32 * 32;
    e = launch_split_y((const double*)Y, m, c->r, rpad, c->ysplit, st);
    if (e == cudaSuccess) {
      TraceScope ts(c, SAS_KERNEL_RECONSTRUCT, st);
      e = launch_reconstruct_mixed(c, c->ysplit, m, (float*)out, st);
    }
  } else if (c->mode == SAS_MODE_MIXED) {
    sas_status s2 = ensure_scratch(c, m, true, st);
    if (s2 != SAS_OK) return s2;
    TraceScope ts(c, SAS_KERNEL_RECONSTRUCT, st);
    if (c->recon_kernel != 1 && reconstruct_x64_supported(c))
      e = launch_reconstruct_x64(c, (const double*)Y, m, (double*)out, c->yx64, st);
    else
      e = launch_reconstruct_f64(c, Y, m, out, st);
  } else {
    TraceScope ts(c, SAS_KERNEL_RECONSTRUCT, st);
    e = launch_reconstruct_f64(c, Y, m, out, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "reconstruct");
  return SAS_OK;
}

sas_status subapsnap_residual(sas_ctx* c, const double* params, int64_t m, const void* Y,
                              double* rho, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!params || !Y || !rho) return fail(SAS_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (c->family == kKernel) {
    // float64 kernel rows, then the residual of the dense M, sub-batch by sub-batch
    const int64_t cap = m < kKernelSubBatch ? m : kKernelSubBatch;
    sas_status s2 = ensure_mbuf(c, cap, st);
    if (s2 != SAS_OK) return s2;
    cudaError_t e = cudaSuccess;
    for (int64_t b0 = 0; b0 < m && e == cudaSuccess; b0 += cap) {
      const int64_t mb = m - b0 < cap ? m - b0 : cap;
      e = launch_krr_assemble(c, params + b0 * 2, mb, c->Mbuf, false, st);
      if (e == cudaSuccess) {
        TraceScope ts(c, SAS_KERNEL_RESIDUAL, st);
        e = launch_residual(c, params + b0 * 2, mb, (const double*)Y + b0 * c->r, rho + b0, st,
                            c->Mbuf);
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "residual");
    return SAS_OK;
  }
  if (c->family != kAffine) return fail(SAS_ENOTSUP, "family not supported");
  TraceScope ts(c, SAS_KERNEL_RESIDUAL, st);
  cudaError_t e = launch_residual(c, params, m, Y, rho, st);
  if (e != cudaSuccess) return cuda_fail(e, "residual");
  return SAS_OK;
}

sas_status subapsnap_true_residual(sas_ctx* c, const double* params, int64_t m, const void* X,
                                   double* rho, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (m < 0) return fail(SAS_EINVAL, "m < 0");
  if (m == 0) return SAS_OK;
  if (!params || !X || !rho) return fail(SAS_EINVAL, "NULL argument");
  if (c->family != kAffine) return fail(SAS_ENOTSUP, "true residual needs the affine family");
  if (m > 65535) return fail(SAS_EINVAL, "at most 65535 parameters per call");
  TraceScope ts(c, SAS_KERNEL_RESIDUAL, (cudaStream_t)stream);
  cudaError_t e = launch_true_residual(c, params, m, X, rho, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "true_residual");
  return SAS_OK;
}

sas_status subapsnap_select_rows_affine(const sas_affine_desc* d, const double* p_sel,
                                        int64_t* J_out, double* gap_out) {
  sas_status st = check_affine_desc(d, false);
  if (st != SAS_OK) return st;
  if (!p_sel || !J_out) return fail(SAS_EINVAL, "p_sel and J_out must be non-NULL");
  return select_rows_affine(d, p_sel, J_out, gap_out);
}

sas_status subapsnap_select_rows_union_affine(const sas_affine_desc* d, const double* points,
                                              int32_t t, int32_t s_each, int64_t* J_out,
                                              int32_t* count_out) {
  if (!d || !points || !J_out || !count_out) return fail(SAS_EINVAL, "NULL argument");
  if (t < 1 || s_each < d->r) return fail(SAS_EINVAL, "need t >= 1 and s_each >= r");
  sas_affine_desc one = *d;
  one.s = s_each;
  sas_status st = check_affine_desc(&one, false);
  if (st != SAS_OK) return st;
  const int dp = d->theta_rule == SAS_THETA_PENCIL ? 1 : d->theta_rule == SAS_THETA_DELAY ? 2 : d->K - 1;
  std::vector<int64_t> picks((size_t)s_each);
  std::vector<char> seen((size_t)d->n, 0);
  int32_t k = 0;
  for (int32_t i = 0; i < t; ++i) {
    st = select_rows_affine(&one, points + (size_t)i * dp, picks.data(), nullptr);
    if (st != SAS_OK) return st;
    for (int64_t j : picks)
      if (!seen[(size_t)j]) {
        seen[(size_t)j] = 1;
        J_out[k++] = j;
      }
  }
  *count_out = k;
  return SAS_OK;
}

sas_status subapsnap_nearest_points(const double* params, int64_t m, int32_t dp,
                                    const double* points, int32_t t, int32_t* idx_out) {
  if (!params || !points || !idx_out) return fail(SAS_EINVAL, "NULL argument");
  if (m < 0 || dp < 1 || t < 1) return fail(SAS_EINVAL, "need m >= 0, dp >= 1, t >= 1");
  for (int64_t q = 0; q < m; ++q) {
    int32_t best = 0;
    double bd = INFINITY;
    for (int32_t i = 0; i < t; ++i) {
      double d2 = 0.0;
      for (int32_t k = 0; k < dp; ++k) {
        const double df = params[q * dp + k] - points[(size_t)i * dp + k];
        d2 += df * df;
      }
      if (d2 < bd) {  // ties go to the lowest index
        bd = d2;
        best = i;
      }
    }
    idx_out[q] = best;
  }
  return SAS_OK;
}

sas_status subapsnap_select_rows_kernel(const sas_kernel_desc* d, const double* p_sel,
                                        int64_t* J_out, double* gap_out) {
  if (!d || !p_sel || !J_out) return fail(SAS_EINVAL, "NULL argument");
  if (d->n < 1 || d->d < 1 || d->d > 16 || d->r < 1 || d->r > kMaxR)
    return fail(SAS_EINVAL, "bad sizes");
  if (d->s < d->r || (int64_t)d->s > d->n) return fail(SAS_EINVAL, "need r <= s <= n");
  if (d->ldS != d->n) return fail(SAS_EINVAL, "select_rows_kernel needs ldS = n");
  if (!is_device_ptr(d->X) || !is_device_ptr(d->S)) return fail(SAS_EINVAL, "X and S must be device pointers");
  if (!(p_sel[0] > 0.0)) return fail(SAS_EINVAL, "sigma must be positive");
  return select_rows_kernel(d, p_sel, J_out, gap_out);
}

sas_status subapsnap_krr_snapshots(const sas_kernel_desc* d, const double* sigma, int32_t ns,
                                   const double* lambda, int32_t nl, double tol, int32_t maxit, double* X,
                                   int64_t ldx, int32_t* iters_out, double* relres_out, void* stream) {
  if (!d || !sigma || !lambda || !X) return fail(SAS_EINVAL, "NULL argument");
  if (d->n < 1 || d->d < 1 || d->d > 16) return fail(SAS_EINVAL, "need n >= 1 and 1 <= d <= 16");
  if (!is_device_ptr(d->X) || !is_device_ptr(d->b) || !is_device_ptr(X))
    return fail(SAS_EINVAL, "X, b and X_out must be device pointers");
  if (ns < 1 || ns > 16 || nl < 1 || nl > 32) return fail(SAS_EINVAL, "need 1 <= nsigma <= 16, 1 <= nlambda <= 32");
  if (ldx < d->n) return fail(SAS_EINVAL, "ldx < N");
  if (!(tol > 0.0) || maxit < 1) return fail(SAS_EINVAL, "need tol > 0 and maxit >= 1");
  for (int i = 0; i < ns; ++i)
    if (!(sigma[i] > 0.0) || !std::isfinite(sigma[i])) return fail(SAS_EINVAL, "sigma must be positive and finite");
  for (int i = 0; i < nl; ++i)
    if (!(lambda[i] > 0.0) || !std::isfinite(lambda[i]))
      return fail(SAS_EINVAL, "lambda must be positive and finite");
  return krr_snapshots(d, sigma, ns, lambda, nl, tol, maxit, X, ldx, iters_out, relres_out,
                       (cudaStream_t)stream);
}

sas_status subapsnap_surrogate_train(sas_ctx* c, const double* P, const double* Y, int64_t ntrain,
                                     int32_t epochs, int32_t batch, double lr, uint64_t seed,
                                     double* loss_out, void* stream) {
  if (!c || !P || !Y) return fail(SAS_EINVAL, "NULL argument");
  if (c->family != kAffine || c->dtype != SAS_REAL64)
    return fail(SAS_ENOTSUP, "the surrogate needs a real affine context");
  if (batch < 1 || ntrain < batch || epochs < 0 || !(lr > 0.0))
    return fail(SAS_EINVAL, "need 1 <= batch <= ntrain, epochs >= 0, lr > 0");
  return surrogate_train(c, P, Y, ntrain, epochs, batch, lr, seed, loss_out, (cudaStream_t)stream);
}

sas_status subapsnap_surrogate_predict(sas_ctx* c, const double* params, int64_t m, double* Yhat,
                                       void* stream) {
  if (!c || !params || !Yhat) return fail(SAS_EINVAL, "NULL argument");
  if (!surrogate_ready(c)) return fail(SAS_EINVAL, "the surrogate is not trained");
  if (m <= 0) return m == 0 ? SAS_OK : fail(SAS_EINVAL, "m < 0");
  cudaStream_t st = (cudaStream_t)stream;
  TraceScope ts(c, SAS_KERNEL_SURROGATE, st);
  cudaError_t e = surrogate_predict(c, params, m, Yhat, st);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate_predict");
  return SAS_OK;
}

sas_status subapsnap_solve_batch_surrogate(sas_ctx* c, const double* params, int64_t m,
                                           int32_t out_kind, void* out, uint32_t* flags,
                                           double* rho, double gate_tol, int64_t* accepted,
                                           void* stream) {
  if (!c || !params || !out) return fail(SAS_EINVAL, "NULL argument");
  if (!surrogate_ready(c)) return fail(SAS_EINVAL, "the surrogate is not trained");
  if (out_kind != SAS_OUT_Y && out_kind != SAS_OUT_QOI)
    return fail(SAS_EINVAL, "the gated solve returns y or the QoI");
  if (out_kind == SAS_OUT_QOI && c->qoi_kind == SAS_QOI_NONE)
    return fail(SAS_EINVAL, "context was set up without a QoI");
  if (m <= 0) {
    if (accepted) *accepted = 0;
    return m == 0 ? SAS_OK : fail(SAS_EINVAL, "m < 0");
  }
  return surrogate_solve(c, params, m, out_kind, out, flags, rho, gate_tol, accepted,
                         (cudaStream_t)stream);
}

sas_status subapsnap_surrogate_reset(sas_ctx* c) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  cudaError_t e = cudaDeviceSynchronize();  // no launch of this context may still read the network
  destroy_surrogate(c);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate_reset");
  return SAS_OK;
}

sas_status subapsnap_surrogate_set_anchors(sas_ctx* c, const double* P, const double* Y, int64_t n) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (c->family != kAffine || c->dtype != SAS_REAL64)
    return fail(SAS_ENOTSUP, "the surrogate needs a real affine context");
  if (n < 0 || (n > 0 && (!P || !Y))) return fail(SAS_EINVAL, "anchors: n < 0 or NULL buffers");
  return surrogate_set_anchors(c, P, Y, n);
}

sas_status subapsnap_surrogate_weights(sas_ctx* c, int32_t get, float* theta, double* norm,
                                       int64_t* nparam) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  if (c->family != kAffine || c->dtype != SAS_REAL64)
    return fail(SAS_ENOTSUP, "the surrogate needs a real affine context");
  if (!c->surrogate) {
    if (get) return fail(SAS_EINVAL, "no surrogate network in this context");
    sas_status s2 = surrogate_create(c, 0);
    if (s2 != SAS_OK) return s2;
  }
  if (nparam) *nparam = surrogate_nparam(c);
  if (!theta && !norm) return SAS_OK;
  return surrogate_io(c, get, theta, norm);
}

sas_status subapsnap_surrogate_grad(sas_ctx* c, const double* X, const double* Yn, int64_t B,
                                    double* loss, float* grads) {
  if (!c || !X || !Yn || !loss || !grads) return fail(SAS_EINVAL, "NULL argument");
  if (!c->surrogate) return fail(SAS_EINVAL, "no surrogate network in this context");
  if (B < 1) return fail(SAS_EINVAL, "B must be positive");
  return surrogate_grad(c, X, Yn, B, loss, grads, 0);
}

struct sas_multi_plan {
  sas::MultiPlan p;
};

sas_status subapsnap_multi_plan_create(sas_ctx* const* ctxs, int32_t nctx,
                                       const double* const* params, const int64_t* m,
                                       int32_t out_kind, void* const* outs,
                                       uint32_t* const* flags, double* const* rho,
                                       sas_multi_plan** plan) {
  if (!plan) return fail(SAS_EINVAL, "plan is NULL");
  *plan = nullptr;
  if (!ctxs || nctx < 1 || !params || !m || !outs) return fail(SAS_EINVAL, "NULL argument");
  if (out_kind != SAS_OUT_Y && out_kind != SAS_OUT_QOI)
    return fail(SAS_EINVAL, "multi plans return y or the QoI");
  for (int i = 0; i < nctx; ++i) {
    const sas_ctx* c = ctxs[i];
    if (!c || c->family != kAffine) return fail(SAS_EINVAL, "every context must be affine");
    if (c->mode != ctxs[0]->mode || c->dtype != ctxs[0]->dtype)
      return fail(SAS_EINVAL, "every context needs the same mode and dtype");
    if (m[i] < 0 || (m[i] > 0 && (!params[i] || !outs[i]))) return fail(SAS_EINVAL, "bad batch");
    if (out_kind == SAS_OUT_QOI && c->qoi_kind == SAS_QOI_NONE)
      return fail(SAS_EINVAL, "a context was set up without a QoI");
  }
  sas_multi_plan* pl = new (std::nothrow) sas_multi_plan();
  if (!pl) return fail(SAS_ENOMEM, "host allocation failed");
  cudaError_t e = multi_plan_build(&pl->p, ctxs, nctx, params, m, out_kind, outs, flags, rho);
  if (e != cudaSuccess) {
    subapsnap_multi_plan_destroy(pl);
    return cuda_fail(e, "multi_plan_create");
  }
  *plan = pl;
  return SAS_OK;
}

sas_status subapsnap_multi_plan_launch(sas_multi_plan* pl, int32_t use_graph, void* stream) {
  if (!pl) return fail(SAS_EINVAL, "plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!use_graph) {
    e = multi_plan_enqueue(&pl->p, st);
  } else {
    if (!pl->p.exec) {
      if (!pl->p.graph_stream) e = cudaStreamCreateWithFlags(&pl->p.graph_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(pl->p.graph_stream, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        cudaError_t e2 = multi_plan_enqueue(&pl->p, pl->p.graph_stream);
        e = cudaStreamEndCapture(pl->p.graph_stream, &pl->p.graph);
        if (e2 != cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->p.exec, pl->p.graph, 0);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(pl->p.exec, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "multi_plan_launch");
  return SAS_OK;
}

void subapsnap_multi_plan_destroy(sas_multi_plan* pl) {
  if (!pl) return;
  if (pl->p.exec) cudaGraphExecDestroy(pl->p.exec);
  if (pl->p.graph) cudaGraphDestroy(pl->p.graph);
  if (pl->p.graph_stream) cudaStreamDestroy(pl->p.graph_stream);
  cudaFree(pl->p.d_probs);
  cudaFree(pl->p.d_offs);
  cudaFree(pl->p.d_counter);
  delete pl;
}

void subapsnap_destroy(sas_ctx* c) { free_ctx(c); }

namespace sas {
static std::string tune_key(const sas_ctx* c, int64_t m) {
  std::ostringstream k;
  k << "family=" << c->family << " mode=" << c->mode << " dtype=" << c->dtype << " s=" << c->s
    << " r=" << c->r << " K=" << c->K << " m=" << m;
  return k.str();
}
static int tune_cache_lookup(const std::string& key) {
  const char* path = std::getenv("SAS_TUNE_CACHE");
  if (!path) return -1;
  std::ifstream f(path);
  std::string line;
  int found = -1;
  while (std::getline(f, line)) {
    const size_t bar = line.rfind(" variant=");
    if (bar != std::string::npos && line.compare(0, bar, key) == 0)
      found = std::atoi(line.c_str() + bar + 9);
  }
  return found;
}
static void tune_cache_store(const std::string& key, int v) {
  const char* path = std::getenv("SAS_TUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " variant=" << v << "\n";
}
}  // namespace sas

sas_status subapsnap_autotune(sas_ctx* c, const double* params, int64_t m, int32_t reps,
                              double* times_ms, int32_t* chosen, void* stream) {
  if (!c || !params) return fail(SAS_EINVAL, "NULL argument");
  if (m < 1) return fail(SAS_EINVAL, "m must be positive");
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  const bool mixed = c->mode == SAS_MODE_MIXED;
  int* var = mixed ? &c->ls_variant_mixed : &c->ls_variant_plain;
  const int nv = ls_num_variants(mixed);
  if (times_ms)
    for (int v = 0; v < SAS_MAX_VARIANTS; ++v) times_ms[v] = -1.0;
  const std::string key = tune_key(c, m);
  const int cached = tune_cache_lookup(key);
  if (cached >= 0 && cached < nv) {
    *var = cached;
    if (chosen) *chosen = cached;
    return SAS_OK;
  }
  void* Y = nullptr;
  const size_t es = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  cudaError_t e = cudaMalloc(&Y, (size_t)m * c->r * es);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int keep = *var;
  int best = keep;
  double best_ms = 1e300;
  const int tr = c->tracing;
  c->tracing = 0;
  for (int v = 0; v < nv; ++v) {
    *var = v;
    sas_status s0 = subapsnap_solve_batch(c, params, m, SAS_OUT_Y, Y, nullptr, nullptr, st);
    if (s0 != SAS_OK || cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps; ++k) subapsnap_solve_batch(c, params, m, SAS_OUT_Y, Y, nullptr, nullptr, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / reps;
    if (times_ms && v < SAS_MAX_VARIANTS) times_ms[v] = per;
    if (per < best_ms) {
      best_ms = per;
      best = v;
    }
  }
  c->tracing = tr;
  *var = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Y);
  if (chosen) *chosen = best;
  if (best_ms < 1e300) tune_cache_store(key, best);
  return SAS_OK;
}

sas_status subapsnap_output_row_bytes(const sas_ctx* c, int32_t out_kind, int64_t* bytes) {
  if (!c || !bytes) return fail(SAS_EINVAL, "NULL argument");
  const int64_t elt = c->dtype == SAS_COMPLEX128 ? 16 : 8;
  switch (out_kind) {
    case SAS_OUT_Y: *bytes = (int64_t)c->r * elt; return SAS_OK;
    case SAS_OUT_QOI: *bytes = elt; return SAS_OK;
    case SAS_OUT_XHAT:
      *bytes = c->n * (c->mode == SAS_MODE_MIXED && c->xhat_f32 ? 4 : elt);
      return SAS_OK;
    default:
      return fail(SAS_EINVAL, "bad out_kind");
  }
}

sas_status subapsnap_set_option(sas_ctx* c, int32_t key, double value) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  switch (key) {
    case SAS_OPT_RECON_KERNEL:
      if (!(value >= 0.0 && value <= 6.0 && value == (double)(int)value))
        return fail(SAS_EINVAL, "recon kernel must be an integer in [0, 6]");
      c->recon_kernel = (int)value;
      return SAS_OK;
    case SAS_OPT_MAX_REFINE:
      if (!(value >= 0.0 && value <= 16.0)) return fail(SAS_EINVAL, "max refine must be in [0, 16]");
      c->max_refine = (int)value;
      return SAS_OK;
    case SAS_OPT_REFINE_TOL:
      if (!(value > 0.0 && value < 1.0)) return fail(SAS_EINVAL, "refine tol must be in (0, 1)");
      c->refine_tol = value;
      return SAS_OK;
    case SAS_OPT_RECON_STORE:
      if (value != 0.0 && value != 1.0) return fail(SAS_EINVAL, "recon store must be 0 or 1");
      c->recon_store = (int)value;
      return SAS_OK;
    case SAS_OPT_XHAT_F32:
      if (value != 0.0 && value != 1.0) return fail(SAS_EINVAL, "xhat f32 must be 0 or 1");
      if (value == 1.0 && c->mode == SAS_MODE_MIXED && c->dtype == SAS_REAL64 && !c->Shi)
        return fail(SAS_ENOTSUP, "this context has no float32 copy of S");
      c->xhat_f32 = (int)value;
      return SAS_OK;
    case SAS_OPT_SURROGATE_F32_OUT:
      if (value != 0.0 && value != 1.0) return fail(SAS_EINVAL, "surrogate f32 out must be 0 or 1");
      c->surr_f32_out = (int)value;
      return SAS_OK;
    case SAS_OPT_HOST_CHUNK:
      if (!(value >= 1.0 && value <= 1099511627776.0)) return fail(SAS_EINVAL, "host chunk must be in [1, 2^40] bytes");
      c->host_chunk = (size_t)value;
      return SAS_OK;
    case SAS_OPT_ASSEMBLY_SEGMENT:
      if (!(value >= 32.0 && value <= 1048576.0) || std::fmod(value, 32.0) != 0.0)
        return fail(SAS_EINVAL, "assembly segment must be a multiple of 32 in [32, 2^20]");
      c->krr_seg_points = (int)value;
      return SAS_OK;
    case SAS_OPT_ASSEMBLY_KERNEL:
      if (value != 0.0 && value != 1.0 && value != 2.0)
        return fail(SAS_EINVAL, "assembly kernel must be 0, 1 or 2");
      c->krr_kernel = (int)value;
      return SAS_OK;
    case SAS_OPT_LS_VARIANT: {
      const bool mixed = c->mode == SAS_MODE_MIXED;
      const int nv = ls_num_variants(mixed);
      if (!(value >= 0.0 && value < nv)) return fail(SAS_EINVAL, "ls variant out of range");
      (mixed ? c->ls_variant_mixed : c->ls_variant_plain) = (int)value;
      return SAS_OK;
    }
    default:
      return fail(SAS_EINVAL, "unknown option");
  }
}

sas_status subapsnap_set_tracing(sas_ctx* c, int32_t enable) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  c->tracing = enable ? 1 : 0;
  return SAS_OK;
}

sas_status subapsnap_trace_read(sas_ctx* c, int32_t cls, double* total_ms, int64_t* launches) {
  if (!c || !total_ms || !launches) return fail(SAS_EINVAL, "NULL argument");
  if (cls < 0 || cls >= SAS_KERNEL_CLASSES) return fail(SAS_EINVAL, "bad kernel class");
  *total_ms = 0.0;
  *launches = 0;
  if (!c->trace) return SAS_OK;
  std::vector<sas_ctx::TraceRec> keep;
  for (auto& t : *c->trace) {
    if (t.cls != cls) {
      keep.push_back(t);
      continue;
    }
    cudaError_t e = cudaEventSynchronize(t.b);
    if (e != cudaSuccess) return cuda_fail(e, "trace_read");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    *total_ms += ms;
    *launches += 1;
    c->event_pool->push_back(t.a);
    c->event_pool->push_back(t.b);
  }
  c->trace->swap(keep);
  return SAS_OK;
}

sas_status subapsnap_device_status(sas_ctx* c, void* stream) {
  if (!c) return fail(SAS_EINVAL, "context is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device_status");
  int v = 0;
  e = cudaMemcpy(&v, c->dev_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "device_status");
  cudaMemset(c->dev_status, 0, sizeof(int));
  return (sas_status)v;
}

}  // extern "C"
