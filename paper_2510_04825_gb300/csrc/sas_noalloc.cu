// subapsnap_solve_batch_xhat_noalloc: the plain float64 solve with x_hat
// output, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at solve time: a host framework that
// reserves all device memory up front and hands out nothing else, or a
// latency-critical loop where a device allocation (which may synchronise the
// whole device) is not allowed.  The regular entry point grows a scratch
// buffer for the m x r coefficient vectors between the least-squares kernel
// and the reconstruction kernel; this variant stages them in the fixed
// device array below instead, so the call itself allocates nothing (the
// context was set up, and allocated, beforehand).
//
// The array lives in every device that loads the library until the process
// exits (SAS_NOALLOC_MAX_Y doubles = 512 KiB).  Host code only ever sees the
// array's name as a host-side stand-in, so its device address is looked up
// with cudaGetSymbolAddress, with the device current: once at context set-up
// (which also brings the array onto the device, so that no later call makes
// the driver load it) and again at every call, which allocates nothing and
// stays right after a device reset or a new primary context.  Make the first
// call after set-up and before any stream capture.  All calls share the array
// and it keeps the last call's contents; every call overwrites the m x r
// entries it uses before reading them, so nothing has to start at zero.
// Calls whose work overlaps on the GPU (other streams, other host threads)
// race on the array.
#include "sas_internal.cuh"

namespace sas {

static __device__ __align__(256) double g_noalloc_y[SAS_NOALLOC_MAX_Y];

// Device address of g_noalloc_y on the current device.
static cudaError_t noalloc_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_y);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// Context set-up: look the array up once on the current device.
cudaError_t noalloc_prepare() {
  double* p = nullptr;
  return noalloc_address(&p);
}

}  // namespace sas

using namespace sas;

extern "C" sas_status subapsnap_solve_batch_xhat_noalloc(sas_ctx* c, const double* params,
                                                         int64_t m, double* out, uint32_t* flags,
                                                         double* rho, void* stream) {
  if (!c) {
    set_error("context is NULL");
    return SAS_EINVAL;
  }
  if (m < 0) {
    set_error("m < 0");
    return SAS_EINVAL;
  }
  if (m == 0) return SAS_OK;
  if (!params || !out) {
    set_error("params and out must be non-NULL");
    return SAS_EINVAL;
  }
  if (c->family != kAffine || c->dtype != SAS_REAL64) {
    set_error("solve_batch_xhat_noalloc: needs a real affine context");
    return SAS_ENOTSUP;
  }
  if (m * (int64_t)c->r > (int64_t)SAS_NOALLOC_MAX_Y) {
    set_error("solve_batch_xhat_noalloc: m * r = " + std::to_string(m * (int64_t)c->r) +
              " exceeds the fixed scratch of " + std::to_string((int64_t)SAS_NOALLOC_MAX_Y) +
              " coefficients; split the batch");
    return SAS_EINVAL;
  }
  double* ybuf = nullptr;
  cudaError_t e = noalloc_address(&ybuf);
  if (e == cudaSuccess) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = launch_ls_plain(c, params, m, ybuf, nullptr, flags, rho, st);
    if (e == cudaSuccess) e = launch_reconstruct_f64(c, ybuf, m, out, st);
  }
  if (e != cudaSuccess) {
    set_error(std::string("solve_batch_xhat_noalloc: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  return SAS_OK;
}
