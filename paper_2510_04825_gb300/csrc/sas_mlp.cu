// Learned surrogate of the online stage (not in the paper): an MLP
// p -> y(p), d_in -> 256 -> 256 -> r with the exact GELU, trained on
// coefficient vectors the online stage itself produced.  Its predictions are
// accepted only when the subsampled relative residual
// ||M(p) y_hat - b_J|| / ||b_J|| (Sec. 4.3.1's online estimate) is below a
// threshold; the rest fall back to the exact least-squares solve.
//
// Arithmetic: float32 master weights and Adam moments; every matrix product
// (forward, input gradients, weight gradients) runs on the tensor cores
// (tcgen05 kind::f16, bfloat16 operands, float32 accumulation; sas_mlp_tc.cu)
// with bfloat16 copies of the weights and float32 activations split into two
// bfloat16 terms.  Option: the output layer takes its float32 weights (split
// the same way).  Inputs are normalised to [-1, 1] per parameter, outputs
// standardised per component, both from the training set.  Optional anchors
// (parameter points with their coefficient vectors, e.g. the snapshots): the
// network then learns the deviation of y(p) from the coefficient vector of the
// nearest anchor, and predicts that anchor's vector plus its output.
//
// Kernels here: GELU backward, column sums, MSE loss, Adam with the bfloat16
// cast, nearest anchor, and the gather/normalisation helpers.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "sas_internal.cuh"

namespace sas {

namespace mlp {

__device__ inline float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// dZ = dH * gelu'(Z)
__global__ void gelu_backward_kernel(const float* Z, float* dH, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dH[i] *= gelu_grad_f(Z[i]);
}

// db[j] = sum_b dZ[b*ld + j]  (fixed order)
__global__ void colsum_kernel(const float* dZ, int B, int N, int64_t ld, float* db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * ld + j];
  db[j] = s;
}

// dOut = 2 (out - y) / (B r); loss accumulated in double
__global__ void mse_kernel(const float* out, const float* y, int64_t count, float scale, float* dout,
                           double* loss) {
  __shared__ double red[8];
  double part = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = out[i] - y[i];
    dout[i] = 2.0f * d * scale;
    part += (double)d * d;
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w];
    atomicAdd(loss, t * scale);
  }
}

// Adam with bias correction on the float32 masters; refresh the bfloat16 copies.
__global__ void adam_kernel(float* theta, const float* g, float* m, float* v, int64_t count,
                            float lr, float b1, float b2, float eps, float c1, float c2,
                            const int64_t* woff, const int64_t* wlen, int nw, __nv_bfloat16* wbf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[i] = th;
    int64_t acc = 0;
    for (int w = 0; w < nw; ++w) {
      if (i >= woff[w] && i < woff[w] + wlen[w]) wbf[acc + (i - woff[w])] = __float2bfloat16(th);
      acc += wlen[w];
    }
  }
}

__global__ void cast_weights_kernel(const float* theta, const int64_t* woff, const int64_t* wlen,
                                    int nw, int64_t total, __nv_bfloat16* wbf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t acc = 0;
    for (int w = 0; w < nw; ++w) {
      if (i < acc + wlen[w]) {
        wbf[i] = __float2bfloat16(theta[woff[w] + (i - acc)]);
        break;
      }
      acc += wlen[w];
    }
  }
}

// X[b][k] = (P[idx[b]][k] - center[k]) / scale[k] (float32); Yn likewise with mean/std
__global__ void gather_normalise_kernel(const double* src, int64_t ld, const int64_t* idx, int B,
                                        int cols, const double* shift, const double* scale,
                                        float* dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)B * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / cols), k = (int)(t % cols);
    const int64_t row = idx ? idx[b] : b;
    dst[t] = (float)((src[row * ld + k] - shift[k]) / scale[k]);
  }
}

// y_hat[b][k] = mean[k] + std[k] * out[b][k] (float64), plus the nearest anchor's
// coefficient vector aY[nn[b]][k] when anchors are in use
__global__ void denormalise_kernel(const float* out, int B, int cols, const double* mean,
                                   const double* sd, const int64_t* nn, const double* aY, double* y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)B * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / cols;
    const int k = (int)(t % cols);
    double v = mean[k] + sd[k] * (double)out[t];
    if (nn) v += aY[nn[b] * cols + k];
    y[t] = v;
  }
}

// nn[b] = the anchor a nearest to P[b] in the network's input scaling:
// argmin_a sum_k ((P[b][k] - A[a][k]) / scale[k])^2, the lowest index on ties.
__global__ void nearest_anchor_kernel(const double* P, int64_t m, int din, const double* A,
                                      int64_t na, const double* scale, int64_t* nn) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
       b += (int64_t)gridDim.x * blockDim.x) {
    double best = 0.0;
    int64_t arg = -1;
    for (int64_t a = 0; a < na; ++a) {
      double d2 = 0.0;
      for (int k = 0; k < din; ++k) {
        const double d = (P[b * din + k] - A[a * din + k]) / scale[k];
        d2 += d * d;
      }
      if (arg < 0 || d2 < best) {
        best = d2;
        arg = a;
      }
    }
    nn[b] = arg;
  }
}

// D[b][k] = Y[b][k] - aY[nn[b]][k]
__global__ void deviation_kernel(const double* Y, int64_t m, int cols, const int64_t* nn,
                                 const double* aY, double* D) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m * cols;
       t += (int64_t)gridDim.x * blockDim.x)
    D[t] = Y[t] - aY[nn[t / cols] * cols + (t % cols)];
}

}  // namespace mlp

// ------------------------------------------------------------------ state
struct Surrogate {
  int din = 0, h = 256, dout = 0;
  int64_t nparam = 0;
  int64_t off[6] = {};  // W1 b1 W2 b2 W3 b3 in theta
  float* theta = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wbf = nullptr;  // W1 | W2 | W3
  int64_t* woff = nullptr;       // device: offsets of W1, W2, W3 in theta
  int64_t* wlen = nullptr;
  double* norm = nullptr;        // device: in_center[din], in_scale[din], out_mean[dout], out_sd[dout]
  int64_t t = 0;
  // activation buffers for up to cap rows
  int64_t cap = 0;
  float *X = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *O = nullptr;
  float *Yn = nullptr, *dO = nullptr, *dH = nullptr;
  int64_t* idx = nullptr;  // nearest anchor of each row of a prediction chunk
  double* loss = nullptr;
  bool trained = false;
  int f32_out = 0;              // output layer with the float32 weights (hi + lo bfloat16)
  float* part = nullptr;        // split-K partial tiles of the weight gradients
  int64_t part_cap = 0;
  int* status = nullptr;        // the context's device status word (bounded waits)
  double* aP = nullptr;         // anchors the network was trained with: na x din, na x dout
  double* aY = nullptr;
  int64_t na = 0;
};

static void free_surrogate(Surrogate* s) {
  if (!s) return;
  for (void* p : {(void*)s->theta, (void*)s->grad, (void*)s->m, (void*)s->v, (void*)s->wbf,
                  (void*)s->woff, (void*)s->wlen, (void*)s->norm, (void*)s->X, (void*)s->Z1,
                  (void*)s->H1, (void*)s->Z2, (void*)s->H2, (void*)s->O, (void*)s->Yn,
                  (void*)s->dO, (void*)s->dH, (void*)s->idx, (void*)s->loss, (void*)s->part,
                  (void*)s->aP, (void*)s->aY})
    cudaFree(p);
  delete s;
}

void destroy_surrogate(sas_ctx* c) {
  free_surrogate(static_cast<Surrogate*>(c->surrogate));
  c->surrogate = nullptr;
}

static cudaError_t ensure_acts(Surrogate* s, int64_t rows) {
  if (rows <= s->cap) return cudaSuccess;
  for (float** p : {&s->X, &s->Z1, &s->H1, &s->Z2, &s->H2, &s->O, &s->Yn, &s->dO, &s->dH}) {
    cudaFree(*p);
    *p = nullptr;
  }
  cudaFree(s->idx);
  s->idx = nullptr;
  const int64_t hw = std::max<int64_t>(s->h, std::max(s->din, s->dout));
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&s->X, sizeof(float) * rows * s->din);
  e = e ? e : cudaMalloc(&s->Z1, sizeof(float) * rows * s->h);
  e = e ? e : cudaMalloc(&s->H1, sizeof(float) * rows * s->h);
  e = e ? e : cudaMalloc(&s->Z2, sizeof(float) * rows * s->h);
  e = e ? e : cudaMalloc(&s->H2, sizeof(float) * rows * s->h);
  e = e ? e : cudaMalloc(&s->O, sizeof(float) * rows * s->dout);
  e = e ? e : cudaMalloc(&s->Yn, sizeof(float) * rows * s->dout);
  e = e ? e : cudaMalloc(&s->dO, sizeof(float) * rows * s->dout);
  e = e ? e : cudaMalloc(&s->dH, sizeof(float) * rows * hw);
  e = e ? e : cudaMalloc(&s->idx, sizeof(int64_t) * rows);
  if (e == cudaSuccess) s->cap = rows;
  return e;
}

static cudaError_t refresh_bf16(Surrogate* s, cudaStream_t st) {
  const int64_t total = (int64_t)s->h * s->din + (int64_t)s->h * s->h + (int64_t)s->dout * s->h;
  mlp::cast_weights_kernel<<<256, 256, 0, st>>>(s->theta, s->woff, s->wlen, 3, total, s->wbf);
  return cudaGetLastError();
}

// Create the network with N(0, 1/fan_in) weights and zero biases (host RNG, seeded).
sas_status surrogate_create(sas_ctx* c, uint64_t seed) {
  destroy_surrogate(c);
  Surrogate* s = new Surrogate();
  s->din = c->dp;
  s->dout = c->r;
  const int din = s->din, h = s->h, dout = s->dout;
  const int64_t sizes[6] = {(int64_t)h * din, h, (int64_t)h * h, h, (int64_t)dout * h, dout};
  int64_t o = 0;
  for (int k = 0; k < 6; ++k) {
    s->off[k] = o;
    o += sizes[k];
  }
  s->nparam = o;
  std::vector<float> host(o, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  const int fan[3] = {din, h, h};
  for (int l = 0; l < 3; ++l)
    for (int64_t i = 0; i < sizes[2 * l]; ++i)
      host[s->off[2 * l] + i] = (float)(nd(rng) / std::sqrt((double)fan[l]));
  const int64_t woff[3] = {s->off[0], s->off[2], s->off[4]};
  const int64_t wlen[3] = {sizes[0], sizes[2], sizes[4]};
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&s->theta, sizeof(float) * o);
  e = e ? e : cudaMalloc(&s->grad, sizeof(float) * o);
  e = e ? e : cudaMalloc(&s->m, sizeof(float) * o);
  e = e ? e : cudaMalloc(&s->v, sizeof(float) * o);
  e = e ? e : cudaMalloc(&s->wbf, sizeof(__nv_bfloat16) * (wlen[0] + wlen[1] + wlen[2]));
  e = e ? e : cudaMalloc(&s->woff, sizeof(woff));
  e = e ? e : cudaMalloc(&s->wlen, sizeof(wlen));
  e = e ? e : cudaMalloc(&s->norm, sizeof(double) * 2 * (din + dout));
  e = e ? e : cudaMalloc(&s->loss, sizeof(double));
  s->part_cap = 32 * std::max<int64_t>((int64_t)h * h, std::max<int64_t>((int64_t)h * din, (int64_t)dout * h));
  e = e ? e : cudaMalloc(&s->part, sizeof(float) * s->part_cap);
  s->status = c->dev_status;
  e = e ? e : cudaMemcpy(s->theta, host.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  e = e ? e : cudaMemset(s->m, 0, sizeof(float) * o);
  e = e ? e : cudaMemset(s->v, 0, sizeof(float) * o);
  e = e ? e : cudaMemcpy(s->woff, woff, sizeof(woff), cudaMemcpyHostToDevice);
  e = e ? e : cudaMemcpy(s->wlen, wlen, sizeof(wlen), cudaMemcpyHostToDevice);
  std::vector<double> norm(2 * (din + dout));
  for (int k = 0; k < din; ++k) {
    norm[k] = 0.0;
    norm[din + k] = 1.0;
  }
  for (int k = 0; k < dout; ++k) {
    norm[2 * din + k] = 0.0;
    norm[2 * din + dout + k] = 1.0;
  }
  e = e ? e : cudaMemcpy(s->norm, norm.data(), sizeof(double) * norm.size(), cudaMemcpyHostToDevice);
  e = e ? e : refresh_bf16(s, 0);
  e = e ? e : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_surrogate(s);
    set_error(std::string("surrogate: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
  }
  c->surrogate = s;
  return SAS_OK;
}

// C = A B on the tensor cores (A float32; B float32 or bfloat16 by tb).
static cudaError_t mm(Surrogate* s, cudaStream_t st, int M, int N, int K, const float* A, int64_t lai,
                      int64_t lak, const void* B, int tb, int64_t lbk, int64_t lbj, float* C,
                      int64_t ldc, int epi = 0, const float* bias = nullptr, float* H = nullptr) {
  return mlp_gemm_tc(st, s->part, s->part_cap, s->status, M, N, K, A, kMlpF32, lai, lak, B, tb, lbk,
                     lbj, C, ldc, epi, bias, H);
}

// The output layer's weights as the products read them: the bfloat16 copy, or the float32
// masters when the float32 output layer is chosen.
static const void* w3_operand(const Surrogate* s, int* tb) {
  *tb = s->f32_out ? kMlpF32 : kMlpBF16;
  if (s->f32_out) return s->theta + s->off[4];
  return s->wbf + (int64_t)s->h * s->din + (int64_t)s->h * s->h;
}

// Forward pass on rows already normalised in s->X (float32); output in s->O.  keep_z: also
// store the pre-activations Z1, Z2 (training needs them; inference writes H1, H2 only).
static cudaError_t forward(Surrogate* s, int64_t B, cudaStream_t st, bool keep_z = true) {
  const __nv_bfloat16* W1 = s->wbf;
  const __nv_bfloat16* W2 = W1 + (int64_t)s->h * s->din;
  int t3 = kMlpBF16;
  const void* W3 = w3_operand(s, &t3);
  const int din = s->din, h = s->h, dout = s->dout;
  const int ep = keep_z ? 1 : 3;
  cudaError_t e = mm(s, st, (int)B, h, din, s->X, din, 1, W1, kMlpBF16, 1, din, keep_z ? s->Z1 : s->H1,
                     h, ep, s->theta + s->off[1], s->H1);
  if (e == cudaSuccess)
    e = mm(s, st, (int)B, h, h, s->H1, h, 1, W2, kMlpBF16, 1, h, keep_z ? s->Z2 : s->H2, h, ep,
           s->theta + s->off[3], s->H2);
  if (e == cudaSuccess)
    e = mm(s, st, (int)B, dout, h, s->H2, h, 1, W3, t3, 1, h, s->O, dout, 2, s->theta + s->off[5]);
  return e;
}

// Loss and gradients (into s->grad) for the normalised batch in s->X / s->Yn.
static cudaError_t forward_backward(Surrogate* s, int64_t B, cudaStream_t st) {
  const __nv_bfloat16* W1 = s->wbf;
  const __nv_bfloat16* W2 = W1 + (int64_t)s->h * s->din;
  int t3 = kMlpBF16;
  const void* W3 = w3_operand(s, &t3);
  const int din = s->din, h = s->h, dout = s->dout;
  float* g = s->grad;
  cudaError_t e = forward(s, B, st);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(s->loss, 0, sizeof(double), st);
  mlp::mse_kernel<<<64, 256, 0, st>>>(s->O, s->Yn, B * dout, 1.0f / (float)(B * dout), s->dO, s->loss);
  // layer 3: dW3 = dO^T H2, db3 = colsum dO, dH2 = dO W3
  e = mm(s, st, dout, h, (int)B, s->dO, 1, dout, s->H2, kMlpF32, h, 1, g + s->off[4], h);
  if (e != cudaSuccess) return e;
  mlp::colsum_kernel<<<(dout + 255) / 256, 256, 0, st>>>(s->dO, (int)B, dout, dout, g + s->off[5]);
  e = mm(s, st, (int)B, h, dout, s->dO, dout, 1, W3, t3, h, 1, s->dH, h);
  if (e != cudaSuccess) return e;
  mlp::gelu_backward_kernel<<<256, 256, 0, st>>>(s->Z2, s->dH, B * h);
  // layer 2: dW2 = dZ2^T H1, db2 = colsum dZ2
  e = mm(s, st, h, h, (int)B, s->dH, 1, h, s->H1, kMlpF32, h, 1, g + s->off[2], h);
  if (e != cudaSuccess) return e;
  mlp::colsum_kernel<<<(h + 255) / 256, 256, 0, st>>>(s->dH, (int)B, h, h, g + s->off[3]);
  // dH1 = dZ2 W2 (into H2, whose values are no longer needed)
  e = mm(s, st, (int)B, h, h, s->dH, h, 1, W2, kMlpBF16, h, 1, s->H2, h);
  if (e != cudaSuccess) return e;
  mlp::gelu_backward_kernel<<<256, 256, 0, st>>>(s->Z1, s->H2, B * h);
  // layer 1: dW1 = dZ1^T X, db1 = colsum dZ1
  e = mm(s, st, h, din, (int)B, s->H2, 1, h, s->X, kMlpF32, din, 1, g + s->off[0], din);
  if (e != cudaSuccess) return e;
  mlp::colsum_kernel<<<(h + 255) / 256, 256, 0, st>>>(s->H2, (int)B, h, h, g + s->off[1]);
  return cudaGetLastError();
}

sas_status surrogate_train(sas_ctx* c, const double* P, const double* Y, int64_t ntrain,
                           int epochs, int batch, double lr, uint64_t seed, double* loss_out,
                           cudaStream_t st) {
  Surrogate* s = static_cast<Surrogate*>(c->surrogate);
  if (!s) {
    sas_status r = surrogate_create(c, seed);
    if (r != SAS_OK) return r;
    s = static_cast<Surrogate*>(c->surrogate);
  }
  const int din = s->din, dout = s->dout;
  s->f32_out = c->surr_f32_out;
  // the network keeps its own copy of the context's anchors (none: it learns y itself)
  cudaError_t e = cudaSuccess;
  cudaFree(s->aP);
  cudaFree(s->aY);
  s->aP = s->aY = nullptr;
  s->na = 0;
  if (c->surr_na > 0) {
    e = cudaMalloc(&s->aP, sizeof(double) * c->surr_na * din);
    if (e == cudaSuccess) e = cudaMalloc(&s->aY, sizeof(double) * c->surr_na * dout);
    if (e == cudaSuccess)
      e = cudaMemcpy(s->aP, c->surr_aP, sizeof(double) * c->surr_na * din, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(s->aY, c->surr_aY, sizeof(double) * c->surr_na * dout, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) s->na = c->surr_na;
  }
  // normalisation of the inputs from the training set (host pass over P)
  std::vector<double> hp((size_t)ntrain * din), hy((size_t)ntrain * dout);
  if (e == cudaSuccess) e = cudaMemcpy(hp.data(), P, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost);
  std::vector<double> norm(2 * (din + dout));
  for (int k = 0; k < din && e == cudaSuccess; ++k) {
    double lo = hp[k], hi = hp[k];
    for (int64_t i = 0; i < ntrain; ++i) {
      lo = std::min(lo, hp[i * din + k]);
      hi = std::max(hi, hp[i * din + k]);
    }
    norm[k] = 0.5 * (lo + hi);
    norm[din + k] = hi > lo ? 0.5 * (hi - lo) : 1.0;
  }
  // targets: y, or its deviation from the nearest anchor's coefficient vector
  const double* Yt = Y;
  double* dev = nullptr;
  int64_t* dnn = nullptr;
  if (e == cudaSuccess && s->na > 0) {
    e = cudaMemcpy(s->norm, norm.data(), sizeof(double) * 2 * din, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&dnn, sizeof(int64_t) * ntrain);
    if (e == cudaSuccess) e = cudaMalloc(&dev, sizeof(double) * ntrain * dout);
    if (e == cudaSuccess) {
      mlp::nearest_anchor_kernel<<<(int)std::min<int64_t>(1024, (ntrain + 127) / 128), 128>>>(
          P, ntrain, din, s->aP, s->na, s->norm + din, dnn);
      mlp::deviation_kernel<<<256, 256>>>(Y, ntrain, dout, dnn, s->aY, dev);
      e = cudaGetLastError();
    }
    Yt = dev;
  }
  if (e == cudaSuccess) e = cudaMemcpy(hy.data(), Yt, sizeof(double) * hy.size(), cudaMemcpyDeviceToHost);
  cudaFree(dnn);
  if (e != cudaSuccess) {
    cudaFree(dev);
    set_error(std::string("surrogate_train: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
  }
  for (int k = 0; k < dout; ++k) {
    double mu = 0.0, sq = 0.0;
    for (int64_t i = 0; i < ntrain; ++i) mu += hy[i * dout + k];
    mu /= (double)ntrain;
    for (int64_t i = 0; i < ntrain; ++i) sq += (hy[i * dout + k] - mu) * (hy[i * dout + k] - mu);
    const double sd = std::sqrt(sq / (double)ntrain);
    norm[2 * din + k] = mu;
    norm[2 * din + dout + k] = sd > 0.0 ? sd : 1.0;
  }
  e = cudaMemcpy(s->norm, norm.data(), sizeof(double) * norm.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ensure_acts(s, batch);
  if (e != cudaSuccess) {
    cudaFree(dev);
    set_error(std::string("surrogate_train: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
  }
  const double* in_c = s->norm;
  const double* in_s = s->norm + din;
  const double* out_m = s->norm + 2 * din;
  const double* out_s = s->norm + 2 * din + dout;
  std::vector<int64_t> perm(ntrain);
  std::iota(perm.begin(), perm.end(), 0);
  std::mt19937_64 rng(seed ^ 0x9e3779b97f4a7c15ull);
  int64_t* dperm = nullptr;
  e = cudaMalloc(&dperm, sizeof(int64_t) * ntrain);
  const float b1 = 0.9f, b2 = 0.999f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    e = cudaMemcpyAsync(dperm, perm.data(), sizeof(int64_t) * ntrain, cudaMemcpyHostToDevice, st);
    double ep_loss = 0.0;
    int64_t nb = 0;
    for (int64_t b0 = 0; b0 + batch <= ntrain && e == cudaSuccess; b0 += batch, ++nb) {
      mlp::gather_normalise_kernel<<<128, 256, 0, st>>>(P, din, dperm + b0, batch, din, in_c, in_s, s->X);
      mlp::gather_normalise_kernel<<<128, 256, 0, st>>>(Yt, dout, dperm + b0, batch, dout, out_m, out_s,
                                                         s->Yn);
      e = forward_backward(s, batch, st);
      if (e != cudaSuccess) break;
      s->t += 1;
      const float c1 = 1.f - std::pow(b1, (float)s->t), c2 = 1.f - std::pow(b2, (float)s->t);
      mlp::adam_kernel<<<256, 256, 0, st>>>(s->theta, s->grad, s->m, s->v, s->nparam, (float)lr, b1, b2,
                                            1e-8f, c1, c2, s->woff, s->wlen, 3, s->wbf);
      e = cudaGetLastError();
      if (loss_out) {
        double l = 0.0;
        cudaMemcpyAsync(&l, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        ep_loss += l;
      }
    }
    if (loss_out) loss_out[ep] = nb ? ep_loss / nb : 0.0;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dperm);
  cudaFree(dev);
  if (e != cudaSuccess) {
    set_error(std::string("surrogate_train: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  s->trained = true;
  return SAS_OK;
}

cudaError_t surrogate_predict(sas_ctx* c, const double* params, int64_t m, double* Yhat,
                              cudaStream_t st) {
  Surrogate* s = static_cast<Surrogate*>(c->surrogate);
  const int din = s->din, dout = s->dout;
  s->f32_out = c->surr_f32_out;
  const int64_t chunk = 65536;
  cudaError_t e = ensure_acts(s, std::min<int64_t>(m, chunk));
  for (int64_t b0 = 0; b0 < m && e == cudaSuccess; b0 += chunk) {
    const int64_t B = std::min<int64_t>(chunk, m - b0);
    mlp::gather_normalise_kernel<<<256, 256, 0, st>>>(params + b0 * din, din, nullptr, (int)B, din,
                                                       s->norm, s->norm + din, s->X);
    if (s->na > 0)
      mlp::nearest_anchor_kernel<<<(int)std::min<int64_t>(1024, (B + 127) / 128), 128, 0, st>>>(
          params + b0 * din, B, din, s->aP, s->na, s->norm + din, s->idx);
    e = forward(s, B, st, false);
    if (e != cudaSuccess) break;
    mlp::denormalise_kernel<<<1024, 256, 0, st>>>(s->O, (int)B, dout, s->norm + 2 * din,
                                                  s->norm + 2 * din + dout, s->na > 0 ? s->idx : nullptr,
                                                  s->aY, Yhat + b0 * dout);
    e = cudaGetLastError();
  }
  return e;
}

// One forward/backward on a given normalised batch (device float64 X, Yn) for
// gradient checks: loss (host) and gradients (host, float32, theta layout).
sas_status surrogate_grad(sas_ctx* c, const double* X, const double* Yn, int64_t B, double* loss,
                          float* grads_host, cudaStream_t st) {
  Surrogate* s = static_cast<Surrogate*>(c->surrogate);
  if (!s) return SAS_EINVAL;
  s->f32_out = c->surr_f32_out;
  cudaError_t e = ensure_acts(s, B);
  if (e == cudaSuccess) {
    std::vector<double> zero(std::max(s->din, s->dout), 0.0), one(std::max(s->din, s->dout), 1.0);
    double *dz = nullptr, *d1 = nullptr;
    e = cudaMalloc(&dz, sizeof(double) * zero.size());
    if (e == cudaSuccess) e = cudaMalloc(&d1, sizeof(double) * one.size());
    if (e == cudaSuccess) e = cudaMemcpy(dz, zero.data(), sizeof(double) * zero.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d1, one.data(), sizeof(double) * one.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      mlp::gather_normalise_kernel<<<64, 256, 0, st>>>(X, s->din, nullptr, (int)B, s->din, dz, d1, s->X);
      mlp::gather_normalise_kernel<<<64, 256, 0, st>>>(Yn, s->dout, nullptr, (int)B, s->dout, dz, d1, s->Yn);
      e = forward_backward(s, B, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(grads_host, s->grad, sizeof(float) * s->nparam, cudaMemcpyDeviceToHost);
    cudaFree(dz);
    cudaFree(d1);
  }
  if (e != cudaSuccess) {
    set_error(std::string("surrogate_grad: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  return SAS_OK;
}

// Copy parameters (float32 masters, theta layout) and the normalisation
// (float64: in_center, in_scale, out_mean, out_sd) out of or into the network.
sas_status surrogate_io(sas_ctx* c, int get, float* theta, double* norm) {
  Surrogate* s = static_cast<Surrogate*>(c->surrogate);
  if (!s) return SAS_EINVAL;
  cudaError_t e = cudaSuccess;
  const size_t nn = 2 * (size_t)(s->din + s->dout);
  if (get) {
    if (theta) e = cudaMemcpy(theta, s->theta, sizeof(float) * s->nparam, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && norm) e = cudaMemcpy(norm, s->norm, sizeof(double) * nn, cudaMemcpyDeviceToHost);
  } else {
    if (theta) e = cudaMemcpy(s->theta, theta, sizeof(float) * s->nparam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && norm) e = cudaMemcpy(s->norm, norm, sizeof(double) * nn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = refresh_bf16(s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    s->trained = true;
  }
  if (e != cudaSuccess) {
    set_error(std::string("surrogate weights: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  return SAS_OK;
}

// Anchors for the next training: device P (n x dp) and Y (n x r), copied into buffers the
// context owns; n = 0 clears them.
sas_status surrogate_set_anchors(sas_ctx* c, const double* P, const double* Y, int64_t n) {
  cudaFree(c->surr_aP);
  cudaFree(c->surr_aY);
  c->surr_aP = c->surr_aY = nullptr;
  c->surr_na = 0;
  if (n == 0) return SAS_OK;
  cudaError_t e = cudaMalloc(&c->surr_aP, sizeof(double) * n * c->dp);
  if (e == cudaSuccess) e = cudaMalloc(&c->surr_aY, sizeof(double) * n * c->r);
  if (e == cudaSuccess) e = cudaMemcpy(c->surr_aP, P, sizeof(double) * n * c->dp, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->surr_aY, Y, sizeof(double) * n * c->r, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    cudaFree(c->surr_aP);
    cudaFree(c->surr_aY);
    c->surr_aP = c->surr_aY = nullptr;
    set_error(std::string("surrogate anchors: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SAS_ENOMEM : SAS_ECUDA;
  }
  c->surr_na = n;
  return SAS_OK;
}

int64_t surrogate_nparam(const sas_ctx* c) {
  const Surrogate* s = static_cast<const Surrogate*>(c->surrogate);
  return s ? s->nparam : 0;
}

bool surrogate_ready(const sas_ctx* c) {
  const Surrogate* s = static_cast<const Surrogate*>(c->surrogate);
  return s && s->trained;
}

}  // namespace sas

// ---------------------------------------------------------------- the gate
namespace sas {

namespace gate {

// Rejected indices (rho > tol or not finite) in increasing order; count in *nrej.
__global__ void compact_kernel(const double* rho, int64_t m, double tol, int64_t* rej, int64_t* nrej) {
  __shared__ int64_t scan[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t per = (m + T - 1) / T;
  const int64_t a = (int64_t)t * per, b = a + per < m ? a + per : m;
  int64_t cnt = 0;
  for (int64_t i = a; i < b; ++i) cnt += !(rho[i] <= tol);
  scan[t] = cnt;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {  // inclusive scan (Hillis-Steele)
    const int64_t v = t >= o ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int64_t pos = scan[t] - cnt;
  for (int64_t i = a; i < b; ++i)
    if (!(rho[i] <= tol)) rej[pos++] = i;
  if (t == T - 1) *nrej = scan[T - 1];
}

__global__ void gather_rows_kernel(const double* src, int cols, const int64_t* idx, int64_t n,
                                   double* dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * cols;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[idx[t / cols] * cols + t % cols];
}

// scatter compact results back: Y rows, rho and flags (flags marks fallbacks)
__global__ void scatter_kernel(const double* Yc, const double* rhoc, const uint32_t* flc, int cols,
                               const int64_t* idx, int64_t n, double* Y, double* rho,
                               uint32_t* flags) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / cols;
    const int k = (int)(t % cols);
    Y[idx[q] * cols + k] = Yc[t];
    if (k == 0) {
      if (rho) rho[idx[q]] = rhoc[q];
      if (flags) flags[idx[q]] = flc[q] | SAS_FLAG_FALLBACK;
    }
  }
}

__global__ void mark_accepted_kernel(const double* rho, int64_t m, double tol, uint32_t* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    if (rho[i] <= tol) flags[i] = SAS_FLAG_SURROGATE;
}

// h_q = w . y_q (real)
__global__ void qoi_kernel(const double* Y, int64_t m, int r, const double* w, double* h) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m;
       q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += w[k] * Y[q * r + k];
    h[q] = s;
  }
}

}  // namespace gate

// Gated solve: predict, gate by the float64 subsampled residual, exact LS for
// the rejected parameters.  Returns the number accepted.
sas_status surrogate_solve(sas_ctx* c, const double* params, int64_t m, int32_t out_kind, void* out,
                           uint32_t* flags, double* rho_out, double tol, int64_t* accepted,
                           cudaStream_t st) {
  const int r = c->r, dp = c->dp;
  // scratch: Yhat (m x r), rho (m), rejected list, compact params / Y / rho / flags
  double *Yh = nullptr, *rh = nullptr, *Pc = nullptr, *Yc = nullptr, *rc = nullptr;
  int64_t *rej = nullptr, *nrej_d = nullptr;
  uint32_t* fc = nullptr;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMallocAsync((void**)&Yh, sizeof(double) * m * r, st);
  e = e ? e : cudaMallocAsync((void**)&rh, sizeof(double) * m, st);
  e = e ? e : cudaMallocAsync((void**)&rej, sizeof(int64_t) * m, st);
  e = e ? e : cudaMallocAsync((void**)&nrej_d, sizeof(int64_t), st);
  if (e == cudaSuccess) {
    TraceScope ts(c, SAS_KERNEL_SURROGATE, st);
    e = surrogate_predict(c, params, m, Yh, st);
  }
  if (e == cudaSuccess) {
    TraceScope ts(c, SAS_KERNEL_RESIDUAL, st);
    e = launch_residual(c, params, m, Yh, rh, st);
  }
  int64_t nrej = 0;
  if (e == cudaSuccess) {
    gate::compact_kernel<<<1, 1024, 0, st>>>(rh, m, tol, rej, nrej_d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nrej, nrej_d, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess && flags) {
    cudaMemsetAsync(flags, 0, sizeof(uint32_t) * m, st);
    gate::mark_accepted_kernel<<<256, 256, 0, st>>>(rh, m, tol, flags);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && nrej > 0) {
    e = e ? e : cudaMallocAsync((void**)&Pc, sizeof(double) * nrej * dp, st);
    e = e ? e : cudaMallocAsync((void**)&Yc, sizeof(double) * nrej * r, st);
    e = e ? e : cudaMallocAsync((void**)&rc, sizeof(double) * nrej, st);
    e = e ? e : cudaMallocAsync((void**)&fc, sizeof(uint32_t) * nrej, st);
    if (e == cudaSuccess) {
      gate::gather_rows_kernel<<<256, 256, 0, st>>>(params, dp, rej, nrej, Pc);
      TraceScope ts(c, SAS_KERNEL_LS, st);
      e = c->mode == SAS_MODE_MIXED
              ? launch_ls_mixed(c, Pc, nrej, Yc, nullptr, nullptr, fc, rc, st)
              : launch_ls_plain(c, Pc, nrej, Yc, nullptr, fc, rc, st);
    }
    if (e == cudaSuccess) {
      gate::scatter_kernel<<<256, 256, 0, st>>>(Yc, rc, fc, r, rej, nrej, Yh, rh, flags);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && rho_out) e = cudaMemcpyAsync(rho_out, rh, sizeof(double) * m, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    if (out_kind == SAS_OUT_Y) {
      e = cudaMemcpyAsync(out, Yh, sizeof(double) * m * r, cudaMemcpyDeviceToDevice, st);
    } else if (out_kind == SAS_OUT_QOI) {
      gate::qoi_kernel<<<256, 256, 0, st>>>(Yh, m, r, (const double*)c->wq, (double*)out);
      e = cudaGetLastError();
    } else {
      e = cudaErrorInvalidValue;
    }
  }
  for (void* p : {(void*)Yh, (void*)rh, (void*)rej, (void*)nrej_d, (void*)Pc, (void*)Yc, (void*)rc, (void*)fc})
    if (p) cudaFreeAsync(p, st);
  if (e != cudaSuccess) {
    set_error(std::string("solve_batch_surrogate: ") + cudaGetErrorString(e));
    return SAS_ECUDA;
  }
  if (accepted) *accepted = m - nrej;
  return SAS_OK;
}

}  // namespace sas
