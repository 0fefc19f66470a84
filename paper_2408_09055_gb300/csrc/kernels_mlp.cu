// Learned kernel-cost model: a three-layer perceptron that predicts the log
// run time of a kernel from its features.  FP32-accumulate training kernels
// (forward, backpropagation of the mean squared error, Adam) and BF16
// inference (BF16 weights and activations, FP32 accumulation).
//
// Parameter layout (flat FP32 vector): W1 [F x H], b1 [H], W2 [H x H],
// b2 [H], W3 [H], b3 [1]; layer l computes x @ W_l + b_l.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "internal.hpp"

struct qs_mlp {
  int F = 0, H = 0;
  size_t np = 0;
  float* theta = nullptr;   // device FP32 parameters
  float* grad = nullptr;    // device gradient
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  __nv_bfloat16* wbf = nullptr;  // BF16 copy of the parameters
  bool bf_stale = true;
  int64_t step = 0;
  // loss: expectile of ln(time), weight 2 tau on underestimates (y < t) and
  // 2 (1 - tau) on overestimates; tau = 0.5 is the mean squared error
  float tau = 0.5f;
  // activations for a batch (grown on demand)
  int cap = 0;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dz = nullptr, *dh = nullptr, *loss = nullptr;
};

namespace qs {

namespace {

constexpr int kT = 256;

struct Off {
  size_t W1, b1, W2, b2, W3, b3;
};
Off offsets(int F, int H) {
  Off o;
  o.W1 = 0;
  o.b1 = o.W1 + (size_t)F * H;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + (size_t)H * H;
  o.W3 = o.b2 + H;
  o.b3 = o.W3 + H;
  return o;
}

// out[b, o] = sum_i in[b, i] W[i, o] + bias[o]  (pre-activation); the input
// is relu(in) when relu_in is set
__global__ void linear_fwd(const float* in, int B, int I, const float* W, const float* bias, int O,
                           bool relu_in, float* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * O) return;
  const int b = idx / O, o = idx % O;
  float acc = bias[o];
  for (int i = 0; i < I; ++i) {
    float xv = in[(size_t)b * I + i];
    if (relu_in) xv = fmaxf(xv, 0.0f);
    acc = fmaf(xv, W[(size_t)i * O + o], acc);
  }
  out[idx] = acc;
}

// output layer: y[b] = relu(z2[b]) . W3 + b3; with d = y - t and the
// expectile weight w = 2 tau (d < 0) or 2 (1 - tau): loss partial w d^2 / B,
// dz[b] = 2 w d / B
__global__ void output_fwd_bwd(const float* z2, int B, int H, const float* W3, const float* b3,
                               const float* t, float tau, float* y, float* dz, float* loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float acc = b3[0];
  for (int h = 0; h < H; ++h) acc = fmaf(fmaxf(z2[(size_t)b * H + h], 0.0f), W3[h], acc);
  y[b] = acc;
  if (t) {
    const float d = acc - t[b];
    const float w = 2.0f * (d < 0.0f ? tau : 1.0f - tau);
    dz[b] = 2.0f * w * d / (float)B;
    atomicAdd(loss, w * d * d / (float)B);
  }
}

// gradient of a weight matrix: gW[i, o] = sum_b act(in[b, i]) * g[b, o]
__global__ void weight_grad(const float* in, int B, int I, bool relu_in, const float* g, int O,
                            float* gW, float* gb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= I * O) return;
  const int i = idx / O, o = idx % O;
  float acc = 0.0f;
  for (int b = 0; b < B; ++b) {
    float xv = in[(size_t)b * I + i];
    if (relu_in) xv = fmaxf(xv, 0.0f);
    acc = fmaf(xv, g[(size_t)b * O + o], acc);
  }
  gW[idx] = acc;
  if (i == 0 && gb) {
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += g[(size_t)b * O + o];
    gb[o] = s;
  }
}

// gradient through a ReLU layer: dh[b, i] = (sum_o g[b, o] W[i, o]) * [z[b, i] > 0]
__global__ void input_grad(const float* g, int B, int O, const float* W, int I, const float* z,
                           float* dh) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * I) return;
  const int b = idx / I, i = idx % I;
  float acc = 0.0f;
  for (int o = 0; o < O; ++o) acc = fmaf(g[(size_t)b * O + o], W[(size_t)i * O + o], acc);
  dh[idx] = z[idx] > 0.0f ? acc : 0.0f;
}

// dz2[b, h] = dz[b] * W3[h] * [z2 > 0]; also dW3 and db3
__global__ void output_grad(const float* dz, int B, const float* W3, const float* z2, int H,
                            float* dh2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * H) return;
  const int b = idx / H, h = idx % H;
  dh2[idx] = z2[idx] > 0.0f ? dz[b] * W3[h] : 0.0f;
}

__global__ void adam_step(float* p, const float* g, float* m, float* v, size_t n, float lr,
                          float b1, float b2, float eps, float c1, float c2) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16(const float* a, __nv_bfloat16* b, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// BF16 inference: one CTA of H threads per sample; hidden activations are
// rounded to BF16 between layers, every product accumulates in FP32.
__global__ void infer_bf16(const float* x, int B, int F, int H, const __nv_bfloat16* w, Off o,
                           float* y) {
  extern __shared__ __nv_bfloat16 act[];  // 2H
  const int b = blockIdx.x, h = threadIdx.x;
  if (b >= B) return;
  __nv_bfloat16* a1 = act;
  __nv_bfloat16* a2 = act + H;
  if (h < H) {
    float acc = __bfloat162float(w[o.b1 + h]);
    for (int f = 0; f < F; ++f)
      acc = fmaf(__bfloat162float(__float2bfloat16_rn(x[(size_t)b * F + f])),
                 __bfloat162float(w[o.W1 + (size_t)f * H + h]), acc);
    a1[h] = __float2bfloat16_rn(fmaxf(acc, 0.0f));
  }
  __syncthreads();
  if (h < H) {
    float acc = __bfloat162float(w[o.b2 + h]);
    for (int i = 0; i < H; ++i)
      acc = fmaf(__bfloat162float(a1[i]), __bfloat162float(w[o.W2 + (size_t)i * H + h]), acc);
    a2[h] = __float2bfloat16_rn(fmaxf(acc, 0.0f));
  }
  __syncthreads();
  if (h == 0) {
    float acc = __bfloat162float(w[o.b3]);
    for (int i = 0; i < H; ++i) acc = fmaf(__bfloat162float(a2[i]), __bfloat162float(w[o.W3 + i]), acc);
    y[b] = acc;
  }
}

unsigned blocks(size_t n) { return (unsigned)((n + kT - 1) / kT); }

int ensure_batch(qs_mlp* M, int B) {
  if (B <= M->cap) return QS_OK;
  for (float* p : {M->z1, M->z2, M->y, M->dz, M->dh, M->loss})
    if (p) cudaFree(p);
  const int H = M->H;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&M->z1, sizeof(float) * (size_t)B * H);
  if (e == cudaSuccess) e = cudaMalloc(&M->z2, sizeof(float) * (size_t)B * H);
  if (e == cudaSuccess) e = cudaMalloc(&M->y, sizeof(float) * B);
  if (e == cudaSuccess) e = cudaMalloc(&M->dz, sizeof(float) * B);
  if (e == cudaSuccess) e = cudaMalloc(&M->dh, sizeof(float) * (size_t)B * H * 2);
  if (e == cudaSuccess) e = cudaMalloc(&M->loss, sizeof(float));
  if (e != cudaSuccess) {
    M->cap = 0;
    return cuda_status(e);
  }
  M->cap = B;
  return QS_OK;
}

// forward + backward into M->grad; loss written to M->loss (device)
int run_gradient(qs_mlp* M, const float* x, const float* t, int B, cudaStream_t s) {
  int rc = ensure_batch(M, B);
  if (rc != QS_OK) return rc;
  const int F = M->F, H = M->H;
  const Off o = offsets(F, H);
  const float* th = M->theta;
  cudaMemsetAsync(M->loss, 0, sizeof(float), s);
  linear_fwd<<<blocks((size_t)B * H), kT, 0, s>>>(x, B, F, th + o.W1, th + o.b1, H, false, M->z1);
  linear_fwd<<<blocks((size_t)B * H), kT, 0, s>>>(M->z1, B, H, th + o.W2, th + o.b2, H, true, M->z2);
  output_fwd_bwd<<<blocks(B), kT, 0, s>>>(M->z2, B, H, th + o.W3, th + o.b3, t, M->tau, M->y, M->dz,
                                          M->loss);
  float* g = M->grad;
  float* dh2 = M->dh;
  float* dh1 = M->dh + (size_t)B * H;
  // dW3 = relu(z2)^T dz, db3 = sum dz (a weight gradient with O = 1)
  weight_grad<<<blocks(H), kT, 0, s>>>(M->z2, B, H, true, M->dz, 1, g + o.W3, g + o.b3);
  output_grad<<<blocks((size_t)B * H), kT, 0, s>>>(M->dz, B, th + o.W3, M->z2, H, dh2);
  weight_grad<<<blocks((size_t)H * H), kT, 0, s>>>(M->z1, B, H, true, dh2, H, g + o.W2, g + o.b2);
  input_grad<<<blocks((size_t)B * H), kT, 0, s>>>(dh2, B, H, th + o.W2, H, M->z1, dh1);
  weight_grad<<<blocks((size_t)F * H), kT, 0, s>>>(x, B, F, false, dh1, H, g + o.W1, g + o.b1);
  return cuda_status(cudaGetLastError());
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

int qs_mlp_create(int32_t features, int32_t hidden, uint64_t seed, qs_mlp** out) {
  if (!out || features < 1 || features > 4096 || hidden < 1 || hidden > 1024) return QS_EINVAL;
  *out = nullptr;
  qs_mlp* M = new (std::nothrow) qs_mlp();
  if (!M) return QS_ENOMEM;
  M->F = features;
  M->H = hidden;
  M->np = (size_t)features * hidden + hidden + (size_t)hidden * hidden + hidden + hidden + 1;
  cudaError_t e = cudaMalloc(&M->theta, sizeof(float) * M->np);
  if (e == cudaSuccess) e = cudaMalloc(&M->grad, sizeof(float) * M->np);
  if (e == cudaSuccess) e = cudaMalloc(&M->m, sizeof(float) * M->np);
  if (e == cudaSuccess) e = cudaMalloc(&M->v, sizeof(float) * M->np);
  if (e == cudaSuccess) e = cudaMalloc(&M->wbf, sizeof(__nv_bfloat16) * M->np);
  if (e != cudaSuccess) {
    qs_mlp_free(M);
    return cuda_status(e);
  }
  // He-uniform weights, zero biases
  std::vector<float> h(M->np, 0.0f);
  std::mt19937_64 rng(seed);
  const Off o = offsets(features, hidden);
  auto fill = [&](size_t at, size_t count, int fan_in) {
    std::uniform_real_distribution<float> d(-std::sqrt(6.0f / fan_in), std::sqrt(6.0f / fan_in));
    for (size_t i = 0; i < count; ++i) h[at + i] = d(rng);
  };
  fill(o.W1, (size_t)features * hidden, features);
  fill(o.W2, (size_t)hidden * hidden, hidden);
  fill(o.W3, hidden, hidden);
  int rc = qs_mlp_set_params(M, h.data(), M->np);
  if (rc != QS_OK) {
    qs_mlp_free(M);
    return rc;
  }
  *out = M;
  return QS_OK;
}

void qs_mlp_free(qs_mlp* M) {
  if (!M) return;
  for (float* p : {M->theta, M->grad, M->m, M->v, M->z1, M->z2, M->y, M->dz, M->dh, M->loss})
    if (p) cudaFree(p);
  if (M->wbf) cudaFree(M->wbf);
  delete M;
}

int64_t qs_mlp_num_params(const qs_mlp* M) { return M ? (int64_t)M->np : QS_EINVAL; }

int qs_mlp_set_expectile(qs_mlp* M, float tau) {
  if (!M || !(tau > 0.0f && tau < 1.0f)) return QS_EINVAL;
  M->tau = tau;
  return QS_OK;
}

int qs_mlp_shape(const qs_mlp* M, int32_t* features, int32_t* hidden) {
  if (!M || !features || !hidden) return QS_EINVAL;
  *features = M->F;
  *hidden = M->H;
  return QS_OK;
}

int qs_mlp_get_params(const qs_mlp* M, float* out, uint64_t n) {
  if (!M || !out || n != M->np) return QS_EINVAL;
  return cuda_status(cudaMemcpy(out, M->theta, sizeof(float) * n, cudaMemcpyDeviceToHost));
}

int qs_mlp_set_params(qs_mlp* M, const float* in, uint64_t n) {
  if (!M || !in || n != M->np) return QS_EINVAL;
  cudaError_t e = cudaMemcpy(M->theta, in, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMemset(M->v, 0, sizeof(float) * n);
  M->step = 0;
  M->bf_stale = true;
  return cuda_status(e);
}

int qs_mlp_gradient(qs_mlp* M, const float* x, const float* t, int32_t batch, float* grad_out,
                    float* loss_out, void* stream) {
  if (!M || !x || !t || batch < 1) return QS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = run_gradient(M, x, t, batch, s);
  if (rc != QS_OK) return rc;
  cudaError_t e = cudaSuccess;
  if (grad_out) e = cudaMemcpyAsync(grad_out, M->grad, sizeof(float) * M->np, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

int qs_mlp_train_step(qs_mlp* M, const float* x, const float* t, int32_t batch, float lr,
                      float* loss_out, void* stream) {
  if (!M || !x || !t || batch < 1 || !(lr > 0)) return QS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = run_gradient(M, x, t, batch, s);
  if (rc != QS_OK) return rc;
  M->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)M->step), c2 = 1.0f - std::pow(b2, (float)M->step);
  adam_step<<<blocks(M->np), kT, 0, s>>>(M->theta, M->grad, M->m, M->v, M->np, lr, b1, b2, 1e-8f, c1, c2);
  M->bf_stale = true;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss_out) {
    e = cudaMemcpyAsync(loss_out, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return cuda_status(e);
}

int qs_mlp_forward(qs_mlp* M, const float* x, int32_t batch, float* y, int32_t bf16, void* stream) {
  if (!M || !x || !y || batch < 1) return QS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const Off o = offsets(M->F, M->H);
  if (bf16) {
    if (M->bf_stale) {
      to_bf16<<<blocks(M->np), kT, 0, s>>>(M->theta, M->wbf, M->np);
      M->bf_stale = false;
    }
    const int threads = ((M->H + 31) / 32) * 32;
    infer_bf16<<<batch, threads, sizeof(__nv_bfloat16) * 2 * M->H, s>>>(x, batch, M->F, M->H, M->wbf, o, y);
    return cuda_status(cudaGetLastError());
  }
  int rc = ensure_batch(M, batch);
  if (rc != QS_OK) return rc;
  const float* th = M->theta;
  linear_fwd<<<blocks((size_t)batch * M->H), kT, 0, s>>>(x, batch, M->F, th + o.W1, th + o.b1, M->H, false, M->z1);
  linear_fwd<<<blocks((size_t)batch * M->H), kT, 0, s>>>(M->z1, batch, M->H, th + o.W2, th + o.b2, M->H, true, M->z2);
  output_fwd_bwd<<<blocks(batch), kT, 0, s>>>(M->z2, batch, M->H, th + o.W3, th + o.b3, nullptr, 0.5f, y, nullptr,
                                              nullptr);
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
