// The launch-parameter predictor's network on the GPU: forward pass,
// mean-squared-error loss with its backward pass, and the Adam update, all
// in fp32.  The network maps features (log2 n, log2 batch, dtype,
// residency), normalised, to (log2 m, log2 S, log2 chunk), normalised:
//
//   z1 = X W1^T + b1, h1 = relu(z1); z2 = h1 W2^T + b2, h2 = relu(z2);
//   y = h2 W3^T + b3;   L = mean over batch and outputs of (y - t)^2
//
// Parameters are one flat fp32 array [W1 (64x4), b1, W2 (64x64), b2,
// W3 (3x64), b3], weights row-major [out][in].  relu'(z) = 1 for z > 0.
// Adam: Kingma and Ba, 2015.  The paper fits its stream model by linear
// regression and curve fitting instead (Sec. 2.4).
#include <cuda_runtime.h>

#include "tps_internal.h"

namespace {

constexpr int kIn = TPS_MLP_IN, kH = TPS_MLP_HIDDEN, kOut = TPS_MLP_OUT;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH,
              oW3 = oB2 + kH, oB3 = oW3 + kOut * kH, kNParams = oB3 + kOut;
static_assert(kNParams == TPS_MLP_NPARAMS, "parameter count");

// Z[b][o] = sum_i X[b][i] W[o][i] + bias[o]; H = relu(Z) when relu != 0.
__global__ void k_linear(int B, int in, int out, const float* __restrict__ X,
                         const float* __restrict__ W, const float* __restrict__ bias,
                         float* __restrict__ Z, float* __restrict__ H) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * out) return;
  const int b = idx / out, o = idx % out;
  float s = bias[o];
  for (int i = 0; i < in; ++i) s = fmaf(X[b * in + i], W[o * in + i], s);
  Z[idx] = s;
  if (H) H[idx] = s > 0.0f ? s : 0.0f;
}

// dY = 2 (Y - T) / (B * out); loss (sum of squares / (B * out)) added to *loss.
__global__ void k_mse(int B, int out, const float* __restrict__ Y, const float* __restrict__ T,
                      float* __restrict__ dY, float* __restrict__ loss) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (idx < B * out) {
    const float e = Y[idx] - T[idx];
    dY[idx] = 2.0f * e / (float)(B * out);
    l = e * e / (float)(B * out);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// dX[b][i] = (sum_o dZ[b][o] W[o][i]) * relu'(Zprev[b][i]).
__global__ void k_back_input(int B, int in, int out, const float* __restrict__ dZ,
                             const float* __restrict__ W, const float* __restrict__ Zprev,
                             float* __restrict__ dX) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * in) return;
  const int b = idx / in, i = idx % in;
  float s = 0.0f;
  for (int o = 0; o < out; ++o) s = fmaf(dZ[b * out + o], W[o * in + i], s);
  dX[idx] = Zprev[idx] > 0.0f ? s : 0.0f;
}

// dW[o][i] = sum_b dZ[b][o] X[b][i]; db[o] = sum_b dZ[b][o].
__global__ void k_back_weight(int B, int in, int out, const float* __restrict__ dZ,
                              const float* __restrict__ X, float* __restrict__ dW,
                              float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= out * (in + 1)) return;
  const int o = idx / (in + 1), i = idx % (in + 1);
  float s = 0.0f;
  if (i < in) {
    for (int b = 0; b < B; ++b) s = fmaf(dZ[b * out + o], X[b * in + i], s);
    dW[o * in + i] = s;
  } else {
    for (int b = 0; b < B; ++b) s += dZ[b * out + o];
    db[o] = s;
  }
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float beta1,
                       float beta2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned blocks(int n) { return (unsigned)((n + 127) / 128); }

// Activation scratch (floats): z1, h1, z2, h2, y, dy, d2, d1.
inline size_t act_floats(int B) { return (size_t)B * (4 * kH + 2 * kOut + 2 * kH); }

}  // namespace

extern "C" {

size_t tps_mlp_workspace_floats(int32_t batch) {
  return batch > 0 ? act_floats(batch) : 0;
}

tps_status tps_mlp_forward(const float* params, int32_t batch, const float* X, float* Y,
                           float* work, void* stream) {
  if (!params || !X || !Y || !work || batch <= 0) return TPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int B = batch;
  float* z1 = work;
  float* h1 = z1 + (size_t)B * kH;
  float* z2 = h1 + (size_t)B * kH;
  float* h2 = z2 + (size_t)B * kH;
  k_linear<<<blocks(B * kH), 128, 0, s>>>(B, kIn, kH, X, params + oW1, params + oB1, z1, h1);
  k_linear<<<blocks(B * kH), 128, 0, s>>>(B, kH, kH, h1, params + oW2, params + oB2, z2, h2);
  k_linear<<<blocks(B * kOut), 128, 0, s>>>(B, kH, kOut, h2, params + oW3, params + oB3, Y,
                                           nullptr);
  return cudaGetLastError() == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

tps_status tps_mlp_loss_backward(const float* params, int32_t batch, const float* X,
                                 const float* T, float* grads, float* loss, float* work,
                                 void* stream) {
  if (!params || !X || !T || !grads || !work || batch <= 0) return TPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int B = batch;
  float* z1 = work;
  float* h1 = z1 + (size_t)B * kH;
  float* z2 = h1 + (size_t)B * kH;
  float* h2 = z2 + (size_t)B * kH;
  float* y = h2 + (size_t)B * kH;
  float* dy = y + (size_t)B * kOut;
  float* d2 = dy + (size_t)B * kOut;
  float* d1 = d2 + (size_t)B * kH;
  tps_status st = tps_mlp_forward(params, batch, X, y, work, stream);
  if (st != TPS_OK) return st;
  if (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return TPS_ERR_CUDA;
  k_mse<<<blocks(B * kOut), 128, 0, s>>>(B, kOut, y, T, dy, loss);
  k_back_weight<<<blocks(kOut * (kH + 1)), 128, 0, s>>>(B, kH, kOut, dy, h2, grads + oW3,
                                                        grads + oB3);
  k_back_input<<<blocks(B * kH), 128, 0, s>>>(B, kH, kOut, dy, params + oW3, z2, d2);
  k_back_weight<<<blocks(kH * (kH + 1)), 128, 0, s>>>(B, kH, kH, d2, h1, grads + oW2,
                                                      grads + oB2);
  k_back_input<<<blocks(B * kH), 128, 0, s>>>(B, kH, kH, d2, params + oW2, z1, d1);
  k_back_weight<<<blocks(kH * (kIn + 1)), 128, 0, s>>>(B, kIn, kH, d1, X, grads + oW1,
                                                       grads + oB1);
  return cudaGetLastError() == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

tps_status tps_mlp_adam_step(float* params, const float* grads, float* m, float* v, int32_t t,
                             float lr, float beta1, float beta2, float eps, void* stream) {
  if (!params || !grads || !m || !v || t < 1) return TPS_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  k_adam<<<blocks(kNParams), 128, 0, (cudaStream_t)stream>>>(kNParams, params, grads, m, v, lr,
                                                             beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}

}  // extern "C"
