// k_mlp.cu -- the learned selector's network: 16 features -> 64 hidden (ReLU)
// -> 8 logits, one per candidate (interpolation x axis order), masked softmax
// cross-entropy, trained by plain gradient descent.  Hand-written kernels:
//   mlp_fwd_bwd_kernel   one thread per example: standardised input z, hidden
//                        h, logits, softmax, loss, dlogits, dh
//   mlp_grad_kernel      one thread per parameter: the batch sum of its
//                        gradient (a fixed summation order, no atomics)
//   mlp_sgd_kernel       w -= lr * g
// Weights, packed as floats (SZ3G_MLP_WEIGHTS of them):
//   mu[16], sd[16]      feature standardisation (not trained)
//   W1[64][16], b1[64], W2[8][64], b2[8]
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace sz3g {

constexpr int kIn = 16, kHid = 64, kOut = 8;
constexpr int kOffMu = 0, kOffSd = 16, kOffW1 = 32, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kOut * kHid, kWeights = kOffB2 + kOut;
static_assert(kWeights == SZ3G_MLP_WEIGHTS, "weight layout");
constexpr int kPer = kIn + kHid + kOut + kHid;  // scratch floats per example: z, h, dlogit, dh
constexpr int kMlpThreads = 128;

// Forward (and, with labels, backward) of example i.  Masked logits are
// -inf; a masked label is an error (loss NaN).
__global__ void __launch_bounds__(kMlpThreads) mlp_fwd_bwd_kernel(const float* __restrict__ w,
                                                                  const float* __restrict__ feat,
                                                                  const uint8_t* __restrict__ mask,
                                                                  const int32_t* __restrict__ label, uint32_t B,
                                                                  float* logits, float* scratch, float* loss_i) {
  __shared__ float sw[kWeights];
  for (int k = threadIdx.x; k < kWeights; k += blockDim.x) sw[k] = w[k];
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  float z[kIn], h[kHid], lg[kOut];
  for (int k = 0; k < kIn; ++k) z[k] = (feat[(size_t)i * kIn + k] - sw[kOffMu + k]) / sw[kOffSd + k];
  for (int j = 0; j < kHid; ++j) {
    float a = sw[kOffB1 + j];
    for (int k = 0; k < kIn; ++k) a += sw[kOffW1 + j * kIn + k] * z[k];
    h[j] = a > 0.0f ? a : 0.0f;
  }
  float mx = -INFINITY;
  for (int o = 0; o < kOut; ++o) {
    float a = sw[kOffB2 + o];
    for (int j = 0; j < kHid; ++j) a += sw[kOffW2 + o * kHid + j] * h[j];
    lg[o] = mask[(size_t)i * kOut + o] ? a : -INFINITY;
    mx = fmaxf(mx, lg[o]);
  }
  if (logits)
    for (int o = 0; o < kOut; ++o) logits[(size_t)i * kOut + o] = lg[o];
  if (!label) return;
  float e[kOut], sum = 0.0f;
  for (int o = 0; o < kOut; ++o) {
    e[o] = lg[o] == -INFINITY ? 0.0f : expf(lg[o] - mx);
    sum += e[o];
  }
  const int y = label[i];
  float* sc = scratch + (size_t)i * kPer;
  const bool ok = y >= 0 && y < kOut && mask[(size_t)i * kOut + y];
  loss_i[i] = ok ? -(lg[y] - mx - logf(sum)) : NAN;
  float dl[kOut];
  for (int o = 0; o < kOut; ++o) dl[o] = (e[o] / sum - (o == y ? 1.0f : 0.0f)) / (float)B;
  for (int k = 0; k < kIn; ++k) sc[k] = z[k];
  for (int j = 0; j < kHid; ++j) sc[kIn + j] = h[j];
  for (int o = 0; o < kOut; ++o) sc[kIn + kHid + o] = dl[o];
  for (int j = 0; j < kHid; ++j) {
    float a = 0.0f;
    for (int o = 0; o < kOut; ++o) a += sw[kOffW2 + o * kHid + j] * dl[o];
    sc[kIn + kHid + kOut + j] = h[j] > 0.0f ? a : 0.0f;
  }
}

// Gradient of parameter k summed over the batch, in example order; k ==
// kWeights sums the loss (the mean over the batch).
__global__ void mlp_grad_kernel(const float* scratch, const float* loss_i, uint32_t B, float* grad, float* loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kWeights) return;
  float g = 0.0f;
  if (k == kWeights) {
    for (uint32_t i = 0; i < B; ++i) g += loss_i[i];
    *loss = g / (float)B;
    return;
  }
  if (k < kOffW1) {  // standardisation is not trained
    grad[k] = 0.0f;
    return;
  }
  int src_a, src_b;  // product of two scratch entries, or one (a bias)
  if (k < kOffB1) {
    const int j = (k - kOffW1) / kIn, q = (k - kOffW1) % kIn;
    src_a = kIn + kHid + kOut + j;  // dh_j
    src_b = q;                      // z_q
  } else if (k < kOffW2) {
    src_a = kIn + kHid + kOut + (k - kOffB1);
    src_b = -1;
  } else if (k < kOffB2) {
    const int o = (k - kOffW2) / kHid, j = (k - kOffW2) % kHid;
    src_a = kIn + kHid + o;  // dlogit_o
    src_b = kIn + j;         // h_j
  } else {
    src_a = kIn + kHid + (k - kOffB2);
    src_b = -1;
  }
  for (uint32_t i = 0; i < B; ++i) {
    const float* sc = scratch + (size_t)i * kPer;
    g += src_b < 0 ? sc[src_a] : sc[src_a] * sc[src_b];
  }
  grad[k] = g;
}

__global__ void mlp_sgd_kernel(float* w, const float* grad, float lr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kOffW1 && k < kWeights) w[k] -= lr * grad[k];
}

static int mlp_gradient(const float* w, const float* feat, const uint8_t* mask, const int32_t* label, uint32_t B,
                        float* grad, float* loss, float* scratch, float* loss_i, cudaStream_t s) {
  SZ3G_LAUNCH(kKMlp, s,
              mlp_fwd_bwd_kernel<<<(B + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, s>>>(w, feat, mask, label, B,
                                                                                            nullptr, scratch, loss_i));
  SZ3G_LAUNCH(kKMlp, s, mlp_grad_kernel<<<(kWeights + 1 + 127) / 128, 128, 0, s>>>(scratch, loss_i, B, grad, loss));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int launch_mlp_forward(const float* w, const float* feat, const uint8_t* mask, uint32_t B, float* logits,
                       cudaStream_t s) {
  SZ3G_LAUNCH(kKMlp, s,
              mlp_fwd_bwd_kernel<<<(B + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, s>>>(w, feat, mask, nullptr, B,
                                                                                            logits, nullptr, nullptr));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

}  // namespace sz3g

using namespace sz3g;

namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
}  // namespace

extern "C" {

int sz3g_mlp_forward(const float* d_w, const float* d_feat, const uint8_t* d_mask, uint32_t n, float* d_logits,
                     void* stream) {
  if (!d_w || !d_feat || !d_mask || !d_logits || n < 1) return SZ3G_E_INVAL;
  return launch_mlp_forward(d_w, d_feat, d_mask, n, d_logits, (cudaStream_t)stream);
}

int sz3g_mlp_gradient(const float* d_w, const float* d_feat, const uint8_t* d_mask, const int32_t* d_label,
                      uint32_t n, float* d_grad, float* h_loss, void* stream) {
  if (!d_w || !d_feat || !d_mask || !d_label || !d_grad || n < 1) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf sc, li, ls;
  if (cudaMalloc(&sc.p, (size_t)n * kPer * 4) != cudaSuccess || cudaMalloc(&li.p, (size_t)n * 4) != cudaSuccess ||
      cudaMalloc(&ls.p, 4) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_NOMEM;
  }
  int rc = mlp_gradient(d_w, d_feat, d_mask, d_label, n, d_grad, (float*)ls.p, (float*)sc.p, (float*)li.p, s);
  if (rc) return rc;
  float l = 0.0f;
  if (cudaMemcpyAsync(&l, ls.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return SZ3G_E_CUDA;
  if (h_loss) *h_loss = l;
  return SZ3G_OK;
}

int sz3g_mlp_train(float* d_w, const float* d_feat, const uint8_t* d_mask, const int32_t* d_label, uint32_t n,
                   float lr, uint32_t steps, float* h_loss, void* stream) {
  if (!d_w || !d_feat || !d_mask || !d_label || n < 1 || !(lr > 0.0f)) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf sc, li, ls, gr;
  if (cudaMalloc(&sc.p, (size_t)n * kPer * 4) != cudaSuccess || cudaMalloc(&li.p, (size_t)n * 4) != cudaSuccess ||
      cudaMalloc(&ls.p, 4) != cudaSuccess || cudaMalloc(&gr.p, (size_t)kWeights * 4) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_NOMEM;
  }
  for (uint32_t t = 0; t < steps; ++t) {
    int rc = mlp_gradient(d_w, d_feat, d_mask, d_label, n, (float*)gr.p, (float*)ls.p, (float*)sc.p, (float*)li.p, s);
    if (rc) return rc;
    SZ3G_LAUNCH(kKMlp, s, mlp_sgd_kernel<<<(kWeights + 127) / 128, 128, 0, s>>>(d_w, (const float*)gr.p, lr));
  }
  float l = 0.0f;
  if (cudaMemcpyAsync(&l, ls.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return SZ3G_E_CUDA;
  if (h_loss) *h_loss = l;
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

}  // extern "C"
