// Learned configuration predictors: 3-layer MLPs, 8 -> 64 -> 64 -> OUT with
// ReLU, FP32, trained and evaluated on the GPU by the kernels below: OUT = 6
// for the grouped plans' configurations, OUT = 39 for single-call schedules.
//
// The paper chooses its micro-kernel parameters by hand and notes the
// trade-off between input and output ratios (Section III-C); here a small
// network learns, from the autotuner's own timings, which configuration
// (path and tile shape) is cheapest for a shape, so that grouped plans can
// skip timing every problem.
//
// Parameters (one flat FP32 array of GBGEMM_MLP_PARAMS, or
// GBGEMM_SCHED_MLP_PARAMS for the schedule network):
//   W1[64][8], b1[64], W2[64][64], b2[64], W3[OUT][64], b3[OUT]   (row = output)
// Inputs x[8]: log2 m/14, log2 n/14, log2 k/14, transa, transb, and the
// 16-byte alignment class of A, B, C (0/1).  Outputs: predicted
// log2(cost_c / cost_best) of every configuration (or schedule) c.
// Loss: mean over (sample, legal configuration) of (output - target)^2.
#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "mlp.h"

namespace gbg {
namespace {

constexpr int kIn = 8, kH = 64;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH;
// Layout of a network with OUT outputs (the hidden layers are the same for every OUT).
template <int OUT>
struct Net {
  static constexpr int kOut = OUT;
  static constexpr int oB3 = oW3 + OUT * kH;
  static constexpr int kParams = oB3 + OUT;
  static constexpr int kLegalBytes = (OUT + 7) / 8;  // legal-mask bytes per sample
};
static_assert(Net<GBGEMM_NUM_CONFIGS>::kParams == GBGEMM_MLP_PARAMS, "parameter count");
static_assert(Net<GBGEMM_NUM_SCHEDULES>::kParams == GBGEMM_SCHED_MLP_PARAMS, "parameter count");
constexpr int kTrainBatch = 256;  // samples per mini-batch = threads of the training kernel

// Forward pass of one sample held by one thread; writes h1, h2 (post-ReLU)
// and the outputs.
template <int OUT>
__device__ __forceinline__ void forward_one(const float* __restrict__ P, const float* x, float* h1, float* h2,
                                            float* out) {
  constexpr int kOut = OUT, oB3 = Net<OUT>::oB3;
  for (int j = 0; j < kH; ++j) {
    float a = P[oB1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a = fmaf(P[oW1 + j * kIn + i], x[i], a);
    h1[j] = a > 0.f ? a : 0.f;
  }
  for (int j = 0; j < kH; ++j) {
    float a = P[oB2 + j];
    for (int i = 0; i < kH; ++i) a = fmaf(P[oW2 + j * kH + i], h1[i], a);
    h2[j] = a > 0.f ? a : 0.f;
  }
  for (int j = 0; j < kOut; ++j) {
    float a = P[oB3 + j];
    for (int i = 0; i < kH; ++i) a = fmaf(P[oW3 + j * kH + i], h2[i], a);
    out[j] = a;
  }
}

// Batched inference: scores (optional) and the masked argmin per sample
// (ties to the lower configuration index; -1 when no configuration is legal).
// legal: kLegalBytes bytes per sample, bit c % 8 of byte c / 8 for output c.
template <int OUT>
__global__ void mlp_predict_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                   const uint8_t* __restrict__ legal, int64_t n, float* __restrict__ scores,
                                   int* __restrict__ configs) {
  constexpr int kOut = OUT, kParams = Net<OUT>::kParams, kLB = Net<OUT>::kLegalBytes;
  __shared__ float sp[kParams];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float x[kIn], h1[kH], h2[kH], out[kOut];
#pragma unroll
    for (int i = 0; i < kIn; ++i) x[i] = X[s * kIn + i];
    forward_one<OUT>(sp, x, h1, h2, out);
    int best = -1;
    for (int c = 0; c < kOut; ++c) {
      if (scores) scores[s * kOut + c] = out[c];
      if (legal && !((legal[s * kLB + (c >> 3)] >> (c & 7)) & 1)) continue;
      if (best < 0 || out[c] < out[best]) best = c;
    }
    if (configs) configs[s] = best;
  }
}

// One mini-batch (up to kTrainBatch samples, one thread each): forward,
// masked MSE, backward; writes the gradient of the mean loss into G and the
// loss sum / legal count into loss2[0..1].
template <int OUT>
__global__ void __launch_bounds__(kTrainBatch) mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                              const float* __restrict__ Y, const float* __restrict__ M,
                                                              const int* __restrict__ idx, int nb,
                                                              float* __restrict__ G, float* __restrict__ loss2) {
  constexpr int kOut = OUT, kParams = Net<OUT>::kParams, oB3 = Net<OUT>::oB3;
  extern __shared__ float sm[];
  float* sp = sm;                                  // kParams
  float* sh1 = sp + kParams;                       // [nb][kH]
  float* sh2 = sh1 + kTrainBatch * kH;             // [nb][kH]
  float* sd = sh2 + kTrainBatch * kH;              // output deltas [nb][kOut]
  float* sx = sd + kTrainBatch * kOut;             // inputs [nb][kIn]
  __shared__ float red[2];
  const int t = threadIdx.x;
  for (int i = t; i < kParams; i += blockDim.x) sp[i] = P[i];
  if (t < 2) red[t] = 0.f;
  __syncthreads();
  float lsum = 0.f, lcnt = 0.f;
  if (t < nb) {
    const int s = idx ? idx[t] : t;
    float x[kIn], out[kOut];
#pragma unroll
    for (int i = 0; i < kIn; ++i) { x[i] = X[(int64_t)s * kIn + i]; sx[t * kIn + i] = x[i]; }
    forward_one<OUT>(sp, x, sh1 + t * kH, sh2 + t * kH, out);
    for (int c = 0; c < kOut; ++c) {
      const float m = M[(int64_t)s * kOut + c];
      const float d = (out[c] - Y[(int64_t)s * kOut + c]) * m;
      lsum += d * d;
      lcnt += m;
      sd[t * kOut + c] = d;  // scaled below by 2 / count
    }
  }
  atomicAdd(&red[0], lsum);
  atomicAdd(&red[1], lcnt);
  __syncthreads();
  const float cnt = red[1] > 0.f ? red[1] : 1.f;
  const float scale = 2.f / cnt;
  if (t < nb)
    for (int c = 0; c < kOut; ++c) sd[t * kOut + c] *= scale;
  __syncthreads();
  // layer 3: dW3[c][i] = sum_s d[s][c] h2[s][i]; db3[c] = sum_s d[s][c]
  for (int w = t; w < kOut * kH + kOut; w += blockDim.x) {
    float g = 0.f;
    if (w < kOut * kH) {
      const int c = w / kH, i = w % kH;
      for (int s = 0; s < nb; ++s) g = fmaf(sd[s * kOut + c], sh2[s * kH + i], g);
      G[oW3 + w] = g;
    } else {
      const int c = w - kOut * kH;
      for (int s = 0; s < nb; ++s) g += sd[s * kOut + c];
      G[oB3 + c] = g;
    }
  }
  __syncthreads();
  // delta2[s][i] = (sum_c W3[c][i] d[s][c]) * [h2 > 0], stored in place of h2
  // after dW3 has used h2 (h2 itself is only needed as the ReLU mask).
  float d2[kH];
  if (t < nb) {
    for (int i = 0; i < kH; ++i) {
      float a = 0.f;
      for (int c = 0; c < kOut; ++c) a = fmaf(sp[oW3 + c * kH + i], sd[t * kOut + c], a);
      d2[i] = sh2[t * kH + i] > 0.f ? a : 0.f;
    }
  }
  __syncthreads();
  if (t < nb)
    for (int i = 0; i < kH; ++i) sh2[t * kH + i] = d2[i];
  __syncthreads();
  // layer 2: dW2[j][i] = sum_s delta2[s][j] h1[s][i]; db2[j] = sum_s delta2[s][j]
  for (int w = t; w < kH * kH + kH; w += blockDim.x) {
    float g = 0.f;
    if (w < kH * kH) {
      const int j = w / kH, i = w % kH;
      for (int s = 0; s < nb; ++s) g = fmaf(sh2[s * kH + j], sh1[s * kH + i], g);
      G[oW2 + w] = g;
    } else {
      const int j = w - kH * kH;
      for (int s = 0; s < nb; ++s) g += sh2[s * kH + j];
      G[oB2 + j] = g;
    }
  }
  __syncthreads();
  // delta1[s][i] = (sum_j W2[j][i] delta2[s][j]) * [h1 > 0]
  float d1[kH];
  if (t < nb) {
    for (int i = 0; i < kH; ++i) {
      float a = 0.f;
      for (int j = 0; j < kH; ++j) a = fmaf(sp[oW2 + j * kH + i], sh2[t * kH + j], a);
      d1[i] = sh1[t * kH + i] > 0.f ? a : 0.f;
    }
  }
  __syncthreads();
  if (t < nb)
    for (int i = 0; i < kH; ++i) sh1[t * kH + i] = d1[i];
  __syncthreads();
  // layer 1: dW1[j][i] = sum_s delta1[s][j] x[s][i]; db1[j] = sum_s delta1[s][j]
  for (int w = t; w < kH * kIn + kH; w += blockDim.x) {
    float g = 0.f;
    if (w < kH * kIn) {
      const int j = w / kIn, i = w % kIn;
      for (int s = 0; s < nb; ++s) g = fmaf(sh1[s * kH + j], sx[s * kIn + i], g);
      G[oW1 + w] = g;
    } else {
      const int j = w - kH * kIn;
      for (int s = 0; s < nb; ++s) g += sh1[s * kH + j];
      G[oB1 + j] = g;
    }
  }
  if (t == 0 && loss2) {
    loss2[0] = red[0];
    loss2[1] = red[1];
  }
}

// Adam (Kingma and Ba, 2015) on the flat parameter array.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m1,
                            float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float v = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  P[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

template <int OUT>
constexpr size_t grad_smem_bytes() {
  return (size_t)(Net<OUT>::kParams + 2 * kTrainBatch * kH + kTrainBatch * OUT + kTrainBatch * kIn) * sizeof(float);
}

// The shared-memory opt-in of the training kernel, once per process and OUT.
template <int OUT>
cudaError_t ensure_grad_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel<OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)grad_smem_bytes<OUT>());
  done = e == cudaSuccess;
  return e;
}

// He-uniform initialisation (zero biases) of a network with OUT outputs.
template <int OUT>
std::vector<float> he_init(std::mt19937_64& rng) {
  std::vector<float> p(Net<OUT>::kParams, 0.f);
  auto init = [&](int off, int fan_out, int fan_in) {
    const double b = std::sqrt(6.0 / fan_in);
    std::uniform_real_distribution<double> u(-b, b);
    for (int i = 0; i < fan_out * fan_in; ++i) p[off + i] = (float)u(rng);
  };
  init(oW1, kH, kIn);
  init(oW2, kH, kH);
  init(oW3, OUT, kH);
  return p;
}

}  // namespace

void predictor_features(const gbgemm_problem& q, float* x) {
  auto l2 = [](int64_t v) { return (float)(std::log2((double)(v > 0 ? v : 1)) / 14.0); };
  auto al = [](int64_t ld, const void* p) {
    return ((ld & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) ? 1.f : 0.f;
  };
  x[0] = l2(q.m);
  x[1] = l2(q.n);
  x[2] = l2(q.k);
  x[3] = (q.transa == 'N' || q.transa == 'n') ? 0.f : 1.f;
  x[4] = (q.transb == 'N' || q.transb == 'n') ? 0.f : 1.f;
  x[5] = al(q.lda, q.A);
  x[6] = al(q.ldb, q.B);
  x[7] = al(q.ldc, q.C);
}

namespace {

template <int OUT>
int predict_impl(const float* P, const float* dx, const uint8_t* dlegal, int64_t n, float* dscores, int* dconfigs,
                 cudaStream_t s) {
  const int64_t blocks = (n + 127) / 128;
  mlp_predict_kernel<OUT><<<(unsigned)(blocks < 1024 ? blocks : 1024), 128, 0, s>>>(P, dx, dlegal, n, dscores,
                                                                                   dconfigs);
  return cudaGetLastError() == cudaSuccess ? GBGEMM_OK : GBGEMM_ERR_CUDA;
}

template <int OUT>
int loss_grad_impl(const float* P, const float* dx, const float* dy, const float* dmask, int64_t n, float* host_loss,
                   float* dgrad, cudaStream_t s) {
  if (ensure_grad_attr<OUT>() != cudaSuccess) return GBGEMM_ERR_CUDA;
  float* dl = nullptr;
  if (cudaMalloc(&dl, 2 * sizeof(float)) != cudaSuccess) return GBGEMM_ERR_ALLOC;
  mlp_grad_kernel<OUT><<<1, kTrainBatch, grad_smem_bytes<OUT>(), s>>>(P, dx, dy, dmask, nullptr, (int)n, dgrad, dl);
  float l2[2] = {0.f, 0.f};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(l2, dl, sizeof(l2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dl);
  if (e != cudaSuccess) return GBGEMM_ERR_CUDA;
  if (host_loss) *host_loss = l2[1] > 0.f ? l2[0] / l2[1] : 0.f;
  return GBGEMM_OK;
}

// Adam on mini-batches from the parameters at P (updated in place).
template <int OUT>
int train_impl(float* P, const float* dx, const float* dy, const float* dmask, int64_t n, int epochs, int batch,
               float lr, std::mt19937_64& rng, float* host_loss, cudaStream_t s) {
  constexpr int kParams = Net<OUT>::kParams;
  if (ensure_grad_attr<OUT>() != cudaSuccess) return GBGEMM_ERR_CUDA;
  // work buffers: gradient, Adam moments, epoch permutation, loss
  float* work = nullptr;
  const size_t nperm = (size_t)n;
  const size_t bytes = 3 * kParams * sizeof(float) + nperm * sizeof(int) + 2 * sizeof(float);
  if (cudaMalloc(&work, bytes) != cudaSuccess) return GBGEMM_ERR_ALLOC;
  float* G = work;
  float* m1 = G + kParams;
  float* m2 = m1 + kParams;
  int* perm = reinterpret_cast<int*>(m2 + kParams);
  float* dl = reinterpret_cast<float*>(perm + nperm);
  cudaError_t e = cudaMemsetAsync(m1, 0, 2 * kParams * sizeof(float), s);
  std::vector<int> hp(nperm);
  for (size_t i = 0; i < nperm; ++i) hp[i] = (int)i;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int64_t step = 0;
  double last_epoch_loss = 0.0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    std::shuffle(hp.begin(), hp.end(), rng);
    e = cudaMemcpyAsync(perm, hp.data(), nperm * sizeof(int), cudaMemcpyHostToDevice, s);
    for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
      const int nb = (int)((n - b0) < batch ? (n - b0) : batch);
      mlp_grad_kernel<OUT><<<1, kTrainBatch, grad_smem_bytes<OUT>(), s>>>(P, dx, dy, dmask, perm + b0, nb, G, dl);
      ++step;
      const float c1 = 1.f - (float)std::pow(b1, (double)step), c2 = 1.f - (float)std::pow(b2, (double)step);
      adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(P, G, m1, m2, kParams, lr, b1, b2, eps, c1, c2);
      e = cudaGetLastError();
    }
    // stream order keeps the host copy of the epoch permutation alive until use
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  // loss of the final parameters over the whole set, in batches
  if (e == cudaSuccess) {
    double lsum = 0.0, lcnt = 0.0;
    for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += kTrainBatch) {
      const int nb = (int)((n - b0) < kTrainBatch ? (n - b0) : kTrainBatch);
      for (int i = 0; i < nb; ++i) hp[i] = (int)(b0 + i);
      e = cudaMemcpy(perm, hp.data(), nb * sizeof(int), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) break;
      mlp_grad_kernel<OUT><<<1, kTrainBatch, grad_smem_bytes<OUT>(), s>>>(P, dx, dy, dmask, perm, nb, G, dl);
      float l2[2];
      e = cudaMemcpyAsync(l2, dl, sizeof(l2), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      lsum += l2[0];
      lcnt += l2[1];
    }
    last_epoch_loss = lcnt > 0 ? lsum / lcnt : 0.0;
  }
  cudaFree(work);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return GBGEMM_ERR_CUDA;
  }
  if (host_loss) *host_loss = (float)last_epoch_loss;
  return GBGEMM_OK;
}

}  // namespace

Predictor::Predictor(int outputs) : out_(outputs == GBGEMM_NUM_SCHEDULES ? GBGEMM_NUM_SCHEDULES : GBGEMM_NUM_CONFIGS) {}

Predictor::~Predictor() {
  if (dparams_) cudaFree(dparams_);
}

int Predictor::params() const {
  return out_ == GBGEMM_NUM_SCHEDULES ? Net<GBGEMM_NUM_SCHEDULES>::kParams : Net<GBGEMM_NUM_CONFIGS>::kParams;
}

int Predictor::set(const float* host_params) {
  const size_t bytes = (size_t)params() * sizeof(float);
  if (!dparams_ && cudaMalloc(&dparams_, bytes) != cudaSuccess) {
    cudaGetLastError();
    dparams_ = nullptr;
    return GBGEMM_ERR_ALLOC;
  }
  if (cudaMemcpy(dparams_, host_params, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return GBGEMM_ERR_CUDA;
  ready_ = true;
  return GBGEMM_OK;
}

int Predictor::get(float* host_params) const {
  if (!ready_) return GBGEMM_ERR_NOT_INITIALIZED;
  return cudaMemcpy(host_params, dparams_, (size_t)params() * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
             ? GBGEMM_OK
             : GBGEMM_ERR_CUDA;
}

int Predictor::predict(const float* dx, const uint8_t* dlegal, int64_t n, float* dscores, int* dconfigs,
                       cudaStream_t s) const {
  if (!ready_) return GBGEMM_ERR_NOT_INITIALIZED;
  if (n <= 0) return GBGEMM_OK;
  return out_ == GBGEMM_NUM_SCHEDULES
             ? predict_impl<GBGEMM_NUM_SCHEDULES>(dparams_, dx, dlegal, n, dscores, dconfigs, s)
             : predict_impl<GBGEMM_NUM_CONFIGS>(dparams_, dx, dlegal, n, dscores, dconfigs, s);
}

int Predictor::loss_grad(const float* dx, const float* dy, const float* dmask, int64_t n, float* host_loss,
                         float* dgrad, cudaStream_t s) const {
  if (!ready_) return GBGEMM_ERR_NOT_INITIALIZED;
  if (n <= 0 || n > kTrainBatch) return GBGEMM_ERR_INVALID_VALUE;
  return out_ == GBGEMM_NUM_SCHEDULES
             ? loss_grad_impl<GBGEMM_NUM_SCHEDULES>(dparams_, dx, dy, dmask, n, host_loss, dgrad, s)
             : loss_grad_impl<GBGEMM_NUM_CONFIGS>(dparams_, dx, dy, dmask, n, host_loss, dgrad, s);
}

int Predictor::train(const float* dx, const float* dy, const float* dmask, int64_t n, int epochs, int batch, float lr,
                     uint64_t seed, float* host_loss, cudaStream_t s) {
  if (n <= 0 || epochs < 1 || batch < 1 || batch > kTrainBatch || !(lr > 0.f)) return GBGEMM_ERR_INVALID_VALUE;
  if (n > 0x7FFFFFFF) return GBGEMM_ERR_INVALID_VALUE;
  std::mt19937_64 rng(seed);
  if (!ready_) {
    const std::vector<float> p = out_ == GBGEMM_NUM_SCHEDULES ? he_init<GBGEMM_NUM_SCHEDULES>(rng)
                                                              : he_init<GBGEMM_NUM_CONFIGS>(rng);
    const int rc = set(p.data());
    if (rc != GBGEMM_OK) return rc;
  }
  return out_ == GBGEMM_NUM_SCHEDULES
             ? train_impl<GBGEMM_NUM_SCHEDULES>(dparams_, dx, dy, dmask, n, epochs, batch, lr, rng, host_loss, s)
             : train_impl<GBGEMM_NUM_CONFIGS>(dparams_, dx, dy, dmask, n, epochs, batch, lr, rng, host_loss, s);
}

}  // namespace gbg
