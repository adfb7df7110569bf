// Learned cost model: a 3-layer perceptron with ReLU activations,
//   h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  f = W3 h2 + b3,
// trained on measured plan timings (mean squared error on log time) with
// the Adam update (Kingma and Ba, Algorithm 1).  It ranks fusion plans in
// place of (or beside) the paper's additive predictor (Section 3.2).
//
// Parameters are one flat FP32 array in the order W1 (H x D, row major),
// b1 (H), W2 (H x H), b2 (H), W3 (1 x H), b3 (1).  H = 64; D <= 32.
// Kernels (FP32 FMA; there is no dense contraction large enough for the
// tensor cores):
//   forward   : a block of 64 threads (one per hidden unit) runs 32 samples
//               at a time through the three layers, activations in shared
//               memory;
//   loss/grad : the same forward, then the chain rule; each thread owns the
//               parameters of its hidden unit and accumulates their
//               gradient in registers over the samples its block visits;
//               per-block partial gradients are then added in block order
//               by a second kernel (deterministic);
//   adam      : element-wise update with bias correction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/kf.h"
#include "kf_device.cuh"

namespace kf {
const char* set_error_message(const std::string& msg);
int device_sm_count();

namespace {

constexpr int H = 64;
constexpr int DMAX = 32;
constexpr int SB = 32;  // samples per tile

__host__ __device__ constexpr int n_params(int d) { return H * d + H + H * H + H + H + 1; }

struct Layout {
  int w1, b1, w2, b2, w3, b3;
};
__host__ __device__ inline Layout layout(int d) {
  Layout L;
  L.w1 = 0;
  L.b1 = H * d;
  L.w2 = L.b1 + H;
  L.b2 = L.w2 + H * H;
  L.w3 = L.b2 + H;
  L.b3 = L.w3 + H;
  return L;
}

// Forward of one tile of samples: fills z1, h1, z2, h2 (shared) and f.
__device__ void tile_forward(const float* __restrict__ P, int d, const float* __restrict__ X, int s0, int batch,
                             float (*xs)[DMAX], float (*z1)[H], float (*z2)[H], float* f) {
  const Layout L = layout(d);
  const int j = threadIdx.x;  // hidden unit
  for (int i = j; i < SB * d; i += H) {
    const int s = i / d, c = i % d;
    xs[s][c] = (s0 + s < batch) ? X[(int64_t)(s0 + s) * d + c] : 0.f;
  }
  __syncthreads();
  for (int s = 0; s < SB; ++s) {
    float a = P[L.b1 + j];
    for (int c = 0; c < d; ++c) a = fmaf(P[L.w1 + j * d + c], xs[s][c], a);
    z1[s][j] = a;
  }
  __syncthreads();
  for (int s = 0; s < SB; ++s) {
    float a = P[L.b2 + j];
    for (int k = 0; k < H; ++k) a = fmaf(P[L.w2 + j * H + k], fmaxf(z1[s][k], 0.f), a);
    z2[s][j] = a;
  }
  __syncthreads();
  if (j < SB) {
    float a = P[L.b3];
    for (int k = 0; k < H; ++k) a = fmaf(P[L.w3 + k], fmaxf(z2[j][k], 0.f), a);
    f[j] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(H) mlp_forward_kernel(const float* __restrict__ P, int d, const float* __restrict__ X,
                                                         int batch, float* __restrict__ out) {
  __shared__ float xs[SB][DMAX];
  __shared__ float z1[SB][H], z2[SB][H];
  __shared__ float f[SB];
  for (int s0 = blockIdx.x * SB; s0 < batch; s0 += gridDim.x * SB) {
    tile_forward(P, d, X, s0, batch, xs, z1, z2, f);
    if (threadIdx.x < SB && s0 + threadIdx.x < batch) out[s0 + threadIdx.x] = f[threadIdx.x];
    __syncthreads();
  }
}

// Per-block partial gradient of L = mean_s (f_s - y_s)^2 and partial loss.
__global__ void __launch_bounds__(H) mlp_grad_kernel(const float* __restrict__ P, int d, const float* __restrict__ X,
                                                      const float* __restrict__ Y, int batch,
                                                      float* __restrict__ part, float* __restrict__ lpart) {
  __shared__ float xs[SB][DMAX];
  __shared__ float z1[SB][H], z2[SB][H];
  __shared__ float f[SB], df[SB];
  __shared__ float dz2[SB][H];
  const Layout L = layout(d);
  const int np = n_params(d);
  const int j = threadIdx.x;
  float gw1[DMAX], gw2[H];
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
#pragma unroll
  for (int c = 0; c < DMAX; ++c) gw1[c] = 0.f;
#pragma unroll
  for (int k = 0; k < H; ++k) gw2[k] = 0.f;
  const float inv_b = 1.f / (float)batch;
  for (int s0 = blockIdx.x * SB; s0 < batch; s0 += gridDim.x * SB) {
    tile_forward(P, d, X, s0, batch, xs, z1, z2, f);
    if (j < SB) {
      const bool ok = s0 + j < batch;
      const float e = ok ? f[j] - Y[s0 + j] : 0.f;
      df[j] = 2.f * e * inv_b;
      loss += e * e;
    }
    __syncthreads();
    // layer 3 and dz2 (thread j: hidden unit j of layer 2)
    for (int s = 0; s < SB; ++s) {
      const float h2 = fmaxf(z2[s][j], 0.f);
      gw3 = fmaf(df[s], h2, gw3);
      dz2[s][j] = z2[s][j] > 0.f ? df[s] * P[L.w3 + j] : 0.f;
    }
    if (j == 0)
      for (int s = 0; s < SB; ++s) gb3 += df[s];
    __syncthreads();
    // layer 2: dW2[j][k] += dz2[s][j] h1[s][k]
    for (int s = 0; s < SB; ++s) {
      const float g = dz2[s][j];
      gb2 += g;
#pragma unroll
      for (int k = 0; k < H; ++k) gw2[k] = fmaf(g, fmaxf(z1[s][k], 0.f), gw2[k]);
    }
    // layer 1 (thread j: hidden unit j of layer 1): dz1 = (W2^T dz2) * [z1 > 0]
    for (int s = 0; s < SB; ++s) {
      float dh = 0.f;
      for (int k = 0; k < H; ++k) dh = fmaf(P[L.w2 + k * H + j], dz2[s][k], dh);
      const float g = z1[s][j] > 0.f ? dh : 0.f;
      gb1 += g;
#pragma unroll
      for (int c = 0; c < DMAX; ++c)
        if (c < d) gw1[c] = fmaf(g, xs[s][c], gw1[c]);
    }
    __syncthreads();
  }
  float* out = part + (int64_t)blockIdx.x * np;
  for (int c = 0; c < d; ++c) out[L.w1 + j * d + c] = gw1[c];
  out[L.b1 + j] = gb1;
#pragma unroll
  for (int k = 0; k < H; ++k) out[L.w2 + j * H + k] = gw2[k];
  out[L.b2 + j] = gb2;
  out[L.w3 + j] = gw3;
  if (j == 0) out[L.b3] = gb3;
  // loss: lanes < SB hold per-sample sums; combine in a fixed order
  __shared__ float lsh[H];
  lsh[j] = loss;
  __syncthreads();
  if (j == 0) {
    float t = 0.f;
    for (int k = 0; k < SB; ++k) t += lsh[k];
    lpart[blockIdx.x] = t;
  }
}

// grad[p] = sum over blocks (in order) of part[b][p]; loss likewise.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, const float* __restrict__ lpart, int nblocks, int np,
                                  int batch, float* __restrict__ grad, float* __restrict__ loss) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * np + p];
    grad[p] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss != nullptr) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += lpart[b];
    *loss = s / (float)batch;
  }
}

__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                                float* __restrict__ V, int n, float lr, float b1, float b2, float eps, float c1,
                                float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    const float mh = m / c1, vh = v / c2;
    P[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

int grad_blocks(int batch) {
  const int tiles = (batch + SB - 1) / SB;
  return std::max(1, std::min(tiles, device_sm_count() * 2));
}

}  // namespace
}  // namespace kf

using namespace kf;

extern "C" {

kf_status kf_mlp_param_count(int d_in, int hidden, int* count) {
  if (count == nullptr || hidden != H || d_in < 1 || d_in > DMAX) {
    set_error_message("the cost model has 64 hidden units and 1..32 inputs");
    return KF_ERR_INVALID_ARG;
  }
  *count = n_params(d_in);
  return KF_OK;
}

kf_status kf_mlp_workspace_size(int d_in, int hidden, int batch, size_t* bytes) {
  int np = 0;
  kf_status st = kf_mlp_param_count(d_in, hidden, &np);
  if (st != KF_OK) return st;
  if (bytes == nullptr || batch < 0) { set_error_message("bad arguments"); return KF_ERR_INVALID_ARG; }
  const int nb = grad_blocks(batch);
  *bytes = ((size_t)nb * np + nb + 64) * sizeof(float);
  return KF_OK;
}

kf_status kf_mlp_forward(const float* params, int d_in, int hidden, const float* X, int batch, float* out,
                         void* stream) {
  int np = 0;
  kf_status st = kf_mlp_param_count(d_in, hidden, &np);
  if (st != KF_OK) return st;
  if (batch < 0 || (batch > 0 && (params == nullptr || X == nullptr || out == nullptr))) {
    set_error_message("bad arguments");
    return KF_ERR_INVALID_ARG;
  }
  if (batch == 0) return KF_OK;
  const int tiles = (batch + SB - 1) / SB;
  const int grid = std::min(tiles, device_sm_count() * 8);
  mlp_forward_kernel<<<grid, H, 0, (cudaStream_t)stream>>>(params, d_in, X, batch, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  return KF_OK;
}

kf_status kf_mlp_loss_grad(const float* params, int d_in, int hidden, const float* X, const float* y, int batch,
                           float* grad, float* loss, void* ws, size_t ws_bytes, void* stream) {
  int np = 0;
  kf_status st = kf_mlp_param_count(d_in, hidden, &np);
  if (st != KF_OK) return st;
  if (batch <= 0 || params == nullptr || X == nullptr || y == nullptr || grad == nullptr) {
    set_error_message("bad arguments");
    return KF_ERR_INVALID_ARG;
  }
  size_t need = 0;
  kf_mlp_workspace_size(d_in, hidden, batch, &need);
  if (ws == nullptr || ws_bytes < need) { set_error_message("workspace too small"); return KF_ERR_WORKSPACE; }
  const int nb = grad_blocks(batch);
  float* part = static_cast<float*>(ws);
  float* lpart = part + (size_t)nb * np;
  mlp_grad_kernel<<<nb, H, 0, (cudaStream_t)stream>>>(params, d_in, X, y, batch, part, lpart);
  mlp_reduce_kernel<<<(np + 255) / 256, 256, 0, (cudaStream_t)stream>>>(part, lpart, nb, np, batch, grad, loss);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  return KF_OK;
}

kf_status kf_mlp_adam(float* params, const float* grad, float* m, float* v, int count, int step, float lr, float b1,
                      float b2, float eps, void* stream) {
  if (params == nullptr || grad == nullptr || m == nullptr || v == nullptr || count <= 0 || step < 1) {
    set_error_message("bad arguments");
    return KF_ERR_INVALID_ARG;
  }
  const float c1 = 1.f - powf(b1, (float)step);
  const float c2 = 1.f - powf(b2, (float)step);
  mlp_adam_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, b1, b2, eps,
                                                                          c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  return KF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- training

namespace kf {
namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used counter-style: the key
// of stream (seed, id) is mix(mix(seed) + id), element i is
// mix(key + (i + 1) * GAMMA); its top 24 bits b give b * 2^-23 - 1 in [-1, 1).
constexpr uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;
uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t INIT_STREAM_ID = 15;  // the network's stream

float sm_uniform(uint64_t key, uint64_t i) {
  const uint64_t b = sm_mix(key + (i + 1) * SM_GAMMA) >> 40;
  return (float)b * (1.0f / 8388608.0f) - 1.0f;
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct TrainLayout {
  size_t xs, y, grad, m, v, loss, mlpws, total;
};

TrainLayout train_layout(int count, int d) {
  TrainLayout L{};
  const size_t np = (size_t)n_params(d);
  size_t mlp = 0;
  kf_mlp_workspace_size(d, H, count, &mlp);
  size_t off = 0;
  L.xs = off; off += al256((size_t)count * d * sizeof(float));
  L.y = off; off += al256((size_t)count * sizeof(float));
  L.grad = off; off += al256(np * sizeof(float));
  L.m = off; off += al256(np * sizeof(float));
  L.v = off; off += al256(np * sizeof(float));
  L.loss = off; off += 256;
  L.mlpws = off; off += al256(mlp);
  L.total = off;
  return L;
}

}  // namespace
}  // namespace kf

extern "C" {

kf_status kf_planner_train_workspace_size(int count, int d_in, size_t* bytes) {
  if (bytes == nullptr || count < 1 || d_in != KF_PLAN_NFEATURES) {
    set_error_message("count >= 1 samples of KF_PLAN_NFEATURES features expected");
    return KF_ERR_INVALID_ARG;
  }
  *bytes = train_layout(count, d_in).total;
  return KF_OK;
}

kf_status kf_planner_train(const float* features, const double* measured_ms, const double* analytic_us,
                           const int64_t* script_ids, int count, int d_in, const kf_train_options* opt,
                           const float* params_init, float* params, void* ws, size_t ws_bytes, void* stream,
                           kf_cost_model* model, float* loss_out, int loss_cap, int* n_loss) {
  if (features == nullptr || measured_ms == nullptr || analytic_us == nullptr || opt == nullptr ||
      params == nullptr || model == nullptr || count < 1 || d_in != KF_PLAN_NFEATURES) {
    set_error_message("null argument, no samples, or not KF_PLAN_NFEATURES features");
    return KF_ERR_INVALID_ARG;
  }
  if (opt->epochs < 1 || !(opt->lr > 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) ||
      !(opt->beta2 >= 0.f && opt->beta2 < 1.f) || !(opt->eps > 0.f) || opt->loss_every < 0 ||
      (opt->centre_per_script && script_ids == nullptr) || (loss_cap > 0 && loss_out == nullptr)) {
    set_error_message("bad training options");
    return KF_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    if (!(measured_ms[i] > 0.0) || !std::isfinite(measured_ms[i]) || !std::isfinite(analytic_us[i])) {
      set_error_message("measured times must be positive and finite");
      return KF_ERR_INVALID_ARG;
    }
  }
  const int d = d_in;
  const TrainLayout L = train_layout(count, d);
  if (ws == nullptr || ws_bytes < L.total) {
    set_error_message("workspace missing or smaller than kf_planner_train_workspace_size()");
    return KF_ERR_WORKSPACE;
  }
  const int np = n_params(d);
  cudaStream_t st = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  float* dX = reinterpret_cast<float*>(w + L.xs);
  float* dy = reinterpret_cast<float*>(w + L.y);
  float* dg = reinterpret_cast<float*>(w + L.grad);
  float* dm = reinterpret_cast<float*>(w + L.m);
  float* dv = reinterpret_cast<float*>(w + L.v);
  float* dloss = reinterpret_cast<float*>(w + L.loss);
  void* dmlp = w + L.mlpws;
  size_t mlp_bytes = L.total - L.mlpws;

  // Feature standardisation: (f - mean) / (population std + 1e-6), in double.
  std::vector<double> mean(d, 0.0), sd(d, 0.0);
  for (int i = 0; i < count; ++i)
    for (int c = 0; c < d; ++c) mean[c] += features[(size_t)i * d + c];
  for (int c = 0; c < d; ++c) mean[c] /= count;
  for (int i = 0; i < count; ++i)
    for (int c = 0; c < d; ++c) {
      const double t = features[(size_t)i * d + c] - mean[c];
      sd[c] += t * t;
    }
  std::vector<double> inv(d);
  for (int c = 0; c < d; ++c) inv[c] = 1.0 / (std::sqrt(sd[c] / count) + 1e-6);
  std::vector<float> Xs((size_t)count * d);
  for (int i = 0; i < count; ++i)
    for (int c = 0; c < d; ++c) Xs[(size_t)i * d + c] = (float)((features[(size_t)i * d + c] - mean[c]) * inv[c]);
  // Targets: ln(measured ms) - w ln(analytic ms) (analytic floored at 1 ns),
  // centred per script when asked (only differences between one script's
  // plans decide a choice).
  std::vector<double> tgt(count);
  for (int i = 0; i < count; ++i)
    tgt[i] = std::log(measured_ms[i]) - (double)opt->analytic_weight * std::log(std::max(analytic_us[i], 1e-3) * 1e-3);
  if (opt->centre_per_script) {
    std::map<int64_t, std::pair<double, int>> acc;
    for (int i = 0; i < count; ++i) {
      auto& a = acc[script_ids[i]];
      a.first += tgt[i];
      a.second += 1;
    }
    for (int i = 0; i < count; ++i) {
      const auto& a = acc[script_ids[i]];
      tgt[i] -= a.first / a.second;
    }
  }
  std::vector<float> y(count);
  for (int i = 0; i < count; ++i) y[i] = (float)tgt[i];

  cudaError_t e = cudaMemcpyAsync(dX, Xs.data(), Xs.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y.data(), y.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  // Initial weights: the caller's, or He-uniform (u * sqrt(6 / fan_in), u from
  // the SplitMix64 stream (seed, 15) at the parameter's index) with zero biases.
  std::vector<float> init;
  if (e == cudaSuccess) {
    if (params_init != nullptr) {
      e = cudaMemcpyAsync(params, params_init, (size_t)np * sizeof(float), cudaMemcpyDeviceToDevice, st);
    } else {
      init.assign(np, 0.f);
      const uint64_t key = sm_mix(sm_mix(opt->seed) + INIT_STREAM_ID);
      const Layout Lp = layout(d);
      auto fill = [&](int off, int count_w, int fan_in) {
        const double g = std::sqrt(6.0 / fan_in);
        for (int k = 0; k < count_w; ++k)
          init[off + k] = (float)((double)sm_uniform(key, (uint64_t)(off + k)) * g);
      };
      fill(Lp.w1, H * d, d);
      fill(Lp.w2, H * H, H);
      fill(Lp.w3, H, H);
      e = cudaMemcpyAsync(params, init.data(), (size_t)np * sizeof(float), cudaMemcpyHostToDevice, st);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(dm, 0, (size_t)np * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dv, 0, (size_t)np * sizeof(float), st);
  if (e != cudaSuccess) {
    set_error_message(std::string("training set-up: ") + cudaGetErrorString(e));
    return KF_ERR_CUDA;
  }
  int nl = 0;
  auto record = [&]() -> kf_status {
    float h = 0.f;
    cudaError_t r = cudaMemcpyAsync(&h, dloss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    if (r != cudaSuccess) {
      set_error_message(std::string("reading the loss: ") + cudaGetErrorString(r));
      return KF_ERR_CUDA;
    }
    if (nl < loss_cap) loss_out[nl] = h;
    ++nl;
    return KF_OK;
  };
  // Full-batch Adam (Kingma and Ba, Algorithm 1), every step in the
  // library's kernels.
  for (int t = 1; t <= opt->epochs; ++t) {
    kf_status sst = kf_mlp_loss_grad(params, d, H, dX, dy, count, dg, dloss, dmlp, mlp_bytes, stream);
    if (sst != KF_OK) return sst;
    if (t == 1 || (opt->loss_every > 0 && t % opt->loss_every == 0)) {
      sst = record();
      if (sst != KF_OK) return sst;
    }
    sst = kf_mlp_adam(params, dg, dm, dv, np, t, opt->lr, opt->beta1, opt->beta2, opt->eps, stream);
    if (sst != KF_OK) return sst;
  }
  kf_status sst = kf_mlp_loss_grad(params, d, H, dX, dy, count, dg, dloss, dmlp, mlp_bytes, stream);
  if (sst != KF_OK) return sst;
  sst = record();
  if (sst != KF_OK) return sst;
  if (n_loss != nullptr) *n_loss = nl;
  model->params = params;
  for (int c = 0; c < KF_PLAN_NFEATURES; ++c) {
    model->mean[c] = (float)mean[c];
    model->inv_std[c] = (float)inv[c];
  }
  model->analytic_weight = opt->analytic_weight;
  return KF_OK;
}

}  // extern "C"
