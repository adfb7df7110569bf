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

#include <string>

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
