// Row-scaled quantisation of an FP32 matrix into BF16 or FP8-E4M3 codes.
//
// Not part of the paper (its kernels are FP32 only, Section 4.1); this is
// the storage form of the low-precision matrix passes.  Rule, per row i:
//   s_i  = amax_i / QMAX  (IEEE single division; QMAX = 1 for BF16, 448 for
//          E4M3; s_i = 1 when the row is all zero)
//   Q_ij = round-to-nearest-even of (A_ij / s_i) into the format, saturating
//          to the largest finite E4M3 value.
// The conversions are the hardware's round-to-nearest-even instructions.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kf_device.cuh"
#include "kf_internal.h"

namespace kf {
namespace {

__global__ void __launch_bounds__(256) quantize_rows_kernel(const float* __restrict__ A, int64_t lda,
                                                            int64_t m, int64_t n, int fmt,
                                                            void* __restrict__ Q,
                                                            float* __restrict__ scale) {
  __shared__ float s_max[8];
  __shared__ float s_scale;
  const int64_t i = blockIdx.x;
  if (i >= m) return;
  const float* row = A + i * lda;
  float amax = 0.f;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) amax = fmaxf(amax, fabsf(row[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL_MASK, amax, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, s_max[w]);
    const float qmax = (fmt == FMT_E4M3) ? 448.f : 1.f;
    const float s = (mx > 0.f) ? __fdiv_rn(mx, qmax) : 1.f;
    s_scale = s;
    scale[i] = s;
  }
  __syncthreads();
  const float s = s_scale;
  if (fmt == FMT_E4M3) {
    unsigned char* q = static_cast<unsigned char*>(Q) + i * n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
      q[j] = (unsigned char)__nv_cvt_float_to_fp8(__fdiv_rn(row[j], s), __NV_SATFINITE, __NV_E4M3);
  } else {
    __nv_bfloat16* q = static_cast<__nv_bfloat16*>(Q) + i * n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) q[j] = __float2bfloat16_rn(__fdiv_rn(row[j], s));
  }
}

// out[b] = max_j |v_b[j]|: one block per vector, fixed reduction tree
// (max is exact, so the result does not depend on the order anyway).
struct NormArgs {
  const float* v[4];
};

__global__ void __launch_bounds__(1024) colnorm_kernel(NormArgs a, int64_t n, float* __restrict__ out) {
  __shared__ float s_max[32];
  const float* v = a.v[blockIdx.x];
  float mx = 0.f;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(__ldg(v + j)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL_MASK, mx, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = s_max[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL_MASK, mx, o));
    if (threadIdx.x == 0) out[blockIdx.x] = mx;
  }
}

}  // namespace

int launch_quantize_rows(const float* A, int64_t lda, int64_t m, int64_t n, int fmt, void* Q,
                         float* scale, void* stream, const char** why) {
  if (m == 0) return 0;
  if (m > 0x7fffffffLL) { *why = "too many rows"; return -2; }
  quantize_rows_kernel<<<(unsigned)m, 256, 0, (cudaStream_t)stream>>>(A, lda, m, n, fmt, Q, scale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { *why = cudaGetErrorString(e); return -7; }
  return 0;
}

int launch_colnorms(const float* const* v, int nv, int64_t n, float* out, void* stream, const char** why) {
  if (nv < 1 || nv > 4) { *why = "one to four vectors"; return -1; }
  NormArgs a{};
  for (int k = 0; k < nv; ++k) a.v[k] = v[k];
  colnorm_kernel<<<nv, 1024, 0, (cudaStream_t)stream>>>(a, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { *why = cudaGetErrorString(e); return -7; }
  return 0;
}

}  // namespace kf
