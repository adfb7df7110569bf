// Vector-pass kernels: one read of the input vectors serves every fused
// BLAS-1 call of a fusion (nesting depth 1 in the paper's Section 3.3).
//
// Every map call the library offers for vectors (AXPY, AXPBY, SCAL, WAXPBY,
// VADD, copies) is linear in its vector operands, so the host folds a fused
// chain of them into one coefficient row per stored output and per DOT
// operand (VecProg::C, P, Q).  The kernel reads each input once (16-byte
// streaming loads, grid-stride over a grid that is a multiple of the SM
// count), writes each output once, and reduces the dot products per block;
// the last block to finish adds the per-block partials in block order
// (Section 3.2.2, option (ii)), in double when the vectors are long.
#include <atomic>
#include <map>
#include <string>
#include <vector>
#include <mutex>
#include <tuple>

#include <algorithm>

#include "kf_device.cuh"
#include "kf_internal.h"

namespace kf {
namespace {

// Linear combination sum_k c_k x_k with every product rounded on its own and
// the products added in k order (no fused multiply-add), so that alpha x +
// beta y with beta y = -alpha x is exactly zero.
template <int NIN>
__device__ __forceinline__ float4 lin4(const float (&c)[VP_MAXIN], const float4 (&x)[NIN], int nin) {
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < NIN; ++k) {
    if (k < nin) {
      const float ck = c[k];
      const float4 p = make_float4(__fmul_rn(ck, x[k].x), __fmul_rn(ck, x[k].y), __fmul_rn(ck, x[k].z),
                                   __fmul_rn(ck, x[k].w));
      if (k == 0) {
        r = p;
      } else {
        r.x = __fadd_rn(r.x, p.x); r.y = __fadd_rn(r.y, p.y);
        r.z = __fadd_rn(r.z, p.z); r.w = __fadd_rn(r.w, p.w);
      }
    }
  }
  return r;
}

template <int NIN>
__device__ __forceinline__ float lin1(const float (&c)[VP_MAXIN], const float (&x)[NIN], int nin) {
  float r = 0.f;
#pragma unroll
  for (int k = 0; k < NIN; ++k)
    if (k < nin) r = (k == 0) ? __fmul_rn(c[k], x[k]) : __fadd_rn(r, __fmul_rn(c[k], x[k]));
  return r;
}

template <int NIN, int NOUT, int NDOT, int U>
__global__ void __launch_bounds__(256) vecprog_kernel(const __grid_constant__ VecProg P) {
  pdl_enter();
  constexpr int ND = NDOT > 0 ? NDOT : 1;
  __shared__ float s_red[ND][8];
  __shared__ int s_last;
  const int64_t n = P.n;
  const int nin = P.nin, nout = P.nout, ndot = P.ndot;
  float acc[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d] = 0.f;

  const int64_t n4 = n >> 2;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * U;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x; base < n4; base += step) {
    float4 x[U][NIN];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = base + (int64_t)u * blockDim.x;
#pragma unroll
      for (int k = 0; k < NIN; ++k)
        x[u][k] = (k < nin && c < n4) ? ld_stream_f4(P.in[k] + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = base + (int64_t)u * blockDim.x;
      if (c < n4) {
#pragma unroll
        for (int j = 0; j < NOUT; ++j)
          if (j < nout) st_stream_f4(P.out[j] + 4 * c, lin4<NIN>(P.C[j], x[u], nin));
#pragma unroll
        for (int d = 0; d < NDOT; ++d) {
          if (d < ndot) {
            const float4 a = lin4<NIN>(P.P[d], x[u], nin);
            const float4 b = lin4<NIN>(P.Q[d], x[u], nin);
            float t = a.x * b.x;
            t = fmaf(a.y, b.y, t);
            t = fmaf(a.z, b.z, t);
            t = fmaf(a.w, b.w, t);
            acc[d] += t;
          }
        }
      }
    }
  }
  // Ragged tail (n mod 4 elements) in block 0.
  if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
    const int64_t i = n4 * 4 + threadIdx.x;
    float xs[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) xs[k] = (k < nin) ? P.in[k][i] : 0.f;
#pragma unroll
    for (int j = 0; j < NOUT; ++j)
      if (j < nout) P.out[j][i] = lin1<NIN>(P.C[j], xs, nin);
#pragma unroll
    for (int d = 0; d < NDOT; ++d)
      if (d < ndot) acc[d] += lin1<NIN>(P.P[d], xs, nin) * lin1<NIN>(P.Q[d], xs, nin);
  }

  // the finishing step only when this launch has dot products (the
  // instance may have room for more than it was given)
  if (NDOT > 0 && ndot > 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < NDOT; ++d) {
      const float v = warp_sum(acc[d]);
      if (lane == 0) s_red[d][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int d = 0; d < NDOT; ++d) {
        if (d < ndot) {
          float s = 0.f;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[d][w];
          P.dotpart[(int64_t)d * gridDim.x + blockIdx.x] = s;
        }
      }
      __threadfence();
      s_last = atomicAdd(P.counter, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      // Warp d finishes dot d: lanes stride the block partials, then a fixed
      // shuffle tree; the result does not depend on block timing.
      if (warp < ndot) {
        const float* part = P.dotpart + (int64_t)warp * gridDim.x;
        if (P.fp64_final) {
          double s = 0.0;
          for (unsigned b = lane; b < gridDim.x; b += 32) s += (double)__ldcg(part + b);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
          if (lane == 0) *P.dot_out[warp] = (float)s;
        } else {
          float s = 0.f;
          for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(part + b);
          s = warp_sum(s);
          if (lane == 0) *P.dot_out[warp] = s;
        }
      }
      if (threadIdx.x == 0) *P.counter = 0u;
    }
  }
}

// Element-wise variant for vectors whose base addresses are not 16-byte aligned.
template <int NIN, int NOUT, int NDOT>
__global__ void __launch_bounds__(256) vecprog_scalar_kernel(const __grid_constant__ VecProg P) {
  pdl_enter();
  constexpr int ND = NDOT > 0 ? NDOT : 1;
  __shared__ float s_red[ND][8];
  __shared__ int s_last;
  const int64_t n = P.n;
  const int nin = P.nin, nout = P.nout, ndot = P.ndot;
  float acc[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d] = 0.f;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    float xs[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) xs[k] = (k < nin) ? P.in[k][i] : 0.f;
#pragma unroll
    for (int j = 0; j < NOUT; ++j)
      if (j < nout) P.out[j][i] = lin1<NIN>(P.C[j], xs, nin);
#pragma unroll
    for (int d = 0; d < NDOT; ++d)
      if (d < ndot) acc[d] += lin1<NIN>(P.P[d], xs, nin) * lin1<NIN>(P.Q[d], xs, nin);
  }
  // the finishing step only when this launch has dot products (the
  // instance may have room for more than it was given)
  if (NDOT > 0 && ndot > 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < NDOT; ++d) {
      const float v = warp_sum(acc[d]);
      if (lane == 0) s_red[d][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int d = 0; d < ndot; ++d) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[d][w];
        P.dotpart[(int64_t)d * gridDim.x + blockIdx.x] = s;
      }
      __threadfence();
      s_last = atomicAdd(P.counter, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (warp < ndot) {
        const float* part = P.dotpart + (int64_t)warp * gridDim.x;
        double s = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) s += (double)__ldcg(part + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
        if (lane == 0) *P.dot_out[warp] = (float)s;
      }
      if (threadIdx.x == 0) *P.counter = 0u;
    }
  }
}

struct VEntry {
  const void* fn;
  int nin, nout, ndot, u;
  int occ;
};
using VKey = std::tuple<int, int, int, int, bool>;  // nin nout ndot unroll vec

std::map<VKey, VEntry>& vregistry() {
  static std::map<VKey, VEntry> r;
  return r;
}

template <int NIN, int NOUT, int NDOT, int U>
void vreg() {
  vregistry()[VKey(NIN, NOUT, NDOT, U, true)] =
      VEntry{(const void*)&vecprog_kernel<NIN, NOUT, NDOT, U>, NIN, NOUT, NDOT, U, 0};
}
template <int NIN, int NOUT, int NDOT>
void vreg_s() {
  vregistry()[VKey(NIN, NOUT, NDOT, 1, false)] =
      VEntry{(const void*)&vecprog_scalar_kernel<NIN, NOUT, NDOT>, NIN, NOUT, NDOT, 1, 0};
}

template <int NIN, int NOUT, int NDOT>
void vreg_all() {
  vreg<NIN, NOUT, NDOT, 2>();
  vreg<NIN, NOUT, NDOT, 4>();
  vreg_s<NIN, NOUT, NDOT>();
}

std::once_flag g_vreg_once;
void ensure_vregistry() {
  std::call_once(g_vreg_once, [] {
    // exact fits for the elementaries and the named sequences
    vreg_all<1, 1, 0>();   // SCAL, copy
    vreg_all<2, 1, 0>();   // AXPY, AXPBY, WAXPBY
    vreg_all<3, 1, 0>();   // VADD
    vreg_all<2, 0, 1>();   // DOT
    vreg_all<3, 1, 1>();   // AXPYDOT
    // general fusions of the planner
    vreg_all<4, 2, 1>();
    vreg_all<4, 4, 2>();
    vreg_all<6, 4, 4>();
  });
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

size_t vecprog_workspace_bytes(int ndot) {
  return WS_HEADER + 256 + (size_t)(ndot > 0 ? ndot : 1) * VP_MAXBLOCKS * sizeof(float);
}

std::string vec_cache_key(const VecProg& P);
bool tune_cache_get_vec(const std::string& k, VecTune* t);
extern std::atomic<int> g_autotune_reps;
extern thread_local bool g_in_search;
bool tune_on_first_use(void* stream);
int autotune_vecprog(VecProg& P, void* stream, int reps, VecTune* best, float* best_ms, float* auto_ms);
void tune_cache_put_vec(const std::string& k, const VecTune& t);

int launch_vecprog(VecProg& P, const VecTune& tune_in, void* stream, const char** why) {
  ensure_vregistry();
  VecTune tune = tune_in;
  if (tune.unroll == 0 && !tune_cache_get_vec(vec_cache_key(P), &tune)) {
    bool tuned = false;
    if (tune_on_first_use(stream)) {
      VecTune bt{};
      float bm = 0.f;
      tuned = autotune_vecprog(P, stream, g_autotune_reps.load(), &bt, &bm, nullptr) == 0;
      if (tuned) tune = bt;
    }
    if (!tuned) tune = VecTune{256, 4, 0};
  }
  bool vec = true;
  for (int k = 0; k < P.nin; ++k) vec = vec && al16(P.in[k]);
  for (int j = 0; j < P.nout; ++j) vec = vec && al16(P.out[j]);
  auto& R = vregistry();
  static const int shapes[][3] = {{1, 1, 0}, {2, 1, 0}, {3, 1, 0}, {2, 0, 1}, {3, 1, 1},
                                  {4, 2, 1}, {4, 4, 2}, {6, 4, 4}};
  int u = vec ? (tune.unroll >= 4 ? 4 : 2) : 1;
  const VEntry* e = nullptr;
  for (auto& s : shapes) {
    if (P.nin <= s[0] && P.nout <= s[1] && P.ndot <= s[2]) {
      auto it = R.find(VKey(s[0], s[1], s[2], u, vec));
      if (it != R.end()) { e = &it->second; break; }
    }
  }
  if (e == nullptr) { *why = "vector fusion too large"; return -10; }
  const int threads = 256;
  int64_t blocks = tune.blocks;
  if (blocks <= 0) {
    const int64_t per_block = (int64_t)threads * (vec ? 4 * u : 1);
    const int64_t need = (P.n + per_block - 1) / per_block;
    blocks = std::min<int64_t>((int64_t)device_sm_count() * 4, std::max<int64_t>(1, need));
  }
  blocks = std::min<int64_t>(blocks, VP_MAXBLOCKS);
  void* args[] = {&P};
  cudaError_t err = launch_pdl(e->fn, dim3((unsigned)blocks), dim3(threads), args, 0, stream);
  if (err != cudaSuccess) { *why = cudaGetErrorString(err); return -7; }
  return 0;
}


// Empirical search over rows in flight (2 or 4 chunks per input) and grid
// size (2, 4 or 8 blocks per SM); best to the tuning cache.  Synchronous.
int autotune_vecprog(VecProg& P, void* stream, int reps, VecTune* best, float* best_ms, float* auto_ms) {
  struct Scope {  // no nested first-use tuning inside the search
    bool was;
    Scope() : was(g_in_search) { g_in_search = true; }
    ~Scope() { g_in_search = was; }
  } scope;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // Mean of `reps` back-to-back launches between one pair of events, best of
  // two rounds (host launch latency is not timed).
  auto time_one = [&](const VecTune& t, float* ms) -> int {
    const char* why = nullptr;
    int rc = launch_vecprog(P, t, stream, &why);
    float bestr = 1e30f;
    for (int round = 0; round < 2 && rc == 0; ++round) {
      cudaEventRecord(a, st);
      for (int r = 0; r < reps && rc == 0; ++r) rc = launch_vecprog(P, t, stream, &why);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float x = 0.f;
      cudaEventElapsedTime(&x, a, b);
      bestr = std::min(bestr, x / (float)reps);
    }
    if (rc != 0) return rc;
    *ms = bestr;
    return 0;
  };
  // the current choice: the cache's entry, else the built-in default
  VecTune cur{};
  if (!tune_cache_get_vec(vec_cache_key(P), &cur)) cur = VecTune{256, 4, 0};
  float am = 1e30f;
  {  // warm the GPU with the current choice, then time it
    float ms = 0.f;
    time_one(VecTune{0, 0, 0}, &ms);
    if (time_one(VecTune{0, 0, 0}, &ms) == 0) am = ms;
  }
  float bm = 1e30f;
  VecTune bt{256, 4, 0};
  for (int u : {2, 4})
    for (int k : {2, 4, 8}) {
      VecTune t{256, u, device_sm_count() * k};
      float ms = 0.f;
      if (time_one(t, &ms) == 0 && ms < bm * 0.999f) { bm = ms; bt = t; }
    }
  {
    float ms = 0.f;
    if (time_one(VecTune{0, 0, 0}, &ms) == 0) am = std::min(am, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (bm >= 1e29f) return -7;
  // switch away from the current choice only for a gain of more than 2 %
  if (am < 1e29f && bm > am * 0.98f) {
    bt = cur;
    bm = am;
  }
  tune_cache_put_vec(vec_cache_key(P), bt);
  *best = bt;
  *best_ms = bm;
  if (auto_ms) *auto_ms = am;
  return 0;
}

// C = A + B for matrices with leading dimensions (MADD of Table 1) when the
// rows are not contiguous: a grid-stride map over rows, threads over columns.
namespace {
__global__ void __launch_bounds__(256) madd_strided_kernel(int64_t m, int64_t n, const float* __restrict__ A,
                                                           int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                           float* __restrict__ C, int64_t ldc) {
  pdl_enter();
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    const float* a = A + i * lda;
    const float* b = B + i * ldb;
    float* c = C + i * ldc;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) c[j] = __fadd_rn(__ldg(a + j), __ldg(b + j));
  }
}
}  // namespace

int launch_madd_strided(int64_t m, int64_t n, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                        int64_t ldc, void* stream, const char** why) {
  const int64_t grid = std::min<int64_t>(m, (int64_t)device_sm_count() * 8);
  void* args[] = {(void*)&m, (void*)&n, (void*)&A, (void*)&lda, (void*)&B, (void*)&ldb, (void*)&C, (void*)&ldc};
  cudaError_t e = launch_pdl((const void*)&madd_strided_kernel, dim3((unsigned)grid), dim3(256), args, 0, stream);
  if (e != cudaSuccess) { *why = cudaGetErrorString(e); return -7; }
  return 0;
}

}  // namespace kf
