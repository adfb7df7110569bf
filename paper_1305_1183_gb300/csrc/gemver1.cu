// GEMVER in one launch (Table 1): B = A + u1 v1^T + u2 v2^T;
// x = beta B^T y + z; w = alpha B x.
//
// w needs all of x, which needs every row of B: a global barrier (Section
// 3.2.2).  The two-pass form (abi.cu) ends a kernel there; this form keeps
// one cooperative launch (every block resident, which the launch guarantees)
// and crosses the barrier with a grid-wide barrier on a counter in the
// workspace, the remark of Section 4.2 about persistent threads:
//   phase 1  block (strip, group): rows of its group, B written once, the
//            strip's column sums of B^T y kept in registers -> group partial;
//   barrier, then the column sums finished by the whole grid in two levels
//            (sets of 8 group partials, then the sets in order), x written;
//   phase 2  the same block walks its rows in reverse (the rows it wrote last
//            are the likeliest still in L2) with x, row partial per strip;
//   barrier, then w finished by the whole grid (strip partials in order).
// Every barrier wait is bounded (kf_set_wait_limit_ns): a wait that runs out
// records KF_DEVERR_TIMEOUT in the workspace's error word and the block
// skips the rest of its work.  Results do not depend on block timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "grid_sync.cuh"
#include "kf_device.cuh"
#include "kf_internal.h"

namespace kf {

namespace {

constexpr int G1_WARPS = 8;
constexpr int G1_SW = G1_WARPS * 32 * 4;  // strip width: 1024 columns
constexpr int G1_U_GER = 4;               // rows loaded together: GEMVER (B also written)
constexpr int G1_U_MV = 8;                // SGEMVT (reads only: more rows in flight)
constexpr int G1_SET = 8;                 // group partials per first-level sum

struct GemverArgs {
  int64_t m, n, lda, ldb;  // A (and B) m x n; GEMVER: m = n
  const float* A;
  float* B;
  const float *u1, *v1, *u2, *v2, *y, *z;
  float alpha, beta;
  float* x;
  float* w;
  float* colpart;     // [groups + sets][n]
  float* rowpart;     // [strips][m]
  unsigned* bar;      // [0]: arrivals, [1]: blocks done (zero between launches)
  unsigned* err;      // device error word
  int strips, groups, upg;
  uint64_t wait_ns;
};

// Grid-wide barrier number k (1, 2, ...) on the workspace's counters.
__device__ __forceinline__ bool grid_barrier(const GemverArgs& a, unsigned k) {
  return grid_barrier_bounded(a.bar, k, a.wait_ns, a.err);
}

__device__ __forceinline__ float4 ld_cg4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }

// Row dots of 8 rows held as per-lane partials: afterwards lane L holds the
// warp's total of row (L & 7) (butterfly over the lane quarters, then
// recursive halving over the low three lane bits).
__device__ __forceinline__ float g1_reduce8(float (&d)[8], int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] += __shfl_xor_sync(FULL_MASK, d[i], 16);
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] += __shfl_xor_sync(FULL_MASK, d[i], 8);
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? d[i] : d[i + off];
      const float keep = upper ? d[i + off] : d[i];
      d[i] = keep + __shfl_xor_sync(FULL_MASK, send, off);
    }
  }
  return d[0];
}

// GER: GEMVER (B = A + u1 v1^T + u2 v2^T written in phase 1 and reread in
// phase 2, A read evict-first); !GER: SGEMVT (x = beta A^T y + z,
// w = alpha A x: phase 2 rereads A, which phase 1 reads at normal L2
// priority so that the rows it read last are still in L2).
template <bool GER>
__global__ void __launch_bounds__(G1_WARPS * 32, 3) gemver_single_kernel(const __grid_constant__ GemverArgs a) {
  constexpr int G1_U = GER ? G1_U_GER : G1_U_MV;
  __shared__ float red[G1_WARPS][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int strip = (int)(blockIdx.x % a.strips), group = (int)(blockIdx.x / a.strips);
  const int64_t m = a.m, n = a.n;
  const int64_t col = (int64_t)strip * G1_SW + warp * 128 + lane * 4;  // this lane's four columns
  const bool col_ok = col < n;                                         // n is a multiple of 4
  const int64_t nunits = (m + 7) >> 3;
  const int64_t u0 = std::min<int64_t>(nunits, (int64_t)group * a.upg);
  const int64_t u1e = std::min<int64_t>(nunits, u0 + a.upg);
  const int64_t r0 = u0 << 3, r1 = std::min<int64_t>(m, u1e << 3);
  const uint64_t pol_first = l2_policy_first();
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  unsigned k = 0;  // barriers passed
  bool ok = true;

  // ---- phase 1: B = A + u1 v1^T + u2 v2^T (written once), column sums of B^T y
  {
    const float4 v1c = (GER && col_ok) ? __ldg(reinterpret_cast<const float4*>(a.v1 + col)) : z4;
    const float4 v2c = (GER && col_ok) ? __ldg(reinterpret_cast<const float4*>(a.v2 + col)) : z4;
    float4 t = z4;
    for (int64_t rb = r0 & ~(int64_t)31; rb < r1; rb += 32) {
      // the 32-row block's row scalars, one per lane, shared by shuffles
      const int64_t lr = rb + lane;
      const bool lr_ok = lr >= r0 && lr < r1;
      const float lu1 = (GER && lr_ok) ? __ldg(a.u1 + lr) : 0.f;
      const float lu2 = (GER && lr_ok) ? __ldg(a.u2 + lr) : 0.f;
      const float ly = lr_ok ? __ldg(a.y + lr) : 0.f;
      const int64_t lo = std::max(r0, rb), hi = std::min(r1, rb + 32);
      for (int64_t row = lo; row < hi; row += G1_U) {
        float4 av[G1_U];
#pragma unroll
        for (int u = 0; u < G1_U; ++u) {
          const int64_t rr = row + u;
          if (rr < hi && col_ok) {
            const uint4 q = GER ? ld_stream16_pol(a.A + rr * a.lda + col, pol_first) : ld_stream16(a.A + rr * a.lda + col);
            av[u] = make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w));
          } else {
            av[u] = z4;
          }
        }
#pragma unroll
        for (int u = 0; u < G1_U; ++u) {
          const int64_t rr = row + u;
          const int src = (int)((rr - rb) & 31);
          const float s1 = __shfl_sync(FULL_MASK, lu1, src);
          const float s2 = __shfl_sync(FULL_MASK, lu2, src);
          const float sy = __shfl_sync(FULL_MASK, ly, src);
          if (rr < hi) {
            float4 b = av[u];
            if constexpr (GER) {
              b.x = fmaf(s2, v2c.x, fmaf(s1, v1c.x, av[u].x));
              b.y = fmaf(s2, v2c.y, fmaf(s1, v1c.y, av[u].y));
              b.z = fmaf(s2, v2c.z, fmaf(s1, v1c.z, av[u].z));
              b.w = fmaf(s2, v2c.w, fmaf(s1, v1c.w, av[u].w));
              if (col_ok) st_f4_keep(a.B + rr * a.ldb + col, b);  // reread in phase 2
            }
            t.x = fmaf(b.x, sy, t.x);
            t.y = fmaf(b.y, sy, t.y);
            t.z = fmaf(b.z, sy, t.z);
            t.w = fmaf(b.w, sy, t.w);
          }
        }
      }
    }
    if (col_ok) *reinterpret_cast<float4*>(a.colpart + (int64_t)group * n + col) = t;
  }
  ok = grid_barrier(a, ++k);

  // ---- x = beta * (group partials, added in fixed order) + z, by the whole grid
  const int G = a.groups;
  const int nsets = (G + G1_SET - 1) / G1_SET;
  const int64_t n4 = n >> 2;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  if (ok && nsets > 1) {
    // first level: each set of G1_SET group partials, in group order
    for (int64_t it = gtid; it < n4 * nsets; it += gstride) {
      const int64_t c = (it % n4) * 4;
      const int set = (int)(it / n4);
      const int g0 = set * G1_SET, g1 = std::min(G, g0 + G1_SET);
      float4 s = z4;
      for (int g = g0; g < g1; ++g) {
        const float4 v = ld_cg4(a.colpart + (int64_t)g * n + c);
        s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
      }
      *reinterpret_cast<float4*>(a.colpart + (int64_t)(G + set) * n + c) = s;
    }
    ok = grid_barrier(a, ++k);
  }
  if (ok) {
    const int first = nsets > 1 ? G : 0, count = nsets > 1 ? nsets : G;
    for (int64_t c4 = gtid; c4 < n4; c4 += gstride) {
      const int64_t c = c4 * 4;
      float4 s = z4;
      for (int g = first; g < first + count; ++g) {
        const float4 v = ld_cg4(a.colpart + (int64_t)g * n + c);
        s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
      }
      const float4 zz = __ldg(reinterpret_cast<const float4*>(a.z + c));
      float4 xo;
      xo.x = __fadd_rn(__fmul_rn(a.beta, s.x), zz.x);
      xo.y = __fadd_rn(__fmul_rn(a.beta, s.y), zz.y);
      xo.z = __fadd_rn(__fmul_rn(a.beta, s.z), zz.z);
      xo.w = __fadd_rn(__fmul_rn(a.beta, s.w), zz.w);
      *reinterpret_cast<float4*>(a.x + c) = xo;
    }
    ok = grid_barrier(a, ++k);
  }

  // ---- phase 2: w's row partials over the same rows, walked from the last
  // 8-row unit to the first (GEMVER: this thread reads back what it wrote)
  if (ok) {
    const float4 xv = col_ok ? ld_cg4(a.x + col) : z4;
    const float* M2 = GER ? a.B : a.A;
    const int64_t ld2 = GER ? a.ldb : a.lda;
    for (int64_t un = u1e - 1; un >= u0; --un) {
      float dacc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) dacc[i] = 0.f;
#pragma unroll
      for (int r = 0; r < 8; r += G1_U) {
        float4 bv[G1_U];
#pragma unroll
        for (int u = 0; u < G1_U; ++u) {
          const int64_t rr = (un << 3) + r + u;
          if (rr < m && col_ok) {
            const uint4 q = ld_stream16_pol(M2 + rr * ld2 + col, pol_first);
            bv[u] = make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w));
          } else {
            bv[u] = z4;
          }
        }
#pragma unroll
        for (int u = 0; u < G1_U; ++u) {
          float d0 = fmaf(bv[u].x, xv.x, 0.f), d1 = bv[u].y * xv.y;
          d0 = fmaf(bv[u].z, xv.z, d0);
          d1 = fmaf(bv[u].w, xv.w, d1);
          dacc[r + u] = d0 + d1;
        }
      }
      const float v = g1_reduce8(dacc, lane);
      if (lane < 8) red[warp][lane] = v;
      __syncthreads();
      if (threadIdx.x < 8) {
        const int64_t rr = (un << 3) + threadIdx.x;
        float s = 0.f;
#pragma unroll
        for (int wq = 0; wq < G1_WARPS; ++wq) s += red[wq][threadIdx.x];
        if (rr < m) a.rowpart[(int64_t)strip * m + rr] = s;
      }
      __syncthreads();
    }
    ok = grid_barrier(a, ++k);
  }

  // ---- w = alpha * (strip partials, added in strip order), by the whole grid
  if (ok) {
    for (int64_t i = gtid; i < m; i += gstride) {
      float s = 0.f;
      for (int st = 0; st < a.strips; ++st) s += __ldcg(a.rowpart + (int64_t)st * m + i);
      a.w[i] = __fmul_rn(a.alpha, s);
    }
  }

  // the last block out leaves the barrier counters at zero for the next launch
  grid_exit(a.bar);
}

}  // namespace

// Can the single launch take this call?  FP32, n a multiple of 4, every
// operand 16-byte aligned, B not in place of A (phase 2 rereads B).
bool gemver_single_ok(int64_t n, const float* A, int64_t lda, const float* B, int64_t ldb, const float* const* vecs,
                      int nvec) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (n < 8 || n % 4 != 0 || lda % 4 != 0 || ldb % 4 != 0 || !al(A) || !al(B) || (const void*)A == (const void*)B)
    return false;
  for (int i = 0; i < nvec; ++i)
    if (!al(vecs[i])) return false;
  return true;
}

// The workspace is the matrix pass's layout for an m x n pass with one row
// and one column result (kf_gemver's and kf_sgemvt's): this launch uses its
// row and column partial regions (the counters stay untouched) and two
// barrier words at byte 128 of the header, zero between launches.
namespace {
int launch_single(bool ger, int64_t m, int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                  const float* u2, const float* v2, const float* y, const float* z, float alpha, float beta, float* B,
                  int64_t ldb, float* x, float* w, void* ws, size_t ws_bytes, void* stream, const char** why) {
  MatProg L{};
  L.m = m; L.n = n; L.fmt = FMT_F32; L.nrow_res = 1; L.ncol_res = 1; L.nrow_out = 1; L.ncol_out = 1;
  if (matprog_bind_workspace(L, ws, ws_bytes) != 0) {
    *why = "workspace missing or smaller than kf_workspace_size()";
    return -11;
  }
  const void* fn = ger ? (const void*)&gemver_single_kernel<true> : (const void*)&gemver_single_kernel<false>;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, G1_WARPS * 32, 0) != cudaSuccess || occ < 1) {
    *why = "occupancy query failed";
    return -7;
  }
  GemverArgs a{};
  a.m = m; a.n = n; a.lda = lda; a.ldb = ldb; a.A = A; a.B = B;
  a.u1 = u1; a.v1 = v1; a.u2 = u2; a.v2 = v2; a.y = y; a.z = z;
  a.alpha = alpha; a.beta = beta; a.x = x; a.w = w;
  char* b = static_cast<char*>(ws);
  a.err = reinterpret_cast<unsigned*>(b);
  a.bar = reinterpret_cast<unsigned*>(b + 128);
  a.colpart = L.colpart;  // (MAT_MAXGROUPS + MAT_MAXSETS) x n floats
  a.rowpart = L.rowpart;  // ceil(n / 128) x m floats >= strips x m
  a.strips = (int)((n + G1_SW - 1) / G1_SW);
  // every block resident at once: strips x groups within one wave
  const int64_t slots = (int64_t)device_sm_count() * occ;
  const int64_t nunits = (m + 7) / 8;
  if (a.strips > slots) {
    *why = "matrix too wide for one wave of blocks";
    return -10;
  }
  int64_t G = std::max<int64_t>(1, slots / a.strips);
  G = std::min<int64_t>(G, std::min<int64_t>(nunits, MAT_MAXGROUPS));
  const int64_t upg = (nunits + G - 1) / G;
  G = (nunits + upg - 1) / upg;
  a.groups = (int)G;
  a.upg = (int)upg;
  a.wait_ns = wait_limit_ns();
  void* args[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)(a.strips * G)), dim3(G1_WARPS * 32), args, 0,
                                                    (cudaStream_t)stream);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return -7;
  }
  return 0;
}
}  // namespace

int launch_gemver_single(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1, const float* u2,
                         const float* v2, const float* y, const float* z, float alpha, float beta, float* B,
                         int64_t ldb, float* x, float* w, void* ws, size_t ws_bytes, void* stream, const char** why) {
  return launch_single(true, n, n, A, lda, u1, v1, u2, v2, y, z, alpha, beta, B, ldb, x, w, ws, ws_bytes, stream, why);
}

// SGEMVT in one launch: x = beta A^T y + z, w = alpha A x (A m x n, m >= 8,
// n a multiple of 4, operands 16-byte aligned: sgemvt_single_ok).
bool sgemvt_single_ok(int64_t m, int64_t n, const float* A, int64_t lda, const float* const* vecs, int nvec) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (m < 8 || n < 4 || n % 4 != 0 || lda % 4 != 0 || !al(A)) return false;
  for (int i = 0; i < nvec; ++i)
    if (!al(vecs[i])) return false;
  return true;
}

int launch_sgemvt_single(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                         float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream,
                         const char** why) {
  return launch_single(false, m, n, A, lda, nullptr, nullptr, nullptr, nullptr, y, z, alpha, beta, nullptr, 0, x, w,
                       ws, ws_bytes, stream, why);
}

}  // namespace kf
