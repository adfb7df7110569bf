// Matrix-pass kernel template (included by the instantiation files).
//
// One read of an m x n matrix (or of two same-shaped matrices) serves every
// fused GER / GEMV / GEMVT call of a fusion.  Kernel schema (the paper's
// Algorithm 1, Section 3.3.2, re-derived for a row-major layout on sm_103a):
//   * a block owns a column strip of 32*V 16-byte chunks and a group of
//     32-row blocks; warps of the block take row blocks round robin;
//   * "load invariant data": the column vectors that every row of the strip
//     multiplies (x of GEMV, v of GER) are loaded once into registers;
//   * "clear outputs of accumulated reductions": the GEMVT column sums live
//     in registers across all rows the warp visits and are stored once after
//     the loop (Algorithm 3: s_l accumulated, stored after the loop);
//   * per row, the tile values pass through the ops in script order while
//     they are in registers (GER updates them, GEMV reduces them across the
//     warp with shuffles, GEMVT accumulates them); the updated matrix is
//     written once if a later kernel or the caller needs it;
//   * row results are partial per strip, column results partial per group;
//     the last block of a group (strip) to finish reduces the partials in a
//     fixed order and applies the linear epilogue (Section 3.2.2, option
//     (ii)), so results are deterministic, unlike float atomics.
//
// Staged form (STAGED = true): a warp's part of a row of the strip is 512*V
// contiguous bytes, so each warp streams its rows with one-dimensional bulk
// asynchronous copies (cp.async.bulk, the TMA engine) into its own ring of
// shared-memory stages, `stages` batches of U rows ahead, with completion
// counted in bytes on one mbarrier per stage.  Lanes then read their 16-byte
// chunks from shared memory (conflict free).  Loads in flight no longer
// depend on registers, which is what keeps HBM busy.  Every wait is bounded
// (1 s); a warp whose copy never lands records the error word, stops
// waiting, and the block still takes part in the completion counters.
//
// GEMV is not a dense contraction, so there is nothing for the tensor cores
// here; the bound is HBM bandwidth.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <map>
#include <tuple>

#include "kf_device.cuh"
#include "kf_internal.h"

namespace kf {
namespace mp {

template <int FMT> struct FmtT;
template <> struct FmtT<FMT_F32> { static constexpr int CH = 4; static constexpr int BYTES = 4; };
template <> struct FmtT<FMT_BF16> { static constexpr int CH = 8; static constexpr int BYTES = 2; };
template <> struct FmtT<FMT_E4M3> { static constexpr int CH = 16; static constexpr int BYTES = 1; };

__device__ __forceinline__ float bf16_bits_to_f32(uint32_t h16) {
  return __uint_as_float(h16 << 16);
}

__device__ __forceinline__ void e4m3x2_to_f32(uint32_t two, float& lo, float& hi) {
  __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(two & 0xFFFFu), __NV_E4M3);
  __half2 hv = *reinterpret_cast<__half2*>(&h);
  float2 f = __half22float2(hv);
  lo = f.x;
  hi = f.y;
}

// Decode one 16-byte chunk (CH elements) into floats.
template <int FMT>
__device__ __forceinline__ void decode16(uint4 r, float* o) {
  if constexpr (FMT == FMT_F32) {
    o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
    o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
  } else if constexpr (FMT == FMT_BF16) {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = bf16_bits_to_f32(w[i] & 0xFFFFu);
      o[2 * i + 1] = bf16_bits_to_f32(w[i] >> 16);
    }
  } else {
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      e4m3x2_to_f32(w[i], o[4 * i], o[4 * i + 1]);
      e4m3x2_to_f32(w[i] >> 16, o[4 * i + 2], o[4 * i + 3]);
    }
  }
}

template <int FMT>
__device__ __forceinline__ float load_elem(const void* base, int64_t idx) {
  if constexpr (FMT == FMT_F32) {
    return static_cast<const float*>(base)[idx];
  } else if constexpr (FMT == FMT_BF16) {
    return bf16_bits_to_f32(static_cast<const unsigned short*>(base)[idx]);
  } else {
    const unsigned char b = static_cast<const unsigned char*>(base)[idx];
    float lo, hi;
    e4m3x2_to_f32(b, lo, hi);
    return lo;
  }
}

// Offset inside the strip of value e of chunk v, for this lane.
//  VEC: chunk-contiguous (16-byte loads);  scalar: element-interleaved.
template <int CH, int V, bool VEC>
__device__ __forceinline__ int coff(int v, int e, int lane) {
  return VEC ? (v * 32 + lane) * CH + e : (v * CH + e) * 32 + lane;
}

template <int FMT, int V, bool VEC>
__device__ __forceinline__ void load_row(const void* A, int64_t lda, int64_t row, bool row_ok,
                                         int64_t col0, int64_t n, int lane,
                                         float (&a)[V * FmtT<FMT>::CH]) {
  constexpr int CH = FmtT<FMT>::CH;
  const char* rowp = static_cast<const char*>(A) + (row * lda) * FmtT<FMT>::BYTES;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if constexpr (VEC) {
      const int64_t c = col0 + coff<CH, V, VEC>(v, 0, lane);
      if (row_ok && c + CH <= n) {
        decode16<FMT>(ld_stream16(rowp + c * FmtT<FMT>::BYTES), &a[v * CH]);
      } else {
#pragma unroll
        for (int e = 0; e < CH; ++e)
          a[v * CH + e] = (row_ok && c + e < n) ? load_elem<FMT>(rowp, c + e) : 0.f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const int64_t c = col0 + coff<CH, V, VEC>(v, e, lane);
        a[v * CH + e] = (row_ok && c < n) ? load_elem<FMT>(rowp, c) : 0.f;
      }
    }
  }
}

template <int CH, int V, bool VEC>
__device__ __forceinline__ void store_row(float* B, int64_t ldb, int64_t row, int64_t col0,
                                          int64_t n, int lane, const float (&a)[V * CH]) {
  float* rowp = B + row * ldb;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if constexpr (VEC) {
      const int64_t c = col0 + coff<CH, V, VEC>(v, 0, lane);
      if (c + CH <= n) {
#pragma unroll
        for (int q = 0; q < CH / 4; ++q)
          st_stream_f4(rowp + c + 4 * q, make_float4(a[v * CH + 4 * q], a[v * CH + 4 * q + 1],
                                                     a[v * CH + 4 * q + 2], a[v * CH + 4 * q + 3]));
      } else {
#pragma unroll
        for (int e = 0; e < CH; ++e)
          if (c + e < n) rowp[c + e] = a[v * CH + e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const int64_t c = col0 + coff<CH, V, VEC>(v, e, lane);
        if (c < n) rowp[c] = a[v * CH + e];
      }
    }
  }
}

template <int NR>
__device__ __forceinline__ float pick(const float (&raw)[NR], int s) {
  float v = raw[0];
#pragma unroll
  for (int k = 1; k < NR; ++k)
    if (s == k) v = raw[k];
  return v;
}

template <int NR>
__device__ __forceinline__ void epilogue(const EpiOut* outs, int nout, const float (&raw)[NR],
                                         int64_t i) {
#pragma unroll
  for (int j = 0; j < EPI_MAXOUT; ++j) {
    if (j < nout) {
      const EpiOut& o = outs[j];
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t < EPI_MAXTERM; ++t) {
        if (t < o.nterm) {
          const int s = o.src[t];
          const float v = (s >= 0) ? pick<NR>(raw, s) : __ldg(o.ext[t] + i);
          const float pr = __fmul_rn(o.coef[t], v);
          acc = (t == 0) ? pr : __fadd_rn(acc, pr);
        }
      }
      o.dst[i] = acc;
    }
  }
}


template <int NW, int V, int U, int NOPS, int NMAT, int FMT, bool VEC, bool STAGED>
__global__ void __launch_bounds__(NW * 32)
    matprog_kernel(const __grid_constant__ MatProg P) {
  constexpr int CH = FmtT<FMT>::CH;
  constexpr int BYTES = FmtT<FMT>::BYTES;
  constexpr int W = V * CH;         // values per lane per row
  constexpr int SW = 32 * W;        // strip width in columns
  constexpr int SEG = 32 * V * 16;  // bytes of one warp's part of a row
  constexpr int BATCH = NMAT * U * SEG;
  constexpr int NB = 32 / U;        // batches per 32-row block
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ __align__(8) uint64_t bars[STAGED ? NW * MAT_MAXSTAGES : 1];
  __shared__ int s_last[2];

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int strip = blockIdx.x;
  const int group = blockIdx.y;
  const int64_t m = P.m, n = P.n;
  const int64_t col0 = (int64_t)strip * SW;
  const int nops = P.nops;

  const int64_t nrb = (m + 31) >> 5;
  const int64_t rb_begin = (int64_t)group * P.blocks_per_group;
  const int64_t rb_end = min(nrb, rb_begin + P.blocks_per_group);

  // ---- bulk-copy ring (staged form, full strips only; block-uniform choice)
  const int S = STAGED ? P.stages : 1;
  const bool ring = STAGED && (col0 + SW <= n);
  char* myring = reinterpret_cast<char*>(smem4) + (size_t)warp * S * BATCH;
  uint64_t* mybar = bars + (STAGED ? warp * MAT_MAXSTAGES : 0);
  const int64_t my_rbs = (rb_end > rb_begin + warp) ? (rb_end - rb_begin - warp + NW - 1) / NW : 0;
  const int64_t nbatch = my_rbs * NB;
  bool dead = false;  // warp-uniform: a copy never completed
  int64_t jdead = 0;  // first batch whose copy never completed

  auto issue = [&](int64_t jj) {  // lane 0 only: batch jj into stage jj % S
    const int s = (int)(jj % S);
    const int64_t rbx = rb_begin + warp + (jj / NB) * NW;
    const int64_t rowb = (rbx << 5) + (int64_t)(jj % NB) * U;
    unsigned bytes = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (rowb + u < m) bytes += NMAT * SEG;
    mbar_expect_tx(&mybar[s], bytes);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (rowb + u < m) {
#pragma unroll
        for (int t = 0; t < NMAT; ++t) {
          const char* src = static_cast<const char*>(P.A[t]) + ((rowb + u) * P.lda[t] + col0) * BYTES;
          bulk_g2s(myring + (size_t)s * BATCH + (size_t)(t * U + u) * SEG, src, SEG, &mybar[s]);
        }
      }
    }
  };

  if (ring) {
    if (lane == 0) {
      for (int s = 0; s < S; ++s) mbar_init(&mybar[s], 1);
      fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0)
      for (int64_t j = 0; j < S && j < nbatch; ++j) issue(j);
  }

  // Invariant column vectors (GER v, GEMV x) or GEMVT accumulators.
  float cv[NOPS][W];
#pragma unroll
  for (int k = 0; k < NOPS; ++k) {
    const int kind = (k < nops) ? P.ops[k].kind : MOP_NONE;
    const float* src = (kind == MOP_GER || kind == MOP_GEMV) ? P.ops[k].colvec : nullptr;
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const int64_t c = col0 + coff<CH, V, VEC>(v, e, lane);
        cv[k][v * CH + e] = (src != nullptr && c < n) ? __ldg(src + c) : 0.f;
      }
  }

  int64_t j = 0;  // batch counter of this warp
  for (int64_t rb = rb_begin + warp; rb < rb_end; rb += NW) {
    const int64_t row0 = rb << 5;
    const bool lane_row_ok = row0 + lane < m;
    float rv[NOPS];    // per-lane row scalar (GER u, GEMVT y) for row row0+lane
    float rres[NOPS];  // per-lane GEMV result for row row0+lane
#pragma unroll
    for (int k = 0; k < NOPS; ++k) {
      const int kind = (k < nops) ? P.ops[k].kind : MOP_NONE;
      const float* rs = (kind == MOP_GER || kind == MOP_GEMVT) ? P.ops[k].rowvec : nullptr;
      rv[k] = (rs != nullptr && lane_row_ok) ? __ldg(rs + row0 + lane) : 0.f;
      rres[k] = 0.f;
    }
    float rsc[NMAT];
#pragma unroll
    for (int t = 0; t < NMAT; ++t)
      rsc[t] = (FMT != FMT_F32 && lane_row_ok) ? __ldg(P.rscale[t] + row0 + lane) : 1.f;

#pragma unroll 1
    for (int r = 0; r < 32; r += U) {
      float a[NMAT][U][W];
      if (ring) {
        const int s = (int)(j % S);
        bool ok = dead ? false : mbar_wait_bounded(&mybar[s], (unsigned)((j / S) & 1));
        ok = __all_sync(FULL_MASK, ok);
        if (!ok && !dead) {
          dead = true;
          jdead = j;
          if (lane == 0 && P.errword != nullptr) atomicOr(P.errword, KF_DEVERR_TIMEOUT);
        }
        const char* stage = myring + (size_t)s * BATCH;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool row_ok = !dead && (row0 + r + u < m);
#pragma unroll
          for (int t = 0; t < NMAT; ++t)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              if (row_ok) {
                const uint4 q = *reinterpret_cast<const uint4*>(stage + (size_t)(t * U + u) * SEG +
                                                                 (size_t)(v * 32 + lane) * 16);
                decode16<FMT>(q, &a[t][u][v * CH]);
              } else {
#pragma unroll
                for (int e = 0; e < CH; ++e) a[t][u][v * CH + e] = 0.f;
              }
            }
        }
        __syncwarp();
        if (lane == 0 && !dead && j + S < nbatch) {
          fence_proxy_async_smem();
          issue(j + S);
        }
        ++j;
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t row = row0 + r + u;
#pragma unroll
          for (int t = 0; t < NMAT; ++t)
            load_row<FMT, V, VEC>(P.A[t], P.lda[t], row, row < m, col0, n, lane, a[t][u]);
        }
      }
      if constexpr (FMT != FMT_F32) {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int t = 0; t < NMAT; ++t) {
            const float s = __shfl_sync(FULL_MASK, rsc[t], r + u);
#pragma unroll
            for (int e = 0; e < W; ++e) a[t][u][e] *= s;
          }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int rr = r + u;
#pragma unroll
        for (int k = 0; k < NOPS; ++k) {
          if (k < nops) {
            const MatOp& op = P.ops[k];
            const int kind = op.kind;
            auto apply = [&](float (&t)[W]) {
              if (kind == MOP_GER) {
                const float s = op.alpha * __shfl_sync(FULL_MASK, rv[k], rr);
#pragma unroll
                for (int e = 0; e < W; ++e) t[e] = fmaf(s, cv[k][e], t[e]);
              } else if (kind == MOP_GEMV) {
                float d0 = 0.f, d1 = 0.f;
#pragma unroll
                for (int e = 0; e < W; e += 2) {
                  d0 = fmaf(t[e], cv[k][e], d0);
                  d1 = fmaf(t[e + 1], cv[k][e + 1], d1);
                }
                const float d = warp_sum(d0 + d1);
                if (lane == rr) rres[k] = d;
              } else if (kind == MOP_GEMVT) {
                const float y = __shfl_sync(FULL_MASK, rv[k], rr);
#pragma unroll
                for (int e = 0; e < W; ++e) cv[k][e] = fmaf(t[e], y, cv[k][e]);
              }
            };
            if (NMAT == 1 || op.mat == 0) apply(a[0][u]);
            else apply(a[NMAT - 1][u]);
          }
        }
        const int64_t row = row0 + rr;
        if (row < m) {
#pragma unroll
          for (int t = 0; t < NMAT; ++t)
            if (P.Bout[t] != nullptr)
              store_row<CH, V, VEC>(P.Bout[t], P.ldb[t], row, col0, n, lane, a[t][u]);
        }
      }
    }
    // Partial row results of this strip, one coalesced store per GEMV.
#pragma unroll
    for (int k = 0; k < NOPS; ++k) {
      if (k < nops && P.ops[k].kind == MOP_GEMV && lane_row_ok)
        P.rowpart[((int64_t)P.ops[k].res * P.n_strips + strip) * m + row0 + lane] = rres[k];
    }
  }
  if (ring && dead && lane == 0) {
    // let copies already in flight land before the block's shared memory is reused
    for (int64_t q = jdead; q < nbatch && q < jdead + S; ++q)
      (void)mbar_wait_bounded(&mybar[q % S], (unsigned)((q / S) & 1));
  }

  // Column partials of this group: combine the warps in a fixed order.
  // (The staging area aliases the copy ring, so wait for every warp first.)
  if (P.ncol_res > 0) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NOPS; ++k) {
      if (k < nops && P.ops[k].kind == MOP_GEMVT) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int e = 0; e < CH; ++e) smem[warp * SW + coff<CH, V, VEC>(v, e, lane)] = cv[k][v * CH + e];
        __syncthreads();
        for (int c = threadIdx.x; c < SW; c += NW * 32) {
          float s = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) s += smem[w * SW + c];
          const int64_t col = col0 + c;
          if (col < n) P.colpart[((int64_t)P.ops[k].res * P.n_groups + group) * n + col] = s;
        }
        __syncthreads();
      }
    }
  }

  // Last-block completion of the cross-block reductions.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ls = 0, lg = 0;
    if (P.ncol_out > 0) ls = atomicAdd(&P.counters[strip], 1u) == (unsigned)P.n_groups - 1u;
    if (P.nrow_out > 0)
      lg = atomicAdd(&P.counters[P.n_strips + group], 1u) == (unsigned)P.n_strips - 1u;
    s_last[0] = ls;
    s_last[1] = lg;
  }
  __syncthreads();
  if (s_last[0]) {
    __threadfence();
    for (int c = threadIdx.x; c < SW; c += NW * 32) {
      const int64_t col = col0 + c;
      if (col >= n) continue;
      float raw[NOPS];
#pragma unroll
      for (int q = 0; q < NOPS; ++q) {
        float s = 0.f;
        if (q < P.ncol_res) {
          const float* part = P.colpart + (int64_t)q * P.n_groups * n + col;
          for (int g = 0; g < P.n_groups; ++g) s += __ldcg(part + (int64_t)g * n);
        }
        raw[q] = s;
      }
      epilogue<NOPS>(P.col_out, P.ncol_out, raw, col);
    }
    if (threadIdx.x == 0) P.counters[strip] = 0u;
  }
  if (s_last[1]) {
    __threadfence();
    const int64_t r0 = rb_begin << 5;
    const int64_t r1 = min(m, rb_end << 5);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += NW * 32) {
      float raw[NOPS];
#pragma unroll
      for (int q = 0; q < NOPS; ++q) {
        float s = 0.f;
        if (q < P.nrow_res) {
          const float* part = P.rowpart + (int64_t)q * P.n_strips * m + i;
          int st = 0;
          for (; st + 8 <= P.n_strips; st += 8) {
            float t[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) t[jj] = __ldcg(part + (int64_t)(st + jj) * m);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) s += t[jj];
          }
          for (; st < P.n_strips; ++st) s += __ldcg(part + (int64_t)st * m);
        }
        raw[q] = s;
      }
      epilogue<NOPS>(P.row_out, P.nrow_out, raw, i);
    }
    if (threadIdx.x == 0) P.counters[P.n_strips + group] = 0u;
  }
}

// ---------------------------------------------------------------- registry

struct Entry {
  const void* fn;
  int nw, v, u, nops, nmat, fmt;
  bool vec, staged;
};

// (warps, vec, unroll, nops, nmat, fmt, vec-path, staged)
using Key = std::tuple<int, int, int, int, int, int, bool, bool>;

std::map<Key, Entry>& registry();

template <int NW, int V, int U, int NOPS, int NMAT, int FMT, bool VEC, bool STAGED>
void reg() {
  registry()[Key(NW, V, U, NOPS, NMAT, FMT, VEC, STAGED)] =
      Entry{(const void*)&matprog_kernel<NW, V, U, NOPS, NMAT, FMT, VEC, STAGED>, NW, V, U, NOPS,
            NMAT, FMT, VEC, STAGED};
}

// the five op shapes: (nops, nmat) = (1,1) (2,1) (4,1) (2,2) (4,2)
template <int NW, int V, int U, int FMT, bool STAGED>
void reg_shapes() {
  reg<NW, V, U, 1, 1, FMT, true, STAGED>();
  reg<NW, V, U, 2, 1, FMT, true, STAGED>();
  reg<NW, V, U, 4, 1, FMT, true, STAGED>();
  reg<NW, V, U, 2, 2, FMT, true, STAGED>();
  reg<NW, V, U, 4, 2, FMT, true, STAGED>();
}

void register_f32_staged();
void register_f32_plain();
void register_lowp();

}  // namespace mp
}  // namespace kf
