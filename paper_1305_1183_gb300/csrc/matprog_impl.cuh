// Matrix-pass kernel template (included by the instantiation files).
//
// One read of an m x n matrix (or of two same-shaped matrices) serves every
// fused GER / GEMV / GEMVT call of a fusion.  Kernel schema (the paper's
// Algorithm 1, Section 3.3.2, re-derived for a row-major layout on sm_103a):
//   * a block owns a column strip and a group of consecutive 8-row units
//     (so the groups of a full-chip grid differ by at most one unit); its NW
//     consumer warps sit side by side across the strip (each owns 32*V
//     16-byte chunks of every row), so the block reads NW*512*V contiguous
//     bytes of each row it visits -- long sequential runs for HBM.  Rows are
//     walked in 32-row blocks of four 8-row quarters; a quarter outside the
//     block's group is skipped (a test every warp takes alike);
//   * "load invariant data": the column vectors that every row multiplies
//     (x of GEMV, v of GER) are loaded once into each warp's registers;
//   * "clear outputs of accumulated reductions": GEMVT column sums live in
//     registers across all rows of the group and are stored once at the end
//     (Algorithm 3: s_l accumulated, stored after the loop);
//   * per row, the values pass through the ops in script order while in
//     registers (GER updates them, GEMV accumulates per-lane row partials,
//     GEMVT accumulates column sums); an updated matrix is written once;
//   * row dots: each lane keeps a partial per row of an 8-row quarter,
//     reduced across the warp once per quarter (23 shuffles), then across
//     the warps through shared memory once per 32 rows;
//   * row results are partial per strip, column results partial per group;
//     the last block of a group (strip) to finish reduces the partials in a
//     fixed order and applies the linear epilogue (Section 3.2.2, option
//     (ii)), so results are deterministic, unlike float atomics.
//
// Staged form (STAGED = true): one extra producer warp streams the block's
// rows with one-dimensional bulk asynchronous copies (cp.async.bulk, the TMA
// engine; one copy per row and matrix) into a ring of shared-memory stages,
// `stages` batches of U rows ahead; a "full" mbarrier per stage counts the
// bytes, an "empty" mbarrier per stage counts the consumer warps that have
// read it.  Every wait is bounded (P.wait_ns, 1 s by default): on a timeout
// the block records the error word, stops waiting, lets its in-flight copies
// land (bounded by the default 1 s) and still takes part in the completion
// counters.
//
// GEMV is not a dense contraction, so there is nothing for the tensor cores
// here; the bound is HBM bandwidth.
#pragma once

#include <cuda_bf16.h>
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
                                         float (&a)[V * FmtT<FMT>::CH], uint64_t pol) {
  constexpr int CH = FmtT<FMT>::CH;
  const char* rowp = static_cast<const char*>(A) + (row * lda) * FmtT<FMT>::BYTES;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if constexpr (VEC) {
      const int64_t c = col0 + coff<CH, V, VEC>(v, 0, lane);
      if (row_ok && c + CH <= n) {
        decode16<FMT>(ld_stream16_pol(rowp + c * FmtT<FMT>::BYTES, pol), &a[v * CH]);
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

// Raw 16-byte chunks of a row (low-precision formats, 16-byte loads): the
// codes stay packed until the row is used, so a batch of rows in flight
// costs 4 registers per chunk instead of CH.  Chunks past the end of the
// row are assembled element by element (code 0 beyond n).
template <int FMT, int V>
__device__ __forceinline__ void load_row_raw(const void* A, int64_t lda, int64_t row, bool row_ok, int64_t col0,
                                             int64_t n, int lane, uint4 (&q)[V], uint64_t pol) {
  constexpr int CH = FmtT<FMT>::CH;
  constexpr int BYTES = FmtT<FMT>::BYTES;
  const char* rowp = static_cast<const char*>(A) + (row * lda) * BYTES;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int64_t c = col0 + coff<CH, V, true>(v, 0, lane);
    if (row_ok && c + CH <= n) {
      q[v] = ld_stream16_pol(rowp + c * BYTES, pol);
    } else {
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (row_ok) {
#pragma unroll
        for (int e = 0; e < CH; ++e) {
          if (c + e < n) {
            const uint32_t code = BYTES == 2 ? (uint32_t) reinterpret_cast<const unsigned short*>(rowp)[c + e]
                                             : (uint32_t) reinterpret_cast<const unsigned char*>(rowp)[c + e];
            w[e * BYTES / 4] |= code << (8 * ((e * BYTES) & 3));
          }
        }
      }
      q[v] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

template <int CH, int V, bool VEC>
__device__ __forceinline__ void store_row(float* B, int64_t ldb, int64_t row, int64_t col0,
                                          int64_t n, int lane, const float (&a)[V * CH], bool keep) {
  float* rowp = B + row * ldb;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    if constexpr (VEC) {
      const int64_t c = col0 + coff<CH, V, VEC>(v, 0, lane);
      if (c + CH <= n) {
#pragma unroll
        for (int q = 0; q < CH / 4; ++q)
        {
          const float4 t4 = make_float4(a[v * CH + 4 * q], a[v * CH + 4 * q + 1], a[v * CH + 4 * q + 2],
                                        a[v * CH + 4 * q + 3]);
          if (keep) st_f4_keep(rowp + c + 4 * q, t4);
          else st_stream_f4(rowp + c + 4 * q, t4);
        }
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

// Low-precision matrix output (a GER chain stored in the input's format with
// a per-row scale sB): code = round-to-nearest-even of b * (1 / sB) into the
// format (E4M3 saturating), then b is replaced by sB * code, the value later
// readers of the stored matrix see.  One 16-byte chunk of codes per CH
// values, the layout the loads decode.
template <int FMT>
__device__ __forceinline__ uint32_t encode1(float t) {
  if constexpr (FMT == FMT_BF16) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(t));
  } else {
    return (uint32_t)__nv_cvt_float_to_fp8(t, __NV_SATFINITE, __NV_E4M3);
  }
}

template <int FMT>
__device__ __forceinline__ float decode1(uint32_t c) {
  if constexpr (FMT == FMT_BF16) {
    return bf16_bits_to_f32(c);
  } else {
    float lo, hi;
    e4m3x2_to_f32(c, lo, hi);
    return lo;
  }
}

template <int FMT, int V, bool VEC>
__device__ __forceinline__ void quant_store_row(void* B, int64_t ldb, int64_t row, bool row_ok, int64_t col0,
                                                int64_t n, int lane, float (&a)[V * FmtT<FMT>::CH], float sB,
                                                float isB, bool keep) {
  constexpr int CH = FmtT<FMT>::CH;
  constexpr int BYTES = FmtT<FMT>::BYTES;
  char* rowp = static_cast<char*>(B) + (row * ldb) * BYTES;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    uint32_t code[CH];
    if constexpr (FMT == FMT_E4M3) {
      // two values per conversion each way (the paired E4M3 forms round
      // each element exactly as the single ones do)
#pragma unroll
      for (int e = 0; e < CH; e += 2) {
        const float2 t = make_float2(__fmul_rn(a[v * CH + e], isB), __fmul_rn(a[v * CH + e + 1], isB));
        const uint32_t pr = (uint32_t)__nv_cvt_float2_to_fp8x2(t, __NV_SATFINITE, __NV_E4M3);
        code[e] = pr & 0xFFu;
        code[e + 1] = (pr >> 8) & 0xFFu;
        float lo, hi;
        e4m3x2_to_f32(pr, lo, hi);
        a[v * CH + e] = __fmul_rn(sB, lo);
        a[v * CH + e + 1] = __fmul_rn(sB, hi);
      }
    } else {
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        code[e] = encode1<FMT>(__fmul_rn(a[v * CH + e], isB));
        a[v * CH + e] = __fmul_rn(sB, decode1<FMT>(code[e]));
      }
    }
    if (!row_ok) continue;
    if constexpr (VEC) {
      const int64_t c = col0 + coff<CH, V, VEC>(v, 0, lane);
      if (c + CH <= n) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if constexpr (FMT == FMT_BF16) w[q] = code[2 * q] | (code[2 * q + 1] << 16);
          else w[q] = code[4 * q] | (code[4 * q + 1] << 8) | (code[4 * q + 2] << 16) | (code[4 * q + 3] << 24);
        }
        st_u4(rowp + c * BYTES, w[0], w[1], w[2], w[3], keep);
      } else {
#pragma unroll
        for (int e = 0; e < CH; ++e) {
          if (c + e < n) {
            if constexpr (FMT == FMT_BF16) reinterpret_cast<unsigned short*>(rowp)[c + e] = (unsigned short)code[e];
            else reinterpret_cast<unsigned char*>(rowp)[c + e] = (unsigned char)code[e];
          }
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const int64_t c = col0 + coff<CH, V, VEC>(v, e, lane);
        if (c < n) {
          if constexpr (FMT == FMT_BF16) reinterpret_cast<unsigned short*>(rowp)[c] = (unsigned short)code[e];
          else reinterpret_cast<unsigned char*>(rowp)[c] = (unsigned char)code[e];
        }
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


// Row dots of 8 rows, each spread over the 32 lanes as per-lane partials
// d[0..7]: after the call every lane L holds the total of row (L & 7).
// Two butterfly steps (xor 16, xor 8) add the four lane quarters, then
// recursive halving over lane bits 2..0 leaves each lane the row its bits
// select: 23 shuffles per 8 rows, no per-row chain of dependent shuffles.
__device__ __forceinline__ float reduce8_rows(float (&d)[8], int lane) {
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Compile-time op signatures.  A signature fixes the kind and matrix of
// every op of a fusion (3 bits per op: kind in bits 0-1, matrix in bit 2;
// bit 12 marks a specialised signature), so the per-row dispatch over the
// op list folds away.  SIG = 0 keeps the runtime dispatch for any fusion.
constexpr int SIG_SPEC = 1 << 12;
constexpr int sig_op(int kind, int mat) { return kind | (mat << 2); }
constexpr int sig_kind(int sig, int k) { return (sig >> (3 * k)) & 3; }
constexpr int sig_mat(int sig, int k) { return (sig >> (3 * k + 2)) & 1; }
constexpr int SIG_GEMV = SIG_SPEC | sig_op(MOP_GEMV, 0);
constexpr int SIG_GEMVT = SIG_SPEC | sig_op(MOP_GEMVT, 0);
constexpr int SIG_GER = SIG_SPEC | sig_op(MOP_GER, 0);
constexpr int SIG_BICGK = SIG_SPEC | sig_op(MOP_GEMV, 0) | (sig_op(MOP_GEMVT, 0) << 3);
constexpr int SIG_GEMVER1 = SIG_SPEC | sig_op(MOP_GER, 0) | (sig_op(MOP_GER, 0) << 3) | (sig_op(MOP_GEMVT, 0) << 6);
constexpr int SIG_GESUMMV = SIG_SPEC | sig_op(MOP_GEMV, 0) | (sig_op(MOP_GEMV, 1) << 3);

// Index of the last GER of a specialised signature (-1: none).  A
// low-precision instance with such a signature stores the GER chain's result
// as codes with per-row scales (the kernel quantises right after that op).
constexpr int sig_last_ger(int sig) {
  int last = -1;
  if (sig & SIG_SPEC)
    for (int k = 0; k < 4; ++k)
      if (sig_kind(sig, k) == MOP_GER) last = k;
  return last;
}

// Resident blocks per SM asked of the register allocator: the one-chunk
// FP32 forms are latency bound and need four blocks of eight warps.
template <int NW, int V, int NMAT, int FMT, bool VEC, int U>
constexpr int min_blocks() {
  return (NW == 8 && V == 1 && NMAT == 1 && FMT == FMT_F32)   ? (U >= 8 ? 3 : 4)
         : (NW == 8 && V == 1 && NMAT == 2 && FMT == FMT_F32) ? (U >= 8 ? 2 : 3)
                                                                : ((FMT != FMT_F32 && VEC) ? 2 : 1);
}

// BF16 GEMVER passes (GER chain + GEMVT, and GEMV) with 8 rows in flight
// run at three blocks per SM: a few spilled bytes cost less than the extra
// warps gain (measured 310 -> 289 us for GEMVER at n = 16384); BiCGK and
// E4M3 spill too much at that bound and keep two.
template <int NW, int V, int NMAT, int FMT, bool VEC, int U, int SIG>
constexpr int min_blocks_sig() {
  return (FMT == FMT_BF16 && VEC && V == 1 && U == 8 && NMAT == 1 &&
          (SIG == SIG_GEMVER1 || SIG == SIG_GEMV))
             ? 3
             : min_blocks<NW, V, NMAT, FMT, VEC, U>();
}

// Registers of one batch of rows: decoded floats, or packed chunks.
template <bool RAW, int NMAT, int U, int V, int W> struct BatchOf { using type = float[NMAT][U][W]; };
template <int NMAT, int U, int V, int W> struct BatchOf<true, NMAT, U, V, W> { using type = uint4[NMAT][U][V]; };

template <int NW, int V, int U, int NOPS, int NMAT, int NG, int FMT, bool VEC, bool STAGED, int SIG>
__global__ void __launch_bounds__((NW + (STAGED ? 1 : 0)) * 32, (min_blocks_sig<NW, V, NMAT, FMT, VEC, U, SIG>()))
    matprog_kernel(const __grid_constant__ MatProg P) {
  constexpr int CH = FmtT<FMT>::CH;
  constexpr int BYTES = FmtT<FMT>::BYTES;
  constexpr int W = V * CH;          // values per lane per row
  constexpr int SWW = 32 * W;        // columns of one warp's slice
  constexpr int SW = NW * SWW;       // strip width in columns
  constexpr int SEGW = 32 * V * 16;  // bytes of one warp's slice of a row
  constexpr int SEG = NW * SEGW;     // bytes of the block's part of a row
  constexpr int BATCH = NMAT * U * SEG;
  static_assert(U == 1 || U == 2 || U == 4 || U == 8, "U must divide 8");
  constexpr int NGA = NG > 0 ? NG : 1;
  constexpr bool SPEC = (SIG & SIG_SPEC) != 0;
  constexpr int LASTGER = sig_last_ger(SIG);
  constexpr bool QOUT = FMT != FMT_F32 && LASTGER >= 0;  // low-precision matrix output
  static_assert(!QOUT || NMAT == 1, "low-precision output: one matrix");
  constexpr float QMAX = FMT == FMT_E4M3 ? 448.f : 1.f;
  // low-precision 16-byte loads keep their chunks packed until the row is used
  constexpr bool RAW = FMT != FMT_F32 && VEC;
  // Without a GER the row scale is applied once per row (to the row dot and
  // to the GEMVT row value) instead of once per element.
  constexpr bool FOLD = RAW && SPEC && LASTGER < 0;
  using BatchT = typename BatchOf<RAW, NMAT, U, V, W>::type;
  extern __shared__ float4 smem4[];
  __shared__ __align__(8) uint64_t full[STAGED ? MAT_MAXSTAGES : 1];
  __shared__ __align__(8) uint64_t empty[STAGED ? MAT_MAXSTAGES : 1];
  __shared__ float red[2][NGA][NW][32];
  __shared__ int s_last[2];
  __shared__ int s_abort;

  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int strip = blockIdx.x;
  const int group = blockIdx.y;
  const int64_t m = P.m, n = P.n;
  const int64_t col0 = (int64_t)strip * SW;
  const int64_t wcol0 = col0 + (int64_t)min(warp, NW - 1) * SWW;
  const int nops = P.nops;

  // the group's rows: 8-row units [u_begin, u_end), walked by 32-row blocks
  constexpr int NBU = 8 / U;         // batches per 8-row unit
  const int64_t nunits = (m + 7) >> 3;
  const int64_t u_begin = min(nunits, (int64_t)group * P.units_per_group);
  const int64_t u_end = min(nunits, u_begin + P.units_per_group);
  const int64_t rb_begin = u_begin >> 2;
  const int64_t rb_end = (u_end + 3) >> 2;
  const int64_t nbatch = (u_end - u_begin) * NBU;

  const int S = STAGED ? P.stages : 1;
  // column partial slots per result: one per group, then (more than
  // MAT_COLSET groups) one per set of MAT_COLSET groups
  const int nsets = (P.n_groups + MAT_COLSET - 1) / MAT_COLSET;
  const int64_t cslots = (int64_t)P.n_groups + (nsets > 1 ? nsets : 0);
  unsigned* setcnt = P.counters + P.n_strips + MAT_MAXGROUPS;  // [n_strips][MAT_MAXSETS]
  const bool rev = P.reverse_rows != 0;
  // matrix loads stream with the evict-first hint; a matrix output the next
  // pass reads is stored plainly (normal L2 priority), else streamed
  const uint64_t lpol = l2_policy_first();
  const bool keep_out = P.l2_keep_out != 0;
  const bool ring = STAGED && (col0 + SW <= n);  // block-uniform
  char* ringp = reinterpret_cast<char*>(smem4);

  if (threadIdx.x == 0) {
    s_abort = 0;
    if (ring) {
      for (int s = 0; s < S; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], NW);
      }
      fence_mbar_init();
    }
  }
  __syncthreads();

  if (STAGED && warp == NW) {
    // ------------------------------------------------------------ producer
    if (ring && lane == 0) {
      int64_t issued = 0;
      for (int64_t jj = 0; jj < nbatch; ++jj) {
        const int s = (int)(jj % S);
        if (jj >= S) {
          bool ok = false;
          if (!*(volatile int*)&s_abort) ok = mbar_wait_bounded(&empty[s], (unsigned)(((jj / S) - 1) & 1), P.wait_ns);
          if (!ok) {
            *(volatile int*)&s_abort = 1;
            if (P.errword != nullptr) atomicOr(P.errword, KF_DEVERR_TIMEOUT);
            break;
          }
        }
        const int64_t unit = rev ? u_end - 1 - jj / NBU : u_begin + jj / NBU;
        const int64_t rowb = (unit << 3) + (jj % NBU) * U;
        unsigned bytes = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (rowb + u < m) bytes += NMAT * SEG;
        mbar_expect_tx(&full[s], bytes);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (rowb + u < m) {
#pragma unroll
            for (int t = 0; t < NMAT; ++t) {
              const char* src = static_cast<const char*>(P.A[t]) + ((rowb + u) * P.lda[t] + col0) * BYTES;
              bulk_g2s(ringp + (size_t)s * BATCH + (size_t)(t * U + u) * SEG, src, SEG, &full[s]);
            }
          }
        }
        issued = jj + 1;
      }
      if (*(volatile int*)&s_abort) {
        // let the copies that may still be in flight land before exiting
        for (int64_t q = issued - S < 0 ? 0 : issued - S; q < issued; ++q)
          (void)mbar_wait_bounded(&full[q % S], (unsigned)((q / S) & 1), WAIT_DRAIN_NS);
      }
    }
    __syncwarp();  // reconverge the producer warp before the block barrier below
  } else {
    // ------------------------------------------------------------ consumers
    float cv[NOPS][W];  // invariant column vectors (GER v, GEMV x) or GEMVT sums
#pragma unroll
    for (int k = 0; k < NOPS; ++k) {
      const int kind = SPEC ? sig_kind(SIG, k) : ((k < nops) ? P.ops[k].kind : MOP_NONE);
      const float* src = (kind == MOP_GER || kind == MOP_GEMV) ? P.ops[k].colvec : nullptr;
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int e = 0; e < CH; ++e) {
          const int64_t c = wcol0 + coff<CH, V, VEC>(v, e, lane);
          cv[k][v * CH + e] = (src != nullptr && c < n) ? __ldg(src + c) : 0.f;
        }
    }
    bool dead = false;  // block-uniform in effect: set from s_abort

    auto load_batch = [&](int64_t row0, int r, int64_t jj, BatchT& a) {
      if (ring) {
        const int s = (int)(jj % S);
        bool ok = false;
        if (!dead && !*(volatile int*)&s_abort) ok = mbar_wait_bounded(&full[s], (unsigned)((jj / S) & 1), P.wait_ns);
        ok = __all_sync(FULL_MASK, ok);
        if (!ok && !dead) {
          dead = true;
          if (lane == 0) {
            *(volatile int*)&s_abort = 1;
            if (P.errword != nullptr) atomicOr(P.errword, KF_DEVERR_TIMEOUT);
          }
        }
        const char* stage = ringp + (size_t)s * BATCH + (size_t)warp * SEGW;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool row_ok = !dead && (row0 + r + u < m);
#pragma unroll
          for (int t = 0; t < NMAT; ++t)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              if constexpr (RAW) {
                a[t][u][v] = row_ok ? *reinterpret_cast<const uint4*>(stage + (size_t)(t * U + u) * SEG +
                                                                        (size_t)(v * 32 + lane) * 16)
                                    : make_uint4(0u, 0u, 0u, 0u);
              } else if (row_ok) {
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
        if (lane == 0 && !dead) mbar_arrive(&empty[s]);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t row = row0 + r + u;
#pragma unroll
          for (int t = 0; t < NMAT; ++t) {
            if constexpr (RAW) load_row_raw<FMT, V>(P.A[t], P.lda[t], row, row < m, wcol0, n, lane, a[t][u], lpol);
            else load_row<FMT, V, VEC>(P.A[t], P.lda[t], row, row < m, wcol0, n, lane, a[t][u], lpol);
          }
        }
      }
    };

    int64_t j = 0;  // batch counter (every consumer warp visits every batch)
    for (int64_t ri = 0; ri < rb_end - rb_begin; ++ri) {
      const int64_t rb = rev ? rb_end - 1 - ri : rb_begin + ri;
      const int64_t row0 = rb << 5;
      const bool lane_row_ok = row0 + lane < m;
      // this lane's row (row0 + lane) belongs to the group: its partials are ours to store
      const int64_t lane_unit = (rb << 2) + (lane >> 3);
      const bool lane_in = lane_row_ok && lane_unit >= u_begin && lane_unit < u_end;
      float rv[NOPS];  // per-lane row scalar (GER u, GEMVT y) for row row0+lane
#pragma unroll
      for (int k = 0; k < NOPS; ++k) {
        const int kind = SPEC ? sig_kind(SIG, k) : ((k < nops) ? P.ops[k].kind : MOP_NONE);
        const float* rs = (kind == MOP_GER || kind == MOP_GEMVT) ? P.ops[k].rowvec : nullptr;
        rv[k] = (rs != nullptr && lane_row_ok) ? __ldg(rs + row0 + lane) : 0.f;
      }
      float rsc[NMAT];
#pragma unroll
      for (int t = 0; t < NMAT; ++t)
        rsc[t] = (FMT != FMT_F32 && lane_row_ok) ? __ldg(P.rscale[t] + row0 + lane) : 1.f;
      // Per-row scale of a low-precision output: a bound on |B_ij| over the
      // row, sA_i * QMAX + sum over the GERs of |alpha u_i| * max_j |v_j|,
      // divided by QMAX (1 for an all-zero bound), in this order.
      float sbrow = 1.f, isbrow = 1.f;
      if constexpr (QOUT) {
        float bound = __fmul_rn(rsc[0], QMAX);
#pragma unroll
        for (int k = 0; k <= LASTGER; ++k)
          if (sig_kind(SIG, k) == MOP_GER)
            bound = __fadd_rn(bound, __fmul_rn(fabsf(P.ops[k].alpha * rv[k]), __ldg(P.ops[k].vnorm)));
        sbrow = bound > 0.f ? __fdiv_rn(bound, QMAX) : 1.f;
        isbrow = __fdiv_rn(1.f, sbrow);
        if (strip == 0 && warp == 0 && lane_in) P.Bscale[0][row0 + lane] = sbrow;
      }
      float rowdot[NGA];  // this warp's partial of row row0+lane
#pragma unroll
      for (int g = 0; g < NGA; ++g) rowdot[g] = 0.f;

#pragma unroll 1
      for (int hi = 0; hi < 4; ++hi) {  // four quarters of 8 rows
        const int h = rev ? 3 - hi : hi;
        const int64_t unit = (rb << 2) + h;
        if (unit < u_begin || unit >= u_end) continue;  // another group's rows
        float dacc[NGA][8];          // per-lane partial dot of each row of the quarter
#pragma unroll
        for (int g = 0; g < NGA; ++g)
#pragma unroll
          for (int i = 0; i < 8; ++i) dacc[g][i] = 0.f;
#pragma unroll
        for (int r16 = 0; r16 < 8; r16 += U) {
          const int r = h * 8 + r16;
          BatchT a;
          load_batch(row0, r, j, a);
          ++j;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int rr = r + u;
            // the row's values: decoded, then scaled by the row's scale
            float ar[NMAT][W];
            float rowfac[NMAT];  // scale still to apply to this row's results (FOLD)
#pragma unroll
            for (int t = 0; t < NMAT; ++t) {
              rowfac[t] = 1.f;
              if constexpr (RAW) {
                const float sc = __shfl_sync(FULL_MASK, rsc[t], rr);
#pragma unroll
                for (int v = 0; v < V; ++v) decode16<FMT>(a[t][u][v], &ar[t][v * CH]);
                if constexpr (FOLD) {
                  rowfac[t] = sc;
                } else {
#pragma unroll
                  for (int e = 0; e < W; ++e) ar[t][e] = __fmul_rn(ar[t][e], sc);
                }
              } else {
#pragma unroll
                for (int e = 0; e < W; ++e) ar[t][e] = a[t][u][e];
                if constexpr (FMT != FMT_F32) {
                  const float sc = __shfl_sync(FULL_MASK, rsc[t], rr);
#pragma unroll
                  for (int e = 0; e < W; ++e) ar[t][e] *= sc;
                }
              }
            }
#pragma unroll
            for (int k = 0; k < NOPS; ++k) {
              if (SPEC || k < nops) {
                const MatOp& op = P.ops[k];
                const int kind = SPEC ? sig_kind(SIG, k) : op.kind;
                const int opmat = SPEC ? sig_mat(SIG, k) : op.mat;
                auto apply = [&](float (&t)[W]) {
                  if (kind == MOP_GER) {
                    const float sc = op.alpha * __shfl_sync(FULL_MASK, rv[k], rr);
#pragma unroll
                    for (int e = 0; e < W; ++e) t[e] = fmaf(sc, cv[k][e], t[e]);
                  } else if (kind == MOP_GEMV) {
                    if constexpr (NG > 0) {
                      float d0 = 0.f, d1 = 0.f;
#pragma unroll
                      for (int e = 0; e < W; e += 2) {
                        d0 = fmaf(t[e], cv[k][e], d0);
                        d1 = fmaf(t[e + 1], cv[k][e + 1], d1);
                      }
                      int slot0;
                      if constexpr (SPEC) {
                        int c = 0;
#pragma unroll
                        for (int q = 0; q < k; ++q) c += sig_kind(SIG, q) == MOP_GEMV;
                        slot0 = (c == 0);
                      } else {
                        slot0 = (op.res == 0);
                      }
                      float d = d0 + d1;
                      if constexpr (FOLD) d *= rowfac[NMAT == 1 ? 0 : opmat];
                      if (NG == 1 || slot0) dacc[0][r16 + u] += d;
                      else dacc[NGA - 1][r16 + u] += d;
                    }
                  } else if (kind == MOP_GEMVT) {
                    float y = __shfl_sync(FULL_MASK, rv[k], rr);
                    if constexpr (FOLD) y *= rowfac[NMAT == 1 ? 0 : opmat];
#pragma unroll
                    for (int e = 0; e < W; ++e) cv[k][e] = fmaf(t[e], y, cv[k][e]);
                  }
                };
                if (NMAT == 1 || opmat == 0) apply(ar[0]);
                else apply(ar[NMAT - 1]);
                if constexpr (QOUT) {
                  if (k == LASTGER) {
                    const int64_t row = row0 + rr;
                    quant_store_row<FMT, V, VEC>(P.Bout[0], P.ldb[0], row, row < m, wcol0, n, lane, ar[0],
                                                 __shfl_sync(FULL_MASK, sbrow, rr),
                                                 __shfl_sync(FULL_MASK, isbrow, rr), keep_out);
                  }
                }
              }
            }
            const int64_t row = row0 + rr;
            if (!QOUT && row < m) {
#pragma unroll
              for (int t = 0; t < NMAT; ++t)
                if (P.Bout[t] != nullptr)
                  store_row<CH, V, VEC>(P.Bout[t], P.ldb[t], row, wcol0, n, lane, ar[t], keep_out);
            }
          }
        }
        if constexpr (NG > 0) {
#pragma unroll
          for (int g = 0; g < NGA; ++g) {
            const float v = reduce8_rows(dacc[g], lane);
            if ((lane >> 3) == h) rowdot[g] = v;
          }
        }
      }
      // Row dots across the warps of the strip (fixed warp order), one
      // coalesced store of the strip's partial per GEMV result.
      if constexpr (NG > 0) {
        const int buf = (int)(rb & 1);
#pragma unroll
        for (int g = 0; g < NGA; ++g) red[buf][g][warp][lane] = rowdot[g];
        consumer_sync(NW * 32);
        if (warp < NGA && warp < P.nrow_res && lane_in) {
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) sum += red[buf][warp][w][lane];
          P.rowpart[((int64_t)warp * P.n_strips + strip) * m + row0 + lane] = sum;
        }
      }
    }
    // GEMVT: each warp owns its columns; one store of the group's partial.
#pragma unroll
    for (int k = 0; k < NOPS; ++k) {
      if ((SPEC ? sig_kind(SIG, k) : (k < nops ? P.ops[k].kind : 0)) == MOP_GEMVT) {
        float* part = P.colpart + ((int64_t)P.ops[k].res * cslots + group) * n;
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int e = 0; e < CH; ++e) {
            const int64_t c = wcol0 + coff<CH, V, VEC>(v, e, lane);
            if (c < n) part[c] = cv[k][v * CH + e];
          }
      }
    }
  }

  // Cross-block completion (Section 3.2.2, option (ii), in a fixed order).
  // Row results: the last block of a group adds the strips' partials in
  // strip order.  Column results: with at most MAT_COLSET groups the last
  // block of a strip adds the groups' partials in group order; with more, the
  // last block of each set of MAT_COLSET groups adds its set's partials in
  // group order into a set partial, and the last set of the strip to finish
  // adds the set partials in set order, so the sets finish side by side
  // instead of one block adding every group's partial.
  const int G = P.n_groups;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ls = 0, lg = 0;
    if (P.ncol_out > 0) {
      if (nsets == 1) {
        ls = atomicAdd(&P.counters[strip], 1u) == (unsigned)G - 1u ? 2 : 0;
      } else {
        const int set = group / MAT_COLSET;
        const int ssize = min(MAT_COLSET, G - set * MAT_COLSET);
        ls = atomicAdd(&setcnt[strip * MAT_MAXSETS + set], 1u) == (unsigned)ssize - 1u ? 1 : 0;
      }
    }
    if (P.nrow_out > 0)
      lg = atomicAdd(&P.counters[P.n_strips + group], 1u) == (unsigned)P.n_strips - 1u;
    s_last[0] = ls;
    s_last[1] = lg;
  }
  __syncthreads();
  // Sum of column partial slots [first, first + count) in slot order for the
  // strip's columns, four adjacent columns per thread and eight loads in
  // flight; into slot `to`, or (to < 0) through the column epilogue.
  auto col_sum = [&](int first, int count, int to) {
    const bool v4 = (n & 3) == 0;
    const int step = v4 ? 4 : 1;
    for (int c = threadIdx.x * step; c < SW; c += blockDim.x * step) {
      const int64_t col = col0 + c;
      if (col >= n) continue;
      float raw[4][NOPS];
#pragma unroll
      for (int q = 0; q < NOPS; ++q) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < P.ncol_res) {
          const float* part = P.colpart + ((int64_t)q * cslots + first) * n + col;
          int g = 0;
          if (v4) {
            for (; g + 8 <= count; g += 8) {
              float4 t[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) t[jj] = __ldcg(reinterpret_cast<const float4*>(part + (int64_t)(g + jj) * n));
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) { acc.x += t[jj].x; acc.y += t[jj].y; acc.z += t[jj].z; acc.w += t[jj].w; }
            }
            for (; g < count; ++g) {
              const float4 t = __ldcg(reinterpret_cast<const float4*>(part + (int64_t)g * n));
              acc.x += t.x; acc.y += t.y; acc.z += t.z; acc.w += t.w;
            }
          } else {
            for (; g + 8 <= count; g += 8) {
              float t[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) t[jj] = __ldcg(part + (int64_t)(g + jj) * n);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) acc.x += t[jj];
            }
            for (; g < count; ++g) acc.x += __ldcg(part + (int64_t)g * n);
          }
          if (to >= 0) {
            float* dst = P.colpart + ((int64_t)q * cslots + to) * n + col;
            if (v4) {
              *reinterpret_cast<float4*>(dst) = acc;
            } else {
              dst[0] = acc.x;
            }
          }
        }
        raw[0][q] = acc.x; raw[1][q] = acc.y; raw[2][q] = acc.z; raw[3][q] = acc.w;
      }
      if (to < 0)
        for (int e = 0; e < step; ++e)
          if (col + e < n) epilogue<NOPS>(P.col_out, P.ncol_out, raw[e], col + e);
    }
  };
  if (s_last[0] == 1) {
    // first level: this block closes its set of groups
    __threadfence();
    const int set = group / MAT_COLSET;
    col_sum(set * MAT_COLSET, min(MAT_COLSET, G - set * MAT_COLSET), G + set);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      setcnt[strip * MAT_MAXSETS + set] = 0u;
      s_last[0] = atomicAdd(&P.counters[strip], 1u) == (unsigned)nsets - 1u ? 2 : 0;
    }
    __syncthreads();
  }
  if (s_last[0] == 2) {
    // the strip's column results
    __threadfence();
    if (nsets == 1) col_sum(0, G, -1);
    else col_sum(G, nsets, -1);
    if (threadIdx.x == 0) P.counters[strip] = 0u;
  }
  if (s_last[1]) {
    __threadfence();
    // Row results of this group: sum the strips' partials in strip order.
    const int64_t r0 = u_begin << 3;
    const int64_t r1 = min(m, u_end << 3);
    const bool v4 = (m & 3) == 0;
    const int step = v4 ? 4 : 1;
    for (int64_t i = r0 + threadIdx.x * step; i < r1; i += (int64_t)blockDim.x * step) {
      float raw[4][NOPS];
#pragma unroll
      for (int q = 0; q < NOPS; ++q) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < P.nrow_res) {
          const float* part = P.rowpart + (int64_t)q * P.n_strips * m + i;
          int st = 0;
          if (v4) {
            for (; st + 8 <= P.n_strips; st += 8) {
              float4 t[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) t[jj] = __ldcg(reinterpret_cast<const float4*>(part + (int64_t)(st + jj) * m));
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) { acc.x += t[jj].x; acc.y += t[jj].y; acc.z += t[jj].z; acc.w += t[jj].w; }
            }
            for (; st < P.n_strips; ++st) {
              const float4 t = __ldcg(reinterpret_cast<const float4*>(part + (int64_t)st * m));
              acc.x += t.x; acc.y += t.y; acc.z += t.z; acc.w += t.w;
            }
          } else {
            for (; st + 8 <= P.n_strips; st += 8) {
              float t[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) t[jj] = __ldcg(part + (int64_t)(st + jj) * m);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) acc.x += t[jj];
            }
            for (; st < P.n_strips; ++st) acc.x += __ldcg(part + (int64_t)st * m);
          }
        }
        raw[0][q] = acc.x; raw[1][q] = acc.y; raw[2][q] = acc.z; raw[3][q] = acc.w;
      }
      for (int e = 0; e < step; ++e)
        if (i + e < r1) epilogue<NOPS>(P.row_out, P.nrow_out, raw[e], i + e);
    }
    if (threadIdx.x == 0) P.counters[P.n_strips + group] = 0u;
  }
}

// ---------------------------------------------------------------- registry

struct Entry {
  const void* fn;
  int nw, v, u, nops, nmat, ng, fmt;
  bool vec, staged;
  int sig;
};

// (warps, vec, unroll, nops, nmat, ngemv, fmt, vec-path, staged, signature)
using Key = std::tuple<int, int, int, int, int, int, int, bool, bool, int>;

std::map<Key, Entry>& registry();

template <int NW, int V, int U, int NOPS, int NMAT, int NG, int FMT, bool VEC, bool STAGED, int SIG = 0>
void reg() {
  registry()[Key(NW, V, U, NOPS, NMAT, NG, FMT, VEC, STAGED, SIG)] =
      Entry{(const void*)&matprog_kernel<NW, V, U, NOPS, NMAT, NG, FMT, VEC, STAGED, SIG>, NW, V, U,
            NOPS, NMAT, NG, FMT, VEC, STAGED, SIG};
}

// Runtime-dispatch op shapes (ops, matrices, GEMV results):
//   (1,1,0) GER or GEMVT alone   (1,1,1) GEMV alone       (2,1,1) BiCGK-like
//   (2,2,2) GESUMMV-like          (4,1,0) GEMVER pass 1    (4,1,1) (4,1,2) (4,2,2) general
template <int NW, int V, int U, int FMT, bool VEC, bool STAGED>
void reg_shapes() {
  reg<NW, V, U, 1, 1, 0, FMT, VEC, STAGED>();
  reg<NW, V, U, 1, 1, 1, FMT, VEC, STAGED>();
  reg<NW, V, U, 2, 1, 1, FMT, VEC, STAGED>();
  reg<NW, V, U, 2, 2, 2, FMT, VEC, STAGED>();
  reg<NW, V, U, 4, 1, 0, FMT, VEC, STAGED>();
  reg<NW, V, U, 4, 1, 1, FMT, VEC, STAGED>();
  reg<NW, V, U, 4, 1, 2, FMT, VEC, STAGED>();
  reg<NW, V, U, 4, 2, 2, FMT, VEC, STAGED>();
}

// Specialised signatures of the sequences' fusions.
template <int NW, int V, int U, int FMT, bool VEC, bool STAGED>
void reg_sigs() {
  reg<NW, V, U, 1, 1, 1, FMT, VEC, STAGED, SIG_GEMV>();
  reg<NW, V, U, 1, 1, 0, FMT, VEC, STAGED, SIG_GEMVT>();
  reg<NW, V, U, 1, 1, 0, FMT, VEC, STAGED, SIG_GER>();
  reg<NW, V, U, 2, 1, 1, FMT, VEC, STAGED, SIG_BICGK>();
  reg<NW, V, U, 3, 1, 0, FMT, VEC, STAGED, SIG_GEMVER1>();
  reg<NW, V, U, 2, 2, 2, FMT, VEC, STAGED, SIG_GESUMMV>();
}

// Signatures a row-scaled matrix takes (BiCGK, GEMV, GEMVT, GEMVER pass 1).
template <int NW, int V, int U, int FMT, bool VEC, bool STAGED>
void reg_lowp_sigs() {
  reg<NW, V, U, 1, 1, 1, FMT, VEC, STAGED, SIG_GEMV>();
  reg<NW, V, U, 1, 1, 0, FMT, VEC, STAGED, SIG_GEMVT>();
  reg<NW, V, U, 2, 1, 1, FMT, VEC, STAGED, SIG_BICGK>();
  reg<NW, V, U, 3, 1, 0, FMT, VEC, STAGED, SIG_GEMVER1>();
}

void register_f32_staged();
void register_f32_plain();
void register_f32_elem();
void register_bf16();
void register_e4m3();
void register_f32_sigs();

}  // namespace mp
}  // namespace kf
