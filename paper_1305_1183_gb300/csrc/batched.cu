// Batched BiCGK / GESUMMV: many independent instances of uneven sizes in one
// persistent launch.
//
// The host cuts every instance into tiles (row bands of `band_rows` rows x
// column strips) and sorts them largest first.  An instance's strip is as
// wide as the instance needs, cw x 128 columns with cw in {1, 2, 4, 8}
// warps side by side; the block's 8 / cw warp rows take turns over the
// band's 32-row blocks, so narrow matrices do not leave warps on masked
// columns.  Blocks pull tiles from an atomic queue; in a tile, row dots are
// kept as per-lane partials of 8 rows, reduced across the cw warps of a warp
// row (a named barrier per warp row), and column sums are added across the
// warp rows in row order at the end of the tile; the tile writes its
// instance's row partial (per strip) and column partial (per band).  The
// last tile of an instance to finish (a per-instance counter) adds the
// partials in strip / band order and writes the outputs (Section 3.2.2,
// option (ii)), so each instance's result does not depend on which block ran
// which tile, and equals the same instance run alone.  The queue and the
// counters reset themselves, so the launch can be replayed from a CUDA graph.
//
// Loads are element-interleaved (lane l of a warp reads columns l, l+32,
// l+64, l+96 of its 128-column slice), so every load instruction covers 128
// contiguous bytes for any row length and alignment; a warp keeps 8 rows
// of one matrix (BiCGK) or 4 rows of two (GESUMMV) in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/kf.h"
#include "kf_device.cuh"
#include "kf_internal.h"

namespace kf {
const char* set_error_message(const std::string& msg);
int device_sm_count();

namespace {

struct BDesc {
  int64_t m, n, lda;
  const float* A;
  const float* B;
  const float* x;   // BiCGK p / GESUMMV x
  const float* r;   // BiCGK r
  float* y;         // BiCGK q / GESUMMV y
  float* s;         // BiCGK s
  float alpha, beta;
  int64_t rowpart_off, colpart_off;
  int ntiles, nstrips, nbands, cw;  // cw: warps side by side across the strip (width-adapted form)
};

struct BTile {
  int inst, band, strip, pad;
};

constexpr int BNW = 8;             // warps per block (side by side)

__device__ __forceinline__ float reduce8(float (&d)[8], int lane) {
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

// KIND 0: BiCGK (q = A p, s = A^T r);  KIND 1: GESUMMV (y = a A x + b B x).
// cw warps side by side across a strip of cw x 128 columns, the 8 / cw warp
// rows taking turns over the band's 32-row blocks; 3 blocks per SM.
template <int KIND>
__global__ void __launch_bounds__(BNW * 32, 3)
    batched_kernel(const BDesc* __restrict__ D, const BTile* __restrict__ T, int ntiles, int band_rows,
                   float* __restrict__ rowpart, float* __restrict__ colpart, unsigned* __restrict__ inst_count,
                   unsigned* __restrict__ queue) {
  constexpr int NM = KIND == 0 ? 1 : 2;   // matrices
  constexpr int NR = KIND == 0 ? 1 : 2;   // row results
  constexpr int BU = KIND == 0 ? 8 : 4;   // rows loaded together (the same bytes in flight for one matrix as for two)
  __shared__ int s_tile;
  __shared__ int s_last;
  __shared__ BDesc s_desc;  // the tile's instance, read field by field (keeps registers free)
  __shared__ float red[2][NR][BNW][32];
  __shared__ float csum[KIND == 0 ? BNW : 1][128];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (;;) {
    __syncthreads();  // previous tile's shared-memory use is over
    if (threadIdx.x == 0) {
      const int tt = (int)atomicAdd(&queue[0], 1u);
      s_tile = tt;
      if (tt < ntiles) s_desc = D[T[tt].inst];
    }
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const BTile tl = T[t];
    const BDesc& d = s_desc;
    const int64_t m = d.m, n = d.n;
    // cw warps side by side cover the strip (cw * 128 columns); the block's
    // rw = 8 / cw warp rows take turns over the band's 32-row blocks
    const int cw = d.cw, rw = BNW / cw;
    const int wcol = warp % cw, wrow = warp / cw;
    const int64_t r0 = (int64_t)tl.band * band_rows;
    const int64_t r1 = min(m, r0 + band_rows);
    const int64_t wc = (int64_t)tl.strip * cw * 128 + wcol * 128;  // this warp's slice

    float xv[4], acc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t c = wc + e * 32 + lane;
      xv[e] = c < n ? __ldg(d.x + c) : 0.f;
      acc[e] = 0.f;
    }
    const int64_t nblk = (r1 - r0 + 31) >> 5;
    const int64_t iters = (nblk + rw - 1) / rw;  // the same for every warp (barriers below)
    for (int64_t it = 0; it < iters; ++it) {
      const int64_t k = it * rw + wrow;
      const bool blk_ok = k < nblk;  // warp-uniform
      const int64_t row0 = r0 + k * 32;
      const bool lane_ok = blk_ok && row0 + lane < r1;
      const float rv = (KIND == 0 && lane_ok) ? __ldg(d.r + row0 + lane) : 0.f;
      float rowdot[NR];
#pragma unroll
      for (int g = 0; g < NR; ++g) rowdot[g] = 0.f;
      if (blk_ok) {
#pragma unroll 1
        for (int h = 0; h < 4; ++h) {
          float dacc[NR][8];
#pragma unroll
          for (int g = 0; g < NR; ++g)
#pragma unroll
            for (int i = 0; i < 8; ++i) dacc[g][i] = 0.f;
#pragma unroll
          for (int b = 0; b < 8; b += BU) {
            float a[NM][BU][4];
#pragma unroll
            for (int u = 0; u < BU; ++u) {
              const int64_t row = row0 + h * 8 + b + u;
              const bool rok = row < r1;
#pragma unroll
              for (int kk = 0; kk < NM; ++kk) {
                const float* rowp = (kk == 0 ? d.A : d.B) + row * d.lda;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const int64_t c = wc + e * 32 + lane;
                  a[kk][u][e] = (rok && c < n) ? __ldcs(rowp + c) : 0.f;
                }
              }
            }
#pragma unroll
            for (int u = 0; u < BU; ++u) {
#pragma unroll
              for (int kk = 0; kk < NM; ++kk) {
                float dd = 0.f;
#pragma unroll
                for (int e = 0; e < 4; ++e) dd = fmaf(a[kk][u][e], xv[e], dd);
                dacc[kk][b + u] += dd;
              }
              if (KIND == 0) {
                const float y = __shfl_sync(FULL_MASK, rv, h * 8 + b + u);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] = fmaf(a[0][u][e], y, acc[e]);
              }
            }
          }
#pragma unroll
          for (int g = 0; g < NR; ++g) {
            const float v = reduce8(dacc[g], lane);
            if ((lane >> 3) == h) rowdot[g] = v;
          }
        }
      }
      // row dots across the cw warps of this warp row, in fixed warp order
      if (cw == 1) {
        if (lane_ok)
#pragma unroll
          for (int g = 0; g < NR; ++g)
            rowpart[d.rowpart_off + ((int64_t)g * d.nstrips + tl.strip) * m + row0 + lane] = rowdot[g];
      } else {
        const int buf = (int)(it & 1);
#pragma unroll
        for (int g = 0; g < NR; ++g) red[buf][g][warp][lane] = rowdot[g];
        asm volatile("bar.sync %0, %1;" ::"r"(1 + wrow), "r"(cw * 32) : "memory");
        if (wcol < NR && lane_ok) {
          float sum = 0.f;
          for (int w = 0; w < cw; ++w) sum += red[buf][wcol][wrow * cw + w][lane];
          rowpart[d.rowpart_off + ((int64_t)wcol * d.nstrips + tl.strip) * m + row0 + lane] = sum;
        }
      }
    }
    if (KIND == 0) {
      // column sums of the strip: the rw warp rows added in row order
      if (rw == 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t c = wc + e * 32 + lane;
          if (c < n) colpart[d.colpart_off + (int64_t)tl.band * n + c] = acc[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) csum[warp][e * 32 + lane] = acc[e];
        __syncthreads();
        if (wrow == 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float sum = 0.f;
            for (int q = 0; q < rw; ++q) sum += csum[q * cw + wcol][e * 32 + lane];
            const int64_t c = wc + e * 32 + lane;
            if (c < n) colpart[d.colpart_off + (int64_t)tl.band * n + c] = sum;
          }
        }
      }
    }
    // last tile of the instance finishes it
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&inst_count[tl.inst], 1u) == (unsigned)d.ntiles - 1u;
    __syncthreads();
    if (s_last) {
      __threadfence();
      // four rows per thread at a time (their strip partials load together),
      // each row's partials added in strip order
      for (int64_t i0 = threadIdx.x; i0 < m; i0 += 4 * (int64_t)blockDim.x) {
        float v[4][NR];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int g = 0; g < NR; ++g) v[q][g] = 0.f;
        for (int st = 0; st < d.nstrips; ++st) {
          float x[4][NR];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t i = i0 + q * (int64_t)blockDim.x;
#pragma unroll
            for (int g = 0; g < NR; ++g)
              x[q][g] = i < m ? __ldcg(rowpart + d.rowpart_off + ((int64_t)g * d.nstrips + st) * m + i) : 0.f;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int g = 0; g < NR; ++g) v[q][g] += x[q][g];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t i = i0 + q * (int64_t)blockDim.x;
          if (i < m) {
            if (KIND == 0) d.y[i] = v[q][0];
            else d.y[i] = __fadd_rn(__fmul_rn(d.alpha, v[q][0]), __fmul_rn(d.beta, v[q][NR - 1]));
          }
        }
      }
      if (KIND == 0) {
        // two columns per thread at a time, each column's band partials
        // loaded eight at a time and added in band order
        for (int64_t j = threadIdx.x; j < n; j += 2 * (int64_t)blockDim.x) {
          const int64_t j2 = j + blockDim.x;
          const float* p0 = colpart + d.colpart_off + j;
          float s0 = 0.f, s1 = 0.f;
          for (int k0 = 0; k0 < d.nbands; k0 += 8) {
            float v0[8], v1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const bool ok = k0 + k < d.nbands;
              v0[k] = ok ? __ldcg(p0 + (int64_t)(k0 + k) * n) : 0.f;
              v1[k] = ok && j2 < n ? __ldcg(p0 + (int64_t)(k0 + k) * n + blockDim.x) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (k0 + k < d.nbands) {
                s0 += v0[k];
                s1 += v1[k];
              }
          }
          d.s[j] = s0;
          if (j2 < n) d.s[j2] = s1;
        }
      }
      if (threadIdx.x == 0) inst_count[tl.inst] = 0u;
    }
  }
  // the last block out resets the queue for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&queue[1], 1u) == gridDim.x - 1u) {
      queue[0] = 0u;
      queue[1] = 0u;
      __threadfence();
    }
  }
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace kf

struct kf_batched {
  int kind = 0;
  int count = 0;
  int band_rows = 128;
  std::vector<kf::BDesc> desc;
  std::vector<kf::BTile> tiles;
  int64_t rowpart_floats = 0, colpart_floats = 0;
  size_t off_queue = 0, off_counts = 0, off_desc = 0, off_tiles = 0, off_row = 0, off_col = 0, total = 0;
  double bytes = 0.0;  // algorithmic bytes of one launch
};

using namespace kf;

extern "C" {

kf_status kf_batched_create(kf_seq seq, const kf_batch_desc* descs, int count, int band_rows, kf_batched** out) {
  if (out == nullptr || count < 0 || (count > 0 && descs == nullptr)) {
    set_error_message("bad arguments");
    return KF_ERR_INVALID_ARG;
  }
  if (seq != KF_SEQ_BICGK && seq != KF_SEQ_GESUMMV) {
    set_error_message("batched form exists for BiCGK and GESUMMV");
    return KF_ERR_UNSUPPORTED;
  }
  if (band_rows <= 0) band_rows = 128;
  if (band_rows % 32 != 0 || band_rows > 4096) {
    set_error_message("band_rows must be a multiple of 32 up to 4096");
    return KF_ERR_INVALID_ARG;
  }
  auto* b = new (std::nothrow) kf_batched();
  if (b == nullptr) { set_error_message("out of host memory"); return KF_ERR_NO_MEM; }
  b->kind = seq == KF_SEQ_BICGK ? 0 : 1;
  b->count = count;
  b->band_rows = band_rows;
  const int nr = b->kind == 0 ? 1 : 2;
  for (int i = 0; i < count; ++i) {
    const kf_batch_desc& u = descs[i];
    const bool bad = u.m < 0 || u.n < 0 || (u.m > 0 && u.lda < u.n) || (u.m > 0 && u.n > 0 && u.A == nullptr) ||
                     (b->kind == 1 && u.m > 0 && u.n > 0 && u.B == nullptr) || (u.n > 0 && u.x == nullptr) ||
                     (u.m > 0 && u.y == nullptr) || (b->kind == 0 && ((u.m > 0 && u.r == nullptr) || (u.n > 0 && u.s == nullptr)));
    if (bad) {
      delete b;
      set_error_message("instance " + std::to_string(i) + ": bad shape or null pointer");
      return KF_ERR_INVALID_ARG;
    }
    BDesc d{};
    d.m = u.m; d.n = u.n; d.lda = u.lda;
    d.A = u.A; d.B = u.B; d.x = u.x; d.r = u.r; d.y = u.y; d.s = u.s;
    d.alpha = u.alpha; d.beta = u.beta;
    // narrow matrices take fewer warps per row and more row blocks at once
    d.cw = u.n <= 128 ? 1 : u.n <= 256 ? 2 : u.n <= 512 ? 4 : BNW;
    d.nstrips = (int)std::max<int64_t>(1, (u.n + d.cw * 128 - 1) / (d.cw * 128));
    d.nbands = (int)std::max<int64_t>(1, (u.m + band_rows - 1) / band_rows);
    d.ntiles = d.nstrips * d.nbands;
    d.rowpart_off = b->rowpart_floats;
    d.colpart_off = b->colpart_floats;
    b->rowpart_floats += (int64_t)nr * d.nstrips * u.m;
    if (b->kind == 0) b->colpart_floats += (int64_t)d.nbands * u.n;
    b->desc.push_back(d);
    for (int bd = 0; bd < d.nbands; ++bd)
      for (int st = 0; st < d.nstrips; ++st) b->tiles.push_back(BTile{i, bd, st, 0});
    b->bytes += 4.0 * (double)(b->kind == 0 ? u.m * u.n + 2 * (u.m + u.n) : 2 * u.m * u.n + u.m + u.n);
  }
  // largest tiles first (balance across the persistent blocks)
  auto tsize = [&](const BTile& t) {
    const BDesc& d = b->desc[t.inst];
    const int64_t rows = std::min<int64_t>(band_rows, d.m - (int64_t)t.band * band_rows);
    const int64_t sw = (int64_t)d.cw * 128;
    const int64_t cols = std::min<int64_t>(sw, d.n - (int64_t)t.strip * sw);
    return rows * cols;
  };
  std::stable_sort(b->tiles.begin(), b->tiles.end(), [&](const BTile& x, const BTile& y) { return tsize(x) > tsize(y); });
  size_t o = WS_HEADER;
  b->off_queue = o; o += 256;
  b->off_counts = o; o += a256((size_t)count * 4);
  b->off_desc = o; o += a256(b->desc.size() * sizeof(BDesc));
  b->off_tiles = o; o += a256(b->tiles.size() * sizeof(BTile));
  b->off_row = o; o += a256((size_t)b->rowpart_floats * 4);
  b->off_col = o; o += a256((size_t)b->colpart_floats * 4);
  b->total = o;
  *out = b;
  return KF_OK;
}

void kf_batched_destroy(kf_batched* b) { delete b; }

kf_status kf_batched_workspace_size(const kf_batched* b, size_t* bytes) {
  if (b == nullptr || bytes == nullptr) { set_error_message("null argument"); return KF_ERR_INVALID_ARG; }
  *bytes = b->total;
  return KF_OK;
}

kf_status kf_batched_info(const kf_batched* b, int* ntiles, double* bytes) {
  if (b == nullptr) { set_error_message("null argument"); return KF_ERR_INVALID_ARG; }
  if (ntiles) *ntiles = (int)b->tiles.size();
  if (bytes) *bytes = b->bytes;
  return KF_OK;
}

kf_status kf_batched_upload(const kf_batched* b, void* ws, size_t ws_bytes, void* stream) {
  if (b == nullptr || ws == nullptr || ws_bytes < b->total) {
    set_error_message("workspace missing or smaller than kf_batched_workspace_size()");
    return KF_ERR_WORKSPACE;
  }
  char* w = static_cast<char*>(ws);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(w, 0, b->off_desc, st);  // header, queue, instance counters
  if (e == cudaSuccess && !b->desc.empty())
    e = cudaMemcpyAsync(w + b->off_desc, b->desc.data(), b->desc.size() * sizeof(BDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !b->tiles.empty())
    e = cudaMemcpyAsync(w + b->off_tiles, b->tiles.data(), b->tiles.size() * sizeof(BTile), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables may change after return
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  return KF_OK;
}

kf_status kf_batched_launch(const kf_batched* b, void* ws, size_t ws_bytes, void* stream) {
  if (b == nullptr || ws == nullptr || ws_bytes < b->total) {
    set_error_message("workspace missing or smaller than kf_batched_workspace_size()");
    return KF_ERR_WORKSPACE;
  }
  if (b->tiles.empty()) return KF_OK;
  char* w = static_cast<char*>(ws);
  const void* fn = b->kind == 0 ? (const void*)&batched_kernel<0> : (const void*)&batched_kernel<1>;
  static int occ[2] = {0, 0};
  if (occ[b->kind] == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, BNW * 32, 0) != cudaSuccess || o < 1) o = 1;
    occ[b->kind] = o;
  }
  const int grid = (int)std::min<int64_t>((int64_t)device_sm_count() * occ[b->kind], (int64_t)b->tiles.size());
  const BDesc* D = reinterpret_cast<const BDesc*>(w + b->off_desc);
  const BTile* T = reinterpret_cast<const BTile*>(w + b->off_tiles);
  int nt = (int)b->tiles.size();
  int br = b->band_rows;
  float* rp = reinterpret_cast<float*>(w + b->off_row);
  float* cp = reinterpret_cast<float*>(w + b->off_col);
  unsigned* cnt = reinterpret_cast<unsigned*>(w + b->off_counts);
  unsigned* q = reinterpret_cast<unsigned*>(w + b->off_queue);
  void* args[] = {(void*)&D, (void*)&T, (void*)&nt, (void*)&br, (void*)&rp, (void*)&cp, (void*)&cnt, (void*)&q};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(BNW * 32), args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  return KF_OK;
}

kf_status kf_batched_graph_create(const kf_batched* b, void* ws, size_t ws_bytes, void** graph_exec) {
  if (graph_exec == nullptr) { set_error_message("null argument"); return KF_ERR_INVALID_ARG; }
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    set_error_message("cudaStreamCreate failed");
    return KF_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  kf_status rc = KF_OK;
  if (e == cudaSuccess) {
    rc = kf_batched_launch(b, ws, ws_bytes, st);
    e = cudaStreamEndCapture(st, &g);
  }
  if (e == cudaSuccess && rc == KF_OK) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(st);
  if (rc != KF_OK) return rc;
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  *graph_exec = ge;
  return KF_OK;
}

kf_status kf_batched_graph_launch(void* graph_exec, void* stream) {
  if (graph_exec == nullptr) { set_error_message("null graph"); return KF_ERR_INVALID_ARG; }
  cudaError_t e = cudaGraphLaunch((cudaGraphExec_t)graph_exec, (cudaStream_t)stream);
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return KF_ERR_CUDA; }
  return KF_OK;
}

void kf_batched_graph_destroy(void* graph_exec) {
  if (graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)graph_exec);
}


// Tile height for a batch: every candidate band height is uploaded into the
// workspace and launched `reps` times; the fastest median wins.  The
// workspace must hold the largest candidate (kf_batched_workspace_bound).
static const int kBandCandidates[] = {32, 64, 128, 256, 512};

kf_status kf_batched_workspace_bound(kf_seq seq, const kf_batch_desc* descs, int count, size_t* bytes) {
  if (bytes == nullptr) { set_error_message("null argument"); return KF_ERR_INVALID_ARG; }
  size_t mx = 0;
  for (int br : kBandCandidates) {
    kf_batched* b = nullptr;
    kf_status st = kf_batched_create(seq, descs, count, br, &b);
    if (st != KF_OK) return st;
    mx = std::max(mx, b->total);
    kf_batched_destroy(b);
  }
  *bytes = mx;
  return KF_OK;
}

kf_status kf_batched_autotune(kf_seq seq, const kf_batch_desc* descs, int count, void* ws, size_t ws_bytes,
                              void* stream, int reps, int* best_band_rows, float* best_ms) {
  if (best_band_rows == nullptr || reps <= 0) { set_error_message("bad arguments"); return KF_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a, e;
  cudaEventCreate(&a);
  cudaEventCreate(&e);
  float bm = 1e30f;
  int bb = 128;
  kf_status rc = KF_OK;
  for (int br : kBandCandidates) {
    kf_batched* b = nullptr;
    rc = kf_batched_create(seq, descs, count, br, &b);
    if (rc != KF_OK) break;
    rc = kf_batched_upload(b, ws, ws_bytes, stream);
    std::vector<float> v;
    if (rc == KF_OK) rc = kf_batched_launch(b, ws, ws_bytes, stream);
    for (int r = 0; r < reps && rc == KF_OK; ++r) {
      cudaEventRecord(a, st);
      rc = kf_batched_launch(b, ws, ws_bytes, stream);
      cudaEventRecord(e, st);
      cudaEventSynchronize(e);
      float x = 0.f;
      cudaEventElapsedTime(&x, a, e);
      v.push_back(x);
    }
    kf_batched_destroy(b);
    if (rc != KF_OK) break;
    std::sort(v.begin(), v.end());
    if (!v.empty() && v[v.size() / 2] < bm * 0.999f) { bm = v[v.size() / 2]; bb = br; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(e);
  if (rc != KF_OK) return rc;
  *best_band_rows = bb;
  if (best_ms) *best_ms = bm;
  return KF_OK;
}

}  // extern "C"
