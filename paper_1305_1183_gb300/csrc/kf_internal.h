// Internal descriptors shared by the host side of libkf and its kernels.
//
// A fused kernel is described by a small "program" that the host fills and
// passes by value (__grid_constant__) to one of two kernel families:
//
//  * MatProg: one pass over one or two m x n matrices (nesting depth 2 in the
//    paper's terms, Section 3.3).  Ops run per matrix tile in script order:
//    GER updates the tile in registers, GEMV takes row dot products (nested
//    map-reduce over rows), GEMVT accumulates column sums (the same function
//    on A viewed as a list of columns).  Row and column reductions that cross
//    thread blocks are finished by the last block to arrive (Section 3.2.2,
//    option (ii)) in a fixed order, followed by a linear epilogue.
//
//  * VecProg: one pass over vectors (depth 1).  Every map call of BLAS-1
//    (AXPY, SCAL, WAXPBY, VADD, copy) is linear, so a fused chain of them is
//    a linear combination of the input vectors; the host folds the chain into
//    coefficient rows and the kernel evaluates them.  DOT products of such
//    combinations are per-block partial reductions finished by the last block.
#pragma once

#include <cstddef>
#include <cstdint>

namespace kf {

constexpr int MAT_MAXOPS = 4;
constexpr int EPI_MAXTERM = 4;
constexpr int EPI_MAXOUT = 4;
constexpr int MAT_MAXGROUPS = 128;     // bound on row groups (workspace sizing)
constexpr int MAT_COLSET = 8;          // column partials added per first-level finisher
constexpr int MAT_MAXSETS = MAT_MAXGROUPS / MAT_COLSET;
constexpr int MAT_MAXSTAGES = 8;       // bound on the per-warp copy ring depth
constexpr size_t WS_HEADER = 256;      // every workspace starts with a 256-byte header (error word at 0)
constexpr size_t WS_AUX = 64;          // header offset of per-launch device scalars (vector norms)

constexpr int VP_MAXIN = 6;
constexpr int VP_MAXOUT = 4;
constexpr int VP_MAXDOT = 4;
constexpr int VP_MAXBLOCKS = 4096;     // bound on vector-kernel blocks (workspace)

enum MatOpKind : int { MOP_NONE = 0, MOP_GER = 1, MOP_GEMV = 2, MOP_GEMVT = 3 };

// Storage format of a matrix operand.
enum MatFmt : int { FMT_F32 = 0, FMT_BF16 = 1, FMT_E4M3 = 2 };

struct MatOp {
  int kind;              // MatOpKind
  int mat;               // matrix operand (0 or 1)
  int res;               // GEMV: row-result id; GEMVT: column-result id
  float alpha;           // GER: coefficient of u v^T
  const float* colvec;   // GER: v (length n); GEMV: x (length n)
  const float* rowvec;   // GER: u (length m); GEMVT: y (length m)
  const float* vnorm;    // GER into a low-precision matrix: device max_j |colvec_j|
};

// One epilogue output: dst[i] = sum_t coef[t] * (src[t] >= 0 ? raw_src[t][i] : ext[t][i])
// where raw_k is the finished k-th row (or column) reduction.
struct EpiOut {
  float* dst;
  int nterm;
  int src[EPI_MAXTERM];
  const float* ext[EPI_MAXTERM];
  float coef[EPI_MAXTERM];
};

struct MatProg {
  int64_t m, n;
  int nmat;
  int fmt;                       // MatFmt of A[] (both operands share it)
  const void* A[2];
  const float* rscale[2];        // per-row scales (low-precision formats)
  int64_t lda[2];
  float* Bout[2];                // updated matrix output or nullptr (codes when fmt is low precision)
  int64_t ldb[2];
  float* Bscale[2];              // per-row scales written with a low-precision Bout
  int nops;
  MatOp ops[MAT_MAXOPS];
  int nrow_res, ncol_res;
  int nrow_out, ncol_out;
  EpiOut row_out[EPI_MAXOUT];
  EpiOut col_out[EPI_MAXOUT];
  // geometry
  int n_strips, n_groups;
  int stages;                    // per-warp bulk-copy ring depth (staged kernels)
  int64_t units_per_group;       // 8-row units per row group
  // workspace
  float* rowpart;                // [nrow_res][n_strips][m]
  float* colpart;                // [ncol_res][n_groups + sets][n] (group partials, then set partials)
  unsigned* counters;            // [n_strips + MAT_MAXGROUPS + n_strips * MAT_MAXSETS], zero between launches
  unsigned* errword;             // device error word (bounded waits that ran out)
  uint64_t wait_ns;              // bound of every wait on data (set by launch_matprog)
  // L2 use: the matrix output stored at normal priority (read again by the
  // next pass) instead of streamed, and rows walked from the last 8-row unit
  // of each group to the first (reading first what an earlier pass over the
  // same rows wrote last).  Matrix loads always stream (evict-first).
  int l2_keep_out;
  int reverse_rows;
};

struct VecProg {
  int64_t n;
  int nin, nout, ndot;
  const float* in[VP_MAXIN];
  float* out[VP_MAXOUT];
  float C[VP_MAXOUT][VP_MAXIN];   // out_j = sum_k C[j][k] in_k
  float* dot_out[VP_MAXDOT];      // device scalars
  float P[VP_MAXDOT][VP_MAXIN];   // dot_d = (sum_k P[d][k] in_k) . (sum_k Q[d][k] in_k)
  float Q[VP_MAXDOT][VP_MAXIN];
  int fp64_final;                 // finish the cross-block sum in double
  float* dotpart;                 // [ndot][gridDim]
  unsigned* counter;              // one word, zero between launches
};

// Tuning knobs of a matrix-pass launch (chosen by the autotuner or defaults).
struct MatTune {
  int warps;      // warps per block: 4 or 8
  int vec;        // 16-byte chunks per lane per row: 1, 2 or 4
  int unroll;     // rows loaded together: 1, 2 or 4
  int groups;     // row groups (0 = automatic)
  int stages;     // bulk-copy ring depth per warp; 0 = direct 16-byte loads
};

// Tuning knobs of a vector-pass launch.
struct VecTune {
  int threads;    // 128 or 256 or 512
  int unroll;     // float4 chunks per thread per input per iteration
  int blocks;     // 0 = automatic (a multiple of the SM count)
};

// Status codes mirror kf.h.
int launch_matprog(MatProg& P, const MatTune& t, void* stream, const char** why);
bool matprog_sig_compiled(const int* kinds, const int* mats, int nops, int fmt);
// The tuning an automatic launch would take without running a search: the
// fixed tuning when its warps field is set, else the tuning cache's entry for
// P's op signature and size class, else the built-in tuning.
MatTune matprog_tuning_nosearch(const MatProg& P, const MatTune& fixed);
// The matrix tuning fixed by kf_set_matrix_tuning (warps = 0: automatic).
MatTune current_matrix_tuning();
// cudaLaunchKernelExC with programmatic stream serialization (the kernel
// must begin with pdl_enter()).
cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, void* stream);
// out[k] = max_j |v_k[j]| for the nv <= 4 vectors v_k of length n (device).
int launch_colnorms(const float* const* v, int nv, int64_t n, float* out, void* stream, const char** why);
int launch_vecprog(VecProg& P, const VecTune& t, void* stream, const char** why);
size_t matprog_workspace_bytes(int64_t m, int64_t n, int nrow_res, int ncol_res, int fmt);
size_t vecprog_workspace_bytes(int ndot);
int matprog_bind_workspace(MatProg& P, void* ws, size_t bytes);
void matprog_geometry(MatProg& P, const MatTune& t, int sm_count, int* threads, size_t* smem);

int device_sm_count();

// ATAX, y = scale * A^T (A x): the single pass when the shape and pointers
// allow it, else the two matrix passes; workspace as kf_workspace_size's
// KF_SEQ_ATAX (atax_plan_workspace_bytes).
// Returns a kf_status; the calling thread's error message is set on failure.
int atax_run(int64_t m, int64_t n, const float* A, int64_t lda, const float* x, float* y, float scale, void* ws,
             size_t ws_bytes, void* stream);
size_t atax_plan_workspace_bytes(int64_t m, int64_t n);

// Bound of the kernels' waits on data (kf_set_wait_limit_ns; 1 s by default).
uint64_t wait_limit_ns();

}  // namespace kf
