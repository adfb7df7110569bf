// BiCGK without caller-provided workspace, for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they need BiCGK: code running inside a CUDA-graph-building
// framework that forbids allocation, a host that has handed its memory
// budget to another allocator, or a plain C program that has no device
// allocator of its own.  This variant takes only the inputs and outputs.
// Its scratch (completion counters and cross-block partial sums of the
// matrix pass) lives in a fixed array in the library's device image instead
// of in a workspace.
//
// Properties:
//   * the array is KF_BICGK_NOALLOC_SCRATCH_BYTES (8 MiB) on every GPU that
//     loads the library, held until the process exits;
//   * a shape whose matrix-pass scratch would not fit is rejected with
//     KF_ERR_SHAPE before anything is enqueued;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it; make
//     that first call before any stream capture;
//   * every call clears the array's completion counters on `stream` before
//     the launch (cudaMemsetAsync), since the array keeps the last call's
//     contents;
//   * the matrix pass always takes its direct-load form here (16-byte loads
//     into registers, no bulk-copy ring), which waits on nothing, so no
//     bounded wait can run out and there is no device error word to report;
//   * the kernel shape is the one kf_bicgk would take without a search: a
//     tuning fixed by kf_set_matrix_tuning (its ring depth ignored), else the
//     tuning cache's entry, else the built-in shape; this call never runs
//     the first-use tuning search;
//   * every call on a device shares the one array, so calls whose execution
//     overlaps on the GPU (different streams without ordering, concurrent
//     host threads) race and give wrong results; order them on one stream.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/kf.h"
#include "kf_internal.h"

namespace kf {
const char* set_error_message(const std::string& msg);
}

namespace {

constexpr size_t SCRATCH_BYTES = KF_BICGK_NOALLOC_SCRATCH_BYTES;

// The scratch array.  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char kf_bicgk_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch[MAX_DEVICES] = {nullptr};

// Per-device set-up: the device address of the scratch array (current device).
kf_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    kf::set_error_message(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return KF_ERR_CUDA;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    kf::set_error_message("device index out of range");
    return KF_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> g(g_mu);
  if (g_scratch[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, kf_bicgk_scratch);
    if (e != cudaSuccess || p == nullptr) {
      kf::set_error_message(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return KF_ERR_CUDA;
    }
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return KF_OK;
}

}  // namespace

extern "C" kf_status kf_bicgk_noalloc(int64_t m, int64_t n, const float* A, int64_t lda,
                                      const float* p, const float* r, float* q, float* s,
                                      void* stream) {
  using namespace kf;
  if (m < 0 || n < 0) { set_error_message("negative size"); return KF_ERR_INVALID_ARG; }
  if ((m > 0 && n > 0 && A == nullptr) || (n > 0 && (p == nullptr || s == nullptr)) ||
      (m > 0 && (r == nullptr || q == nullptr))) {
    set_error_message("null pointer");
    return KF_ERR_INVALID_ARG;
  }
  if (m > 0 && lda < n) { set_error_message("leading dimension smaller than the row length"); return KF_ERR_SHAPE; }
  if (m == 0 && n == 0) return KF_OK;
  const size_t need = matprog_workspace_bytes(m, n, 1, 1, FMT_F32);
  if (need > SCRATCH_BYTES) {
    set_error_message("shape needs " + std::to_string(need) + " bytes of scratch; the fixed array holds " +
                      std::to_string(SCRATCH_BYTES) + " (use kf_bicgk with a workspace)");
    return KF_ERR_SHAPE;
  }
  void* ws = nullptr;
  kf_status st = scratch_address(&ws);
  if (st != KF_OK) return st;

  MatProg P;
  std::memset(&P, 0, sizeof(P));
  P.m = m; P.n = n;
  P.nmat = 1; P.fmt = FMT_F32; P.A[0] = A; P.lda[0] = lda;
  P.nops = 2;
  P.ops[0].kind = MOP_GEMV; P.ops[0].mat = 0; P.ops[0].res = 0; P.ops[0].colvec = p;
  P.ops[1].kind = MOP_GEMVT; P.ops[1].mat = 0; P.ops[1].res = 0; P.ops[1].rowvec = r;
  P.nrow_res = 1; P.ncol_res = 1;
  P.nrow_out = m > 0 ? 1 : 0;
  P.row_out[0].dst = q; P.row_out[0].nterm = 1; P.row_out[0].src[0] = 0; P.row_out[0].coef[0] = 1.f;
  P.ncol_out = n > 0 ? 1 : 0;
  P.col_out[0].dst = s; P.col_out[0].nterm = 1; P.col_out[0].src[0] = 0; P.col_out[0].coef[0] = 1.f;
  if (matprog_bind_workspace(P, ws, SCRATCH_BYTES) != 0) {
    set_error_message("scratch binding failed");
    return KF_ERR_WORKSPACE;
  }
  // The array keeps the previous call's contents: clear the completion
  // counters (they sit between the header and the partial sums, which every
  // launch overwrites before reading).
  const size_t clear = static_cast<size_t>(reinterpret_cast<char*>(P.rowpart) - reinterpret_cast<char*>(P.counters));
  cudaError_t e = cudaMemsetAsync(P.counters, 0, clear, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_error_message(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    return KF_ERR_CUDA;
  }
  // kf_bicgk's kernel shape without a search, in its direct-load form
  MatTune t = matprog_tuning_nosearch(P, current_matrix_tuning());
  t.stages = 0;
  const char* why = nullptr;
  const int rc = launch_matprog(P, t, stream, &why);
  if (rc != 0) {
    set_error_message(why ? why : "launch failed");
    return rc;
  }
  return KF_OK;
}
