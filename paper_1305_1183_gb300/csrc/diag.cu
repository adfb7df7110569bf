// Bound of the device waits, and a probe of what happens when one runs out.
//
// Every wait of the library's kernels on data (the bulk-copy rings of the
// staged matrix pass and of ATAX) is bounded: after the limit the block
// records KF_DEVERR_TIMEOUT in the workspace's error word, stops waiting,
// lets the copies already in flight land (bounded) and returns, and the host
// reads the word with kf_workspace_status.  kf_wait_probe exercises that
// failure path on demand, without a fault: one thread waits on an mbarrier
// phase that nothing ever completes (no arrival is made and no copy counts
// bytes on it), so the wait runs out after the given limit.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "../../include/kf.h"
#include "kf_device.cuh"
#include "kf_internal.h"

namespace kf {

const char* set_error_message(const std::string& msg);

namespace {
std::atomic<uint64_t> g_wait_ns{WAIT_LIMIT_NS};

__global__ void wait_probe_kernel(unsigned* err, uint64_t limit_ns, unsigned long long* waited) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const uint64_t t0 = global_ns();
  // phase 0 completes only when one arrival is made: none is
  const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
  const uint64_t t1 = global_ns();
  if (!ok) atomicOr(err, KF_DEVERR_TIMEOUT);
  if (waited != nullptr) *waited = (unsigned long long)(t1 - t0);
}
}  // namespace

uint64_t wait_limit_ns() { return g_wait_ns.load(); }

}  // namespace kf

extern "C" {

kf_status kf_set_wait_limit_ns(uint64_t limit_ns) {
  if (limit_ns < KF_WAIT_LIMIT_MIN_NS || limit_ns > KF_WAIT_LIMIT_MAX_NS) {
    kf::set_error_message("wait limit out of range");
    return KF_ERR_INVALID_ARG;
  }
  kf::g_wait_ns.store(limit_ns);
  return KF_OK;
}

kf_status kf_get_wait_limit_ns(uint64_t* limit_ns) {
  if (limit_ns == nullptr) {
    kf::set_error_message("null output");
    return KF_ERR_INVALID_ARG;
  }
  *limit_ns = kf::g_wait_ns.load();
  return KF_OK;
}

kf_status kf_wait_probe(uint64_t limit_ns, void* ws, size_t ws_bytes, unsigned long long* waited_ns,
                        void* stream) {
  if (ws == nullptr || ws_bytes < 256) {
    kf::set_error_message("workspace of at least 256 bytes required");
    return KF_ERR_WORKSPACE;
  }
  if (limit_ns < KF_WAIT_LIMIT_MIN_NS || limit_ns > KF_WAIT_LIMIT_MAX_NS) {
    kf::set_error_message("wait limit out of range");
    return KF_ERR_INVALID_ARG;
  }
  kf::wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(static_cast<unsigned*>(ws), limit_ns, waited_ns);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    kf::set_error_message(std::string("launch: ") + cudaGetErrorString(e));
    return KF_ERR_CUDA;
  }
  return KF_OK;
}

}  // extern "C"
