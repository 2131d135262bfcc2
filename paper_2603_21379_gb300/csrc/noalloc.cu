// noalloc.cu - an entry point for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc around this library: code that runs
// while a stream is being captured into a CUDA graph (allocation is not a
// stream operation and is refused in global capture mode), frameworks that
// reserve nearly all device memory up front and hand out memory only from
// their own pools, and latency-critical loops that must not hit the implicit
// device synchronisation a cudaMalloc/cudaFree can cause.  The handle-based
// entry points allocate a workspace on first use, so they are closed to such
// callers.
//
// rhtucker_root_transfer_noalloc computes the root transfer tensor of an
// H-Tucker format, B_R(0, j, k) = sum_{a,b} X[a nr + b] U_l[a][j] U_r[b][k],
// with the tiled root kernel (the one rhtucker_decompose uses for shapes the
// streaming kernel does not take; it has no waits and so needs no status word;
// rhtucker_decompose takes the streaming kernel where it can, and the two agree to
// float32 rounding),
// but its scratch (one partial r_l x r_r block per CTA) lives in the file-scope
// device array below
// instead of a workspace.  The array has a fixed capacity; every GPU that
// loads the library holds it until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/rtucker.h"
#include "rt_common.cuh"
#include "rt_host.h"

namespace {

// Capacity of the static scratch, in floats (4 MiB).
constexpr size_t NOALLOC_ROOT_FLOATS = RT_ROOT_NOALLOC_MAX_PARTIALS;

static __device__ __align__(256) float g_root_scratch[NOALLOC_ROOT_FLOATS];

// Device address of g_root_scratch per device.  In host code the symbol is a
// host-side stand-in, not a device address, so it is resolved once per device
// with cudaGetSymbolAddress while that device is current.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
float* g_addr[MAX_DEVICES] = {nullptr};

rt_status scratch_for_current_device(float** out) {
  int dev = 0;
  // Failures are returned as RT_ECUDA and left in the runtime's error state (no
  // cudaGetLastError here: it would also clear an error the caller had pending).
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return RT_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_root_scratch);
    if (e != cudaSuccess || !p) return RT_ECUDA;
    g_addr[dev] = static_cast<float*>(p);
  }
  *out = g_addr[dev];
  return RT_OK;
}

}  // namespace

extern "C" rt_status rhtucker_root_transfer_noalloc(const void* X, rt_dtype dtype, int64_t nl, int64_t nr,
                                                    const float* Ul, int32_t rl, const float* Ur, int32_t rr,
                                                    float* BR, void* stream) {
  if (!X || !Ul || !Ur || !BR) return RT_EINVAL;
  if (dtype != RT_F32 && dtype != RT_F64 && dtype != RT_BF16) return RT_EINVAL;
  if (nl < 1 || nr < 1 || rl < 1 || rr < 1 || nl > ((int64_t)1 << 31) || nr > ((int64_t)1 << 40)) return RT_EINVAL;
  if (rr > 12) return RT_ENOTSUP;
  if (rt::root_scratch_floats(nl, nr, rl, rr) > NOALLOC_ROOT_FLOATS) return RT_ENOTSUP;
  float* scratch = nullptr;
  const rt_status st = scratch_for_current_device(&scratch);
  if (st != RT_OK) return st;
  // The partial blocks are all overwritten by the first kernel; nothing in the
  // scratch has to start at zero.  The launch errors come back from the launches
  // themselves, so an error the caller left pending in the runtime is neither
  // reported as ours nor cleared.
  cudaError_t e = cudaSuccess;
  rt::launch_root_tiled(X, (int)dtype, nl, nr, Ul, rl, Ur, rr, BR, scratch, static_cast<cudaStream_t>(stream), &e);
  return e == cudaSuccess ? RT_OK : RT_ECUDA;
}
