// pat_forward_noalloc: the forward map without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// forward map: plug-ins whose host framework owns every device buffer and
// hands the plug-in only its inputs and outputs, or hard-real-time loops that
// must not call into the allocator.  pat_forward needs a caller-supplied
// workspace for the time-stepping state; this variant keeps that state in a
// fixed array that lives in this library's device image instead.
#include <cuda_runtime.h>

#include <mutex>

#include "pat_internal.h"
#include "pat_solver.cuh"

namespace {

// 8 MiB of time-stepping state per device that loads the library, held until
// the process exits.  Sized for pat_workspace_bytes(mesh, 0, K) of small and
// mid-size problems (N*K <= 524,288 for FP32 meshes, 262,144 for FP64 meshes).
constexpr size_t kScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_forward_scratch[kScratchBytes];

// Host code must not use g_forward_scratch directly: on the host that name is a
// stand-in object, not a device address.  The device address is looked up once
// per device, with that device current, and cached here for the life of the
// process (a cudaDeviceReset, which reloads the module, is not supported).
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

pat_status scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pat::cuda_check(e, "pat_forward_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    pat::set_error("pat_forward_noalloc: device index %d is beyond the %d supported", dev, kMaxDevices);
    return PAT_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_forward_scratch);
    if (e != cudaSuccess || p == nullptr)
      return pat::cuda_check(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "pat_forward_noalloc: cudaGetSymbolAddress of the scratch array");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PAT_OK;
}

}  // namespace

extern "C" pat_status pat_forward_noalloc(const pat_mesh* mesh, const void* p0, int32_t K, void* Y, double scale,
                                          void* stream) {
  using namespace pat;
  clear_error();
  if (!mesh || !p0 || !Y) {
    set_error("pat_forward_noalloc: NULL argument");
    return PAT_EINVAL;
  }
  // the same argument rules as pat_forward
  if (bad_K(K, "pat_forward_noalloc") || !check_device(mesh, "pat_forward_noalloc")) return PAT_EINVAL;
  const size_t need = state_bytes(mesh->d, K);
  if (need > kScratchBytes) {
    set_error("pat_forward_noalloc: N*K = %lld needs %zu bytes of time-stepping state, more than the fixed "
              "%zu-byte scratch array; use pat_forward with a workspace",
              (long long)(mesh->d.N * (int64_t)K), need, kScratchBytes);
    return PAT_EINVAL;
  }
  void* scratch = nullptr;
  pat_status s = scratch_for_current_device(&scratch);
  if (s) return s;
  // Every state the time loop reads is written earlier in the same call, so the
  // previous call's leftovers in the shared array need no clearing.
  return forward(mesh->d, p0, K, Y, scale, scratch, (cudaStream_t)stream);
}
