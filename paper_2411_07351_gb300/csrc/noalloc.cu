// fht_forward_noalloc: the forward transform with its workspace taken from a
// fixed array inside this library instead of a caller-provided buffer.
//
// Some callers cannot allocate device memory when they run the transform:
// a real-time loop that must never block (cudaMalloc can synchronise the
// whole device), a plugin whose host framework owns every allocation and
// hands it only input and output buffers, or a process that has already
// given all free device memory to its own pool.  Such a caller creates the
// plan once at start-up and then calls fht_forward_noalloc, which allocates
// nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/fht.h"
#include "fht_launch.hpp"

namespace {

// Scratch for fht_forward_noalloc.  Every GPU that loads this library holds
// these bytes until the process exits.
constexpr size_t kScratchBytes = FHT_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

}  // namespace

// Defined in capi.cpp; fills the thread's last-error message.
fht_status fht_capi_fail(fht_status st, const std::string& msg);

struct fht_plan_s;
const fht::DevicePlan* fht_capi_device_plan(fht_plan_t plan);

// The array's device address on `device` (looked up once, with that device
// current; the caller has made it current).
static cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = cudaSuccess;
  if (!g_scratch_ptr[device]) {
    e = cudaGetSymbolAddress(&g_scratch_ptr[device], g_noalloc_scratch);
    if (e != cudaSuccess) g_scratch_ptr[device] = nullptr;
  }
  *out = g_scratch_ptr[device];
  return e;
}

extern "C" fht_status fht_forward_noalloc(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out,
                                          void* stream) {
  const fht::DevicePlan* D = fht_capi_device_plan(plan);
  if (!D) return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: plan is NULL");
  const fht::HostPlan& P = *D->host;
  if (D->device < 0) return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: host-only plan (device < 0)");
  if (D->device >= kMaxDevices) return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: device index too large");
  if (!d_in || !d_out) return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: NULL buffer");
  if (in_pitch < P.cfg.w) return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: in_pitch < w");
  if (((uintptr_t)d_out) % P.acc_size || ((uintptr_t)d_in) % P.in_size)
    return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: misaligned input or output");
  if (P.ws_bytes > kScratchBytes)
    return fht_capi_fail(FHT_ERR_INVALID, "fht_forward_noalloc: the plan needs " + std::to_string(P.ws_bytes) +
                                              " bytes of workspace; the built-in scratch holds " +
                                              std::to_string(kScratchBytes) + " (use fht_forward)");
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_forward_noalloc: ") + cudaGetErrorString(e));
  if (prev != D->device && (e = cudaSetDevice(D->device)) != cudaSuccess)
    return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_forward_noalloc: ") + cudaGetErrorString(e));
  // one-time set-up per device, with that device current: the array's
  // device address (its name in host code is only a host-side stand-in)
  void* scratch = nullptr;
  e = scratch_address(D->device, &scratch);
  // Nothing in the scratch needs clearing here: the first launch of every
  // forward resets the status word at its start, and every other byte is
  // written before it is read within the same forward.
  if (e == cudaSuccess && scratch)
    e = fht::launch_forward(*D, d_in, in_pitch, d_out, scratch, (cudaStream_t)stream);
  if (prev >= 0 && prev != D->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_forward_noalloc: ") + cudaGetErrorString(e));
  if (!scratch) return fht_capi_fail(FHT_ERR_CUDA, "fht_forward_noalloc: scratch address unavailable");
  return FHT_OK;
}

// The device-side status word of the last fht_forward_noalloc on `device`
// (the same word fht_ws_status reads from a caller's workspace).
extern "C" fht_status fht_noalloc_status(int device, void* stream) {
  if (device < 0 || device >= kMaxDevices) return fht_capi_fail(FHT_ERR_INVALID, "fht_noalloc_status: bad device");
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_noalloc_status: ") + cudaGetErrorString(e));
  if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess)
    return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_noalloc_status: ") + cudaGetErrorString(e));
  void* scratch = nullptr;
  e = scratch_address(device, &scratch);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess || !scratch)
    return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_noalloc_status: ") + cudaGetErrorString(e));
  return fht_ws_status(scratch, stream);
}
