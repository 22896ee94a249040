// Device-side copy of a plan and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "plan.hpp"

namespace fht {

// Shared-memory geometry of the fused forward kernel.
struct FusedGeometry {
  int32_t RP = 0, Fm = 1;  // generic path: row pitch and rows per buffer
  int32_t RS = 0, RA = 0;  // 64-row fast path: pitches of the two buffers
  size_t smem = 0;         // dynamic shared memory (bytes)
  size_t gsmem = 0;        // generic subtrees alone (their own launch on the register-tiled path)
  size_t vsmem = 0;        // register-tiled 64-row block launch
};

struct DevicePlan {
  const HostPlan* host = nullptr;
  int device = 0;
  FusedItem* fused = nullptr;
  MergeOp* ops = nullptr;
  RowJob* rows = nullptr;
  FusedItem* band_items = nullptr;
  SpineRow* spine_rows = nullptr;
  SpineTerm* spine_terms = nullptr;
  SpineSeg* spine_segs = nullptr;
  SpineGrp* spine_grps = nullptr;
  AdjRow* arows = nullptr;
  AdjTerm* aterms = nullptr;
  int32_t* aptr = nullptr;
  MergeOp* aops = nullptr;
  FusedGeometry geo;
};

void fused_geometry(const HostPlan& P, FusedGeometry& g);

// Raises the dynamic shared-memory limit of `kernel` on the current device to
// at least `bytes`, calling the runtime only when the limit must grow (it is
// never lowered; occupancy follows the shared memory a launch requests, not
// the limit).  Setting the attribute on every launch would take the driver's
// lock on every call, which threads building plans at the same time wait on.
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);
template <typename K>
cudaError_t raise_smem_limit(K* kernel, size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(kernel), bytes);
}

// Enqueues the forward transform.  When `events` is non-null, events[2k] and
// events[2k + 1] are recorded just before and after the k-th kernel launch.
cudaError_t launch_forward(const DevicePlan& D, const void* in, int64_t in_pitch, void* out, void* ws,
                           cudaStream_t st, cudaEvent_t* events = nullptr);

// Shared-memory geometry of the fused adjoint kernel.
void adjoint_geometry(const HostPlan& P, int32_t& rp, int32_t& padl, size_t& smem);

// Enqueues the adjoint: gin (h x w, pitch gin_pitch) = transpose of the forward applied to gout.
cudaError_t launch_adjoint(const DevicePlan& D, const void* gout, void* gin, int64_t gin_pitch, void* ws,
                           cudaStream_t st);

// Kernel launches of one forward transform, and the kind of launch k
// (LAUNCH_FUSED, LAUNCH_UPPER, LAUNCH_BAND, LAUNCH_SPINE, LAUNCH_BLOCK) with
// its model bytes.
int32_t forward_launches(const HostPlan& P);
void forward_launch_info(const HostPlan& P, int32_t k, int32_t& kind, int64_t& bytes);

}  // namespace fht
