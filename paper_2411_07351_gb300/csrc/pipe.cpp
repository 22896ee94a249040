// Host-memory pipeline: forward transforms of images that live in host
// memory, with the copies in and out as part of every call.
//
// Each fht_pipe_submit uses the next of `depth` device buffer sets (input,
// output, workspace) and enqueues, without blocking the host:
//   input stream:  wait until the set's previous output copies are done,
//                  host -> device copy of the image;
//   compute stream: wait for that copy, fht_forward;
//   output streams: wait for the transform, device -> host copy of the output,
//                  split into equal pieces over `copy_streams` streams.
// Consecutive submits therefore overlap: the output copy of image i runs with
// the transform of image i + 1 and the input copy of image i + 2, and the
// throughput is that of the slowest stage rather than of their sum.  All
// streams are created blocking, so work on the legacy default stream orders
// with them (events recorded there bracket a run of submits).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/fht.h"
#include "fht_launch.hpp"
#include "plan.hpp"

fht_status fht_capi_fail(fht_status st, const std::string& msg);
const fht::DevicePlan* fht_capi_device_plan(fht_plan_t plan);

struct fht_pipe_s {
  fht_plan_t plan = nullptr;
  int device = 0;
  int32_t depth = 0, ncopy = 0;
  int32_t h = 0, w = 0;
  size_t in_size = 0, in_bytes = 0, out_bytes = 0, ws_bytes = 0;
  std::vector<void*> d_in, d_out, d_ws;
  cudaStream_t s_in = nullptr, s_comp = nullptr;
  std::vector<cudaStream_t> s_out;
  std::vector<cudaEvent_t> ev_in, ev_comp;  // per set
  std::vector<cudaEvent_t> ev_part;         // per set x output stream
  int64_t next = 0;
};

namespace {

struct PipeDeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit PipeDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~PipeDeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void pipe_free(fht_pipe_s* p) {
  for (void* b : p->d_in) cudaFree(b);
  for (void* b : p->d_out) cudaFree(b);
  for (void* b : p->d_ws) cudaFree(b);
  for (cudaEvent_t e : p->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_comp) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_part) cudaEventDestroy(e);
  for (cudaStream_t s : p->s_out) cudaStreamDestroy(s);
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_comp) cudaStreamDestroy(p->s_comp);
}

fht_status cuda_fail(cudaError_t e, const char* where) {
  return fht_capi_fail(e == cudaErrorMemoryAllocation ? FHT_ERR_NOMEM : FHT_ERR_CUDA,
                       std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

fht_status fht_pipe_create(fht_pipe_t* out, fht_plan_t plan, int32_t depth, int32_t copy_streams) {
  if (!out) return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_create: out is NULL");
  *out = nullptr;
  const fht::DevicePlan* D = fht_capi_device_plan(plan);
  if (!D) return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_create: plan is NULL");
  if (D->device < 0) return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_create: host-only plan (device < 0)");
  if (depth < 1 || depth > 8 || copy_streams < 1 || copy_streams > 8)
    return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_create: depth and copy_streams must be in [1, 8]");
  const fht::HostPlan& P = *D->host;
  fht_pipe_s* p = new (std::nothrow) fht_pipe_s();
  if (!p) return fht_capi_fail(FHT_ERR_NOMEM, "fht_pipe_create: host allocation failed");
  p->plan = plan;
  p->device = D->device;
  p->depth = depth;
  p->ncopy = copy_streams;
  p->h = P.cfg.h;
  p->w = P.cfg.w;
  p->in_size = (size_t)P.in_size;
  p->in_bytes = (size_t)P.cfg.h * P.cfg.w * P.in_size;
  p->out_bytes = (size_t)P.out_elems * P.acc_size;
  p->ws_bytes = P.ws_bytes;
  PipeDeviceGuard g(p->device);
  if (!g.ok) {
    delete p;
    return fht_capi_fail(FHT_ERR_CUDA, "fht_pipe_create: cannot select the plan's device");
  }
  cudaError_t e = cudaSuccess;
  auto add_event = [&](std::vector<cudaEvent_t>& v) {
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) v.push_back(ev);
  };
  auto add_buffer = [&](std::vector<void*>& v, size_t bytes) {
    void* b = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&b, std::max<size_t>(bytes, 256));
    if (e == cudaSuccess) v.push_back(b);
  };
  e = cudaStreamCreate(&p->s_in);
  if (e == cudaSuccess) e = cudaStreamCreate(&p->s_comp);
  for (int32_t c = 0; c < copy_streams && e == cudaSuccess; c++) {
    cudaStream_t s = nullptr;
    e = cudaStreamCreate(&s);
    if (e == cudaSuccess) p->s_out.push_back(s);
  }
  for (int32_t k = 0; k < depth && e == cudaSuccess; k++) {
    add_buffer(p->d_in, p->in_bytes);
    add_buffer(p->d_out, p->out_bytes);
    add_buffer(p->d_ws, p->ws_bytes);
    add_event(p->ev_in);
    add_event(p->ev_comp);
    for (int32_t c = 0; c < copy_streams; c++) add_event(p->ev_part);
  }
  if (e != cudaSuccess) {
    pipe_free(p);
    delete p;
    return cuda_fail(e, "fht_pipe_create");
  }
  *out = p;
  return FHT_OK;
}

fht_status fht_pipe_submit(fht_pipe_t p, const void* h_in, int64_t in_pitch, void* h_out) {
  if (!p) return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_submit: pipe is NULL");
  if (!h_in || !h_out || in_pitch < p->w) return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_submit: bad argument");
  PipeDeviceGuard g(p->device);
  if (!g.ok) return fht_capi_fail(FHT_ERR_CUDA, "fht_pipe_submit: cannot select the pipe's device");
  const int32_t k = (int32_t)(p->next % p->depth);
  cudaError_t e = cudaSuccess;
  // the set is free once its previous output copies have finished (an event
  // never recorded counts as complete)
  for (int32_t c = 0; c < p->ncopy && e == cudaSuccess; c++)
    e = cudaStreamWaitEvent(p->s_in, p->ev_part[(size_t)k * p->ncopy + c], 0);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(p->d_in[k], (size_t)p->w * p->in_size, h_in, (size_t)in_pitch * p->in_size,
                          (size_t)p->w * p->in_size, (size_t)p->h, cudaMemcpyHostToDevice, p->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[k], p->s_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_comp, p->ev_in[k], 0);
  if (e != cudaSuccess) return cuda_fail(e, "fht_pipe_submit");
  const fht_status st = fht_forward(p->plan, p->d_in[k], p->w, p->d_out[k], p->d_ws[k], p->ws_bytes, p->s_comp);
  if (st != FHT_OK) return st;
  e = cudaEventRecord(p->ev_comp[k], p->s_comp);
  // output copy in equal pieces (multiples of 4 KiB) over the output streams
  const size_t piece = ((p->out_bytes + p->ncopy - 1) / p->ncopy + 4095) & ~(size_t)4095;
  for (int32_t c = 0; c < p->ncopy && e == cudaSuccess; c++) {
    const size_t off = (size_t)c * piece;
    const size_t len = off < p->out_bytes ? std::min(piece, p->out_bytes - off) : 0;
    e = cudaStreamWaitEvent(p->s_out[c], p->ev_comp[k], 0);
    if (e == cudaSuccess && len > 0)
      e = cudaMemcpyAsync(static_cast<unsigned char*>(h_out) + off, static_cast<unsigned char*>(p->d_out[k]) + off,
                          len, cudaMemcpyDeviceToHost, p->s_out[c]);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_part[(size_t)k * p->ncopy + c], p->s_out[c]);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fht_pipe_submit");
  p->next++;
  return FHT_OK;
}

fht_status fht_pipe_sync(fht_pipe_t p) {
  if (!p) return fht_capi_fail(FHT_ERR_INVALID, "fht_pipe_sync: pipe is NULL");
  PipeDeviceGuard g(p->device);
  if (!g.ok) return fht_capi_fail(FHT_ERR_CUDA, "fht_pipe_sync: cannot select the pipe's device");
  cudaError_t e = cudaStreamSynchronize(p->s_in);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->s_comp);
  for (size_t c = 0; c < p->s_out.size() && e == cudaSuccess; c++) e = cudaStreamSynchronize(p->s_out[c]);
  if (e != cudaSuccess) return cuda_fail(e, "fht_pipe_sync");
  return FHT_OK;
}

fht_status fht_pipe_destroy(fht_pipe_t p) {
  if (!p) return FHT_OK;
  PipeDeviceGuard g(p->device);
  if (p->s_comp) cudaStreamSynchronize(p->s_comp);
  for (cudaStream_t s : p->s_out) cudaStreamSynchronize(s);
  if (p->s_in) cudaStreamSynchronize(p->s_in);
  pipe_free(p);
  delete p;
  return FHT_OK;
}

}  // extern "C"
