// extern "C" entry points of libfht.so (declared in include/fht.h).
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>

#include "../../include/fht.h"
#include "fht_launch.hpp"
#include "plan.hpp"
#include "table_arena.hpp"

struct fht_plan_s {
  fht::HostPlan host;
  fht::DevicePlan dev;
  void* d_tables = nullptr;  // one device range (table arena) holding every table of the plan
  size_t d_tables_bytes = 0;
  std::mutex mu;             // serialises the lazy adjoint build and the host-table restore
  // Once uploaded, a device plan keeps on the host only what launches read
  // there (work lists and pass boundaries): the merge programs, row jobs,
  // spine and adjoint tables live on the device alone, so that a server
  // holding thousands of plans does not hold their tables twice.  Their
  // lengths are kept for fht_plan_table and fht_plan_check, which copy them
  // back on demand.
  bool host_released = false;
  int64_t released[10] = {};
};

namespace {

thread_local std::string g_last_error;

fht_status fail(fht_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

fht_status cuda_fail(cudaError_t e, const char* where) {
  return fail(FHT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Packs every table of the plan into one device allocation (sections aligned
// to 256 bytes) with a single copy.
struct TablePacker {
  std::vector<unsigned char> host;
  std::vector<std::pair<void**, size_t>> fix;  // (device pointer to set, offset)
  template <typename T>
  void add(T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return;
    size_t off = (host.size() + 255) / 256 * 256;
    host.resize(off + sizeof(T) * v.size());
    memcpy(host.data() + off, v.data(), sizeof(T) * v.size());
    fix.emplace_back(reinterpret_cast<void**>(dst), off);
  }
};

cudaError_t upload_tables(fht_plan_s* p) {
  fht::DevicePlan& d = p->dev;
  const fht::HostPlan& h = p->host;
  TablePacker tp;
  tp.add(&d.fused, h.fused);
  tp.add(&d.ops, h.ops);
  tp.add(&d.rows, h.rows);
  tp.add(&d.band_items, h.band_items);
  tp.add(&d.spine_rows, h.spine_rows);
  tp.add(&d.spine_terms, h.spine_terms);
  tp.add(&d.spine_segs, h.spine_segs);
  tp.add(&d.spine_grps, h.spine_grps);
  if (h.has_adjoint) {
    tp.add(&d.arows, h.arows);
    tp.add(&d.aterms, h.aterms);
    tp.add(&d.aptr, h.aptr);
    tp.add(&d.aops, h.aops);
  } else {
    d.arows = nullptr;
    d.aterms = nullptr;
    d.aptr = nullptr;
    d.aops = nullptr;
  }
  const int dev = p->dev.device;
  void* buf = nullptr;
  const size_t bytes = std::max<size_t>(tp.host.size(), 256);
  cudaError_t e = fht::table_arena_alloc(dev, bytes, &buf);
  if (e != cudaSuccess) return e;
  // The copy runs on a non-blocking stream of this thread (one per device),
  // so that it waits for nothing but itself: a plan built while the device
  // is busy (a serving loop's builder threads) does not queue behind the
  // work on the legacy default stream.  It leaves from this thread's pinned
  // staging buffer (grown when a plan needs more, freed at thread exit).
  static thread_local cudaStream_t upload_stream[64] = {};
  struct Staging {
    void* p = nullptr;
    size_t n = 0;
    ~Staging() {
      if (p) cudaFreeHost(p);
    }
  };
  static thread_local Staging staging;
  cudaStream_t us = nullptr;
  if (dev >= 0 && dev < 64) {
    if (!upload_stream[dev] && cudaStreamCreateWithFlags(&upload_stream[dev], cudaStreamNonBlocking) != cudaSuccess)
      upload_stream[dev] = nullptr;
    us = upload_stream[dev];
  }
  if (us && staging.n < tp.host.size()) {
    if (staging.p) cudaFreeHost(staging.p);
    staging.p = nullptr;
    staging.n = 0;
    const size_t want = std::max<size_t>(tp.host.size(), size_t(1) << 20);
    if (cudaMallocHost(&staging.p, want) == cudaSuccess) {
      staging.n = want;
    } else {
      staging.p = nullptr;
      cudaGetLastError();  // clear the failed allocation; the copy below goes from pageable memory
    }
  }
  if (us) {
    const void* src = tp.host.data();
    if (staging.n >= tp.host.size()) {
      memcpy(staging.p, tp.host.data(), tp.host.size());
      src = staging.p;
    }
    e = cudaMemcpyAsync(buf, src, tp.host.size(), cudaMemcpyHostToDevice, us);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
  } else {
    e = cudaMemcpy(buf, tp.host.data(), tp.host.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    fht::table_arena_free(dev, buf, bytes);
    return e;
  }
  for (auto& f : tp.fix) *f.first = static_cast<unsigned char*>(buf) + f.second;
  p->d_tables = buf;
  p->d_tables_bytes = bytes;
  return cudaSuccess;
}

void free_dev(fht_plan_s* p) {
  if (p->d_tables) {
    // launches that may still read the tables end first (as a cudaFree
    // would wait for them): the range can be handed to another plan at once
    cudaDeviceSynchronize();
    fht::table_arena_free(p->dev.device, p->d_tables, p->d_tables_bytes);
  }
  p->d_tables = nullptr;
  p->d_tables_bytes = 0;
  fht::DevicePlan& d = p->dev;
  d.fused = nullptr;
  d.ops = nullptr;
  d.rows = nullptr;
  d.arows = nullptr;
  d.aterms = nullptr;
  d.aptr = nullptr;
  d.aops = nullptr;
  d.band_items = nullptr;
  d.spine_rows = nullptr;
  d.spine_terms = nullptr;
  d.spine_segs = nullptr;
  d.spine_grps = nullptr;
}

// A table is released only where the device holds a copy (n = its length);
// a table that was not uploaded (the adjoint tables of a forward-only plan)
// stays on the host (n = -1).
template <typename T>
void drop_table(std::vector<T>& v, const T* d, int64_t& n) {
  if (!d) {
    n = -1;
    return;
  }
  n = (int64_t)v.size();
  std::vector<T>().swap(v);
}

void release_host_tables(fht_plan_s* p) {
  fht::HostPlan& h = p->host;
  const fht::DevicePlan& d = p->dev;
  int64_t* n = p->released;
  drop_table(h.ops, d.ops, n[0]);
  drop_table(h.rows, d.rows, n[1]);
  drop_table(h.spine_rows, d.spine_rows, n[2]);
  drop_table(h.spine_terms, d.spine_terms, n[3]);
  drop_table(h.spine_segs, d.spine_segs, n[4]);
  drop_table(h.spine_grps, d.spine_grps, n[5]);
  drop_table(h.arows, d.arows, n[6]);
  drop_table(h.aterms, d.aterms, n[7]);
  drop_table(h.aptr, d.aptr, n[8]);
  drop_table(h.aops, d.aops, n[9]);
  p->host_released = true;
}

template <typename T>
cudaError_t fetch_table(std::vector<T>& v, const T* d, int64_t n) {
  if (n < 0) return cudaSuccess;  // kept on the host
  v.resize((size_t)n);
  if (n == 0) return cudaSuccess;
  return cudaMemcpy(v.data(), d, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost);
}

// The released host tables copied back from the device (caller holds p->mu).
cudaError_t restore_host_tables(fht_plan_s* p) {
  if (!p->host_released) return cudaSuccess;
  DeviceGuard g(p->dev.device);
  if (!g.ok) return cudaErrorInvalidDevice;
  fht::HostPlan& h = p->host;
  const fht::DevicePlan& d = p->dev;
  const int64_t* n = p->released;
  cudaError_t e;
  if ((e = fetch_table(h.ops, d.ops, n[0])) != cudaSuccess || (e = fetch_table(h.rows, d.rows, n[1])) != cudaSuccess ||
      (e = fetch_table(h.spine_rows, d.spine_rows, n[2])) != cudaSuccess ||
      (e = fetch_table(h.spine_terms, d.spine_terms, n[3])) != cudaSuccess ||
      (e = fetch_table(h.spine_segs, d.spine_segs, n[4])) != cudaSuccess ||
      (e = fetch_table(h.spine_grps, d.spine_grps, n[5])) != cudaSuccess ||
      (e = fetch_table(h.arows, d.arows, n[6])) != cudaSuccess ||
      (e = fetch_table(h.aterms, d.aterms, n[7])) != cudaSuccess ||
      (e = fetch_table(h.aptr, d.aptr, n[8])) != cudaSuccess || (e = fetch_table(h.aops, d.aops, n[9])) != cudaSuccess)
    return e;
  p->host_released = false;
  return cudaSuccess;
}

}  // namespace

// Shared with noalloc.cu.
fht_status fht_capi_fail(fht_status st, const std::string& msg) { return fail(st, msg); }
const fht::DevicePlan* fht_capi_device_plan(fht_plan_t plan) { return plan ? &plan->dev : nullptr; }

extern "C" {

fht_status fht_plan(fht_plan_t* out, int32_t h, int32_t w, fht_dtype dtype, uint32_t quadrants,
                    fht_boundary boundary, fht_split split, int device, const fht_tuning_t* tuning) {
  if (!out) return fail(FHT_ERR_INVALID, "fht_plan: out is NULL");
  *out = nullptr;
  if ((int)split != 0 && (int)split != 1) return fail(FHT_ERR_INVALID, "fht_plan: unknown split rule");
  fht::PlanConfig cfg;
  cfg.h = h;
  cfg.w = w;
  cfg.dtype = (int32_t)dtype;
  cfg.quads = quadrants;
  cfg.ext = (int32_t)boundary;
  cfg.split = split == FHT_SPLIT_S ? fht::Split::S : fht::Split::T;
  cfg.F = 64;
  cfg.TW = 0;       // the planner's default launch shape
  cfg.threads = 0;
  if (tuning) {
    if (tuning->fused_rows) cfg.F = tuning->fused_rows;
    if (tuning->tile_cols) cfg.TW = tuning->tile_cols;
    if (tuning->threads) cfg.threads = tuning->threads;
    cfg.with_adjoint = tuning->with_adjoint != 0;
    cfg.rounding = tuning->rounding;
    if (tuning->spine_chunk) cfg.spine_chunk = tuning->spine_chunk;
    cfg.generic_cols = tuning->generic_cols;
    if (cfg.spine_chunk < 1) return fail(FHT_ERR_INVALID, "fht_plan: spine_chunk must be >= 1");
    if (cfg.threads > 512) return fail(FHT_ERR_INVALID, "fht_plan: threads must be <= 512");
  }
  fht_plan_s* p = new (std::nothrow) fht_plan_s();
  if (!p) return fail(FHT_ERR_NOMEM, "fht_plan: host allocation failed");
  std::string err;
  try {
    err = fht::build_plan(cfg, p->host);
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(FHT_ERR_NOMEM, "fht_plan: host allocation failed while building tables");
  }
  if (!err.empty()) {
    delete p;
    return fail(FHT_ERR_INVALID, "fht_plan: " + err);
  }
  p->dev.host = &p->host;
  p->dev.device = device;
  fht::fused_geometry(p->host, p->dev.geo);
  if (device < 0) {  // host-only plan: tables and sizes for inspection, no device copy
    *out = p;
    return FHT_OK;
  }
  int max_smem = 0;
  {
    DeviceGuard g(device);
    if (!g.ok) {
      delete p;
      return fail(FHT_ERR_CUDA, "fht_plan: cannot select device " + std::to_string(device));
    }
    cudaError_t e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "fht_plan: cudaDeviceGetAttribute");
    }
    int32_t arp = 0, apad = 0;
    size_t asmem = 0;
    fht::adjoint_geometry(p->host, arp, apad, asmem);
    if ((size_t)max_smem < std::max(p->dev.geo.smem, asmem)) {
      const std::string need = std::to_string(std::max(p->dev.geo.smem, asmem));
      delete p;
      return fail(FHT_ERR_INVALID,
                  "fht_plan: fused tile needs " + need + " bytes of shared memory; lower tile_cols or fused_rows");
    }
    if ((e = upload_tables(p)) != cudaSuccess) {
      free_dev(p);
      delete p;
      if (e == cudaErrorMemoryAllocation) return fail(FHT_ERR_NOMEM, "fht_plan: device allocation failed");
      return cuda_fail(e, "fht_plan: upload");
    }
    release_host_tables(p);
  }
  *out = p;
  return FHT_OK;
}

fht_status fht_plan_info(fht_plan_t plan, fht_plan_info_t* info) {
  if (!plan || !info) return fail(FHT_ERR_INVALID, "fht_plan_info: NULL argument");
  const fht::HostPlan& P = plan->host;
  memset(info, 0, sizeof(*info));
  info->h = P.cfg.h;
  info->w = P.cfg.w;
  for (int q = 0; q < 4; q++) {
    if (P.cfg.quads & (1u << q)) {
      info->rows[q] = P.quad[q].n;
      info->cols[q] = P.quad[q].W;
      info->out_offset[q] = P.quad[q].out_off;
    } else {
      info->out_offset[q] = -1;
    }
  }
  info->out_elems = P.out_elems;
  info->workspace_bytes = P.ws_bytes;
  info->adjoint_workspace_bytes = P.adj_ws_bytes;
  info->adds = P.adds;
  info->model_bytes = P.model_bytes;
  info->ideal_bytes = P.ideal_bytes;
  info->fused_rows = P.cfg.F;
  info->tile_cols = P.cfg.TW;
  info->upper_passes = P.upper_heights;
  return FHT_OK;
}

static fht_status forward_impl(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out, void* d_ws,
                               size_t ws_bytes, void* stream, void** events, int32_t nevents) {
  if (!plan) return fail(FHT_ERR_INVALID, "fht_forward: plan is NULL");
  if (events && nevents < 2 * fht::forward_launches(plan->host))
    return fail(FHT_ERR_INVALID, "fht_forward_timed: need two events per kernel launch");
  const fht::HostPlan& P = plan->host;
  if (!d_in || !d_out || !d_ws) return fail(FHT_ERR_INVALID, "fht_forward: NULL buffer");
  if (in_pitch < P.cfg.w) return fail(FHT_ERR_INVALID, "fht_forward: in_pitch < w");
  if (ws_bytes < P.ws_bytes)
    return fail(FHT_ERR_INVALID, "fht_forward: workspace too small (need " + std::to_string(P.ws_bytes) + " bytes)");
  if (((uintptr_t)d_ws) % 256) return fail(FHT_ERR_INVALID, "fht_forward: workspace must be 256-byte aligned");
  if (((uintptr_t)d_out) % P.acc_size) return fail(FHT_ERR_INVALID, "fht_forward: misaligned output");
  if (((uintptr_t)d_in) % P.in_size) return fail(FHT_ERR_INVALID, "fht_forward: misaligned input");
  if (plan->dev.device < 0) return fail(FHT_ERR_INVALID, "fht_forward: host-only plan (device < 0)");
  DeviceGuard g(plan->dev.device);
  if (!g.ok) return fail(FHT_ERR_CUDA, "fht_forward: cannot select the plan's device");
  cudaError_t e = fht::launch_forward(plan->dev, d_in, in_pitch, d_out, d_ws, (cudaStream_t)stream,
                                      reinterpret_cast<cudaEvent_t*>(events));
  if (e != cudaSuccess) return cuda_fail(e, "fht_forward");
  return FHT_OK;
}

fht_status fht_forward(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out, void* d_ws,
                       size_t ws_bytes, void* stream) {
  return forward_impl(plan, d_in, in_pitch, d_out, d_ws, ws_bytes, stream, nullptr, 0);
}

fht_status fht_forward_timed(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out, void* d_ws,
                             size_t ws_bytes, void* stream, void** events, int32_t nevents) {
  if (!events) return fail(FHT_ERR_INVALID, "fht_forward_timed: events is NULL");
  return forward_impl(plan, d_in, in_pitch, d_out, d_ws, ws_bytes, stream, events, nevents);
}

fht_status fht_plan_launches(fht_plan_t plan, int32_t* count) {
  if (!plan || !count) return fail(FHT_ERR_INVALID, "fht_plan_launches: NULL argument");
  *count = fht::forward_launches(plan->host);
  return FHT_OK;
}

fht_status fht_plan_launch_info(fht_plan_t plan, int32_t k, int32_t* kind, int64_t* model_bytes) {
  if (!plan || !kind || !model_bytes) return fail(FHT_ERR_INVALID, "fht_plan_launch_info: NULL argument");
  if (k < 0 || k >= fht::forward_launches(plan->host)) return fail(FHT_ERR_INVALID, "fht_plan_launch_info: k");
  fht::forward_launch_info(plan->host, k, *kind, *model_bytes);
  return FHT_OK;
}

fht_status fht_adjoint(fht_plan_t plan, const void* d_gout, void* d_gin, int64_t gin_pitch, void* d_ws,
                       size_t ws_bytes, void* stream) {
  if (!plan) return fail(FHT_ERR_INVALID, "fht_adjoint: plan is NULL");
  const fht::HostPlan& P = plan->host;
  if (plan->dev.device < 0) return fail(FHT_ERR_INVALID, "fht_adjoint: host-only plan (device < 0)");
  if (!d_gout || !d_gin || !d_ws) return fail(FHT_ERR_INVALID, "fht_adjoint: NULL buffer");
  if (gin_pitch < P.cfg.w) return fail(FHT_ERR_INVALID, "fht_adjoint: gin_pitch < w");
  if (((uintptr_t)d_ws) % 256) return fail(FHT_ERR_INVALID, "fht_adjoint: workspace must be 256-byte aligned");
  if (((uintptr_t)d_gout) % P.acc_size || ((uintptr_t)d_gin) % P.acc_size)
    return fail(FHT_ERR_INVALID, "fht_adjoint: misaligned buffer");
  DeviceGuard g(plan->dev.device);
  if (!g.ok) return fail(FHT_ERR_CUDA, "fht_adjoint: cannot select the plan's device");
  {
    // the adjoint tables are built on first use (plans made for the forward
    // transform only never pay for them)
    std::lock_guard<std::mutex> lock(plan->mu);
    if (!plan->host.has_adjoint) {
      fht::PlanConfig cfg = plan->host.cfg;
      cfg.with_adjoint = true;
      fht::HostPlan hp;
      std::string err;
      try {
        err = fht::build_plan(cfg, hp);
      } catch (const std::bad_alloc&) {
        return fail(FHT_ERR_NOMEM, "fht_adjoint: host allocation failed while building tables");
      }
      if (!err.empty()) return fail(FHT_ERR_INVALID, "fht_adjoint: " + err);
      free_dev(plan);
      plan->host = std::move(hp);
      plan->host_released = false;
      fht::fused_geometry(plan->host, plan->dev.geo);
      cudaError_t e = upload_tables(plan);
      if (e != cudaSuccess) return cuda_fail(e, "fht_adjoint: table upload");
      release_host_tables(plan);
    }
  }
  if (ws_bytes < P.adj_ws_bytes)
    return fail(FHT_ERR_INVALID,
                "fht_adjoint: workspace too small (need " + std::to_string(P.adj_ws_bytes) + " bytes)");
  cudaError_t e = fht::launch_adjoint(plan->dev, d_gout, d_gin, gin_pitch, d_ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "fht_adjoint");
  return FHT_OK;
}

fht_status fht_plan_check(fht_plan_t plan) {
  if (!plan) return fail(FHT_ERR_INVALID, "fht_plan_check: plan is NULL");
  std::lock_guard<std::mutex> lock(plan->mu);
  if (cudaError_t e = restore_host_tables(plan); e != cudaSuccess) return cuda_fail(e, "fht_plan_check: table copy");
  int32_t arp = 0, apad = 0;
  size_t asmem = 0;
  fht::adjoint_geometry(plan->host, arp, apad, asmem);
  std::string err = fht::check_plan(plan->host, plan->dev.geo, arp, apad);
  if (!err.empty()) return fail(FHT_ERR_INVALID, "fht_plan_check: " + err);
  return FHT_OK;
}

fht_status fht_plan_table(fht_plan_t plan, fht_table table, const void** data, int64_t* count, int32_t* elem_size) {
  if (!plan || !data || !count || !elem_size) return fail(FHT_ERR_INVALID, "fht_plan_table: NULL argument");
  {
    std::lock_guard<std::mutex> lock(plan->mu);
    if (cudaError_t e = restore_host_tables(plan); e != cudaSuccess) return cuda_fail(e, "fht_plan_table: table copy");
  }
  const fht::HostPlan& P = plan->host;
  auto give = [&](const auto& v) {
    *data = v.data();
    *count = (int64_t)v.size();
    *elem_size = (int32_t)sizeof(v[0]);
    return FHT_OK;
  };
  switch (table) {
    case FHT_TABLE_QUADS:
      *data = P.quad;
      *count = 4;
      *elem_size = (int32_t)sizeof(P.quad[0]);
      return FHT_OK;
    case FHT_TABLE_FUSED:
      return give(P.fused);
    case FHT_TABLE_OPS:
      return give(P.ops);
    case FHT_TABLE_ROWS:
      return give(P.rows);
    case FHT_TABLE_PASS_BEGIN:
      return give(P.pass_begin);
    case FHT_TABLE_BAND_ITEMS:
      return give(P.band_items);
    case FHT_TABLE_SPINE_ROWS:
      return give(P.spine_rows);
    case FHT_TABLE_SPINE_TERMS:
      return give(P.spine_terms);
    case FHT_TABLE_SPINE_BEGIN:
      return give(P.spine_pass_begin);
    case FHT_TABLE_ADJ_ROWS:
      return give(P.arows);
    case FHT_TABLE_ADJ_TERMS:
      return give(P.aterms);
    case FHT_TABLE_ADJ_BEGIN:
      return give(P.apass_begin);
    case FHT_TABLE_ADJ_PTR:
      return give(P.aptr);
    case FHT_TABLE_ADJ_OPS:
      return give(P.aops);
  }
  return fail(FHT_ERR_INVALID, "fht_plan_table: unknown table");
}

fht_status fht_plan_destroy(fht_plan_t plan) {
  if (!plan) return FHT_OK;
  if (plan->dev.device < 0) {
    delete plan;
    return FHT_OK;
  }
  {
    DeviceGuard g(plan->dev.device);
    free_dev(plan);
  }
  delete plan;
  return FHT_OK;
}

fht_status fht_ws_status(const void* d_ws, void* stream) {
  if (!d_ws) return fail(FHT_ERR_INVALID, "fht_ws_status: NULL workspace");
  int32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, d_ws, sizeof(word), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "fht_ws_status");
  if (word == 0) return FHT_OK;
  return fail(word > 0 && word <= FHT_ERR_DEVICE ? (fht_status)word : FHT_ERR_DEVICE,
              "fht_ws_status: device-side status " + std::to_string(word));
}

const char* fht_status_string(fht_status s) {
  switch (s) {
    case FHT_OK: return "FHT_OK";
    case FHT_ERR_INVALID: return "FHT_ERR_INVALID";
    case FHT_ERR_NOMEM: return "FHT_ERR_NOMEM";
    case FHT_ERR_CUDA: return "FHT_ERR_CUDA";
    case FHT_ERR_TIMEOUT: return "FHT_ERR_TIMEOUT";
    case FHT_ERR_BUSY: return "FHT_ERR_BUSY";
    case FHT_ERR_UNSUPPORTED: return "FHT_ERR_UNSUPPORTED";
    case FHT_ERR_DEVICE: return "FHT_ERR_DEVICE";
  }
  return "FHT_ERR_UNKNOWN";
}

const char* fht_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
