// Batched transform: many images of uneven sizes in one persistent launch.
//
// The host turns every job (a plan + its buffers) into work units -- fused
// subtree tiles, band tiles, spine row groups, or per-height row groups --
// and lists them phase by phase across all jobs (all fused tiles of all jobs
// first, then all band tiles, ...).  Persistent CTAs take units in list order
// from one device counter.  A unit of a later phase of job j first waits until
// job j's earlier-phase units have all finished (a per-job completion
// counter).  Because units are taken in list order and a unit only waits for
// units listed before it, which are already held by running CTAs, the wait
// always ends; it is still bounded by a %globaltimer deadline, after which the
// kernel records FHT_ERR_TIMEOUT in the queue's status word, skips the unit's
// work and carries on, so a lost dependency can never hang the GPU.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fht.h"
#include "fht_desc.h"
#include "fht_block.cuh"
#include "fht_device.cuh"
#include "fht_launch.hpp"
#include "fht_nvtx.hpp"

namespace fht {

struct BatchJob {
  FusedParams fp;                 // input, output, workspace, items, quadrants, geometry
  const FusedItem* band_items;
  const SpineRow* spine_rows;
  const SpineTerm* spine_terms;
  const RowJob* rows;
  int32_t total_units;            // units of this job in the submit
  uint32_t gen;                   // submit generation written to the job's completion flag
  uint32_t* flag;                 // host-mapped completion flag of the job slot
};

enum : int32_t { UNIT_FUSED = 0, UNIT_BAND = 1, UNIT_SPINE = 2, UNIT_UPPER = 3 };

struct BatchUnit {
  int32_t job;
  int32_t kind;
  int32_t index;  // fused / band item, first spine row, or first row job
  int32_t tile;   // first column tile (fused, band), column tile (spine) or row count (upper)
  int32_t need;   // units of this job that must be finished first
  int32_t ntiles; // fused / band: column tiles handled by this unit; spine: rows
  int32_t aux;    // spine: columns per thread (1, 2 or 4)
};

constexpr int kUpperRowsPerUnit = 8;
constexpr int kTilesPerUnit = 4;
constexpr int kBatchThreads = 256;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One register-tiled block or band tile of a job, out of line: its own
// register allocation instead of one shared with every other unit kind.
template <typename InT, typename AccT>
__device__ __noinline__ void batch_vblock(const FusedParams& fp, const FusedItem& it, int32_t tile, AccT* sm) {
  v_block<true, InT, AccT>(fp, it, fp.quad[it.q], tile, sm);
}

template <typename AccT>
__device__ void batch_upper_rows(const RowJob* __restrict__ rows, int32_t first, int32_t count, AccT* ws,
                                 AccT* out) {
  for (int32_t k = first; k < first + count; k++) {
    const RowJob J = rows[k];
    const AccT* top = ws + J.top;
    const AccT* bot = ws + J.bot;
    const bool fin = J.flags & ROW_FINAL;
    const bool ext = J.flags & ROW_EXT;
    AccT* dst = (fin ? out : ws) + J.dst;
    for (int32_t u = threadIdx.x; u < J.wout; u += blockDim.x) {
      AccT a = AccT(0), b = AccT(0);
      if (ext) {
        const int32_t i = u + J.dtop, i2 = u + J.dbot;
        if (i >= 0 && i < J.wtop) a = __ldcg(top + i);
        if (i2 >= 0 && i2 < J.wbot) b = __ldcg(bot + i2);
      } else {
        int32_t i2 = u + J.dbot;
        if (i2 >= J.W) i2 -= J.W;
        a = __ldcg(top + u);
        b = __ldcg(bot + i2);
      }
      store_row(dst, J, fin, u, a + b);
    }
  }
}

template <typename AccT>
__device__ void batch_spine(const BatchJob& jb, int32_t r0, int32_t nr, int32_t tile, int32_t qpt,
                            SpineTerm (*st)[kMaxSpineTerms], SpineRow* sr) {
  AccT* ws = static_cast<AccT*>(jb.fp.ws);
  AccT* out = static_cast<AccT*>(jb.fp.out);
  const int32_t u0 = tile * kBatchThreads * qpt;
  if ((int32_t)threadIdx.x < nr) sr[threadIdx.x] = jb.spine_rows[r0 + threadIdx.x];
  __syncthreads();
  for (int32_t idx = threadIdx.x; idx < nr * kMaxSpineTerms; idx += blockDim.x) {
    const int32_t r = idx / kMaxSpineTerms, c = idx % kMaxSpineTerms;
    if (c < sr[r].term_count) st[r][c] = jb.spine_terms[sr[r].term_begin + c];
  }
  __syncthreads();
  // 256 threads x qpt columns: tiles of 256, 512 or 1024 columns, the narrowest
  // that covers the job's rows in one tile where it can (small images)
  if (qpt == 1) {
    spine_rows_tile<true, kBatchThreads, 1, AccT, false>(sr, st, nr, jb.fp.quad, ws, out, ws, u0);
  } else if (qpt == 2) {
    spine_rows_tile<true, kBatchThreads, 2, AccT, false>(sr, st, nr, jb.fp.quad, ws, out, ws, u0);
  } else {
    spine_rows_tile<true, kBatchThreads, 4, AccT, false>(sr, st, nr, jb.fp.quad, ws, out, ws, u0);
  }
}

// counters[0]: next unit; counters[1 + j]: finished units of job j.
template <typename InT, typename AccT>
__global__ void __launch_bounds__(kBatchThreads, 3) batch_kernel(const BatchJob* __restrict__ jobs,
                                                      const BatchUnit* __restrict__ units, int32_t nunits,
                                                      int32_t* counters,
                                                      int32_t* status, int64_t wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int32_t s_unit;
  __shared__ int32_t s_ok;
  __shared__ SpineTerm st[kSpineRows][kMaxSpineTerms];
  __shared__ SpineRow sr[kSpineRows];
  __shared__ __align__(16) BatchJob s_job;  // the current unit's job descriptor
  AccT* sm = reinterpret_cast<AccT*>(smem_raw);
  int32_t next = 0;  // thread 0: the unit index taken for the following turn
  if (threadIdx.x == 0) s_unit = atomicAdd(&counters[0], 1);
  for (;;) {
    __syncthreads();
    const int32_t ui = s_unit;
    if (ui >= nunits) break;
    // take the next unit now, so the atomic's latency hides behind this unit's work
    if (threadIdx.x == 0) next = atomicAdd(&counters[0], 1);
    const BatchUnit U = units[ui];
    // the job descriptor into shared memory (every field below is read many times)
    static_assert(sizeof(BatchJob) % 4 == 0, "word copy");
    for (int32_t k = threadIdx.x; k < (int32_t)(sizeof(BatchJob) / 4); k += blockDim.x)
      reinterpret_cast<int32_t*>(&s_job)[k] = reinterpret_cast<const int32_t*>(&jobs[U.job])[k];
    if (threadIdx.x == 0) {
      int32_t ok = 1;
      if (U.need > 0) {
        const int32_t* done = &counters[1 + U.job];
        if (ld_acquire(done) < U.need) {
          const uint64_t t0 = global_ns();
          while (ld_acquire(done) < U.need) {
            if (*(volatile int32_t*)status != 0 || global_ns() - t0 > (uint64_t)wait_ns) {
              atomicCAS(status, 0, (int32_t)FHT_ERR_TIMEOUT);
              ok = 0;
              break;
            }
            __nanosleep(200);
          }
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      const BatchJob& jb = s_job;
      switch (U.kind) {
        case UNIT_FUSED:
        case UNIT_BAND: {
          const FusedItem it = (U.kind == UNIT_FUSED ? jb.fp.items : jb.band_items)[U.index];
          const QuadDesc& Q = jb.fp.quad[it.q];
          for (int32_t tile = U.tile; tile < U.tile + U.ntiles && tile < it.ntiles; tile++) {
            if (tile > U.tile) __syncthreads();  // the previous tile's shared reads are done
            if (it.kind != FUSED_GENERIC && jb.fp.vblock) {
              if constexpr (sizeof(AccT) == 4) batch_vblock<InT, AccT>(jb.fp, it, tile, sm);
            } else if (it.kind != FUSED_GENERIC) {
              fused_block_any<true, InT, AccT>(jb.fp, it, Q, tile, sm, sm + (size_t)64 * jb.fp.RS);
            } else {
              fused_generic<InT, AccT>(jb.fp, it, Q, tile, sm, sm + (size_t)jb.fp.Fm * jb.fp.RP);
            }
          }
          break;
        }
        case UNIT_SPINE:
          batch_spine<AccT>(jb, U.index, U.ntiles, U.tile, U.aux, st, sr);
          break;
        default:
          batch_upper_rows<AccT>(jb.rows, U.index, U.tile, static_cast<AccT*>(jb.fp.ws),
                                 static_cast<AccT*>(jb.fp.out));
          break;
      }
    }
    // publish this unit's writes before counting it done (skipped units are
    // counted too, so that nothing waits on them): the barrier orders every
    // thread's writes before thread 0's gpu-scope fence, which is cumulative,
    // and the fence orders them before the count
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const int32_t finished = atomicAdd(&counters[1 + U.job], 1) + 1;
      const BatchJob& jb = jobs[U.job];
      if (finished == jb.total_units) {
        // the job's last unit: tell the host through its mapped completion flag
        __threadfence_system();
        asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(jb.flag), "r"(jb.gen) : "memory");
      }
      s_unit = next;
    }
  }
}

}  // namespace fht

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
fht_status fht_capi_fail(fht_status st, const std::string& msg);
const fht::DevicePlan* fht_capi_device_plan(fht_plan_t plan);

struct fht_queue_s {
  int device = 0;
  int32_t max_jobs = 0;
  int64_t max_units = 0;
  int64_t wait_ns = 2000000000;  // 2 s
  fht::BatchJob* d_jobs = nullptr;
  fht::BatchUnit* d_units = nullptr;
  int32_t* d_counters = nullptr;  // [1 + max_jobs]
  int32_t* d_status = nullptr;
  fht::BatchJob* h_jobs = nullptr;  // pinned staging
  fht::BatchUnit* h_units = nullptr;
  cudaEvent_t staged = nullptr;     // staging buffers free again after this event
  bool staged_pending = false;
  int32_t last_units = 0;
  uint32_t* h_flags = nullptr;      // host-mapped completion flags, one per job slot
  uint32_t* d_flags = nullptr;      // the same memory as seen by the device
  uint32_t gen = 0;                 // generation of the latest submit
  struct Outstanding {
    uint32_t gen;
    std::vector<uint64_t> tags;
    std::vector<char> reported;
  };
  std::vector<Outstanding> outstanding;
  cudaEvent_t done_evt = nullptr;
};

namespace {

struct QueueDeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit QueueDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~QueueDeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void queue_free(fht_queue_s* q) {
  if (q->d_jobs) cudaFree(q->d_jobs);
  if (q->d_units) cudaFree(q->d_units);
  if (q->d_counters) cudaFree(q->d_counters);
  if (q->d_status) cudaFree(q->d_status);
  if (q->h_jobs) cudaFreeHost(q->h_jobs);
  if (q->h_units) cudaFreeHost(q->h_units);
  if (q->staged) cudaEventDestroy(q->staged);
  if (q->done_evt) cudaEventDestroy(q->done_evt);
  if (q->h_flags) cudaFreeHost(q->h_flags);
}

template <typename InT, typename AccT>
cudaError_t launch_batch(fht_queue_s* q, int32_t nunits, size_t smem, cudaStream_t st) {
  auto kfn = fht::batch_kernel<InT, AccT>;
  cudaError_t e = fht::raise_smem_limit(kfn, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, fht::kBatchThreads, smem)) != cudaSuccess)
    return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, q->device)) != cudaSuccess) return e;
  const int grid = std::max(1, std::min<int>(nunits, std::max(1, per_sm) * sms));
  fht::NvtxRange nv("fht batch kernel");
  kfn<<<grid, fht::kBatchThreads, smem, st>>>(q->d_jobs, q->d_units, nunits, q->d_counters, q->d_status,
                                              q->wait_ns);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

fht_status fht_queue_create(fht_queue_t* out, int device, int32_t max_jobs, int64_t max_units) {
  if (!out) return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_create: out is NULL");
  *out = nullptr;
  if (max_jobs < 1 || max_units < 1 || max_units > INT32_MAX)
    return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_create: bad capacity");
  fht_queue_s* q = new (std::nothrow) fht_queue_s();
  if (!q) return fht_capi_fail(FHT_ERR_NOMEM, "fht_queue_create: host allocation failed");
  q->device = device;
  q->max_jobs = max_jobs;
  q->max_units = max_units;
  QueueDeviceGuard g(device);
  if (!g.ok) {
    delete q;
    return fht_capi_fail(FHT_ERR_CUDA, "fht_queue_create: cannot select device");
  }
  cudaError_t e;
  if ((e = cudaMalloc(&q->d_jobs, sizeof(fht::BatchJob) * max_jobs)) != cudaSuccess ||
      (e = cudaMalloc(&q->d_units, sizeof(fht::BatchUnit) * max_units)) != cudaSuccess ||
      (e = cudaMalloc(&q->d_counters, sizeof(int32_t) * (1 + (size_t)max_jobs))) != cudaSuccess ||
      (e = cudaMalloc(&q->d_status, 256)) != cudaSuccess ||
      (e = cudaMallocHost(&q->h_jobs, sizeof(fht::BatchJob) * max_jobs)) != cudaSuccess ||
      (e = cudaMallocHost(&q->h_units, sizeof(fht::BatchUnit) * max_units)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&q->staged, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&q->done_evt, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMemset(q->d_status, 0, 256)) != cudaSuccess ||
      (e = cudaHostAlloc(&q->h_flags, sizeof(uint32_t) * max_jobs, cudaHostAllocMapped)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&q->d_flags, q->h_flags, 0)) != cudaSuccess) {
    queue_free(q);
    delete q;
    return fht_capi_fail(e == cudaErrorMemoryAllocation ? FHT_ERR_NOMEM : FHT_ERR_CUDA,
                         std::string("fht_queue_create: ") + cudaGetErrorString(e));
  }
  memset(q->h_flags, 0, sizeof(uint32_t) * max_jobs);
  *out = q;
  return FHT_OK;
}

fht_status fht_queue_set_wait_limit(fht_queue_t q, int64_t wait_ns) {
  if (!q || wait_ns < 1) return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_set_wait_limit: bad argument");
  q->wait_ns = wait_ns;
  return FHT_OK;
}

fht_status fht_submit(fht_queue_t q, int32_t njobs, const fht_job* jobs, void* stream) {
  if (!q) return fht_capi_fail(FHT_ERR_INVALID, "fht_submit: queue is NULL");
  if (njobs < 1 || !jobs) return fht_capi_fail(FHT_ERR_INVALID, "fht_submit: no jobs");
  if (njobs > q->max_jobs) return fht_capi_fail(FHT_ERR_BUSY, "fht_submit: more jobs than the queue holds");
  cudaStream_t st = (cudaStream_t)stream;
  QueueDeviceGuard g(q->device);
  if (!g.ok) return fht_capi_fail(FHT_ERR_CUDA, "fht_submit: cannot select the queue's device");
  // Under stream capture the copies below become graph nodes that read the
  // staging buffers at every replay: the graph then owns the staging, and no
  // host synchronisation may happen here.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusNone;
  const bool capturing = cap == cudaStreamCaptureStatusActive;
  // the staging buffers of the previous submit must have been copied out
  if (q->staged_pending && !capturing) {
    cudaError_t e = cudaEventSynchronize(q->staged);
    if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_submit: ") + cudaGetErrorString(e));
    q->staged_pending = false;
  }
  int32_t dtype = -1;
  size_t smem = 0;
  int64_t nunits = 0;
  // pass 1: validate and describe the jobs
  for (int32_t j = 0; j < njobs; j++) {
    const fht_job& J = jobs[j];
    const fht::DevicePlan* D = fht_capi_device_plan(J.plan);
    if (!D) return fht_capi_fail(FHT_ERR_INVALID, "fht_submit: job " + std::to_string(j) + " has no plan");
    const fht::HostPlan& P = *D->host;
    if (D->device != q->device)
      return fht_capi_fail(FHT_ERR_INVALID, "fht_submit: job " + std::to_string(j) + " plan is on another device");
    if (dtype < 0) dtype = P.cfg.dtype;
    if (P.cfg.dtype != dtype) return fht_capi_fail(FHT_ERR_INVALID, "fht_submit: jobs of different dtypes");
    if (!J.d_in || !J.d_out || !J.d_ws || J.in_pitch < P.cfg.w || J.ws_bytes < P.ws_bytes ||
        ((uintptr_t)J.d_ws) % 256)
      return fht_capi_fail(FHT_ERR_INVALID, "fht_submit: job " + std::to_string(j) + " buffers");
    fht::BatchJob& B = q->h_jobs[j];
    memset(&B, 0, sizeof(B));
    B.fp.in = J.d_in;
    B.fp.in_pitch = J.in_pitch;
    B.fp.ws = static_cast<unsigned char*>(J.d_ws) + fht::kWsHeader;
    B.fp.out = J.d_out;
    B.fp.items = D->fused;
    B.fp.ops = D->ops;
    for (int k = 0; k < 4; k++) B.fp.quad[k] = P.quad[k];
    B.fp.RP = D->geo.RP;
    B.fp.Fm = D->geo.Fm;
    B.fp.RS = D->geo.RS;
    B.fp.RA = D->geo.RA;
    B.fp.vblock = P.vblock ? 1 : 0;
    B.band_items = D->band_items;
    B.spine_rows = D->spine_rows;
    B.spine_terms = D->spine_terms;
    B.rows = D->rows;
    // the register-tiled path stages into one 64 x kVPitch buffer; the generic
    // subtrees of such a plan use their own (smaller) layout
    smem = std::max(smem, P.vblock ? std::max(D->geo.vsmem, D->geo.gsmem) : D->geo.smem);
  }
  // pass 2: units, phase by phase across all jobs
  std::vector<int32_t> done_before(njobs, 0);
  auto push = [&](int32_t job, int32_t kind, int32_t index, int32_t tile, int32_t need, int32_t ntiles = 1,
                  int32_t aux = 0) -> bool {
    if (nunits >= q->max_units) return false;
    q->h_units[nunits++] = fht::BatchUnit{job, kind, index, tile, need, ntiles, aux};
    return true;
  };
  int32_t max_phase = 0;
  for (int32_t j = 0; j < njobs; j++) {
    const fht::HostPlan& P = *fht_capi_device_plan(jobs[j].plan)->host;
    // bands: fused, band, then one phase per spine chunk (bottom-up)
    max_phase = std::max<int32_t>(max_phase, P.bands ? 1 + (int32_t)P.spine_pass_bytes.size()
                                                     : (int32_t)P.pass_begin.size() - 1);
  }
  std::vector<int32_t> phase_units(njobs, 0);
  for (int32_t phase = 0; phase <= max_phase; phase++) {
    for (int32_t j = 0; j < njobs; j++) {
      const fht::HostPlan& P = *fht_capi_device_plan(jobs[j].plan)->host;
      const int32_t need = done_before[j];
      const bool skip_dep = (jobs[j].flags & FHT_JOB_WITHHOLD_DEPENDENCY) != 0 && phase > 0;
      const int32_t n = need + (skip_dep ? 1 : 0);  // a dependency nothing satisfies
      int32_t count = 0;
      bool ok = true;
      const int32_t tpu = fht::kTilesPerUnit;
      if (phase == 0) {
        for (size_t i = 0; i < P.fused.size() && ok; i++)
          for (int32_t t = 0; t < P.fused[i].ntiles && ok; t += tpu, count++)
            ok = push(j, fht::UNIT_FUSED, (int32_t)i, t, 0, tpu);
      } else if (P.bands) {
        if (phase == 1) {
          for (size_t i = 0; i < P.band_items.size() && ok; i++)
            for (int32_t t = 0; t < P.band_items[i].ntiles && ok; t += tpu, count++)
              ok = push(j, fht::UNIT_BAND, (int32_t)i, t, n, tpu);
        } else if (phase >= 2 && phase - 2 < (int32_t)P.spine_pass_bytes.size()) {
          int32_t maxW = 1;
          for (int k = 0; k < 4; k++)
            if (P.cfg.quads & (1u << k)) maxW = std::max(maxW, P.quad[k].W);
          const int32_t qpt = maxW <= fht::kBatchThreads ? 1 : maxW <= 2 * fht::kBatchThreads ? 2 : 4;
          const int32_t width = fht::kBatchThreads * qpt;
          const int32_t tiles = (maxW + width - 1) / width;
          const int64_t b = P.spine_pass_begin[phase - 2], e = P.spine_pass_begin[phase - 1];
          for (int32_t t = 0; t < tiles && ok; t++)
            for (int64_t r = b; r < e && ok; r += fht::kSpineRows, count++)
              ok = push(j, fht::UNIT_SPINE, (int32_t)r, t, n, (int32_t)std::min<int64_t>(fht::kSpineRows, e - r),
                        qpt);
        }
      } else if (phase < (int32_t)P.pass_begin.size()) {
        const int64_t b = P.pass_begin[phase - 1], e = P.pass_begin[phase];
        for (int64_t r = b; r < e && ok; r += fht::kUpperRowsPerUnit, count++)
          ok = push(j, fht::UNIT_UPPER, (int32_t)r, (int32_t)std::min<int64_t>(fht::kUpperRowsPerUnit, e - r), n);
      }
      if (!ok) return fht_capi_fail(FHT_ERR_BUSY, "fht_submit: more work units than the queue holds");
      done_before[j] += count;
    }
  }
  if (nunits == 0) return FHT_OK;
  q->gen++;
  for (int32_t j = 0; j < njobs; j++) {
    q->h_jobs[j].total_units = done_before[j];
    q->h_jobs[j].gen = q->gen;
    q->h_jobs[j].flag = q->d_flags + j;
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(q->d_jobs, q->h_jobs, sizeof(fht::BatchJob) * njobs, cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(q->d_units, q->h_units, sizeof(fht::BatchUnit) * nunits, cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(q->d_counters, 0, sizeof(int32_t) * (1 + (size_t)njobs), st)) != cudaSuccess ||
      (!capturing && (e = cudaEventRecord(q->staged, st)) != cudaSuccess))
    return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_submit: ") + cudaGetErrorString(e));
  q->staged_pending = !capturing;
  switch (dtype) {
    case 0:
      e = launch_batch<uint8_t, int32_t>(q, (int32_t)nunits, smem, st);
      break;
    case 1:
      e = launch_batch<int32_t, int32_t>(q, (int32_t)nunits, smem, st);
      break;
    case 2:
      e = launch_batch<float, float>(q, (int32_t)nunits, smem, st);
      break;
    default:
      e = launch_batch<double, double>(q, (int32_t)nunits, smem, st);
      break;
  }
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_submit: ") + cudaGetErrorString(e));
  q->last_units = (int32_t)nunits;
  if (capturing) return FHT_OK;
  {
    fht_queue_s::Outstanding o;
    o.gen = q->gen;
    o.tags.reserve(njobs);
    for (int32_t j = 0; j < njobs; j++) o.tags.push_back(jobs[j].tag);
    o.reported.assign(njobs, 0);
    q->outstanding.push_back(std::move(o));
  }
  if ((e = cudaEventRecord(q->done_evt, st)) != cudaSuccess)
    return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_submit: ") + cudaGetErrorString(e));
  return FHT_OK;
}

fht_status fht_queue_ready(fht_queue_t q, int32_t* ready) {
  if (!q || !ready) return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_ready: NULL argument");
  *ready = 1;
  if (!q->staged_pending) return FHT_OK;
  QueueDeviceGuard g(q->device);
  if (!g.ok) return fht_capi_fail(FHT_ERR_CUDA, "fht_queue_ready: cannot select the queue's device");
  const cudaError_t e = cudaEventQuery(q->staged);
  if (e == cudaErrorNotReady) {
    *ready = 0;
    return FHT_OK;
  }
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_queue_ready: ") + cudaGetErrorString(e));
  q->staged_pending = false;
  return FHT_OK;
}

fht_status fht_queue_poll(fht_queue_t q, uint64_t* done_tags, int32_t cap, int32_t* ndone) {
  if (!q || !ndone || (cap > 0 && !done_tags)) return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_poll: bad argument");
  *ndone = 0;
  // per-job completion flags: a job is reported as soon as its last unit has
  // finished, before the rest of its batch
  int32_t n = 0;
  for (size_t k = 0; k < q->outstanding.size() && n < cap; k++) {
    fht_queue_s::Outstanding& o = q->outstanding[k];
    for (size_t j = 0; j < o.tags.size() && n < cap; j++) {
      if (o.reported[j]) continue;
      const uint32_t f = __atomic_load_n(&q->h_flags[j], __ATOMIC_ACQUIRE);
      if ((int32_t)(f - o.gen) >= 0) {
        o.reported[j] = 1;
        done_tags[n++] = o.tags[j];
      }
    }
  }
  // drop submits whose jobs have all been reported
  while (!q->outstanding.empty()) {
    const fht_queue_s::Outstanding& o = q->outstanding.front();
    bool all = true;
    for (char r : o.reported) all = all && r;
    if (!all) break;
    q->outstanding.erase(q->outstanding.begin());
  }
  *ndone = n;
  return FHT_OK;
}

fht_status fht_queue_status(fht_queue_t q, void* stream) {
  if (!q) return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_status: queue is NULL");
  QueueDeviceGuard g(q->device);
  int32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, q->d_status, sizeof(word), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_queue_status: ") + cudaGetErrorString(e));
  if (word == 0) return FHT_OK;
  return fht_capi_fail((fht_status)word, "fht_queue_status: a batch wait gave up (dependency never finished)");
}

fht_status fht_queue_reset_status(fht_queue_t q, void* stream) {
  if (!q) return fht_capi_fail(FHT_ERR_INVALID, "fht_queue_reset_status: queue is NULL");
  QueueDeviceGuard g(q->device);
  cudaError_t e = cudaMemsetAsync(q->d_status, 0, 256, (cudaStream_t)stream);
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_queue_reset_status: ") + cudaGetErrorString(e));
  return FHT_OK;
}

fht_status fht_queue_destroy(fht_queue_t q) {
  if (!q) return FHT_OK;
  {
    QueueDeviceGuard g(q->device);
    cudaDeviceSynchronize();
    queue_free(q);
  }
  delete q;
  return FHT_OK;
}

}  // extern "C"
