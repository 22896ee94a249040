/*
 * fht.h -- C ABI of libfht.so, a GB300 (sm_103a) implementation of the
 * generalised Brady-Yong fast Hough transform FHT2DT (and the FHT2DS variant)
 * of "Generalization of Brady-Yong Algorithm for Fast Hough Transform to
 * Arbitrary Image Size" (arXiv 2411.07351).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Images are row-major I[y][x]: h rows, w columns, a row pitch given in
 *    elements.  The transform splits the ROW range (Algorithm 1 of Section 3
 *    applied to the transposed image), so each Hough row is contiguous.
 *  - Quadrant Q0 sums the patterns pat(h, t) of Algorithm 2 running to the
 *    right:  H0[t][x] = sum_y I[y][(x + pat(h,t)[y]) mod W], t in [0, h).
 *    Q1 runs to the left (x - pat), Q2 / Q3 are Q0 / Q1 of the transposed
 *    image (t in [0, w)).  Quadrants are not in the paper; the paper's
 *    transform is one quadrant.
 *  - Boundary: FHT_CYCLIC is the paper's Rotate (Algorithm 1, W = row length).
 *    FHT_EXTENDED is the cyclic transform of the image zero-padded on the right
 *    to W = length + n - 1, so that every line meeting the image is counted
 *    exactly once; lines entering from the left land in columns [length, W).
 *  - The output holds the requested quadrants packed in the order Q0..Q3,
 *    each a dense row-major block of rows[q] x cols[q] elements starting at
 *    element out_offset[q] (see fht_plan_info).
 *  - Rounding of the child slopes [t (n_P - 1)/(n - 1)] is half to even, in
 *    exact integer arithmetic.
 *  - Device pointers are plain CUDA device addresses; `stream` is a
 *    cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Every call returns an fht_status and never aborts.  On failure a
 *    message is available from fht_last_error() (per thread).
 *  - Calls that take a stream only enqueue work: they never synchronise and
 *    never allocate device memory.  The caller owns every buffer it passes.
 *    One exception: the first fht_adjoint on a plan built without the
 *    adjoint tables (fht_tuning_t.with_adjoint = 0) builds them, frees the
 *    plan's old device tables and uploads new ones, synchronously.  Build
 *    the plan with with_adjoint = 1, or make one adjoint call first, before
 *    capturing adjoint calls into a CUDA graph.
 *  - Threads: a plan may be used by several host threads at once for
 *    fht_forward, fht_forward_timed, fht_plan_info and fht_submit jobs, and
 *    its first fht_adjoint builds the adjoint tables under the plan's lock;
 *    but no other call on the same plan may run while that first adjoint
 *    call does.  A queue (fht_queue_t) or a pipe (fht_pipe_t) belongs to one
 *    thread at a time.  fht_forward_noalloc calls share one scratch array
 *    (see there).
 */
#ifndef FHT_H
#define FHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fht_plan_s* fht_plan_t;
typedef struct fht_queue_s* fht_queue_t;
typedef struct fht_builder_s* fht_builder_t;  /* plan builder pool (fht_builder_create) */

typedef enum {
  FHT_OK = 0,
  FHT_ERR_INVALID = 1,     /* bad argument, shape, dtype or size */
  FHT_ERR_NOMEM = 2,       /* host or device allocation failed (plan creation) */
  FHT_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  FHT_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  FHT_ERR_BUSY = 5,        /* queue full; retry after polling */
  FHT_ERR_UNSUPPORTED = 6, /* valid request this build does not implement */
  FHT_ERR_DEVICE = 7       /* a device-side check failed (status word) */
} fht_status;

/* Input type -> accumulation / output type. */
typedef enum {
  FHT_U8_I32 = 0,  /* uint8 in, int32 out: exact (255 * 65535 < 2^31) */
  FHT_I32_I32 = 1, /* int32 in, int32 out: exact while sums fit in int32 */
  FHT_F32_F32 = 2, /* float in, float out, FP32 accumulation */
  FHT_F64_F64 = 3  /* double in, double out */
} fht_dtype;

enum { FHT_Q0 = 1, FHT_Q1 = 2, FHT_Q2 = 4, FHT_Q3 = 8, FHT_QALL = 15 };

typedef enum { FHT_CYCLIC = 0, FHT_EXTENDED = 1 } fht_boundary;

/* Section 3: Split_T cuts off the largest power of two (FHT2DT, the paper's
 * method); Split_S bisects (FHT2DS, Anikeev et al.). */
typedef enum { FHT_SPLIT_T = 0, FHT_SPLIT_S = 1 } fht_split;

/* Tuning knobs; zero fields take the built-in defaults. */
typedef struct {
  int32_t fused_rows;  /* F: largest subtree merged in shared memory (2..64, power of two) */
  int32_t tile_cols;   /* column tile of the fused pass (multiple of 32) */
  int32_t threads;     /* threads per CTA of the fused pass (multiple of 32, <= 512) */
  int32_t with_adjoint;/* 1: build the adjoint tables now (otherwise on the first fht_adjoint) */
  int32_t rounding;    /* child slopes [t k_P]: 0 = exact, ties to even (default);
                          1 = k_P = (m_P - 1)/(m - 1) in double, then rint(t k_P) (Algorithm 1 read literally) */
  int32_t spine_chunk; /* Split_T roots taller than 64 rows: spine nodes summed per spine launch (default 3);
                          the lower chunks' top nodes are summed first and become single parts of the
                          chunk above.  A value >= the spine length gives one spine launch. */
  int32_t generic_cols;/* column tile of the subtrees under 64 rows that take the generic shared-memory
                          path (multiple of 32; default: 128 with tile_cols 192 and 256 threads, else half
                          of tile_cols rounded down to 32, at least 32) */
  int32_t reserved;
} fht_tuning_t;

typedef struct {
  int32_t h, w;
  int32_t rows[4];       /* per quadrant: number of slopes (h for Q0/Q1, w for Q2/Q3); 0 if absent */
  int32_t cols[4];       /* per quadrant: output row length W */
  int64_t out_offset[4]; /* per quadrant: element offset of its block in the output; -1 if absent */
  int64_t out_elems;     /* total output elements */
  size_t workspace_bytes;/* minimum size of d_ws for fht_forward */
  size_t adjoint_workspace_bytes; /* minimum size of d_ws for fht_adjoint */
  int64_t adds;          /* additions of the transform (Theorem 1's count, all quadrants) */
  int64_t model_bytes;   /* HBM bytes the forward schedule must move (reads + writes) */
  int64_t ideal_bytes;   /* input read once + output written once */
  int32_t fused_rows, tile_cols, upper_passes, reserved;
} fht_plan_info_t;

/* Build a plan: the split tree of Section 3 (Split_T or Split_S applied
 * recursively), the exact merge tables t -> (t1, t2, s) of Algorithm 1, the
 * fused-subtree programs and the pass schedule; upload them to `device`.
 * h, w in [1, 65535]; quadrants a non-zero subset of FHT_QALL.
 * Synchronous; allocates the plan's own device tables (owned by the plan).
 * device < 0 builds a host-only plan (tables, sizes and the byte model for
 * inspection; no CUDA call is made and it cannot be executed).
 * `tuning` may be NULL. */
fht_status fht_plan(fht_plan_t* out, int32_t h, int32_t w, fht_dtype dtype, uint32_t quadrants,
                    fht_boundary boundary, fht_split split, int device, const fht_tuning_t* tuning);

/* Shapes, offsets, workspace size and the byte / addition model of a plan. */
fht_status fht_plan_info(fht_plan_t plan, fht_plan_info_t* info);

/* Forward transform (Algorithm 1, all requested quadrants).
 * d_in: h x w input elements of the plan's input type, row pitch in_pitch
 * (elements, >= w).  d_out: out_elems elements of the output type (packed
 * quadrants).  d_ws: workspace of at least workspace_bytes, 256-byte aligned;
 * its contents on entry are ignored.  Enqueued on `stream`. */
fht_status fht_forward(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out, void* d_ws,
                       size_t ws_bytes, void* stream);

/* Kernel launches one fht_forward of this plan enqueues. */
fht_status fht_plan_launches(fht_plan_t plan, int32_t* count);

/* Kind of the k-th launch of fht_forward (0: fused shared-memory pass over
 * subtrees of at most 64 rows, 1: upper per-height pass, 2: band pass (perfect
 * 2^k bands above the 64-row blocks), 3: spine sum of a Split_T root) and the
 * HBM bytes its schedule must move (compulsory reads + writes of that launch). */
fht_status fht_plan_launch_info(fht_plan_t plan, int32_t k, int32_t* kind, int64_t* model_bytes);

/* fht_forward that also records events[2k] and events[2k + 1] (cudaEvent_t
 * handles created by the caller) on `stream` just before and just after its
 * k-th kernel launch, for per-kernel timing.  nevents >= 2 * launches. */
fht_status fht_forward_timed(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out, void* d_ws,
                             size_t ws_bytes, void* stream, void** events, int32_t nevents);

/* Size of the fixed scratch array used by fht_forward_noalloc (32 MiB). */
#define FHT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/* fht_forward without a caller-provided workspace, for callers that cannot
 * allocate device memory when they run the transform (a real-time loop that
 * must not block on cudaMalloc, a plugin whose host owns all allocations, a
 * process whose free device memory already belongs to its own pool).  The
 * paper has no counterpart: this is an interface choice of this library.
 *  - The workspace is a fixed array of FHT_NOALLOC_SCRATCH_BYTES inside the
 *    library, held on every GPU that loads it until the process exits.  Plans
 *    whose workspace_bytes exceed it are rejected with FHT_ERR_INVALID.
 *  - The call allocates nothing (no cudaMalloc, no cudaFree).  The plan is
 *    created beforehand with fht_plan, which does allocate its tables.
 *  - The first call on a device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents:
 *    calls whose kernels overlap on the GPU (different streams without
 *    ordering between them) race on it.  Order them on one stream.
 *  - The looked-up address is kept for the life of the process: do not
 *    call it on a device after cudaDeviceReset there.
 *  - Arguments, output and errors as for fht_forward; the device-side status
 *    word (a bulk-copy wait that ran out) is read with fht_noalloc_status. */
fht_status fht_forward_noalloc(fht_plan_t plan, const void* d_in, int64_t in_pitch, void* d_out, void* stream);

/* Device-side status of the last fht_forward_noalloc on `device`: what
 * fht_ws_status reports for a caller's own workspace, read from the built-in
 * scratch.  FHT_OK, or FHT_ERR_TIMEOUT when a launch's bounded wait for its
 * bulk copies ran out and left part of the output unwritten.  Synchronises
 * `stream`; allocates nothing. */
fht_status fht_noalloc_status(int device, void* stream);

/* ---- host-memory pipeline ----
 * Forward transforms of images held in host memory, the copies included:
 * for callers whose images arrive in, and whose results go back to, host
 * memory.  The paper has no counterpart (an interface of this library).
 * fht_pipe_create allocates `depth` device sets (input, output, workspace of
 * the plan) and 2 + copy_streams blocking streams on the plan's device.
 * Each fht_pipe_submit takes the next set in turn and enqueues, without
 * blocking the host: the copy of h_in (h x w elements of the plan's input
 * type, row pitch in_pitch elements) to the device once the set's previous
 * output copies have finished; fht_forward; the copy of the packed output
 * (out_elems elements) to h_out, split over the copy streams.  Consecutive
 * submits overlap (output copy of image i, transform of i + 1, input copy of
 * i + 2).  h_in and h_out must stay valid and unchanged (h_in) or unread
 * (h_out) until fht_pipe_sync returns; page-locked host memory gives
 * asynchronous copies, pageable memory still works but copies synchronously.
 * Work recorded on the legacy default stream before (after) a submit runs
 * before (after) it.  Errors: FHT_ERR_INVALID for bad arguments, FHT_ERR_NOMEM
 * or FHT_ERR_CUDA from the runtime; fht_pipe_sync waits for every submit. */
typedef struct fht_pipe_s* fht_pipe_t;
fht_status fht_pipe_create(fht_pipe_t* pipe, fht_plan_t plan, int32_t depth, int32_t copy_streams);
fht_status fht_pipe_submit(fht_pipe_t pipe, const void* h_in, int64_t in_pitch, void* h_out);
fht_status fht_pipe_sync(fht_pipe_t pipe);
/* Waits for outstanding work, then frees the sets and streams.  NULL is accepted. */
fht_status fht_pipe_destroy(fht_pipe_t pipe);

/* Adjoint (back-projection): the exact transpose of fht_forward, i.e.
 * d_gin = sum over quadrants of Q^T(d_gout_q), the transpose of Algorithm 1's
 * merge applied level by level in reverse, as gathers (deterministic).
 * d_gout: out_elems elements of the output type; d_gin: h x w elements of the
 * output type (int32 for integer plans), row pitch gin_pitch, overwritten.
 * d_ws: at least adjoint_workspace_bytes, 256-byte aligned. */
fht_status fht_adjoint(fht_plan_t plan, const void* d_gout, void* d_gin, int64_t gin_pitch, void* d_ws,
                       size_t ws_bytes, void* stream);

/* ---- batched transforms: many images of uneven sizes in one persistent launch ----
 *
 * A job is one image: its plan (any size; all jobs of one submit share the
 * dtype and the queue's device), input, output and workspace (at least the
 * plan's workspace_bytes, 256-byte aligned, not shared with another job of
 * the same submit).  fht_submit lists the work units of every job phase by
 * phase (fused subtree tiles, then band tiles, then spine row groups, or one
 * phase per tree height for per-height plans) and runs them all in one
 * persistent launch: CTAs take units from a device counter; a unit of a later
 * phase waits for the earlier phases of its own job through a per-job
 * completion counter.  Waits are bounded (fht_queue_set_wait_limit, default
 * 2 s); a wait that gives up records FHT_ERR_TIMEOUT in the queue's status
 * word (read with fht_queue_status) and the kernel still returns.
 * Submits to one queue must be ordered (one stream): they share its device
 * tables.  Use one queue per stream for concurrent batches.  A submit made
 * while its stream is being captured into a CUDA graph becomes part of the
 * graph (copies from the queue's staging buffers, counter reset, launch); the
 * graph then owns the queue: replay it instead of submitting again, and do
 * not poll for its tags. */
typedef struct {
  fht_plan_t plan;
  const void* d_in;
  int64_t in_pitch; /* elements */
  void* d_out;
  void* d_ws;
  size_t ws_bytes;
  uint64_t tag;     /* returned by fht_queue_poll when the job's submit has finished */
  uint32_t flags;   /* 0, or FHT_JOB_WITHHOLD_DEPENDENCY */
  uint32_t reserved;
} fht_job;

/* Fault injection for tests of the bounded wait: the job's later-phase units
 * wait for one unit more than the job has, so their waits run out and the
 * submit ends with FHT_ERR_TIMEOUT in the status word (the job's output is
 * then incomplete).  No GPU fault is involved. */
#define FHT_JOB_WITHHOLD_DEPENDENCY 1u

/* Create a queue on `device` holding up to max_jobs jobs and max_units work
 * units per submit (device tables and pinned staging are allocated here). */
fht_status fht_queue_create(fht_queue_t* q, int device, int32_t max_jobs, int64_t max_units);
fht_status fht_queue_set_wait_limit(fht_queue_t q, int64_t wait_ns);
/* Enqueue one persistent launch over all jobs on `stream` (cudaStream_t).
 * FHT_ERR_BUSY when the jobs or their units exceed the queue's capacity.
 * The job tables are staged in the queue's pinned host buffers and copied in
 * stream order, so a submit first waits on the host until the previous
 * submit's copies have run, which is after every launch queued before them
 * on that stream (see fht_queue_ready). */
fht_status fht_submit(fht_queue_t q, int32_t njobs, const fht_job* jobs, void* stream);
/* Non-blocking: *ready = 1 when the queue's staging buffers are free, so
 * that fht_submit will not wait on the host; 0 while the previous submit's
 * table copies are still queued behind earlier work.  A serving loop that
 * submits only to ready queues never stalls on a busy stream. */
fht_status fht_queue_ready(fht_queue_t q, int32_t* ready);
/* Non-blocking: copies up to `cap` tags of finished jobs.  Each job is
 * reported once, as soon as its own last unit has finished (the kernel sets
 * the job's host-mapped completion flag), so early jobs of a batch are seen
 * before the rest of the batch ends.  Their outputs may then be read from
 * another stream. */
fht_status fht_queue_poll(fht_queue_t q, uint64_t* done_tags, int32_t cap, int32_t* ndone);
/* Synchronises `stream` and returns the queue's status word (FHT_OK or FHT_ERR_TIMEOUT). */
fht_status fht_queue_status(fht_queue_t q, void* stream);
fht_status fht_queue_reset_status(fht_queue_t q, void* stream);
fht_status fht_queue_destroy(fht_queue_t q);

/* The accuracy experiment of Sections 4-5: for every n in [n_lo, n_hi], the
 * exact numerator of the maximum orthotropic error of the generating patterns
 * of Algorithm 2 under `split`,
 *   d_num[n - n_lo] = max over t, x in [0, n) of |x t - pat(n,t)(x) (n - 1)|,
 * so that E(n) = d_num / (n - 1) (0 for n = 1).  d_num: device int64 array of
 * n_hi - n_lo + 1 entries, overwritten.  Enqueued on `stream`.  Cost grows as
 * n^2 log n per n (every pattern is generated). */
fht_status fht_pattern_errors(int32_t n_lo, int32_t n_hi, fht_split split, int64_t* d_num, void* stream);

/* Host-side verification of a plan: walks every table entry and checks that
 * each input, workspace, output and shared-memory index the kernels derive
 * from it lies inside its buffer.  Works on host-only plans; on a device plan
 * its first call copies the tables the host does not keep back from the
 * device (see fht_plan_table), nothing else touches the device.
 * FHT_OK, or FHT_ERR_INVALID with the first violation in fht_last_error(). */
fht_status fht_plan_check(fht_plan_t plan);

/* Host copies of a plan's tables, for inspection and host-side tests (no
 * counterpart in the paper).  *data receives a pointer to `*count` elements
 * of `*elem_size` bytes, owned by the plan and valid until fht_plan_destroy
 * (or until a first fht_adjoint rebuilds the tables).  The element layouts
 * are those of the library's internal descriptor header (csrc/fht_desc.h:
 * QuadDesc, FusedItem, MergeOp, RowJob, SpineRow, SpineTerm, AdjRow,
 * AdjTerm) and are not a
 * stable interface.  Offsets in the tables are element offsets into the
 * output, or into the workspace after its 256-byte header.  The adjoint
 * tables are empty until the plan has them (with_adjoint = 1, or after a
 * first fht_adjoint).  A plan built for a device keeps on the host only the
 * tables its launches read there; the first fht_plan_table (or
 * fht_plan_check) on it copies the others back from the device (a
 * synchronous copy) and keeps them for the plan's lifetime.
 * FHT_ERR_INVALID for a NULL argument or an unknown table; FHT_ERR_CUDA if
 * that copy fails. */
typedef enum {
  FHT_TABLE_QUADS = 0,        /* QuadDesc[4] (entries of absent quadrants are unused) */
  FHT_TABLE_FUSED = 1,        /* FusedItem: fused subtrees (64-row blocks and the rest) */
  FHT_TABLE_OPS = 2,          /* MergeOp: the fused subtrees' programs */
  FHT_TABLE_ROWS = 3,         /* RowJob: per-height upper passes, pass after pass */
  FHT_TABLE_PASS_BEGIN = 4,   /* int64: rows of pass p are [begin[p], begin[p + 1]) */
  FHT_TABLE_BAND_ITEMS = 5,   /* FusedItem: band items (band schedule) */
  FHT_TABLE_SPINE_ROWS = 6,   /* SpineRow (band schedule) */
  FHT_TABLE_SPINE_TERMS = 7,  /* SpineTerm */
  FHT_TABLE_SPINE_BEGIN = 8,  /* int64: spine rows of launch k are [begin[k], begin[k + 1]) */
  FHT_TABLE_ADJ_ROWS = 9,     /* AdjRow: adjoint per-height passes, highest first */
  FHT_TABLE_ADJ_TERMS = 10,   /* AdjTerm */
  FHT_TABLE_ADJ_BEGIN = 11,   /* int64: adjoint rows of pass p are [begin[p], begin[p + 1]) */
  FHT_TABLE_ADJ_PTR = 12,     /* int32: fused adjoint programs, row pointers into FHT_TABLE_ADJ_OPS */
  FHT_TABLE_ADJ_OPS = 13      /* MergeOp: (top = forward row, s = shift) terms of the fused adjoint */
} fht_table;

fht_status fht_plan_table(fht_plan_t plan, fht_table table, const void** data, int64_t* count, int32_t* elem_size);

/* Release a plan and its device tables.  NULL is accepted.  Device tables
 * live in ranges of large per-device chunks that the library allocates once
 * and keeps until the process exits (no driver allocation per plan); the
 * destroy waits for the device's outstanding work, as a cudaFree would, and
 * returns the range for reuse by later plans. */
fht_status fht_plan_destroy(fht_plan_t plan);

/* ---- plan builder pool ----
 * fht_plan on native worker threads, for callers that meet new image sizes
 * at run time (a serving loop) and must not block on, or queue behind, plan
 * building.  The paper has no counterpart: this is runtime of this library.
 * fht_builder_create starts `threads` (1..256) workers.  fht_builder_submit
 * queues one fht_plan call with the given arguments (as for fht_plan;
 * `tuning` may be NULL, and is copied) under the caller's `tag`, and returns
 * at once.  fht_builder_poll moves up to `cap` finished builds into tags[],
 * plans[], status[] and sets *n: a plan whose status is FHT_OK is then owned
 * by the caller (fht_plan_destroy), a failed build has plans[k] = NULL (its
 * message is not kept).  fht_builder_pending reports the queued and the
 * finished-but-unpolled builds.  fht_builder_destroy finishes the queued
 * builds, destroys the plans nobody polled and stops the workers.  All
 * functions may be called from any thread; one builder's calls are
 * serialised internally. */
fht_status fht_builder_create(fht_builder_t* out, int32_t threads);
fht_status fht_builder_submit(fht_builder_t b, uint64_t tag, int32_t h, int32_t w, fht_dtype dtype,
                              uint32_t quadrants, fht_boundary boundary, fht_split split, int device,
                              const fht_tuning_t* tuning);
fht_status fht_builder_poll(fht_builder_t b, uint64_t* tags, fht_plan_t* plans, fht_status* status, int32_t cap,
                            int32_t* n);
fht_status fht_builder_pending(fht_builder_t b, int32_t* queued, int32_t* finished);
fht_status fht_builder_destroy(fht_builder_t b);

/* Device status word kept at the start of a workspace: FHT_OK or the first
 * device-side error recorded by a kernel that used it.  Every fht_forward
 * clears it in its first launch; a spine launch whose bounded wait for its
 * bulk copies runs out (1 s) records FHT_ERR_TIMEOUT and leaves its tile
 * unwritten.  Synchronises `stream`. */
fht_status fht_ws_status(const void* d_ws, void* stream);

const char* fht_status_string(fht_status status);
const char* fht_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FHT_H */
