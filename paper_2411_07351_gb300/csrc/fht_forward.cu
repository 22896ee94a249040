// Forward kernels of the generalised Brady-Yong transform (Algorithm 1 of
// Section 3), sm_103a.
//
//  * fused_kernel: one CTA = one subtree of at most F rows x one column tile.
//    The subtree's input rows (a window of tile + m - 1 columns, wrapped or
//    zero-filled) are staged in shared memory and all of its merges run there,
//    level by level, ping-ponging between two shared buffers.  The subtree's
//    Hough rows are written once.
//  * upper_kernel: one pass per tree height above the fused subtrees.  Each
//    output row is Algorithm 1's merge  J(t) = R0(t1) + Rotate(R1(t2), s),
//    a gather-add over a whole row in HBM.  The root's rows are stored into
//    the output with the quadrant's column map.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "../../include/fht.h"
#include "fht_desc.h"
#include "fht_block.cuh"
#include "fht_device.cuh"
#include "fht_launch.hpp"
#include "fht_nvtx.hpp"

namespace fht {

template <typename InT, typename AccT>
__global__ void __launch_bounds__(512, 2) fused_kernel(FusedParams p) {
  pdl_launch_dependents();
  pdl_wait();  // band items read the blocks of the launch before
  // the first launch of a forward clears the workspace status word (later
  // launches record device-side errors there)
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    *reinterpret_cast<int32_t*>(static_cast<unsigned char*>(p.ws) - kWsHeader) = 0;
  const FusedItem it = p.items[blockIdx.x];
  const int32_t tile = blockIdx.y;
  if (tile >= it.ntiles) return;
  const QuadDesc& Q = p.quad[it.q];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AccT* sm = reinterpret_cast<AccT*>(smem_raw);
  if (it.kind != FUSED_GENERIC) {
    fused_block_any<false, InT, AccT>(p, it, Q, tile, sm, sm + (size_t)64 * p.RS);
  } else {
    fused_generic<InT, AccT>(p, it, Q, tile, sm, sm + (size_t)p.Fm * p.RP);
  }
}

// Flags of the register-tiled launches: VB_FIRST, the launch is the first
// of the forward (clears the workspace status word); VB_WAIT_FIRST, it reads
// what the launch before wrote (the band launch), so it waits before its
// first read.  A launch without VB_WAIT_FIRST (the 64-row blocks: they read
// only the input image) starts while the generic subtrees' launch still runs
// and waits for it before it exits, so that its completion still implies
// that launch's, which the next launch relies on.
enum : int32_t { VB_FIRST = 1, VB_WAIT_FIRST = 2 };

template <typename InT, typename AccT>
__global__ void __launch_bounds__(kVThreads, 3) block_kernel(FusedParams p, int32_t flags) {
  pdl_launch_dependents();
  if (flags & VB_WAIT_FIRST) pdl_wait();
  if ((flags & VB_FIRST) && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    *reinterpret_cast<int32_t*>(static_cast<unsigned char*>(p.ws) - kWsHeader) = 0;
  const FusedItem it = p.items[blockIdx.x];
  const int32_t tile = blockIdx.y;
  if (tile < it.ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    v_block<false, InT, AccT>(p, it, p.quad[it.q], tile, reinterpret_cast<AccT*>(smem_raw));
  }
  if (!(flags & VB_WAIT_FIRST)) pdl_wait();
}

// One CTA per output row; every thread keeps U independent element pairs in
// flight (all loads issued before the adds and stores).
template <typename AccT>
__global__ void __launch_bounds__(256) upper_kernel(const RowJob* __restrict__ rows, int64_t nrows,
                                                   const AccT* __restrict__ ws_in, AccT* ws_out, AccT* out) {
  pdl_launch_dependents();
  pdl_wait();
  constexpr int U = 8;
  for (int64_t k = blockIdx.x; k < nrows; k += gridDim.x) {
    const RowJob J = rows[k];
    const AccT* __restrict__ top = ws_in + J.top;
    const AccT* __restrict__ bot = ws_in + J.bot;
    const bool fin = J.flags & ROW_FINAL;
    const bool ext = J.flags & ROW_EXT;
    AccT* dst = (fin ? out : ws_out) + J.dst;
    int32_t u0 = 0;
    if constexpr (sizeof(AccT) == 4) {
      // 16-byte path: every thread four consecutive columns; a chunk runs it
      // when the row is not a root row (no column map) and all of its reads
      // lie inside both child rows with 8 elements to spare (the aligned
      // vector loads read up to 7 past the first wanted element)
      const int32_t C = (int32_t)blockDim.x * 4;
      const int32_t at = (int32_t)((J.top + (ext ? J.dtop : 0)) & 3), ab = (int32_t)((J.bot + J.dbot) & 3);
      const bool vec = !fin && (J.dst & 3) == 0;
      for (; vec && u0 + C <= J.wout; u0 += C) {
        const bool inside = ext ? (u0 + J.dtop >= 0 && u0 + C + J.dtop + 8 <= J.wtop && u0 + J.dbot >= 0 &&
                                   u0 + C + J.dbot + 8 <= J.wbot)
                                : (u0 + C + 8 <= J.W && u0 + C + J.dbot + 8 <= J.W);
        if (!inside) break;
        const int32_t u = u0 + 4 * (int32_t)threadIdx.x;
        AccT a[4], b[4], o[4];
        ldg4_shifted<false, AccT>(top + u + (ext ? J.dtop : 0), at, a);
        ldg4_shifted<false, AccT>(bot + u + J.dbot, ab, b);
#pragma unroll
        for (int q = 0; q < 4; q++) o[q] = a[q] + b[q];
        sts4<AccT>(dst + u, o);
      }
    }
    for (; u0 < J.wout; u0 += (int32_t)blockDim.x * U) {
      AccT a[U], b[U];
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int32_t u = u0 + q * (int32_t)blockDim.x + (int32_t)threadIdx.x;
        a[q] = AccT(0);
        b[q] = AccT(0);
        if (u < J.wout) {
          if (ext) {
            const int32_t i = u + J.dtop, i2 = u + J.dbot;
            if (i >= 0 && i < J.wtop) a[q] = top[i];
            if (i2 >= 0 && i2 < J.wbot) b[q] = bot[i2];
          } else {
            int32_t i2 = u + J.dbot;
            if (i2 >= J.W) i2 -= J.W;
            a[q] = top[u];
            b[q] = bot[i2];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int32_t u = u0 + q * (int32_t)blockDim.x + (int32_t)threadIdx.x;
        if (u < J.wout) store_row(dst, J, fin, u, a[q] + b[q]);
      }
    }
  }
}

// Zeros that stand in for a part row wherever a spine term lies wholly
// outside its part for a column tile (zero-initialised static storage).
__device__ __align__(16) unsigned char g_spine_zero[kSpineTilePlain * sizeof(double)];

// Fast tile of a spine row group: every term of every row is, over this
// column tile, either wholly inside its part row (one contiguous stretch) or
// wholly outside it (zeros), so each load is a plain pointer + constant.
template <bool kMap, int NT, int QPT, typename AccT>
__device__ __forceinline__ void spine_fast_load(const AccT* const* tp, AccT (&v)[NT][QPT]) {
#pragma unroll
  for (int c = 0; c < NT; c++) {
    const AccT* __restrict__ p = tp[c] + threadIdx.x;
#pragma unroll
    for (int q = 0; q < QPT; q++) v[c][q] = __ldg(p + q * 256);
  }
}

template <bool kMap, int NT, int QPT, typename AccT>
__device__ __forceinline__ void spine_fast_group(const SpineRow* sr, const AccT* const (*tp)[kMaxSpineTerms],
                                                 int32_t nr, int32_t W, int32_t sigma, int32_t kappa, AccT* out,
                                                 int32_t u0) {
  AccT a[NT][QPT], b[NT][QPT];
  spine_fast_load<kMap, NT, QPT, AccT>(tp[0], a);
  for (int32_t r = 0; r < nr; r += 2) {
    if (r + 1 < nr) spine_fast_load<kMap, NT, QPT, AccT>(tp[r + 1], b);
    spine_store<kMap, NT, 256, QPT, AccT>(W, sigma, kappa, out + sr[r].dst, u0, a);
    if (r + 1 >= nr) break;
    if (r + 2 < nr) spine_fast_load<kMap, NT, QPT, AccT>(tp[r + 2], a);
    spine_store<kMap, NT, 256, QPT, AccT>(W, sigma, kappa, out + sr[r + 1].dst, u0, b);
  }
}

template <typename AccT>
__global__ void __launch_bounds__(256, sizeof(AccT) > 4 ? 1 : 3) spine_kernel(const SpineRow* __restrict__ rows,
                                                   int64_t nrows, const SpineTerm* __restrict__ terms,
                                                   const AccT* __restrict__ ws, AccT* __restrict__ out, AccT* inner,
                                                   QuadDescs quads, int32_t rpc) {
  // rpc (<= kSpineRows) rows per CTA: a CTA sums its rows one after another,
  // so a short spine takes fewer rows per CTA and more CTAs
  __shared__ SpineTerm st[kSpineRows][kMaxSpineTerms];
  __shared__ SpineRow sr[kSpineRows];
  __shared__ const AccT* tp[kSpineRows][kMaxSpineTerms];
  __shared__ int32_t s_straddle;
  pdl_launch_dependents();
  pdl_wait();
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int32_t u0 = blockIdx.y * kSpineTilePlain;
  const int32_t nr = (int32_t)(nrows - r0 < rpc ? nrows - r0 : rpc);
  if (threadIdx.x < nr) sr[threadIdx.x] = rows[r0 + threadIdx.x];
  if (threadIdx.x == 0) s_straddle = 0;
  __syncthreads();
  for (int32_t idx = threadIdx.x; idx < nr * kMaxSpineTerms; idx += blockDim.x) {
    const int32_t r = idx / kMaxSpineTerms, c = idx % kMaxSpineTerms;
    if (c < sr[r].term_count) st[r][c] = terms[sr[r].term_begin + c];
  }
  // one row geometry for the whole group (same quadrant, kind and term count)
  bool uniform = nr > 0 && sr[0].term_count <= 8;
  for (int32_t r = 1; r < nr; r++)
    uniform = uniform && sr[r].q == sr[0].q && sr[r].term_count == sr[0].term_count && sr[r].flags == sr[0].flags;
  const QuadDesc& Q = quads.q[sr[0].q];
  const bool is_inner = sr[0].flags & SPINE_INNER;
  const int32_t W = is_inner ? sr[0].w : Q.W;
  const bool fast_tile = uniform && u0 + kSpineTilePlain <= W;
  __syncthreads();
  if (fast_tile) {
    // classify every term over this tile: inside its part row, outside it, or across an edge
    const AccT* zero = reinterpret_cast<const AccT*>(g_spine_zero);
    for (int32_t idx = threadIdx.x; idx < nr * kMaxSpineTerms; idx += blockDim.x) {
      const int32_t r = idx / kMaxSpineTerms, c = idx % kMaxSpineTerms;
      if (c >= sr[r].term_count) continue;
      const SpineTerm T = st[r][c];
      const int32_t lo = u0 + T.off, hi = lo + kSpineTilePlain;
      const AccT* p = nullptr;
      if (Q.ext) {
        if (lo >= 0 && hi <= T.wpart) p = ws + T.row + lo;
        else if (hi <= 0 || lo >= T.wpart) p = zero;
      } else {
        if (hi <= W) p = ws + T.row + lo;          // no wrap inside the tile
        else if (lo >= W) p = ws + T.row + lo - W; // the whole tile wraps
      }
      tp[r][c] = p;
      if (!p) s_straddle = 1;
    }
    __syncthreads();
  }
  if (fast_tile && !s_straddle) {
    if (is_inner) {
      switch (sr[0].term_count) {
#define FHT_SPINE_FAST(N)                                                                               \
  case N:                                                                                               \
    spine_fast_group<false, N, kSpineQPT, AccT>(sr, tp, nr, W, 1, 0, inner, u0);                        \
    return;
        FHT_SPINE_FAST(1) FHT_SPINE_FAST(2) FHT_SPINE_FAST(3) FHT_SPINE_FAST(4) FHT_SPINE_FAST(5)
        FHT_SPINE_FAST(6) FHT_SPINE_FAST(7) FHT_SPINE_FAST(8)
#undef FHT_SPINE_FAST
        default:
          break;
      }
    } else {
      switch (sr[0].term_count) {
#define FHT_SPINE_FAST(N)                                                                               \
  case N:                                                                                               \
    spine_fast_group<true, N, kSpineQPT, AccT>(sr, tp, nr, W, Q.sigma, Q.kappa, out, u0);               \
    return;
        FHT_SPINE_FAST(1) FHT_SPINE_FAST(2) FHT_SPINE_FAST(3) FHT_SPINE_FAST(4) FHT_SPINE_FAST(5)
        FHT_SPINE_FAST(6) FHT_SPINE_FAST(7) FHT_SPINE_FAST(8)
#undef FHT_SPINE_FAST
        default:
          break;
      }
    }
  }
  spine_rows_tile<false, 256, kSpineQPT, AccT, kSpinePipe>(sr, st, nr, quads.q, ws, out, inner, u0);
}

// ---- staged spine kernel ----
// One CTA = one 16-row group x one tile of kStageTile columns.  The group's
// segments (distinct part-row windows) are copied into shared memory with
// cp.async: 16-byte chunks whose bytes beyond the part row are zero-filled by
// the copy itself (extended), or element by element with the cyclic wrap;
// then every output element is the sum of its terms read from shared memory.
constexpr int kStageThreads = 256;
constexpr int kStageQPT = kStageTile / kStageThreads;

// Per-row constants of a staged CTA, set once by the prologue.
template <typename AccT>
struct StagedRow {
  AccT* dst;      // output row (root) or inner-node row (workspace)
  int32_t W;      // row length
  int32_t sigma;  // column map X = (sigma u + kappa) mod W; sigma = 0: X = u
  int32_t kappa;
  int32_t pad;
};

// General rows: each row its own geometry and column map.
template <int NT, typename AccT>
__device__ __forceinline__ void staged_rows(const AccT* S, const int32_t (*so)[kMaxSpineTerms],
                                            const StagedRow<AccT>* ri, int32_t nr, int32_t u0) {
  for (int32_t r = 0; r < nr; r++) {
    const StagedRow<AccT> R = ri[r];
    if (u0 >= R.W) continue;
    int32_t o[NT];
#pragma unroll
    for (int c = 0; c < NT; c++) o[c] = so[r][c] + (int32_t)threadIdx.x;
#pragma unroll
    for (int q = 0; q < kStageQPT; q++) {
      const int32_t u = u0 + q * kStageThreads + (int32_t)threadIdx.x;
      AccT acc = S[o[0] + q * kStageThreads];
#pragma unroll
      for (int c = 1; c < NT; c++) acc += S[o[c] + q * kStageThreads];
      if (u < R.W) {
        int32_t X = R.sigma * u + R.kappa;
        if (X < 0) X += R.W;
        if (X >= R.W) X -= R.W;
        R.dst[X] = acc;
      }
    }
  }
}

// Uniform rows (one quadrant, one kind, one term count): the output columns
// X_q of this thread's kStageQPT columns are the same for every row, so they
// are computed once; a row is then NT shared loads and one store per column.
template <int NT, typename AccT>
__device__ __forceinline__ void staged_rows_uniform(const AccT* S, const int32_t (*so)[kMaxSpineTerms],
                                                    const StagedRow<AccT>* ri, int32_t nr, int32_t u0) {
  const StagedRow<AccT> R0 = ri[0];
  int32_t X[kStageQPT];
  bool live[kStageQPT];
#pragma unroll
  for (int q = 0; q < kStageQPT; q++) {
    const int32_t u = u0 + q * kStageThreads + (int32_t)threadIdx.x;
    int32_t x = R0.sigma * u + R0.kappa;
    if (x < 0) x += R0.W;
    if (x >= R0.W) x -= R0.W;
    X[q] = x;
    live[q] = u < R0.W;
  }
  const bool full = u0 + kStageTile <= R0.W;
  for (int32_t r = 0; r < nr; r++) {
    AccT* __restrict__ d = ri[r].dst;
    int32_t o[NT];
#pragma unroll
    for (int c = 0; c < NT; c++) o[c] = so[r][c] + (int32_t)threadIdx.x;
    AccT acc[kStageQPT];
#pragma unroll
    for (int q = 0; q < kStageQPT; q++) {
      acc[q] = S[o[0] + q * kStageThreads];
#pragma unroll
      for (int c = 1; c < NT; c++) acc[q] += S[o[c] + q * kStageThreads];
    }
    if (full) {
#pragma unroll
      for (int q = 0; q < kStageQPT; q++) d[X[q]] = acc[q];
    } else {
#pragma unroll
      for (int q = 0; q < kStageQPT; q++)
        if (live[q]) d[X[q]] = acc[q];
    }
  }
}

template <typename AccT>
__global__ void __launch_bounds__(kStageThreads) spine_staged_kernel(const SpineRow* __restrict__ rows, int64_t nrows,
                                                           const SpineTerm* __restrict__ terms,
                                                           const SpineGrp* __restrict__ grps,
                                                           const SpineSeg* __restrict__ segs,
                                                           const AccT* __restrict__ ws, AccT* __restrict__ out,
                                                           AccT* inner, QuadDescs quads) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AccT* S = reinterpret_cast<AccT*>(smem_raw);
  __shared__ __align__(8) uint64_t bar;
  __shared__ int32_t s_wait_ok;
  __shared__ StagedRow<AccT> ri[kSpineRows];
  __shared__ int32_t tc[kSpineRows], rq[kSpineRows];
  __shared__ __align__(16) int32_t so[kSpineRows][kMaxSpineTerms];
  __shared__ SpineSeg sg[kStageMaxSegs];
  constexpr int32_t EPC = 16 / (int32_t)sizeof(AccT);
  pdl_launch_dependents();
  const int64_t r0 = (int64_t)blockIdx.x * kSpineRows;
  const int32_t u0 = blockIdx.y * kStageTile;
  const int32_t nr = (int32_t)(nrows - r0 < kSpineRows ? nrows - r0 : kSpineRows);
  const SpineGrp G = grps[blockIdx.x];
  if ((int32_t)threadIdx.x < nr) {
    const SpineRow R = rows[r0 + threadIdx.x];
    const QuadDesc& Q = quads.q[R.q];
    const bool is_inner = R.flags & SPINE_INNER;
    StagedRow<AccT> o;
    o.dst = (is_inner ? inner : out) + R.dst;
    o.W = is_inner ? R.w : Q.W;
    o.sigma = is_inner ? 1 : Q.sigma;  // inner rows: X = u
    o.kappa = is_inner ? 0 : Q.kappa;
    o.pad = 0;
    ri[threadIdx.x] = o;
    tc[threadIdx.x] = R.term_count;
    rq[threadIdx.x] = R.q * 2 + (is_inner ? 1 : 0);
    for (int32_t c = 0; c < R.term_count; c++) so[threadIdx.x][c] = terms[R.term_begin + c].sofs;
  }
  for (int32_t s = threadIdx.x; s < G.seg_count; s += blockDim.x) sg[s] = segs[G.seg_begin + s];
  __syncthreads();
  // nothing to do for a tile right of every row of the group
  int32_t wmax = 0;
  bool uniform = true;
  for (int32_t r = 0; r < nr; r++) {
    wmax = ri[r].W > wmax ? ri[r].W : wmax;
    uniform = uniform && tc[r] == tc[0] && rq[r] == rq[0] && ri[r].W == ri[0].W;
  }
  if (u0 >= wmax) return;
  // the tables above are the plan's; the part rows below were written by the launches before
  pdl_wait();
  const bool ext = quads.q[0].ext | quads.q[1].ext | quads.q[2].ext | quads.q[3].ext;
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  if (ext) {
    // Extended: each window's in-row stretch [lo, lo + n) (16-byte multiples: rows are 128-byte
    // aligned, window starts are multiples of 16 bytes) is one bulk copy; the few columns outside
    // it (zeros beyond the part row, up to 15 bytes of tail) are written by the threads.
    if (threadIdx.x == 0) {
      mbar_init(&bar, (uint32_t)G.seg_count);  // one arrival per window
      s_wait_ok = 1;
    }
    __syncthreads();
    if (warp == 0) {
      // lane s announces window s's bytes and issues its copy
      for (int32_t s = lane; s < G.seg_count; s += 32) {
        const SpineSeg& g = sg[s];
        const int32_t A = u0 + g.a_off, lo = A > 0 ? A : 0, hi = A + g.len < g.wpart ? A + g.len : g.wpart;
        const int32_t n = hi > lo ? (hi - lo) / EPC * EPC : 0;
        mbar_arrive_expect_tx(&bar, (uint32_t)n * (uint32_t)sizeof(AccT));
        if (n > 0) bulk_copy_g2s(S + g.smem + (lo - A), ws + g.row + lo, (uint32_t)n * (uint32_t)sizeof(AccT), &bar);
      }
    }
    for (int32_t s = warp; s < G.seg_count; s += nwarps) {
      const SpineSeg g = sg[s];
      const AccT* __restrict__ rowp = ws + g.row;
      const int32_t A = u0 + g.a_off, lo = A > 0 ? A : 0, hi = A + g.len < g.wpart ? A + g.len : g.wpart;
      const int32_t n = hi > lo ? (hi - lo) / EPC * EPC : 0;
      AccT* dst = S + g.smem;
      // columns left of the part row (the whole window when it ends left of column 0)
      const int32_t left = lo - A < g.len ? lo - A : g.len;
      for (int32_t e = lane; e < left; e += 32) dst[e] = AccT(0);
      // the tail of the part row and the columns right of it
      for (int32_t e = (lo - A) + n + lane; e < g.len; e += 32) {
        const int32_t i = A + e;
        dst[e] = i < g.wpart ? __ldg(rowp + i) : AccT(0);
      }
    }
    // bounded wait for the bulk copies (they complete within microseconds)
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(&bar, 0)) {
      if (globaltimer_ns() - t0 > 1000000000ull) {
        s_wait_ok = 0;
        break;
      }
    }
    __syncthreads();
    if (!s_wait_ok) {
      // record the failure in the workspace status word, give the copies a
      // last bounded chance to land, and leave this tile unwritten
      if (threadIdx.x == 0) {
        int32_t* status = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(inner) - kWsHeader);
        atomicCAS(status, 0, (int32_t)FHT_ERR_TIMEOUT);
        const uint64_t t1 = globaltimer_ns();
        while (!mbar_try_wait(&bar, 0) && globaltimer_ns() - t1 < 1000000000ull) {
        }
      }
      __syncthreads();
      return;
    }
  }
  // cyclic: stage the windows with cp.async, one warp per segment, lanes over its 16-byte chunks
  for (int32_t s = warp; s < G.seg_count && !ext; s += nwarps) {
    const SpineSeg g = sg[s];
    const AccT* __restrict__ rowp = ws + g.row;
    const int32_t A = u0 + g.a_off;
    AccT* dst = S + g.smem;
    if (g.wpart % EPC == 0) {
      for (int32_t k = lane; k < g.len / EPC; k += 32) {
        int32_t i0 = A + k * EPC;
        if (i0 >= g.wpart) i0 -= g.wpart;
        if (i0 >= g.wpart) i0 %= g.wpart;  // a tile past this quadrant's rows (mixed groups)
        cp_async_16(dst + k * EPC, rowp + i0, 16);
      }
    } else {
      for (int32_t k = lane; k < g.len; k += 32) {
        int32_t i = A + k;
        if (i >= g.wpart) i -= g.wpart;
        if (i >= g.wpart) i %= g.wpart;
        cp_async_elem_z<AccT>(dst + k, rowp + i, true);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (uniform) {
    switch (tc[0]) {
#define FHT_STAGED(N)                                        \
  case N:                                                    \
    staged_rows_uniform<N, AccT>(S, so, ri, nr, u0);         \
    return;
      FHT_STAGED(1) FHT_STAGED(2) FHT_STAGED(3) FHT_STAGED(4) FHT_STAGED(5) FHT_STAGED(6) FHT_STAGED(7)
      FHT_STAGED(8)
#undef FHT_STAGED
      default:
        break;
    }
  }
  // mixed or long rows: one row at a time
  for (int32_t r = 0; r < nr; r++) {
    switch (tc[r]) {
#define FHT_STAGED1(N)                                                       \
  case N:                                                                    \
    staged_rows<N, AccT>(S, so + r, ri + r, 1, u0);                          \
    break;
      FHT_STAGED1(1) FHT_STAGED1(2) FHT_STAGED1(3) FHT_STAGED1(4) FHT_STAGED1(5) FHT_STAGED1(6)
      FHT_STAGED1(7) FHT_STAGED1(8) FHT_STAGED1(9) FHT_STAGED1(10) FHT_STAGED1(11) FHT_STAGED1(12)
      FHT_STAGED1(13) FHT_STAGED1(14) FHT_STAGED1(15) FHT_STAGED1(16)
#undef FHT_STAGED1
      default:
        break;
    }
  }
}

// ------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------
cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;  // (kernel, device) -> limit set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{kernel, dev}];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

void fused_geometry(const HostPlan& P, FusedGeometry& g) {
  // generic path: a window of tw + m - 1 columns plus room for the largest shifted read
  g.Fm = std::max(P.max_generic_m, 1);
  g.RP = P.generic_tw + g.Fm - 1 + P.generic_shift;
  if (g.RP % 2 == 0) g.RP++;  // odd pitch: column-wise (transposed) staging is conflict-free
  size_t generic = P.max_generic_m > 0 ? (size_t)2 * g.Fm * g.RP * P.acc_size : 0;
  // fast path: staged rows (TW + 63) and level-2 rows (TW + 60)
  g.RS = P.cfg.TW + 63;
  if (g.RS % 2 == 0) g.RS++;
  g.RA = P.cfg.TW + 60;
  if (g.RA % 2 == 0) g.RA++;
  size_t by64 = P.n_by64 > 0 ? (size_t)64 * (g.RS + g.RA) * P.acc_size : 0;
  g.smem = std::max(generic, by64);
  g.gsmem = generic;
  g.vsmem = P.vblock ? (size_t)64 * kVPitch * P.acc_size : 0;
}

// Fused launches of a forward: one, or on the register-tiled path the
// generic subtrees' (if any) and then the 64-row blocks'.
static int32_t fused_launches(const HostPlan& P) { return P.vblock ? 1 + (P.n_generic > 0) : 1; }

static int32_t spine_passes(const HostPlan& P) {
  int32_t n = 0;
  for (size_t k = 0; k + 1 < P.spine_pass_begin.size(); k++) n += P.spine_pass_begin[k + 1] > P.spine_pass_begin[k];
  return n;
}

int32_t forward_launches(const HostPlan& P) {
  const int32_t nf = fused_launches(P);
  if (P.bands) return nf + (P.band_items.empty() ? 0 : 1) + spine_passes(P);
  return nf + (int32_t)P.pass_bytes.size();
}

void forward_launch_info(const HostPlan& P, int32_t k, int32_t& kind, int64_t& bytes) {
  const int32_t nf = fused_launches(P);
  if (k < nf) {
    if (!P.vblock) {
      kind = LAUNCH_FUSED;
      bytes = P.fused_bytes;
    } else if (k + 1 < nf) {
      kind = LAUNCH_FUSED;  // the generic subtrees
      bytes = P.generic_bytes;
    } else {
      kind = LAUNCH_BLOCK;
      bytes = P.by64_bytes;
    }
  } else if (!P.bands) {
    kind = LAUNCH_UPPER;
    bytes = P.pass_bytes[k - nf];
  } else if (k == nf && !P.band_items.empty()) {
    kind = LAUNCH_BAND;
    bytes = P.band_bytes;
  } else {
    kind = LAUNCH_SPINE;
    // the k-th spine launch (empty passes launch nothing)
    int32_t s = k - nf - (P.band_items.empty() ? 0 : 1);
    bytes = 0;
    for (size_t p = 0; p + 1 < P.spine_pass_begin.size(); p++) {
      if (P.spine_pass_begin[p + 1] == P.spine_pass_begin[p]) continue;
      if (s-- == 0) {
        bytes = P.spine_pass_bytes[p];
        break;
      }
    }
  }
}

template <typename InT, typename AccT>
static cudaError_t launch_forward_t(const DevicePlan& D, const void* in, int64_t in_pitch, void* out, void* ws,
                                    cudaStream_t st, cudaEvent_t* ev) {
  int32_t launch = 0;
  auto mark = [&](int which) {
    if (ev) cudaEventRecord(ev[2 * launch + which], st);
  };
  // Every launch after the first of a forward may start while the one before
  // drains (its kernels wait for the data in griddepcontrol.wait); the first
  // launch and the per-launch timing mode serialise normally.
  auto go = [&](auto kernel, dim3 grid, unsigned block, size_t smem, auto... args) -> cudaError_t {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (launch > 0 && !ev) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
  };
  const HostPlan& P = *D.host;
  AccT* wsa = reinterpret_cast<AccT*>(static_cast<unsigned char*>(ws) + kWsHeader);
  FusedParams fp;
  fp.in = in;
  fp.in_pitch = in_pitch;
  fp.ws = wsa;
  fp.out = out;
  fp.items = D.fused;
  fp.ops = D.ops;
  for (int q = 0; q < 4; q++) fp.quad[q] = P.quad[q];
  fp.RP = D.geo.RP;
  fp.Fm = D.geo.Fm;
  fp.RS = D.geo.RS;
  fp.RA = D.geo.RA;
  fp.vblock = 0;  // the plain launches pick their kernels on the host
  const size_t smem = D.geo.smem;
  auto kfn = fused_kernel<InT, AccT>;
  cudaError_t e = raise_smem_limit(kfn, smem);
  if (e != cudaSuccess) return e;
  if (!P.vblock) {
    dim3 grid((unsigned)P.fused.size(), P.max_ntiles);  // tiles <= 131070 / 32 fit in grid.y
    nvtxRangePushA("fht fused subtrees");
    mark(0);
    e = go(kfn, grid, P.cfg.threads, smem, fp);
    mark(1);
    nvtxRangePop();
    launch++;
    if (e != cudaSuccess) return e;
  } else if constexpr (sizeof(AccT) == 4) {
    if (P.n_generic > 0) {
      dim3 grid((unsigned)P.n_generic, P.max_generic_ntiles);
      nvtxRangePushA("fht generic subtrees");
      mark(0);
      e = go(kfn, grid, P.cfg.threads, D.geo.gsmem, fp);
      mark(1);
      nvtxRangePop();
      launch++;
      if (e != cudaSuccess) return e;
    }
    auto kbl = block_kernel<InT, AccT>;
    if ((e = raise_smem_limit(kbl, D.geo.vsmem)) != cudaSuccess)
      return e;
    FusedParams bp = fp;
    bp.items = D.fused + P.n_generic;
    nvtxRangePushA("fht 64-row blocks");
    mark(0);
    e = go(kbl, dim3((unsigned)P.n_by64, P.max_by64_ntiles), kVThreads, D.geo.vsmem, bp,
           (int32_t)(P.n_generic == 0 ? VB_FIRST : 0));
    mark(1);
    nvtxRangePop();
    launch++;
    if (e != cudaSuccess) return e;
  } else {
    return cudaErrorInvalidValue;  // the planner enables the register-tiled path for 4-byte accumulators only
  }
  if (P.bands) {
    if (!P.band_items.empty()) {
      fp.items = D.band_items;
      dim3 bgrid((unsigned)P.band_items.size(), P.max_band_ntiles);
      if constexpr (sizeof(AccT) == 4) {
        if (P.vblock &&
            (e = raise_smem_limit(block_kernel<InT, AccT>, D.geo.vsmem)) != cudaSuccess)
          return e;
      }
      nvtxRangePushA("fht band pass");
      mark(0);
      if constexpr (sizeof(AccT) == 4) {
        if (P.vblock) {
          e = go(block_kernel<InT, AccT>, bgrid, kVThreads, D.geo.vsmem, fp, (int32_t)VB_WAIT_FIRST);
        } else {
          e = go(kfn, bgrid, P.cfg.threads, smem, fp);
        }
      } else {
        e = go(kfn, bgrid, P.cfg.threads, smem, fp);
      }
      mark(1);
      nvtxRangePop();
      launch++;
      if (e != cudaSuccess) return e;
    }
    QuadDescs qd;
    for (int q = 0; q < 4; q++) qd.q[q] = P.quad[q];
    int32_t maxW = 1;
    for (int q = 0; q < 4; q++)
      if (P.cfg.quads & (1u << q)) maxW = std::max(maxW, P.quad[q].W);
    // spine chunks bottom-up: every launch reads the inner nodes the one before wrote
    for (size_t p = 0; p + 1 < P.spine_pass_begin.size(); p++) {
      const int64_t b = P.spine_pass_begin[p], n = P.spine_pass_begin[p + 1] - b;
      if (n <= 0) continue;
      const unsigned groups = (unsigned)((n + kSpineRows - 1) / kSpineRows);
      const size_t ssmem = (size_t)P.spine_pass_smem[p] * sizeof(AccT);
      if (ssmem > 0 && (e = raise_smem_limit(spine_staged_kernel<AccT>, ssmem)) != cudaSuccess)
        return e;
      nvtxRangePushA("fht spine sum");
      mark(0);
      if (ssmem > 0) {
        const size_t smem = ssmem;
        auto kst = spine_staged_kernel<AccT>;
        dim3 sgrid(groups, (unsigned)((maxW + kStageTile - 1) / kStageTile));
        e = go(kst, sgrid, kStageThreads, smem, (const SpineRow*)(D.spine_rows + b), n,
               (const SpineTerm*)D.spine_terms, (const SpineGrp*)(D.spine_grps + P.spine_grp_begin[p]),
               (const SpineSeg*)D.spine_segs, (const AccT*)wsa, static_cast<AccT*>(out), wsa, qd);
      } else {
        // rows per CTA: 16, halved (to 2 at least) while the grid would hold
        // fewer than two CTAs per SM (a 257-row spine: 129 CTAs of 2 rows)
        const unsigned tiles = (unsigned)((maxW + kSpineTilePlain - 1) / kSpineTilePlain);
        int32_t rpc = kSpineRows;
        while (rpc > 2 && (unsigned)((n + rpc - 1) / rpc) * tiles < 2u * 152u) rpc /= 2;
        dim3 sgrid((unsigned)((n + rpc - 1) / rpc), tiles);
        e = go(spine_kernel<AccT>, sgrid, 256, 0, (const SpineRow*)(D.spine_rows + b), n,
               (const SpineTerm*)D.spine_terms, (const AccT*)wsa, static_cast<AccT*>(out), wsa, qd, rpc);
      }
      mark(1);
      nvtxRangePop();
      launch++;
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (size_t p = 0; p + 1 < P.pass_begin.size(); p++) {
    const int64_t b = P.pass_begin[p], n = P.pass_begin[p + 1] - b;
    if (n <= 0) continue;
    const unsigned blocks = (unsigned)std::min<int64_t>(n, 1 << 30);
    nvtxRangePushA("fht upper pass");
    mark(0);
    e = go(upper_kernel<AccT>, dim3(blocks), 256, 0, (const RowJob*)(D.rows + b), n, (const AccT*)wsa, wsa,
           static_cast<AccT*>(out));
    mark(1);
    nvtxRangePop();
    launch++;
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_forward(const DevicePlan& D, const void* in, int64_t in_pitch, void* out, void* ws,
                           cudaStream_t st, cudaEvent_t* ev) {
  switch (D.host->cfg.dtype) {
    case 0:
      return launch_forward_t<uint8_t, int32_t>(D, in, in_pitch, out, ws, st, ev);
    case 1:
      return launch_forward_t<int32_t, int32_t>(D, in, in_pitch, out, ws, st, ev);
    case 2:
      return launch_forward_t<float, float>(D, in, in_pitch, out, ws, st, ev);
    default:
      return launch_forward_t<double, double>(D, in, in_pitch, out, ws, st, ev);
  }
}

}  // namespace fht
