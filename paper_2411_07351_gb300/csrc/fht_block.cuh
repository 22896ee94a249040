// Register-tiled Brady-Yong block path (4-byte accumulators): the 64-row
// blocks of the fused pass with every merge level done in registers.
//
// A perfect block of R = 2^r child blocks of M rows each (the children
// already Brady-Yong transformed) becomes one block of R M rows.  Following
// the merges of Algorithm 1 through r levels (at a power-of-two node t1 = t2 =
// floor(t/2) and the bottom child is shifted by ceil(t/2)), output slope
// t = R k + i (k in [0, M), i in [0, R)) of child e (rows e M + k) is read at
//     column x + e k + p_i(e),
// where p_i is the R-row Brady-Yong pattern:  p^1_0(0) = 0 and
//     p^{2R}_i(e) = p^R_{i/2}(e)               for e <  R,
//     p^{2R}_i(e) = p^R_{i/2}(e - R) + ceil(i/2)  for e >= R.
// A thread owns four consecutive output columns x = j .. j + 3 (j a multiple
// of four) of all R slopes i of one (group, k).  Child e is read over columns
// [j + e k, j + e k + 4 + e) with 16-byte shared loads; their misalignment
// (e k) mod 4 depends only on k mod 4, which is uniform across a warp, so a
// four-way switch on it makes every shifted read a compile-time register
// index.  The R outputs are then built level by level in registers (the
// Brady-Yong sharing: about log2 R additions per output).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fht_desc.h"
#include "fht_device.cuh"

namespace fht {

// Geometry (kVTile, kVThreads, kVPitch: fht_desc.h): the staged window of
// kVTile + 63 columns is merged in place in one shared buffer; kVPitch / 4 is
// odd, so that 8 rows x 4 columns of the transposed staging hit 32 distinct
// banks.
constexpr int kVWin = kVTile + 64;  // staged columns (the window needs kVTile + 63)
static_assert(kVWin <= kVPitch && kVPitch % 4 == 0 && (kVPitch / 4) % 2 == 1, "shared row geometry");

template <int R>
__host__ __device__ constexpr int by_off(int i, int e) {
  if constexpr (R == 1) {
    return 0;
  } else {
    return e < R / 2 ? by_off<R / 2>(i / 2, e) : by_off<R / 2>(i / 2, e - R / 2) + (i + 1) / 2;
  }
}

static_assert(by_off<4>(0, 1) == 0 && by_off<4>(1, 1) == 0 && by_off<4>(2, 1) == 1 && by_off<4>(3, 1) == 1 &&
                  by_off<4>(1, 2) == 1 && by_off<4>(2, 2) == 1 && by_off<4>(3, 2) == 2 && by_off<4>(3, 3) == 3 &&
                  by_off<4>(1, 3) == 1 && by_off<4>(2, 3) == 2,
              "4-row pattern: child 1 at floor(i/2), child 2 at ceil(i/2), child 3 at their sum");
static_assert(by_off<8>(7, 5) == 5 && by_off<8>(0, 7) == 0 && by_off<8>(5, 6) == 4,
              "8-row pattern: the last slope is the diagonal, slope 0 the column");

// Misalignment of child e's first column for k = A (mod 4).
__host__ __device__ constexpr int v_misalign(int e, int A) { return (e * A) & 3; }
// 16-byte vectors that cover child e's columns [0, 4 + e) from that start.
__host__ __device__ constexpr int v_nvec(int e, int A) { return (v_misalign(e, A) + 4 + e + 3) / 4; }

// out[i][x] = sum_e c[E0 + e][a_e + x + p_i(e)], e in [0, R), x in [0, W),
// built as the Brady-Yong recursion: the top half's sub-block at x plus the
// bottom half's at x + ceil(i/2).
template <int R, int W, int E0, int A, typename T>
__device__ __forceinline__ void by_regs(const T (&c)[8][16], T (&out)[R][W]) {
  if constexpr (R == 1) {
    constexpr int a = v_misalign(E0, A);
#pragma unroll
    for (int x = 0; x < W; x++) out[0][x] = c[E0][a + x];
  } else {
    T top[R / 2][W];
    T bot[R / 2][W + R / 2];
    by_regs<R / 2, W, E0, A, T>(c, top);
    by_regs<R / 2, W + R / 2, E0 + R / 2, A, T>(c, bot);
#pragma unroll
    for (int i = 0; i < R; i++)
#pragma unroll
      for (int x = 0; x < W; x++) out[i][x] = top[i / 2][x] + bot[i / 2][x + (i + 1) / 2];
  }
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<int32_t> {
  using type = int4;
};

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T* d) {
  const typename Vec4<T>::type v = *reinterpret_cast<const typename Vec4<T>::type*>(p);
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}

template <typename T>
__device__ __forceinline__ void sts4(T* p, const T* s) {
  typename Vec4<T>::type v;
  v.x = s[0];
  v.y = s[1];
  v.z = s[2];
  v.w = s[3];
  *reinterpret_cast<typename Vec4<T>::type*>(p) = v;
}

// Four consecutive elements p[0..3] of global memory whose first one sits
// `a` (= its element offset mod 4) past a 16-byte boundary: one or two
// aligned 16-byte loads and a selection.  `a` must be the same in every
// thread of a warp for the selection not to diverge; the caller makes sure
// that the aligned span [p - a, p - a + 8) is readable.
template <bool kC, typename T>
__device__ __forceinline__ void ldg4_shifted(const T* p, int32_t a, T (&o)[4]) {
  using V = typename Vec4<T>::type;
  const V* q = reinterpret_cast<const V*>(p - a);
  const V v0 = kC ? __ldcg(q) : __ldg(q);
  if (a == 0) {
    o[0] = v0.x, o[1] = v0.y, o[2] = v0.z, o[3] = v0.w;
    return;
  }
  const V v1 = kC ? __ldcg(q + 1) : __ldg(q + 1);
  switch (a) {
    case 1:
      o[0] = v0.y, o[1] = v0.z, o[2] = v0.w, o[3] = v1.x;
      break;
    case 2:
      o[0] = v0.z, o[1] = v0.w, o[2] = v1.x, o[3] = v1.y;
      break;
    default:
      o[0] = v0.w, o[1] = v1.x, o[2] = v1.y, o[3] = v1.z;
      break;
  }
}

// The R slopes of one (group, k) at columns j .. j + 3: child e is shared
// row `row0 + e * M` (row0 = group * R * M + k), read from column j + e k.
template <int R, int M, int A, typename T>
__device__ __forceinline__ void by_item(const T* S, int32_t row0, int32_t k, int32_t j, T (&out)[R][4]) {
  T c[8][16];
#pragma unroll
  for (int e = 0; e < R; e++) {
    const T* src = S + (row0 + e * M) * kVPitch + j + e * k - v_misalign(e, A);
#pragma unroll
    for (int v = 0; v < v_nvec(e, A); v++) lds4<T>(src + 4 * v, &c[e][4 * v]);
  }
  by_regs<R, 4, 0, A, T>(c, out);
}

// Stage the window of rows [8 w, 8 w + 8) of the block (warp w stages the
// rows its first pass merges, so no CTA barrier is needed before that pass):
// block row r = view row a + r, window column z = view column x0 + z,
// z in [0, kVWin), wrapped (cyclic) or zero outside [0, L) (extended), with
// the quadrant's transpose / column reversal.
template <typename InT, typename AccT>
__device__ __forceinline__ void v_stage(const InT* __restrict__ in, int64_t pitch, const QuadDesc& Q, int32_t a,
                                        int32_t x0, AccT* S) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!Q.transpose) {
    // lanes along the window columns; all 64 loads of a lane in flight
    // before its shared stores
    const bool inside = x0 >= 0 && x0 + kVWin <= Q.L;
    AccT v[8][kVWin / 32];
#pragma unroll
    for (int rr = 0; rr < 8; rr++) {
      const InT* __restrict__ rowp = in + (int64_t)(a + 8 * warp + rr) * pitch;
      if (inside) {
        const InT* __restrict__ src = Q.flip ? rowp + (Q.L - 1 - x0 - lane) : rowp + x0 + lane;
        const int32_t step = Q.flip ? -32 : 32;
#pragma unroll
        for (int c = 0; c < kVWin / 32; c++) v[rr][c] = (AccT)__ldg(src + c * step);
      } else {
#pragma unroll
        for (int c = 0; c < kVWin / 32; c++) v[rr][c] = load_view_elem<InT, AccT>(rowp, Q, x0 + 32 * c + lane);
      }
    }
#pragma unroll
    for (int rr = 0; rr < 8; rr++) {
      AccT* dst = S + (8 * warp + rr) * kVPitch + lane;
#pragma unroll
      for (int c = 0; c < kVWin / 32; c++) dst[32 * c] = v[rr][c];
    }
  } else {
    // transposed view: block row r is image column a + r, window column z an
    // image row.  Lane = (r & 7) + 8 (z & 3): a warp instruction reads 32
    // bytes of four image rows and writes 8 rows x 4 columns of shared memory
    // (distinct banks: kVPitch / 4 is odd).
    const int32_t rl = lane & 7, zl = lane >> 3;
    const int32_t r = 8 * warp + rl;
    const bool inside = x0 >= 0 && x0 + kVWin <= Q.L;
#pragma unroll 1
    for (int zb = 0; zb < kVWin; zb += 128) {
      AccT v[32];
      if (inside) {
        // image rows z0, z0 + 4, ... (reversed for the leftward quadrant)
        const int32_t z0 = x0 + zb + zl;
        const InT* __restrict__ src = in + (int64_t)(Q.flip ? Q.L - 1 - z0 : z0) * pitch + a + r;
        const int64_t step = Q.flip ? -4 * pitch : 4 * pitch;
#pragma unroll
        for (int c = 0; c < 32; c++) v[c] = (AccT)__ldg(src + c * step);
      } else {
#pragma unroll
        for (int c = 0; c < 32; c++) {
          int32_t z = x0 + zb + 4 * c + zl;
          bool ok = true;
          if (Q.ext) {
            ok = z >= 0 && z < Q.L;
          } else if (z >= Q.L) {
            z = z < 2 * Q.L ? z - Q.L : z % Q.L;  // cyclic windows start at column >= 0
          }
          if (Q.flip) z = Q.L - 1 - z;
          v[c] = ok ? (AccT)__ldg(in + (int64_t)z * pitch + a + r) : AccT(0);
        }
      }
#pragma unroll
      for (int c = 0; c < 32; c++) S[r * kVPitch + zb + 4 * c + zl] = v[c];
    }
  }
}

// Band items: staged row r = g B + b holds row K = K0 + g of the band's block
// b, pre-shifted by K b (window column z reads block column x0 + K b + c_src
// + z), so that each group of B rows is then a B-row Brady-Yong transform.
// Warp w stages rows [8 w, 8 w + 8).
// kC: the block rows were written earlier in the same launch by other CTAs
// (persistent batched kernel): read them at L2, past L1.
template <bool kC, typename AccT>
__device__ __forceinline__ void v_stage_band(const AccT* __restrict__ ws, const FusedItem& it, const QuadDesc& Q,
                                             int32_t x0, AccT* S) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t lim = Q.ext ? it.wsrc : Q.W;
  AccT v[8][kVWin / 32];
#pragma unroll
  for (int rr = 0; rr < 8; rr++) {
    const int32_t r = 8 * warp + rr;
    const int32_t g = r / it.B, b = r - g * it.B;
    const int32_t K = it.K0 + g;
    const AccT* __restrict__ row = ws + it.src + (int64_t)(64 * b + K) * it.src_pitch;
    const int32_t base = x0 + K * b + it.c_src;  // >= 0 in the cyclic case
    if (base >= 0 && base + kVWin <= lim) {
#pragma unroll
      for (int c = 0; c < kVWin / 32; c++) v[rr][c] = ld_ws<kC>(row + base + 32 * c + lane);
    } else {
#pragma unroll
      for (int c = 0; c < kVWin / 32; c++) {
        int32_t z = base + 32 * c + lane;
        bool ok = true;
        if (Q.ext) {
          ok = z >= 0 && z < it.wsrc;
        } else if (z >= Q.W) {
          z = z < 2 * Q.W ? z - Q.W : z % Q.W;
        }
        v[rr][c] = ok ? ld_ws<kC>(row + z) : AccT(0);
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < 8; rr++) {
    AccT* dst = S + (8 * warp + rr) * kVPitch + lane;
#pragma unroll
    for (int c = 0; c < kVWin / 32; c++) dst[32 * c] = v[rr][c];
  }
}

// Store the R rows o[i] (slopes row0 + i of the item) at columns j .. j + 3 of
// the tile: 16-byte stores into node-local workspace rows, else element by
// element through the quadrant's column map (a root) and the tile's edge.
template <int R, typename AccT>
__device__ __forceinline__ void v_store(const FusedItem& it, const QuadDesc& Q, AccT* __restrict__ base,
                                        int32_t row0, int32_t u0, int32_t j, int32_t ncols, bool vec_ok,
                                        const AccT (&o)[R][4]) {
  const int64_t pitch = it.dst_pitch;
  AccT* row = base + (int64_t)row0 * pitch;
  if (vec_ok && j + 4 <= ncols) {
#pragma unroll
    for (int i = 0; i < R; i++) sts4<AccT>(row + i * pitch + u0 + j, o[i]);
  } else {
#pragma unroll
    for (int x = 0; x < 4; x++) {
      if (j + x >= ncols) break;
      int32_t X = u0 + j + x;
      if (it.final_) {
        X = Q.sigma * X + Q.kappa;
        if (X < 0) X += Q.W;
        if (X >= Q.W) X -= Q.W;
      }
#pragma unroll
      for (int i = 0; i < R; i++) row[i * pitch + X] = o[i][x];
    }
  }
}

// First pass, in place (groups of B >= 8 rows): the eight 8-row groups of the
// staged window become 8-row Brady-Yong blocks over columns [0, W1).  Warp w
// owns rows [8 w, 8 w + 8) (read and written by no other warp) and walks its
// columns left to right, 128 per step: a step reads up to 8 columns into the
// next step's range, which that step only overwrites later.
template <int W1, typename AccT>
__device__ __forceinline__ void v_pass1(AccT* S) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
  for (int32_t j0 = 0; j0 < W1; j0 += 128) {
    const int32_t j = j0 + 4 * lane;
    AccT o[8][4];
    if (j < W1) by_item<8, 1, 0, AccT>(S, 8 * warp, 0, j, o);
    __syncwarp();  // every lane's reads of this step before any lane's writes
    if (j < W1) {
#pragma unroll
      for (int i = 0; i < 8; i++) sts4<AccT>(S + (8 * warp + i) * kVPitch + j, o[i]);
    }
    __syncwarp();
  }
}

// Groups of B = R1 <= 8 rows: one pass, straight to global memory through
// `st(row0, j, o)` (rows row0 .. row0 + R1 - 1, tile columns j .. j + 3).
template <int R1, typename AccT, typename Store>
__device__ __forceinline__ void v_pass1_out(const AccT* S, int32_t ncols, Store st) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
  for (int32_t j0 = 0; j0 < kVTile; j0 += 128) {
    const int32_t j = j0 + 4 * lane;
    if (j >= ncols) break;
#pragma unroll 1
    for (int32_t sg = 0; sg < 8; sg += R1) {
      AccT o[R1][4];
      by_item<R1, 1, 0, AccT>(S, 8 * warp + sg, 0, j, o);
      st(8 * warp + sg, j, o);
    }
  }
}

// Second pass: in each group g of B = 8 R2 rows the R2 8-row blocks become
// the B-row block; slope R2 k + i reads child e at shared row g B + 8 e + k.
// Warp w computes k = w of every group.
template <int R2, int A, typename AccT, typename Store>
__device__ __forceinline__ void v_pass2_k(const AccT* S, int32_t k, int32_t ncols, Store& st) {
  const int32_t lane = threadIdx.x & 31;
  constexpr int B = 8 * R2;
#pragma unroll 1
  for (int32_t g = 0; g < 64 / B; g++) {
#pragma unroll 1
    for (int32_t j0 = 0; j0 < kVTile; j0 += 128) {
      const int32_t j = j0 + 4 * lane;
      if (j >= ncols) break;
      AccT o[R2][4];
      by_item<R2, 8, A, AccT>(S, g * B + k, k, j, o);
      st(g * B + R2 * k, j, o);
    }
  }
}

template <int R2, typename AccT, typename Store>
__device__ __forceinline__ void v_pass2(const AccT* S, int32_t ncols, Store st) {
  const int32_t k = threadIdx.x >> 5;
  switch (k & 3) {
    case 0:
      v_pass2_k<R2, 0, AccT>(S, k, ncols, st);
      break;
    case 1:
      v_pass2_k<R2, 1, AccT>(S, k, ncols, st);
      break;
    case 2:
      v_pass2_k<R2, 2, AccT>(S, k, ncols, st);
      break;
    default:
      v_pass2_k<R2, 3, AccT>(S, k, ncols, st);
      break;
  }
}

// The merges of a staged window whose groups are 2^L-row Brady-Yong blocks
// (L = 6: one 64-row block), over tile columns [0, ncols), run by kVThreads
// threads (warps 0 .. 7 of the CTA); the results leave through `st`.  `bar`
// synchronises the merging warps between the two passes; it returns false
// if its wait gave up, and then the second pass is skipped.
template <typename AccT, typename Bar, typename Store>
__device__ __forceinline__ bool v_merge_groups(AccT* S, int32_t L, int32_t ncols, Bar bar, Store st) {
  switch (L) {
    case 6:
      v_pass1<kVTile + 56, AccT>(S);
      if (!bar()) return false;
      v_pass2<8, AccT>(S, ncols, st);
      break;
    case 5:
      v_pass1<kVTile + 24, AccT>(S);
      if (!bar()) return false;
      v_pass2<4, AccT>(S, ncols, st);
      break;
    case 4:
      v_pass1<kVTile + 8, AccT>(S);
      if (!bar()) return false;
      v_pass2<2, AccT>(S, ncols, st);
      break;
    case 3:
      v_pass1_out<8, AccT>(S, ncols, st);
      break;
    case 2:
      v_pass1_out<4, AccT>(S, ncols, st);
      break;
    default:
      v_pass1_out<2, AccT>(S, ncols, st);
      break;
  }
  return true;
}

// The forward merges of one staged 64-row block (FUSED_BY64) or band item
// (FUSED_BAND: groups of 2^L rows) x one tile of kVTile columns, stored as
// the item's Hough rows (node-local workspace columns, or the output through
// the quadrant's column map).
template <typename AccT, typename Bar>
__device__ __forceinline__ bool v_merge(const FusedParams& p, const FusedItem& it, const QuadDesc& Q, int32_t tile,
                                        AccT* S, Bar bar) {
  const int32_t u0 = tile * kVTile;
  const int32_t ncols = min(kVTile, it.wn - u0);
  AccT* __restrict__ base = (it.final_ ? static_cast<AccT*>(p.out) : static_cast<AccT*>(p.ws)) + it.dst;
  // 16-byte stores need node-local columns (no output map) on 16-byte aligned rows
  const bool vec_ok = !it.final_ && ((it.dst | (int64_t)it.dst_pitch) & 3) == 0 &&
                      (reinterpret_cast<uintptr_t>(p.ws) & 15) == 0;
  return v_merge_groups<AccT>(S, it.L, ncols, bar, [&](int32_t row0, int32_t j, const auto& o) {
    constexpr int R = sizeof(o) / sizeof(o[0]);
    v_store<R, AccT>(it, Q, base, row0, u0, j, ncols, vec_ok, o);
  });
}

// One item x one tile, staged by the merging warps themselves (each stages
// the rows its first pass merges).
template <bool kC, typename InT, typename AccT>
__device__ __forceinline__ void v_block(const FusedParams& p, const FusedItem& it, const QuadDesc& Q, int32_t tile,
                                        AccT* S) {
  const int32_t x0 = tile * kVTile - it.c;
  if (it.kind == FUSED_BAND) {
    v_stage_band<kC, AccT>(static_cast<const AccT*>(p.ws), it, Q, x0, S);
  } else {
    v_stage<InT, AccT>(static_cast<const InT*>(p.in), p.in_pitch, Q, it.a, x0, S);
  }
  __syncwarp();
  v_merge<AccT>(p, it, Q, tile, S, [] {
    __syncthreads();
    return true;
  });
}

}  // namespace fht
