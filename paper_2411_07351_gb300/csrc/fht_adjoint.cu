// Adjoint (back-projection) kernels: the exact transpose of the forward
// schedule of fht_forward.cu, run in reverse.
//
// Forward merge (Algorithm 1):  J(t)[u] = R0(t1)[u + dtop] + R1(t2)[u + dbot(t)].
// Its transpose sends the gradient of J(t) back to R0(t1) and, shifted the
// other way, to R1(t2).  Written as gathers (no atomics, fixed summation
// order, so results are deterministic):
//   * adj_upper_kernel: one pass per upper tree height, highest first; each
//     child row sums the parent rows that read it (a contiguous range of t).
//   * adj_fused_kernel: each fused subtree's levels in reverse in shared
//     memory, over a window of tile + m - 1 columns with the halo on the
//     left (a pixel is read by outputs at columns up to m - 1 to its left).
//   * adj_sum_kernel: the per-quadrant image gradients are summed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fht_block.cuh"
#include "fht_desc.h"
#include "fht_launch.hpp"
#include "fht_nvtx.hpp"

namespace fht {

struct AdjFusedParams {
  const void* gout;  // AccT output gradient
  void* ws;          // AccT workspace base (after the header)
  const FusedItem* items;
  const int32_t* aptr;
  const MergeOp* aops;
  QuadDesc quad[4];
  int32_t h, w;
  int32_t TW;
  int32_t RP;    // shared row pitch
  int32_t PADL;  // left pad of every shared row (largest shift)
  int32_t Fm;
};

__device__ __forceinline__ int32_t wrap_mod(int32_t x, int32_t W) {
  int32_t r = x % W;
  return r < 0 ? r + W : r;
}

template <typename AccT>
__global__ void __launch_bounds__(512, 1) adj_fused_kernel(AdjFusedParams p) {
  const FusedItem it = p.items[blockIdx.x];
  const int32_t tile = blockIdx.y;
  if (tile >= it.antiles) return;
  const QuadDesc& Q = p.quad[it.q];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AccT* bufA = reinterpret_cast<AccT*>(smem_raw);
  AccT* bufB = bufA + (size_t)p.Fm * p.RP;
  const AccT* __restrict__ gout = static_cast<const AccT*>(p.gout);
  AccT* __restrict__ ws = static_cast<AccT*>(p.ws);

  const int32_t m = it.m;
  const int32_t TZin = p.TW + m - 1;
  const int32_t z0 = tile * p.TW;
  const int32_t xs = z0 - (m - 1);  // window start in node x coordinates
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;

  // ---- stage the gradient of the subtree's Hough rows ----
  constexpr int U = 8;
  for (int32_t r = warp; r < m; r += nwarps) {
    AccT* dst = bufA + (size_t)r * p.RP + p.PADL;
    for (int32_t j0 = 0; j0 < TZin; j0 += 32 * U) {
      AccT v[U];
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int32_t j = j0 + q * 32 + lane;
        v[q] = AccT(0);
        if (j < TZin) {
          int32_t u = xs + j + it.c;
          bool ok = true;
          if (Q.ext) {
            ok = u >= 0 && u < it.wn;
          } else {
            u = wrap_mod(u, Q.W);
          }
          if (ok) {
            if (it.final_) {
              int32_t X = Q.sigma * u + Q.kappa;
              if (X < 0) X += Q.W;
              if (X >= Q.W) X -= Q.W;
              v[q] = gout[it.dst + (int64_t)r * Q.W + X];
            } else {
              v[q] = ws[it.dst + (int64_t)r * it.dst_pitch + u];
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int32_t j = j0 + q * 32 + lane;
        if (j < TZin) dst[j] = v[q];
      }
    }
  }

  // ---- the subtree's merges in reverse ----
  AccT* src = bufA;
  AccT* dst = bufB;
  for (int32_t lev = it.nlev - 1; lev >= 0; lev--) {
    __syncthreads();
    const int32_t* ptr = p.aptr + it.aprog + (size_t)lev * (m + 1);
    for (int32_t k = warp; k < m; k += nwarps) {
      const int32_t b = ptr[k], e = ptr[k + 1];
      AccT* d = dst + (size_t)k * p.RP + p.PADL;
      // one or two parent rows (a Brady-Yong level) with their row pointers
      // taken once; the sum runs over the terms in the same order either way
      if (e - b == 1) {
        const MergeOp o0 = p.aops[b];
        const AccT* s0 = src + (size_t)o0.top * p.RP + p.PADL - o0.s;
        for (int32_t j = lane; j < TZin; j += 32) d[j] = AccT(0) + s0[j];
      } else if (e - b == 2) {
        const MergeOp o0 = p.aops[b], o1 = p.aops[b + 1];
        const AccT* s0 = src + (size_t)o0.top * p.RP + p.PADL - o0.s;
        const AccT* s1 = src + (size_t)o1.top * p.RP + p.PADL - o1.s;
        for (int32_t j = lane; j < TZin; j += 32) d[j] = (AccT(0) + s0[j]) + s1[j];
      } else {
        for (int32_t j = lane; j < TZin; j += 32) {
          AccT acc = AccT(0);
          for (int32_t t = b; t < e; t++) {
            const MergeOp op = p.aops[t];
            acc += src[(size_t)op.top * p.RP + p.PADL + j - op.s];
          }
          d[j] = acc;
        }
      }
    }
    AccT* tmp = src;
    src = dst;
    dst = tmp;
  }
  __syncthreads();

  // ---- leaf gradients: window columns [m - 1, TZin) are view columns [z0, z0 + TW) ----
  AccT* __restrict__ gq = ws + Q.grad_off;
  const int64_t gp = grad_pitch(Q.L);
  for (int32_t r = warp; r < m; r += nwarps) {
    const AccT* s = src + (size_t)r * p.RP + p.PADL + (m - 1);
    AccT* o = gq + (int64_t)(it.a + r) * gp + z0;
    for (int32_t jj = lane; jj < p.TW; jj += 32)
      if (z0 + jj < Q.L) o[jj] = s[jj];
  }
}

// Adjoint of a 64-row Brady-Yong block on the register-tiled path.  The
// forward block is H[t][u] = sum_y V[a + y][u - c + p_t(y)]; its transpose is
// gV[a + y][z] = sum_t g[t][z + c - p_t(y)].  The power-of-two pattern matrix
// is symmetric (p_t(y) = p_y(t)), so with the tile's columns reversed,
// z' = z0 + kVTile - 1 - z and g~[t][v] = g[t][c + z0 + kVTile - 1 - v],
//     gV[a + y][z] = sum_t g~[t][z' + p_y(t)],
// the forward block transform of g~ read at slope y.  One CTA = one block x
// one tile of kVTile view columns: the 64 gradient rows are staged reversed,
// merged exactly as the forward merges its window, and stored back reversed
// into the quadrant's view gradient (a thread's four tile columns j .. j + 3
// are the view columns z0 + kVTile - 4 - j .. z0 + kVTile - 1 - j, one
// 16-byte aligned run of a row).
template <typename AccT>
__device__ __forceinline__ void adj_stage_rev(const AdjFusedParams& p, const FusedItem& it, const QuadDesc& Q,
                                              int32_t z0, AccT* S) {
  const AccT* __restrict__ gout = static_cast<const AccT*>(p.gout);
  const AccT* __restrict__ ws = static_cast<const AccT*>(p.ws);
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t K = it.c + z0 + kVTile - 1;  // u of window column 0
  AccT v[8][kVWin / 32];
#pragma unroll
  for (int rr = 0; rr < 8; rr++) {
    const int32_t t = 8 * warp + rr;
#pragma unroll
    for (int c = 0; c < kVWin / 32; c++) {
      int32_t u = K - (32 * c + lane);
      bool ok = true;
      if (Q.ext) {
        ok = u >= 0 && u < it.wn;
      } else {
        u = wrap_mod(u, Q.W);
      }
      AccT x = AccT(0);
      if (ok) {
        if (it.final_) {
          int32_t X = Q.sigma * u + Q.kappa;
          if (X < 0) X += Q.W;
          if (X >= Q.W) X -= Q.W;
          x = gout[it.dst + (int64_t)t * Q.W + X];
        } else {
          x = ws[it.dst + (int64_t)t * it.dst_pitch + u];
        }
      }
      v[rr][c] = x;
    }
  }
#pragma unroll
  for (int rr = 0; rr < 8; rr++) {
    AccT* dst = S + (8 * warp + rr) * kVPitch + lane;
#pragma unroll
    for (int c = 0; c < kVWin / 32; c++) dst[32 * c] = v[rr][c];
  }
}

template <typename AccT>
__global__ void __launch_bounds__(kVThreads, 3) adj_block_kernel(AdjFusedParams p) {
  const FusedItem it = p.items[blockIdx.x];
  const QuadDesc& Q = p.quad[it.q];
  const int32_t z0 = blockIdx.y * kVTile;
  if (z0 >= Q.L) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AccT* S = reinterpret_cast<AccT*>(smem_raw);
  adj_stage_rev<AccT>(p, it, Q, z0, S);
  __syncwarp();
  AccT* __restrict__ gq = static_cast<AccT*>(p.ws) + Q.grad_off;
  const int64_t gp = grad_pitch(Q.L);
  v_merge_groups<AccT>(S, 6, kVTile, [] {
    __syncthreads();
    return true;
  }, [&](int32_t row0, int32_t j, const auto& o) {
    constexpr int R = sizeof(o) / sizeof(o[0]);
    // z0, kVTile and j are multiples of 4, so zs is; zs < L keeps the run
    // inside the row's grad_pitch(L) elements (a run past L writes slack)
    const int32_t zs = z0 + kVTile - 4 - j;
    if (zs >= Q.L) return;
#pragma unroll
    for (int i = 0; i < R; i++) {
      const AccT v[4] = {o[i][3], o[i][2], o[i][1], o[i][0]};
      sts4<AccT>(gq + (int64_t)(it.a + row0 + i) * gp + zs, v);
    }
  });
}

template <typename AccT>
__global__ void __launch_bounds__(256) adj_upper_kernel(const AdjRow* __restrict__ rows, int64_t nrows,
                                                       const AdjTerm* __restrict__ terms, const AccT* ws_in,
                                                       AccT* ws_out, const AccT* __restrict__ gout) {
  // every thread sums U elements of the row; each term is read once per U
  // elements, and every element still adds its terms in order
  constexpr int U = 4;
  for (int64_t k = blockIdx.x; k < nrows; k += gridDim.x) {
    const AdjRow R = rows[k];
    const bool fin = R.flags & ROW_FINAL;
    const bool ext = R.flags & ROW_EXT;
    const bool neg = R.flags & ROW_NEG;
    const AccT* src = (fin ? gout : ws_in) + R.src;
    AccT* dst = ws_out + R.dst;
    int32_t i0 = 0;
    if constexpr (sizeof(AccT) == 4) {
      // 16-byte path: four consecutive columns per thread, for chunks where
      // every term's columns lie inside its parent row (no cyclic wrap) and,
      // for a root row read through the column map X = (sigma u + kappa) mod W,
      // the chunk's X are one contiguous run (ascending for sigma = +1,
      // descending for sigma = -1) at least 8 elements from either end of the
      // row; the terms are added in the same order as below, so the results
      // are identical
      const int32_t C = (int32_t)blockDim.x * 4;
      const bool vec = (R.dst & 3) == 0;
      for (; vec && i0 + C <= R.wdst; i0 += C) {
        bool inside = true;
        for (int32_t c = 0; c < R.term_count && inside; c++) {
          const int32_t e = terms[R.term_begin + c].e;
          if (ext) {
            inside = i0 + e >= 0 && i0 + C + e + (fin ? 0 : 8) <= R.wsrc;
          } else {
            inside = i0 + C + e + (fin ? 0 : 8) <= R.W;
          }
          if (inside && fin) {
            // X over u in [i0 + e, i0 + e + C): one run shifted by a multiple of W
            const int32_t lo = neg ? R.kappa - (i0 + e + C - 1) : i0 + e + R.kappa;
            const int32_t sh = lo >= R.W ? -R.W : lo < 0 ? R.W : 0;
            inside = lo + sh >= 8 && lo + sh + C + 8 <= R.W;
          }
        }
        if (!inside) break;
        const int32_t i = i0 + 4 * (int32_t)threadIdx.x;
        AccT acc[4] = {AccT(0), AccT(0), AccT(0), AccT(0)};
        for (int32_t c = 0; c < R.term_count; c++) {
          const AdjTerm T = terms[R.term_begin + c];
          const int64_t row = R.src + (int64_t)T.t * R.src_pitch;  // element offset of the parent row
          AccT v[4];
          if (!fin) {
            ldg4_shifted<false, AccT>(src - R.src + row + T.e + i, (int32_t)((row + T.e) & 3), v);
#pragma unroll
            for (int q = 0; q < 4; q++) acc[q] += v[q];
          } else {
            const int32_t lo = neg ? R.kappa - (i0 + T.e + C - 1) : i0 + T.e + R.kappa;
            const int32_t sh = lo >= R.W ? -R.W : lo < 0 ? R.W : 0;
            if (!neg) {
              const int32_t X = i + T.e + R.kappa + sh;  // columns X .. X + 3
              ldg4_shifted<false, AccT>(src - R.src + row + X, (int32_t)((row + R.kappa + sh + T.e) & 3), v);
#pragma unroll
              for (int q = 0; q < 4; q++) acc[q] += v[q];
            } else {
              const int32_t X = R.kappa - (i + T.e) + sh - 3;  // columns X .. X + 3, read backwards
              ldg4_shifted<false, AccT>(src - R.src + row + X, (int32_t)((row + R.kappa + sh - T.e - 3) & 3), v);
#pragma unroll
              for (int q = 0; q < 4; q++) acc[q] += v[3 - q];
            }
          }
        }
        sts4<AccT>(dst + i, acc);
      }
    }
    for (; i0 < R.wdst; i0 += (int32_t)blockDim.x * U) {
      AccT acc[U];
#pragma unroll
      for (int q = 0; q < U; q++) acc[q] = AccT(0);
      for (int32_t c = 0; c < R.term_count; c++) {
        const AdjTerm T = terms[R.term_begin + c];
        const AccT* srow = src + (int64_t)T.t * R.src_pitch;
#pragma unroll
        for (int q = 0; q < U; q++) {
          const int32_t i = i0 + q * (int32_t)blockDim.x + (int32_t)threadIdx.x;
          if (i >= R.wdst) continue;
          int32_t u = i + T.e;
          if (ext) {
            if (u < 0 || u >= R.wsrc) continue;
          } else if (u >= R.W) {
            u -= R.W;
          }
          if (fin) {
            int32_t X = neg ? R.kappa - u : u + R.kappa;
            if (X < 0) X += R.W;
            if (X >= R.W) X -= R.W;
            u = X;
          }
          acc[q] += srow[u];
        }
      }
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int32_t i = i0 + q * (int32_t)blockDim.x + (int32_t)threadIdx.x;
        if (i < R.wdst) dst[i] = acc[q];
      }
    }
  }
}

// The quadrants' view gradients summed into the image gradient.  Quadrant q
// holds gV_q[r][z] (n rows of pitch grad_pitch(L)); image element (y, x) is
// view element (y, x~) of the untransposed quadrants and (x, y~) of the
// transposed ones, with ~ the column reversal of the leftward quadrants.  One
// CTA = one 32 x 32 image tile: untransposed views are read along image rows,
// transposed ones along image columns (coalesced view rows) and turned
// through shared memory.  Every thread issues all its quadrants' loads before
// the one barrier (up to 16 in flight), then every element adds its quadrants
// in order q = 0..3.
struct AdjSumQuad {
  int64_t off;  // element offset of the view gradient in the workspace
  int32_t pitch, L, transpose, flip;
};
struct AdjSumParams {
  AdjSumQuad q[4];
  int32_t nq, h, w;
  int64_t pitch;  // elements between image rows of gin
};

template <typename AccT>
__global__ void __launch_bounds__(256) adj_sum_kernel(const AccT* __restrict__ ws, AdjSumParams sp,
                                                      AccT* __restrict__ gin) {
  __shared__ AccT T[4][32][33];
  const int32_t tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int32_t x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, x = x0 + tx;
  AccT v[4][4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k >= sp.nq) break;
    const AdjSumQuad Q = sp.q[k];
    const AccT* __restrict__ g = ws + Q.off;
    if (!Q.transpose) {
      const int32_t z = Q.flip ? Q.L - 1 - x : x;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int32_t y = y0 + ty + 8 * i;
        v[k][i] = (x < sp.w && y < sp.h) ? g[(int64_t)y * Q.pitch + z] : AccT(0);
      }
    } else {
      // T[k][a][b] = view row x0 + a at the column of image row y0 + b
      const int32_t yb = y0 + tx;
      const int32_t z = Q.flip ? Q.L - 1 - yb : yb;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int32_t xr = x0 + ty + 8 * i;
        T[k][ty + 8 * i][tx] = (xr < sp.w && yb < sp.h) ? g[(int64_t)xr * Q.pitch + z] : AccT(0);
      }
    }
  }
  __syncthreads();
  AccT acc[4] = {AccT(0), AccT(0), AccT(0), AccT(0)};
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k >= sp.nq) break;
#pragma unroll
    for (int i = 0; i < 4; i++) acc[i] += sp.q[k].transpose ? T[k][tx][ty + 8 * i] : v[k][i];
  }
  if (x >= sp.w) return;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int32_t y = y0 + ty + 8 * i;
    if (y < sp.h) gin[(int64_t)y * sp.pitch + x] = acc[i];
  }
}

void adjoint_geometry(const HostPlan& P, int32_t& rp, int32_t& padl, size_t& smem) {
  const int32_t Fm = P.max_fused_m;
  padl = P.max_fused_shift;
  rp = padl + P.adj_tw + Fm - 1;
  if (rp % 2 == 0) rp++;
  smem = (size_t)2 * Fm * rp * P.acc_size;
}

template <typename AccT>
static cudaError_t launch_adjoint_t(const DevicePlan& D, const void* gout, void* gin, int64_t gin_pitch, void* ws,
                                    cudaStream_t st) {
  const HostPlan& P = *D.host;
  NvtxRange nv("fht adjoint");
  AccT* wsa = reinterpret_cast<AccT*>(static_cast<unsigned char*>(ws) + kWsHeader);
  cudaError_t e;
  for (size_t p = 0; p + 1 < P.apass_begin.size(); p++) {
    const int64_t b = P.apass_begin[p], n = P.apass_begin[p + 1] - b;
    if (n <= 0) continue;
    const unsigned blocks = (unsigned)std::min<int64_t>(n, 1 << 30);
    adj_upper_kernel<AccT><<<blocks, 256, 0, st>>>(D.arows + b, n, D.aterms, wsa, wsa,
                                                   static_cast<const AccT*>(gout));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  AdjFusedParams fp;
  fp.gout = gout;
  fp.ws = wsa;
  fp.items = D.fused;
  fp.aptr = D.aptr;
  fp.aops = D.aops;
  for (int q = 0; q < 4; q++) fp.quad[q] = P.quad[q];
  fp.h = P.cfg.h;
  fp.w = P.cfg.w;
  fp.TW = P.adj_tw;
  int32_t rp, padl;
  size_t smem;
  adjoint_geometry(P, rp, padl, smem);
  fp.RP = rp;
  fp.PADL = padl;
  fp.Fm = P.max_fused_m;
  auto kfn = adj_fused_kernel<AccT>;
  if ((e = raise_smem_limit(kfn, smem)) != cudaSuccess)
    return e;
  // 4-byte accumulators: the 64-row blocks on the register-tiled path, the
  // generic subtrees (sorted first) on the shared-memory path
  const bool vblocks = sizeof(AccT) == 4 && P.n_by64 > 0;
  const unsigned nfused = vblocks ? (unsigned)P.n_generic : (unsigned)P.fused.size();
  if (nfused > 0) {
    dim3 grid(nfused, P.max_antiles);
    kfn<<<grid, P.adj_threads, smem, st>>>(fp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if constexpr (sizeof(AccT) == 4) {
    if (vblocks) {
      int32_t maxL = 1;
      for (int q = 0; q < 4; q++)
        if (P.cfg.quads & (1u << q)) maxL = std::max(maxL, P.quad[q].L);
      const size_t vsmem = (size_t)64 * kVPitch * sizeof(AccT);
      auto kbl = adj_block_kernel<AccT>;
      if ((e = raise_smem_limit(kbl, vsmem)) != cudaSuccess) return e;
      AdjFusedParams bp = fp;
      bp.items = D.fused + P.n_generic;
      kbl<<<dim3((unsigned)P.n_by64, (unsigned)((maxL + kVTile - 1) / kVTile)), kVThreads, vsmem, st>>>(bp);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  AdjSumParams sp{};
  for (int q = 0; q < 4; q++) {
    if (!(P.cfg.quads & (1u << q))) continue;
    const QuadDesc& Q = P.quad[q];
    sp.q[sp.nq++] = AdjSumQuad{Q.grad_off, grad_pitch(Q.L), Q.L, Q.transpose, Q.flip};
  }
  sp.h = P.cfg.h;
  sp.w = P.cfg.w;
  sp.pitch = gin_pitch;
  const dim3 grid((unsigned)((P.cfg.w + 31) / 32), (unsigned)((P.cfg.h + 31) / 32));
  adj_sum_kernel<AccT><<<grid, 256, 0, st>>>(wsa, sp, static_cast<AccT*>(gin));
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const DevicePlan& D, const void* gout, void* gin, int64_t gin_pitch, void* ws,
                           cudaStream_t st) {
  switch (D.host->cfg.dtype) {
    case 0:
    case 1:
      return launch_adjoint_t<int32_t>(D, gout, gin, gin_pitch, ws, st);
    case 2:
      return launch_adjoint_t<float>(D, gout, gin, gin_pitch, ws, st);
    default:
      return launch_adjoint_t<double>(D, gout, gin, gin_pitch, ws, st);
  }
}

}  // namespace fht
