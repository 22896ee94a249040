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

#include "fht_desc.h"
#include "fht_launch.hpp"

namespace fht {

struct FusedParams {
  const void* in;
  int64_t in_pitch;
  void* ws;   // AccT workspace base (after the header)
  void* out;  // AccT output
  const FusedItem* items;
  const MergeOp* ops;
  QuadDesc quad[4];
  int32_t TW;
  int32_t RP;  // shared row pitch (elements)
  int32_t Fm;  // rows per shared buffer
};

template <typename InT, typename AccT>
__device__ __forceinline__ AccT view_load(const InT* __restrict__ in, int64_t pitch, const QuadDesc& Q, int32_t i,
                                          int32_t z) {
  // z: view column, already reduced to [0, L) (cyclic) or checked (extended)
  if (Q.flip) z = Q.L - 1 - z;
  const InT v = Q.transpose ? in[(int64_t)z * pitch + i] : in[(int64_t)i * pitch + z];
  return (AccT)v;
}

template <typename InT, typename AccT>
__global__ void __launch_bounds__(512, 1) fused_kernel(FusedParams p) {
  const FusedItem it = p.items[blockIdx.x];
  const int32_t tile = blockIdx.y;
  if (tile >= it.ntiles) return;
  const QuadDesc& Q = p.quad[it.q];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AccT* bufA = reinterpret_cast<AccT*>(smem_raw);
  AccT* bufB = bufA + (size_t)p.Fm * p.RP;
  const InT* __restrict__ in = static_cast<const InT*>(p.in);

  const int32_t m = it.m;
  const int32_t TWin = p.TW + m - 1;
  const int32_t u0 = tile * p.TW;
  const int32_t x0 = u0 - it.c;  // first window column in view coordinates
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;

  // ---- stage the subtree's input rows ----
  // Loads are issued in batches of U per thread before their shared stores so
  // that several global loads are in flight per thread.
  constexpr int U = 8;
  if (!Q.transpose) {
    for (int32_t r = warp; r < m; r += nwarps) {
      AccT* dst = bufA + (size_t)r * p.RP;
      const int32_t row = it.a + r;
      for (int32_t j0 = 0; j0 < TWin; j0 += 32 * U) {
        AccT v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int32_t j = j0 + u * 32 + lane;
          int32_t z = x0 + j;
          bool ok = j < TWin;
          if (Q.ext) {
            ok = ok && z >= 0 && z < Q.L;
          } else if (z >= Q.L) {
            z = z < 2 * Q.L ? z - Q.L : z % Q.L;  // x0 >= 0 in the cyclic case
          }
          v[u] = ok ? view_load<InT, AccT>(in, p.in_pitch, Q, row, z) : AccT(0);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int32_t j = j0 + u * 32 + lane;
          if (j < TWin) dst[j] = v[u];
        }
      }
    }
  } else {
    // transposed view: view row r is image column a + r; lanes run along r so
    // that a warp reads consecutive image columns of one image row.
    for (int32_t j = warp; j < TWin; j += nwarps) {
      int32_t z = x0 + j;
      bool valid = true;
      if (Q.ext) {
        valid = (z >= 0 && z < Q.L);
      } else {
        z %= Q.L;
      }
      for (int32_t r = lane; r < m; r += 32)
        bufA[(size_t)r * p.RP + j] = valid ? view_load<InT, AccT>(in, p.in_pitch, Q, it.a + r, z) : AccT(0);
    }
  }

  // ---- merges, level by level (Algorithm 1's merge on the shared window) ----
  AccT* src = bufA;
  AccT* dst = bufB;
  const MergeOp* prog = p.ops + it.prog;
  for (int32_t lev = 0; lev < it.nlev; lev++) {
    __syncthreads();
    const MergeOp* ops = prog + (size_t)lev * m;
    for (int32_t r = warp; r < m; r += nwarps) {
      const MergeOp op = ops[r];
      AccT* d = dst + (size_t)r * p.RP;
      const AccT* a = src + (size_t)op.top * p.RP;
      if (op.bot >= 0) {
        const AccT* b = src + (size_t)op.bot * p.RP + op.s;
#pragma unroll 4
        for (int32_t j = lane; j < TWin; j += 32) d[j] = a[j] + b[j];
      } else {
#pragma unroll 4
        for (int32_t j = lane; j < TWin; j += 32) d[j] = a[j];
      }
    }
    AccT* tmp = src;
    src = dst;
    dst = tmp;
  }
  __syncthreads();

  // ---- store the subtree's Hough rows (columns [u0, u0 + TW) of the node) ----
  const int32_t ncols = min(p.TW, it.wn - u0);
  if (!it.final_) {
    AccT* __restrict__ ws = static_cast<AccT*>(p.ws) + it.dst;
    for (int32_t r = warp; r < m; r += nwarps) {
      const AccT* s = src + (size_t)r * p.RP;
      AccT* o = ws + (int64_t)r * it.dst_pitch + u0;
      for (int32_t j = lane; j < ncols; j += 32) o[j] = s[j];
    }
  } else {
    AccT* __restrict__ out = static_cast<AccT*>(p.out) + it.dst;
    for (int32_t r = warp; r < m; r += nwarps) {
      const AccT* s = src + (size_t)r * p.RP;
      AccT* o = out + (int64_t)r * it.dst_pitch;
      for (int32_t j = lane; j < ncols; j += 32) {
        int32_t X = Q.sigma * (u0 + j) + Q.kappa;
        if (X < 0) X += Q.W;
        if (X >= Q.W) X -= Q.W;
        o[X] = s[j];
      }
    }
  }
}

template <typename AccT>
__device__ __forceinline__ void store_row(AccT* dst, const RowJob& J, bool fin, int32_t u, AccT v) {
  if (fin) {
    int32_t X = (J.flags & ROW_NEG) ? J.kappa - u : u + J.kappa;
    if (X < 0) X += J.W;
    if (X >= J.W) X -= J.W;
    dst[X] = v;
  } else {
    dst[u] = v;
  }
}

// One CTA per output row; every thread keeps U independent element pairs in
// flight (all loads issued before the adds and stores).
template <typename AccT>
__global__ void __launch_bounds__(256) upper_kernel(const RowJob* __restrict__ rows, int64_t nrows,
                                                   const AccT* __restrict__ ws_in, AccT* ws_out, AccT* out) {
  constexpr int U = 8;
  for (int64_t k = blockIdx.x; k < nrows; k += gridDim.x) {
    const RowJob J = rows[k];
    const AccT* __restrict__ top = ws_in + J.top;
    const AccT* __restrict__ bot = ws_in + J.bot;
    const bool fin = J.flags & ROW_FINAL;
    const bool ext = J.flags & ROW_EXT;
    AccT* dst = (fin ? out : ws_out) + J.dst;
    for (int32_t u0 = 0; u0 < J.wout; u0 += (int32_t)blockDim.x * U) {
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

// ------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------
void fused_geometry(const HostPlan& P, int32_t& rp, size_t& smem) {
  // a window of TW + m - 1 columns, plus room for the largest shifted read
  const int32_t Fm = P.max_fused_m;
  rp = P.cfg.TW + Fm - 1 + P.max_fused_shift;
  if (rp % 2 == 0) rp++;  // odd pitch: column-wise (transposed) staging is conflict-free
  smem = (size_t)2 * Fm * rp * P.acc_size;
}

int32_t forward_launches(const HostPlan& P) { return 1 + (int32_t)P.pass_bytes.size(); }

void forward_launch_info(const HostPlan& P, int32_t k, int32_t& kind, int64_t& bytes) {
  if (k == 0) {
    kind = 0;
    bytes = P.fused_bytes;
  } else {
    kind = 1;
    bytes = P.pass_bytes[k - 1];
  }
}

template <typename InT, typename AccT>
static cudaError_t launch_forward_t(const DevicePlan& D, const void* in, int64_t in_pitch, void* out, void* ws,
                                    cudaStream_t st, cudaEvent_t* ev) {
  int32_t launch = 0;
  auto mark = [&](int which) {
    if (ev) cudaEventRecord(ev[2 * launch + which], st);
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
  fp.TW = P.cfg.TW;
  fp.RP = D.fused_rp;
  fp.Fm = P.max_fused_m;
  const size_t smem = D.fused_smem;
  auto kfn = fused_kernel<InT, AccT>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)P.fused.size(), P.max_ntiles);  // tiles <= 131070 / 32 fit in grid.y
  mark(0);
  kfn<<<grid, P.cfg.threads, smem, st>>>(fp);
  mark(1);
  launch++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (size_t p = 0; p + 1 < P.pass_begin.size(); p++) {
    const int64_t b = P.pass_begin[p], n = P.pass_begin[p + 1] - b;
    if (n <= 0) continue;
    const unsigned blocks = (unsigned)std::min<int64_t>(n, 1 << 30);
    mark(0);
    upper_kernel<AccT><<<blocks, 256, 0, st>>>(D.rows + b, n, wsa, wsa, static_cast<AccT*>(out));
    mark(1);
    launch++;
    e = cudaGetLastError();
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
