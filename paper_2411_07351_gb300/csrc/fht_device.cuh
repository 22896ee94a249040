// Device building blocks of the forward transform, shared by the plain
// kernels (fht_forward.cu) and the batched persistent kernel (batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fht_desc.h"

namespace fht {

// Loads of intermediate (workspace) data.  Plain kernels read data written
// by earlier launches and may use the read-only path; the persistent batch
// kernel reads data written earlier in the same launch by other SMs and must
// bypass L1 (cache at L2 only).
template <bool kCoherent, typename T>
__device__ __forceinline__ T ld_ws(const T* p) {
  if constexpr (kCoherent) {
    return __ldcg(p);
  } else {
    return __ldg(p);
  }
}

struct FusedParams {
  const void* in;
  int64_t in_pitch;
  void* ws;   // AccT workspace base (after the header)
  void* out;  // AccT output
  const FusedItem* items;
  const MergeOp* ops;
  QuadDesc quad[4];
  int32_t RP;  // generic path: shared row pitch (elements)
  int32_t Fm;  // generic path: rows per shared buffer
  int32_t RS;  // fast path: pitch of the staged input / level-4 rows
  int32_t RA;  // fast path: pitch of the level-2 rows
  int32_t vblock;  // the plan's 64-row blocks and bands take the register-tiled path (batched launch)
};

template <typename InT, typename AccT>
__device__ __forceinline__ AccT view_load(const InT* __restrict__ in, int64_t pitch, const QuadDesc& Q, int32_t i,
                                          int32_t z) {
  // z: view column, already reduced to [0, L) (cyclic) or checked (extended)
  if (Q.flip) z = Q.L - 1 - z;
  const InT v = Q.transpose ? in[(int64_t)z * pitch + i] : in[(int64_t)i * pitch + z];
  return (AccT)v;
}

// Stage m view rows [a, a + m) x window columns [x0, x0 + width) into
// buf (row pitch rp): wrapped (cyclic) or zero-filled (extended).  Each lane
// issues the loads of two rows (or four transposed columns) before any shared
// store, so a warp has up to 16 global loads per lane in flight.
template <typename InT, typename AccT>
__device__ __forceinline__ AccT load_view_elem(const InT* __restrict__ rowp, const QuadDesc& Q, int32_t z) {
  // z: window column in view coordinates (any integer)
  if (Q.ext) {
    if (z < 0 || z >= Q.L) return AccT(0);
  } else if (z >= Q.L) {
    z = z < 2 * Q.L ? z - Q.L : z % Q.L;  // z >= 0 in the cyclic case
  }
  if (Q.flip) z = Q.L - 1 - z;
  return (AccT)rowp[z];
}

template <typename InT, typename AccT>
__device__ __forceinline__ void stage_rows(const FusedParams& p, const QuadDesc& Q, int32_t a, int32_t m, int32_t x0,
                                           int32_t width, AccT* buf, int32_t rp) {
  const InT* __restrict__ in = static_cast<const InT*>(p.in);
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  constexpr int NCH = 8;  // 32-column chunks held per row (windows up to 256 columns in one sweep)
  if (!Q.transpose) {
    // the window needs no wrap and no zero fill: plain loads from one pointer
    const bool inside = x0 >= 0 && x0 + width <= Q.L;
    const int32_t step = Q.flip ? -1 : 1;
    for (int32_t jb = 0; jb < width; jb += 32 * NCH) {
      for (int32_t r0 = warp; r0 < m; r0 += 2 * nwarps) {
        AccT v[2][NCH];
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          const int32_t r = r0 + rr * nwarps;
          const InT* __restrict__ rowp = in + (int64_t)(a + min(r, m - 1)) * p.in_pitch;
          const InT* __restrict__ src = rowp + (Q.flip ? Q.L - 1 - x0 : x0) + step * (jb + lane);
#pragma unroll
          for (int c = 0; c < NCH; c++) {
            const int32_t j = jb + c * 32 + lane;
            const bool ok = r < m && j < width;
            if (inside) {
              v[rr][c] = ok ? (AccT)src[step * c * 32] : AccT(0);
            } else {
              v[rr][c] = ok ? load_view_elem<InT, AccT>(rowp, Q, x0 + j) : AccT(0);
            }
          }
        }
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          const int32_t r = r0 + rr * nwarps;
          if (r >= m) continue;
          AccT* dst = buf + (size_t)r * rp;
#pragma unroll
          for (int c = 0; c < NCH; c++) {
            const int32_t j = jb + c * 32 + lane;
            if (j < width) dst[j] = v[rr][c];
          }
        }
      }
    }
  } else {
    // transposed view: view row r is image column a + r, window column j is an
    // image row; lanes run along r so that a warp reads consecutive image
    // columns of one image row.
    constexpr int JB = 4;
    for (int32_t j0 = warp; j0 < width; j0 += JB * nwarps) {
      AccT v[JB][2];
#pragma unroll
      for (int jj = 0; jj < JB; jj++) {
        const int32_t j = j0 + jj * nwarps;
        int32_t z = x0 + j;
        bool valid = j < width;
        if (Q.ext) {
          valid = valid && z >= 0 && z < Q.L;
        } else {
          if (z >= Q.L) z = z < 2 * Q.L ? z - Q.L : z % Q.L;
        }
        if (Q.flip) z = Q.L - 1 - z;
        const InT* __restrict__ rowp = in + (int64_t)(valid ? z : 0) * p.in_pitch + a;
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          const int32_t r = lane + 32 * rr;
          v[jj][rr] = (valid && r < m) ? (AccT)rowp[r] : AccT(0);
        }
      }
#pragma unroll
      for (int jj = 0; jj < JB; jj++) {
        const int32_t j = j0 + jj * nwarps;
        if (j >= width) continue;
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          const int32_t r = lane + 32 * rr;
          if (r < m) buf[(size_t)r * rp + j] = v[jj][rr];
        }
      }
    }
  }
}

// Asynchronous copies into shared memory (cp.async): the copy engine of the
// SM writes shared memory directly, so a thread can have all of its staging
// copies in flight at once without holding them in registers.  With
// src_bytes = 0 nothing is read and the destination is zero-filled.
__device__ __forceinline__ void cp_async_4(void* smem_dst, const void* gmem_src, int32_t src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_8(void* smem_dst, const void* gmem_src, int32_t src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}

// 16-byte copy; the bytes past src_bytes are zero-filled (bypasses L1).
__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gmem_src, int32_t src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}

// ---- programmatic dependent launch ----
// A launch made with programmatic stream serialisation may start while the
// previous kernel on the stream drains; pdl_wait() blocks until that kernel
// has completed and its writes are visible (it returns at once in a launch
// made without the attribute).  pdl_launch_dependents() lets the next such
// launch start once every CTA of this kernel has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" :::); }

// ---- bulk copies (TMA unit) completing on a shared-memory mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrive once and expect `bytes` more from bulk copies before the phase completes.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Global -> shared bulk copy: both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(smem_dst)),
               "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void cp_async_elem_z(T* smem_dst, const T* gmem_src, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  if constexpr (sizeof(T) == 8) {
    cp_async_8(smem_dst, gmem_src, valid ? 8 : 0);
  } else {
    cp_async_4(smem_dst, gmem_src, valid ? 4 : 0);
  }
}

// stage_gathered with cp.async (plain kernels only: the copies go through L1,
// which the persistent batch kernel must not use for data written in the
// same launch).  Same layout as stage_gathered.
template <typename AccT>
__device__ __forceinline__ void stage_gathered_async(const FusedParams& p, const FusedItem& it, const QuadDesc& Q,
                                                     int32_t x0, int32_t width, AccT* buf, int32_t rp) {
  const AccT* __restrict__ ws = static_cast<const AccT*>(p.ws);
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  const int32_t lim = Q.ext ? it.wsrc : Q.W;
  for (int32_t r = warp; r < 64; r += nwarps) {
    const int32_t g = r / it.B, b = r - g * it.B;
    const int32_t K = it.K0 + g;
    const AccT* __restrict__ row = ws + it.src + (int64_t)(64 * b + K) * it.src_pitch;
    const int32_t base = x0 + K * b + it.c_src;  // >= 0 in the cyclic case
    AccT* dst = buf + (size_t)r * rp;
    if (base >= 0 && base + width <= lim) {
      for (int32_t j = lane; j < width; j += 32) cp_async_elem_z<AccT>(dst + j, row + base + j, true);
    } else {
      for (int32_t j = lane; j < width; j += 32) {
        int32_t z = base + j;
        bool ok = true;
        if (Q.ext) {
          ok = z >= 0 && z < it.wsrc;
        } else {
          if (z >= Q.W) z = z < 2 * Q.W ? z - Q.W : z % Q.W;  // z >= 0 in the cyclic case
        }
        cp_async_elem_z<AccT>(dst + j, ok ? row + z : row, ok);
      }
    }
  }
  cp_async_wait_all();
}

// stage_rows for a 64-row block and a compile-time window width: every lane
// issues all of its loads (RB rows x NCH chunks, or JB window columns x 2
// rows transposed) before its first shared store, so the whole window is one
// round trip to memory.  Same layout and boundary rules as stage_rows.
template <typename InT, typename AccT, int WIDTH, int RB>
__device__ __forceinline__ void stage_block_c(const FusedParams& p, const QuadDesc& Q, int32_t a, int32_t x0,
                                              AccT* buf, int32_t rp) {
  const InT* __restrict__ in = static_cast<const InT*>(p.in);
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  constexpr int NCH = (WIDTH + 31) / 32;
  if (!Q.transpose) {
    const bool inside = x0 >= 0 && x0 + WIDTH <= Q.L;
    const int32_t step = Q.flip ? -1 : 1;
    for (int32_t rb = warp * RB; rb < 64; rb += nwarps * RB) {
      AccT v[RB][NCH];
#pragma unroll
      for (int rr = 0; rr < RB; rr++) {
        const InT* __restrict__ rowp = in + (int64_t)(a + rb + rr) * p.in_pitch;
        const InT* __restrict__ src = rowp + (Q.flip ? Q.L - 1 - x0 : x0) + step * lane;
#pragma unroll
        for (int c = 0; c < NCH; c++) {
          const int32_t j = c * 32 + lane;
          const bool ok = (c + 1) * 32 <= WIDTH || j < WIDTH;
          if (inside) {
            v[rr][c] = ok ? (AccT)src[step * c * 32] : AccT(0);
          } else {
            v[rr][c] = ok ? load_view_elem<InT, AccT>(rowp, Q, x0 + j) : AccT(0);
          }
        }
      }
#pragma unroll
      for (int rr = 0; rr < RB; rr++) {
        AccT* dst = buf + (size_t)(rb + rr) * rp;
#pragma unroll
        for (int c = 0; c < NCH; c++) {
          const int32_t j = c * 32 + lane;
          if ((c + 1) * 32 <= WIDTH || j < WIDTH) dst[j] = v[rr][c];
        }
      }
    }
  } else {
    constexpr int JB = 2 * RB;  // window columns per lane and sweep
    for (int32_t j0 = warp; j0 < WIDTH; j0 += JB * nwarps) {
      AccT v[JB][2];
#pragma unroll
      for (int jj = 0; jj < JB; jj++) {
        const int32_t j = j0 + jj * nwarps;
        int32_t z = x0 + j;
        bool valid = j < WIDTH;
        if (Q.ext) {
          valid = valid && z >= 0 && z < Q.L;
        } else {
          if (z >= Q.L) z = z < 2 * Q.L ? z - Q.L : z % Q.L;
        }
        if (Q.flip) z = Q.L - 1 - z;
        const InT* __restrict__ rowp = in + (int64_t)(valid ? z : 0) * p.in_pitch + a;
        v[jj][0] = valid ? (AccT)rowp[lane] : AccT(0);
        v[jj][1] = valid ? (AccT)rowp[lane + 32] : AccT(0);
      }
#pragma unroll
      for (int jj = 0; jj < JB; jj++) {
        const int32_t j = j0 + jj * nwarps;
        if (j >= WIDTH) continue;
        buf[(size_t)lane * rp + j] = v[jj][0];
        buf[(size_t)(lane + 32) * rp + j] = v[jj][1];
      }
    }
  }
}

// Store rows [0, m) x columns [0, ncols) of a shared buffer as the node's
// Hough rows starting at node column u0.
template <typename AccT>
__device__ __forceinline__ void store_rows(const FusedParams& p, const FusedItem& it, const QuadDesc& Q,
                                           const AccT* buf, int32_t rp, int32_t u0, int32_t ncols) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  if (!it.final_) {
    AccT* __restrict__ ws = static_cast<AccT*>(p.ws) + it.dst;
    for (int32_t r = warp; r < it.m; r += nwarps) {
      const AccT* s = buf + (size_t)r * rp;
      AccT* o = ws + (int64_t)r * it.dst_pitch + u0;
      for (int32_t j = lane; j < ncols; j += 32) o[j] = s[j];
    }
  } else {
    AccT* __restrict__ out = static_cast<AccT*>(p.out) + it.dst;
    for (int32_t r = warp; r < it.m; r += nwarps) {
      const AccT* s = buf + (size_t)r * rp;
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

// Generic path: any subtree of at most F rows, run level by level from its
// program, ping-ponging between two shared buffers.
template <typename InT, typename AccT>
__device__ __forceinline__ void fused_generic(const FusedParams& p, const FusedItem& it, const QuadDesc& Q, int32_t tile,
                              AccT* bufA, AccT* bufB) {
  const int32_t m = it.m;
  const int32_t TWin = it.tw + m - 1;
  const int32_t u0 = tile * it.tw;
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  stage_rows<InT, AccT>(p, Q, it.a, m, u0 - it.c, TWin, bufA, p.RP);
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
  store_rows<AccT>(p, it, Q, src, p.RP, u0, min(it.tw, it.wn - u0));
}

// Two Brady-Yong levels at once: four m-row blocks Q0..Q3 (rows base + e m)
// become one 4m-row block.  With t'' = k and t = 4k + i, level by level
// (t' = floor(t/2), child slopes floor(t'/2), shifts ceil(t'/2), ceil(t/2)):
//   out[4k+i][j] = Q0[k][j] + Q1[k][j + k + b] + Q2[k][j + 2k + c]
//                + Q3[k][j + 3k + b + c],   b = floor(i/2), c = ceil(i/2),
// so the four outputs of one k need only ten shifted reads.  `rq` = g m + k
// indexes the 16 (block group, k) pairs of a 64-row block.
template <typename AccT>
__device__ __forceinline__ void merge4_at(const AccT* q0, const AccT* q1, const AccT* q2, const AccT* q3,
                                          int32_t j, AccT o[4]) {
  const AccT a0 = q0[j];
  const AccT b0 = q1[j], b1 = q1[j + 1];
  const AccT c0 = q2[j], c1 = q2[j + 1], c2 = q2[j + 2];
  const AccT d0 = q3[j], d1 = q3[j + 1], d2 = q3[j + 2], d3 = q3[j + 3];
  const AccT ab0 = a0 + b0, ab1 = a0 + b1;
  o[0] = ab0 + (c0 + d0);
  o[1] = ab0 + (c1 + d1);
  o[2] = ab1 + (c1 + d2);
  o[3] = ab1 + (c2 + d3);
}

// Source row pointers of row-quad rq for blocks of M rows (compile-time M).
template <int M, typename AccT>
__device__ __forceinline__ void merge4_ptrs(const AccT* src, int32_t rs, int32_t rq, const AccT*& q0,
                                            const AccT*& q1, const AccT*& q2, const AccT*& q3, int32_t& r0) {
  const int32_t g = rq / M, k = rq % M;  // M is a power of two known at compile time
  q0 = src + (g * 4 * M + k) * rs;
  q1 = q0 + M * rs + k;
  q2 = q0 + 2 * M * rs + 2 * k;
  q3 = q0 + 3 * M * rs + 3 * k;
  r0 = g * 4 * M + 4 * k;
}

template <int M, typename AccT>
__device__ __forceinline__ void merge4_pass(const AccT* src, int32_t rs, AccT* dst, int32_t rd, int32_t width) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  for (int32_t rq = warp; rq < 16; rq += nwarps) {
    const AccT *q0, *q1, *q2, *q3;
    int32_t r0;
    merge4_ptrs<M, AccT>(src, rs, rq, q0, q1, q2, q3, r0);
    AccT* d = dst + r0 * rd;
#pragma unroll 2
    for (int32_t j = lane; j < width; j += 32) {
      AccT o[4];
      merge4_at<AccT>(q0, q1, q2, q3, j, o);
      d[j] = o[0];
      d[rd + j] = o[1];
      d[2 * rd + j] = o[2];
      d[3 * rd + j] = o[3];
    }
  }
}

// One Brady-Yong level: two m-row blocks Q0, Q1 (rows base, base + m) become
// one 2m-row block: t = 2k + i has t1 = t2 = k and shift ceil(t/2) = k + i.
template <int M, typename AccT>
__device__ __forceinline__ void merge2_ptrs(const AccT* src, int32_t rs, int32_t rp, const AccT*& q0,
                                            const AccT*& q1, int32_t& r0) {
  const int32_t g = rp / M, k = rp % M;
  q0 = src + (g * 2 * M + k) * rs;
  q1 = q0 + M * rs + k;
  r0 = g * 2 * M + 2 * k;
}

template <int M, typename AccT>
__device__ __forceinline__ void merge2_pass(const AccT* src, int32_t rs, AccT* dst, int32_t rd, int32_t width) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  for (int32_t rp = warp; rp < 32; rp += nwarps) {
    const AccT *q0, *q1;
    int32_t r0;
    merge2_ptrs<M, AccT>(src, rs, rp, q0, q1, r0);
    AccT* d = dst + r0 * rd;
    for (int32_t j = lane; j < width; j += 32) {
      const AccT a = q0[j];
      d[j] = a + q1[j];
      d[rd + j] = a + q1[j + 1];
    }
  }
}

// Stage the 64 gathered rows of a band item: shared row r = g B + b holds
// row K = K0 + g of block b, pre-shifted by K b.  In a perfect band of B
// blocks the output slope t = K B + i sums, over the blocks, row K of block b
// at offset K b + pat_B(i)(b) (the Brady-Yong pattern of the B-row transform),
// so after this staging the band is a B-row Brady-Yong transform per group.
template <bool kC, typename AccT>
__device__ __forceinline__ void stage_gathered(const FusedParams& p, const FusedItem& it, const QuadDesc& Q,
                                               int32_t x0, int32_t width, AccT* buf, int32_t rp) {
  const AccT* __restrict__ ws = static_cast<const AccT*>(p.ws);
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  constexpr int NCH = 8;
  const int32_t lim = Q.ext ? it.wsrc : Q.W;
  for (int32_t jb = 0; jb < width; jb += 32 * NCH) {
    for (int32_t r0 = warp; r0 < 64; r0 += 2 * nwarps) {
      AccT v[2][NCH];
#pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int32_t r = min(r0 + rr * nwarps, 63);
        const bool rok = r0 + rr * nwarps < 64;
        const int32_t g = r / it.B, b = r - g * it.B;
        const int32_t K = it.K0 + g;
        const AccT* __restrict__ row = ws + it.src + (int64_t)(64 * b + K) * it.src_pitch;
        const int32_t base = x0 + K * b + it.c_src;  // >= 0 in the cyclic case
        const bool inside = base >= 0 && base + width <= lim;
#pragma unroll
        for (int c = 0; c < NCH; c++) {
          const int32_t j = jb + c * 32 + lane;
          int32_t z = base + j;
          bool ok = rok && j < width;
          if (!inside) {
            if (Q.ext) {
              ok = ok && z >= 0 && z < it.wsrc;
            } else {
              if (z >= Q.W) z = z < 2 * Q.W ? z - Q.W : z % Q.W;  // z >= 0 in the cyclic case
            }
          }
          v[rr][c] = ok ? ld_ws<kC>(row + z) : AccT(0);
        }
      }
#pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int32_t r = r0 + rr * nwarps;
        if (r >= 64) continue;
        AccT* dst = buf + (size_t)r * rp;
#pragma unroll
        for (int c = 0; c < NCH; c++) {
          const int32_t j = jb + c * 32 + lane;
          if (j < width) dst[j] = v[rr][c];
        }
      }
    }
  }
}

// Store the four (or two) outputs of one register group into global rows
// r0, r0 + 1, ... of the item's destination at node column u0 + j.
template <typename AccT, int N>
__device__ __forceinline__ void store_group(const FusedItem& it, const QuadDesc& Q, AccT* base, int32_t r0,
                                            int32_t u, const AccT* v) {
  int32_t X = u;
  if (it.final_) {
    X = Q.sigma * u + Q.kappa;
    if (X < 0) X += Q.W;
    if (X >= Q.W) X -= Q.W;
  }
#pragma unroll
  for (int i = 0; i < N; i++) base[(int64_t)(r0 + i) * it.dst_pitch + X] = v[i];
}

// Last two levels (merge4 with blocks of M rows) from shared memory straight
// to global memory.
template <int M, typename AccT>
__device__ __forceinline__ void final_merge4(const FusedItem& it, const QuadDesc& Q, const AccT* src, int32_t rs,
                                             AccT* base, int32_t u0, int32_t ncols) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  for (int32_t rq = warp; rq < 16; rq += nwarps) {
    const AccT *q0, *q1, *q2, *q3;
    int32_t r0;
    merge4_ptrs<M, AccT>(src, rs, rq, q0, q1, q2, q3, r0);
    AccT* o = base + (int64_t)r0 * it.dst_pitch;
    for (int32_t j = lane; j < ncols; j += 32) {
      AccT v[4];
      merge4_at<AccT>(q0, q1, q2, q3, j, v);
      store_group<AccT, 4>(it, Q, o, 0, u0 + j, v);
    }
  }
}

template <typename AccT>
__device__ __forceinline__ void final_merge2_1(const FusedItem& it, const QuadDesc& Q, const AccT* src, int32_t rs,
                                               AccT* base, int32_t u0, int32_t ncols) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  for (int32_t rp = warp; rp < 32; rp += nwarps) {
    const AccT *q0, *q1;
    int32_t r0;
    merge2_ptrs<1, AccT>(src, rs, rp, q0, q1, r0);
    AccT* o = base + (int64_t)r0 * it.dst_pitch;
    for (int32_t j = lane; j < ncols; j += 32) {
      const AccT a = q0[j];
      AccT v[2] = {a + q1[j], a + q1[j + 1]};
      store_group<AccT, 2>(it, Q, o, 0, u0 + j, v);
    }
  }
}

// Brady-Yong block paths: 64 shared rows, G = 64 / 2^L groups, each group a
// 2^L-row Brady-Yong transform done in two-level passes (one single level
// first when L is odd).  The last pass goes from registers to global memory.
// Widths: a pass whose shifts reach `sh` reads sh columns beyond its output,
// so the staged window is TW + 2^L - 1 and each pass narrows it:
//   L=6: merge4<1> (3), merge4<4> (12), final merge4<16> (48)
//   L=5: merge2<1> (1), merge4<2> (6),  final merge4<8>  (24)
//   L=4: merge4<1> (3), final merge4<4> (12)
//   L=3: merge2<1> (1), final merge4<2> (6)
//   L=2: final merge4<1> (3);   L=1: final merge2<1> (1)
template <bool kC, typename InT, typename AccT>
__device__ __forceinline__ void fused_block(const FusedParams& p, const FusedItem& it, const QuadDesc& Q, int32_t tile, AccT* S,
                            AccT* A) {
  const int32_t TW = it.tw;
  const int32_t u0 = tile * TW;
  const int32_t span = (1 << it.L) - 1;
  if (it.kind == FUSED_BY64) {
    stage_rows<InT, AccT>(p, Q, it.a, 64, u0 - it.c, TW + span, S, p.RS);
  } else {
    stage_gathered<kC, AccT>(p, it, Q, u0 - it.c, TW + span, S, p.RS);
  }
  __syncthreads();
  const int32_t ncols = min(TW, it.wn - u0);
  AccT* __restrict__ base = (it.final_ ? static_cast<AccT*>(p.out) : static_cast<AccT*>(p.ws)) + it.dst;
  const int32_t RS = p.RS, RA = p.RA;
  switch (it.L) {
    case 6:
      merge4_pass<1, AccT>(S, RS, A, RA, TW + 60);
      __syncthreads();
      merge4_pass<4, AccT>(A, RA, S, RS, TW + 48);
      __syncthreads();
      final_merge4<16, AccT>(it, Q, S, RS, base, u0, ncols);
      break;
    case 5:
      merge2_pass<1, AccT>(S, RS, A, RA, TW + 30);
      __syncthreads();
      merge4_pass<2, AccT>(A, RA, S, RS, TW + 24);
      __syncthreads();
      final_merge4<8, AccT>(it, Q, S, RS, base, u0, ncols);
      break;
    case 4:
      merge4_pass<1, AccT>(S, RS, A, RA, TW + 12);
      __syncthreads();
      final_merge4<4, AccT>(it, Q, A, RA, base, u0, ncols);
      break;
    case 3:
      merge2_pass<1, AccT>(S, RS, A, RA, TW + 6);
      __syncthreads();
      final_merge4<2, AccT>(it, Q, A, RA, base, u0, ncols);
      break;
    case 2:
      final_merge4<1, AccT>(it, Q, S, RS, base, u0, ncols);
      break;
    default:
      final_merge2_1<AccT>(it, Q, S, RS, base, u0, ncols);
      break;
  }
}

// ---- compile-time tile width: the same block paths with every pitch and
// width a constant, so that shared addresses are base + immediate and the
// column loops unroll without per-iteration bounds or pointer arithmetic ----

template <int M, int RSRC, int RDST, int WIDTH, typename AccT>
__device__ __forceinline__ void merge4_pass_c(const AccT* src, AccT* dst) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  for (int32_t rq = warp; rq < 16; rq += nwarps) {
    const AccT *q0, *q1, *q2, *q3;
    int32_t r0;
    merge4_ptrs<M, AccT>(src, RSRC, rq, q0, q1, q2, q3, r0);
    q0 += lane;
    q1 += lane;
    q2 += lane;
    q3 += lane;
    AccT* d = dst + r0 * RDST + lane;
#pragma unroll
    for (int c = 0; c < (WIDTH + 31) / 32; c++) {
      if (32 * c + 32 <= WIDTH || 32 * c + lane < WIDTH) {
        AccT o[4];
        merge4_at<AccT>(q0, q1, q2, q3, 32 * c, o);
        d[32 * c] = o[0];
        d[RDST + 32 * c] = o[1];
        d[2 * RDST + 32 * c] = o[2];
        d[3 * RDST + 32 * c] = o[3];
      }
    }
  }
}

template <int RSRC, int RDST, int WIDTH, typename AccT>
__device__ __forceinline__ void merge2_pass1_c(const AccT* src, AccT* dst) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  for (int32_t rp = warp; rp < 32; rp += nwarps) {
    const AccT *q0, *q1;
    int32_t r0;
    merge2_ptrs<1, AccT>(src, RSRC, rp, q0, q1, r0);
    q0 += lane;
    q1 += lane;
    AccT* d = dst + r0 * RDST + lane;
#pragma unroll
    for (int c = 0; c < (WIDTH + 31) / 32; c++) {
      if (32 * c + 32 <= WIDTH || 32 * c + lane < WIDTH) {
        const AccT a = q0[32 * c];
        d[32 * c] = a + q1[32 * c];
        d[RDST + 32 * c] = a + q1[32 * c + 1];
      }
    }
  }
}

template <int M, int RSRC, int TW, typename AccT>
__device__ __forceinline__ void final_merge4_c(const FusedItem& it, const QuadDesc& Q, const AccT* src, AccT* base,
                                               int32_t u0, int32_t ncols) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  const int64_t pitch = it.dst_pitch;
  for (int32_t rq = warp; rq < 16; rq += nwarps) {
    const AccT *q0, *q1, *q2, *q3;
    int32_t r0;
    merge4_ptrs<M, AccT>(src, RSRC, rq, q0, q1, q2, q3, r0);
    q0 += lane;
    q1 += lane;
    q2 += lane;
    q3 += lane;
    AccT* o = base + (int64_t)r0 * pitch;
#pragma unroll
    for (int c = 0; c < TW / 32; c++) {
      const int32_t j = 32 * c + lane;
      if (j < ncols) {
        AccT v[4];
        merge4_at<AccT>(q0, q1, q2, q3, 32 * c, v);
        int32_t X = u0 + j;
        if (it.final_) {
          X = Q.sigma * X + Q.kappa;
          if (X < 0) X += Q.W;
          if (X >= Q.W) X -= Q.W;
        }
        AccT* oo = o + X;
        oo[0] = v[0];
        oo[pitch] = v[1];
        oo[2 * pitch] = v[2];
        oo[3 * pitch] = v[3];
      }
    }
  }
}

template <int RSRC, int TW, typename AccT>
__device__ __forceinline__ void final_merge2_1_c(const FusedItem& it, const QuadDesc& Q, const AccT* src, AccT* base,
                                                 int32_t u0, int32_t ncols) {
  const int32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nwarps = blockDim.x >> 5;
  const int64_t pitch = it.dst_pitch;
  for (int32_t rp = warp; rp < 32; rp += nwarps) {
    const AccT *q0, *q1;
    int32_t r0;
    merge2_ptrs<1, AccT>(src, RSRC, rp, q0, q1, r0);
    q0 += lane;
    q1 += lane;
    AccT* o = base + (int64_t)r0 * pitch;
#pragma unroll
    for (int c = 0; c < TW / 32; c++) {
      const int32_t j = 32 * c + lane;
      if (j < ncols) {
        const AccT a = q0[32 * c];
        int32_t X = u0 + j;
        if (it.final_) {
          X = Q.sigma * X + Q.kappa;
          if (X < 0) X += Q.W;
          if (X >= Q.W) X -= Q.W;
        }
        o[X] = a + q1[32 * c];
        o[pitch + X] = a + q1[32 * c + 1];
      }
    }
  }
}

// Shared pitches of the block paths for a tile of TW columns (TW a multiple
// of 32): staged / level-4 rows TW + 63, level-2 rows TW + 61 (both odd).
template <int TW>
struct BlockPitch {
  static constexpr int RS = TW + 63;
  static constexpr int RA = TW + 61;
};

template <bool kC, int TW, typename InT, typename AccT>
__device__ __forceinline__ void fused_block_c(const FusedParams& p, const FusedItem& it, const QuadDesc& Q,
                                              int32_t tile, AccT* S, AccT* A) {
  constexpr int RS = BlockPitch<TW>::RS, RA = BlockPitch<TW>::RA;
  const int32_t u0 = tile * TW;
  const int32_t span = (1 << it.L) - 1;
  if (it.kind == FUSED_BY64) {
    // register staging, all loads of a lane in flight at once (measured
    // faster than cp.async for the input window)
    if (blockDim.x == 512) {
      stage_block_c<InT, AccT, TW + 63, sizeof(AccT) == 8 ? 2 : 4>(p, Q, it.a, u0 - it.c, S, RS);
    } else {
      stage_rows<InT, AccT>(p, Q, it.a, 64, u0 - it.c, TW + span, S, RS);
    }
  } else if constexpr (!kC) {
    stage_gathered_async<AccT>(p, it, Q, u0 - it.c, TW + span, S, RS);
  } else {
    stage_gathered<kC, AccT>(p, it, Q, u0 - it.c, TW + span, S, RS);
  }
  __syncthreads();
  const int32_t ncols = min(TW, it.wn - u0);
  AccT* __restrict__ base = (it.final_ ? static_cast<AccT*>(p.out) : static_cast<AccT*>(p.ws)) + it.dst;
  switch (it.L) {
    case 6:
      merge4_pass_c<1, RS, RA, TW + 60, AccT>(S, A);
      __syncthreads();
      merge4_pass_c<4, RA, RS, TW + 48, AccT>(A, S);
      __syncthreads();
      final_merge4_c<16, RS, TW, AccT>(it, Q, S, base, u0, ncols);
      break;
    case 5:
      merge2_pass1_c<RS, RA, TW + 30, AccT>(S, A);
      __syncthreads();
      merge4_pass_c<2, RA, RS, TW + 24, AccT>(A, S);
      __syncthreads();
      final_merge4_c<8, RS, TW, AccT>(it, Q, S, base, u0, ncols);
      break;
    case 4:
      merge4_pass_c<1, RS, RA, TW + 12, AccT>(S, A);
      __syncthreads();
      final_merge4_c<4, RA, TW, AccT>(it, Q, A, base, u0, ncols);
      break;
    case 3:
      merge2_pass1_c<RS, RA, TW + 6, AccT>(S, A);
      __syncthreads();
      final_merge4_c<2, RA, TW, AccT>(it, Q, A, base, u0, ncols);
      break;
    case 2:
      final_merge4_c<1, RS, TW, AccT>(it, Q, S, base, u0, ncols);
      break;
    default:
      final_merge2_1_c<RS, TW, AccT>(it, Q, S, base, u0, ncols);
      break;
  }
}

// Block path dispatch: the common tile widths run the compile-time variant.
template <bool kC, typename InT, typename AccT>
__device__ __forceinline__ void fused_block_any(const FusedParams& p, const FusedItem& it, const QuadDesc& Q,
                                                int32_t tile, AccT* S, AccT* A) {
  switch (it.tw) {
    case 64:
      fused_block_c<kC, 64, InT, AccT>(p, it, Q, tile, S, A);
      break;
    case 128:
      fused_block_c<kC, 128, InT, AccT>(p, it, Q, tile, S, A);
      break;
    case 256:
      fused_block_c<kC, 256, InT, AccT>(p, it, Q, tile, S, A);
      break;
    default:
      fused_block<kC, InT, AccT>(p, it, Q, tile, S, A);
      break;
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

// Spine sum.  One CTA = kSpineRows consecutive output rows x one column tile
// of kSpineTile columns; every thread owns 4 columns and loads all terms of a
// row before adding (term count fixed at compile time per row).  The rows of
// a CTA read neighbouring rows of the same parts at nearby offsets, so most
// part reads hit L1; consecutive CTAs share rows through L2.
constexpr int kSpineTile = 1024;  // batched kernel: 256 threads x 4 columns
// plain spine kernel: 256 threads x kSpineQPT columns per row tile
constexpr int kSpineQPT = 4;
constexpr bool kSpinePipe = true;
constexpr int kSpineTilePlain = 256 * kSpineQPT;

// One output row x one column tile of BS * QPT columns: every thread owns QPT
// columns spaced BS apart.
template <bool kC, int NT, int BS, int QPT, typename AccT>
__device__ __forceinline__ void spine_tile(const SpineTerm* st, const QuadDesc& Q, const AccT* __restrict__ ws,
                                           AccT* __restrict__ dst, int32_t u0) {
  AccT v[NT][QPT];
  const bool full = u0 + BS * QPT <= Q.W;
#pragma unroll
  for (int c = 0; c < NT; c++) {
    const int32_t off = st[c].off, wpart = st[c].wpart;
    const AccT* __restrict__ row = ws + st[c].row;
    // the whole tile reads one contiguous stretch of the part row
    const bool clean =
        full && (Q.ext ? (u0 + off >= 0 && u0 + BS * QPT - 1 + off < wpart) : (u0 + BS * QPT - 1 + off < Q.W));
    if (clean) {
      const AccT* __restrict__ src = row + u0 + off + (int32_t)threadIdx.x;
#pragma unroll
      for (int q = 0; q < QPT; q++) v[c][q] = ld_ws<kC>(src + q * BS);
    } else {
#pragma unroll
      for (int q = 0; q < QPT; q++) {
        const int32_t u = u0 + q * BS + (int32_t)threadIdx.x;
        int32_t i = u + off;
        bool ok = u < Q.W;
        if (Q.ext) {
          ok = ok && i >= 0 && i < wpart;
        } else if (i >= Q.W) {
          i -= Q.W;
        }
        v[c][q] = ok ? ld_ws<kC>(row + i) : AccT(0);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QPT; q++) {
    AccT acc = v[0][q];
#pragma unroll
    for (int c = 1; c < NT; c++) acc += v[c][q];
    const int32_t u = u0 + q * BS + (int32_t)threadIdx.x;
    if (u < Q.W) {
      int32_t X = Q.sigma * u + Q.kappa;
      if (X < 0) X += Q.W;
      if (X >= Q.W) X -= Q.W;
      dst[X] = acc;
    }
  }
}

// Loads of one spine row's terms for this thread's QPT columns
// u = u0 + tid + q BS of a row of W columns.  Branch-free: for each term the
// columns that read inside the part row (extended) or that wrap (cyclic) form
// one contiguous range of q BS, found from two thresholds; every load uses the
// term's hoisted pointer with a compile-time offset.
template <bool kC, int NT, int BS, int QPT, typename AccT>
__device__ __forceinline__ void spine_load(const SpineTerm* st, int32_t W, bool ext, const AccT* __restrict__ ws,
                                           int32_t u0, AccT (&v)[NT][QPT]) {
  const int32_t base_u = u0 + (int32_t)threadIdx.x;
  const int32_t live = W - base_u;  // column q is inside the row iff q BS < live
  const bool full = u0 + BS * QPT <= W;
#pragma unroll
  for (int c = 0; c < NT; c++) {
    const int32_t off = st[c].off;
    const AccT* __restrict__ src = ws + st[c].row + (base_u + off);
    // CTA-uniform test: the whole tile reads one in-bounds stretch of the part row
    const bool clean = full && (ext ? (u0 + off >= 0 && u0 + BS * QPT + off <= st[c].wpart)
                                    : (u0 + BS * QPT + off <= W));
    if (clean) {
#pragma unroll
      for (int q = 0; q < QPT; q++) v[c][q] = ld_ws<kC>(src + q * BS);
    } else if (ext) {
      const int32_t lo = -(base_u + off), hi = st[c].wpart - (base_u + off);  // valid iff lo <= q BS < hi
#pragma unroll
      for (int q = 0; q < QPT; q++)
        v[c][q] = (q * BS >= lo && q * BS < hi && q * BS < live) ? ld_ws<kC>(src + q * BS) : AccT(0);
    } else {
      const int32_t wrap = W - (base_u + off);  // q BS >= wrap reads W columns back
#pragma unroll
      for (int q = 0; q < QPT; q++) {
        const AccT* p = (q * BS >= wrap) ? src - W : src;
        v[c][q] = (q * BS < live) ? ld_ws<kC>(p + q * BS) : AccT(0);
      }
    }
  }
}

// Sum and store: through the quadrant's column map X = (sigma u + kappa) mod W
// (root rows, kMap) or at u itself (inner spine nodes).
template <bool kMap, int NT, int BS, int QPT, typename AccT>
__device__ __forceinline__ void spine_store(int32_t W, int32_t sigma, int32_t kappa, AccT* __restrict__ dst,
                                            int32_t u0, const AccT (&v)[NT][QPT]) {
#pragma unroll
  for (int q = 0; q < QPT; q++) {
    AccT acc = v[0][q];
#pragma unroll
    for (int c = 1; c < NT; c++) acc += v[c][q];
    const int32_t u = u0 + q * BS + (int32_t)threadIdx.x;
    if (u < W) {
      int32_t X = u;
      if constexpr (kMap) {
        X = sigma * u + kappa;
        if (X < 0) X += W;
        if (X >= W) X -= W;
      }
      dst[X] = acc;
    }
  }
}

// All nr rows share one quadrant, one kind and one term count: the loads of
// row r + 1 are issued before row r is summed and stored, so two rows of
// loads are in flight per thread.
template <bool kC, bool kMap, int NT, int BS, int QPT, typename AccT>
__device__ __forceinline__ void spine_group_pipelined(const SpineRow* sr, SpineTerm (*st)[kMaxSpineTerms],
                                                      int32_t nr, int32_t W, bool ext, int32_t sigma, int32_t kappa,
                                                      const AccT* ws, AccT* out, int32_t u0) {
  AccT a[NT][QPT], b[NT][QPT];
  spine_load<kC, NT, BS, QPT, AccT>(st[0], W, ext, ws, u0, a);
  for (int32_t r = 0; r < nr; r += 2) {
    if (r + 1 < nr) spine_load<kC, NT, BS, QPT, AccT>(st[r + 1], W, ext, ws, u0, b);
    spine_store<kMap, NT, BS, QPT, AccT>(W, sigma, kappa, out + sr[r].dst, u0, a);
    if (r + 1 >= nr) break;
    if (r + 2 < nr) spine_load<kC, NT, BS, QPT, AccT>(st[r + 2], W, ext, ws, u0, a);
    spine_store<kMap, NT, BS, QPT, AccT>(W, sigma, kappa, out + sr[r + 1].dst, u0, b);
  }
}

// The row geometry of a spine row: the quadrant's, or for an inner spine node
// its own width and the identity column map.
__device__ __forceinline__ QuadDesc spine_row_desc(const QuadDesc* quads, const SpineRow& r) {
  QuadDesc Q = quads[r.q];
  if (r.flags & SPINE_INNER) {
    Q.W = r.w;
    Q.sigma = 1;
    Q.kappa = 0;
  }
  return Q;
}

// Rows [r0, r0 + nr) of a spine (terms staged in shared memory by the caller)
// for the column tile starting at u0.  Root rows go to `out`, inner-node rows
// to `inner` (the workspace base; never a region this launch reads).
template <bool kC, int BS, int QPT, typename AccT, bool kPipe = true>
__device__ __forceinline__ void spine_rows_tile(const SpineRow* sr, SpineTerm (*st)[kMaxSpineTerms], int32_t nr,
                                                const QuadDesc* quads, const AccT* ws, AccT* out, AccT* inner,
                                                int32_t u0) {
  bool uniform = kPipe && nr > 0;
  for (int32_t r = 1; r < nr; r++)
    uniform = uniform && sr[r].q == sr[0].q && sr[r].term_count == sr[0].term_count && sr[r].flags == sr[0].flags;
  if constexpr (kPipe) {
  if (uniform) {
    const QuadDesc& Q = quads[sr[0].q];
    if (sr[0].flags & SPINE_INNER) {
      const int32_t W = sr[0].w;
      if (u0 >= W) return;
      switch (sr[0].term_count) {
#define FHT_SPINE_PIPE(N)                                                                             \
  case N:                                                                                             \
    spine_group_pipelined<kC, false, N, BS, QPT, AccT>(sr, st, nr, W, Q.ext, 1, 0, ws, inner, u0);    \
    return;
        FHT_SPINE_PIPE(1) FHT_SPINE_PIPE(2) FHT_SPINE_PIPE(3) FHT_SPINE_PIPE(4) FHT_SPINE_PIPE(5)
        FHT_SPINE_PIPE(6) FHT_SPINE_PIPE(7) FHT_SPINE_PIPE(8)
#undef FHT_SPINE_PIPE
        default:
          break;  // more terms: the row-by-row path below
      }
    } else {
      if (u0 >= Q.W) return;
      switch (sr[0].term_count) {
#define FHT_SPINE_PIPE(N)                                                                                     \
  case N:                                                                                                     \
    spine_group_pipelined<kC, true, N, BS, QPT, AccT>(sr, st, nr, Q.W, Q.ext, Q.sigma, Q.kappa, ws, out, u0); \
    return;
        FHT_SPINE_PIPE(1) FHT_SPINE_PIPE(2) FHT_SPINE_PIPE(3) FHT_SPINE_PIPE(4) FHT_SPINE_PIPE(5)
        FHT_SPINE_PIPE(6) FHT_SPINE_PIPE(7) FHT_SPINE_PIPE(8)
#undef FHT_SPINE_PIPE
        default:
          break;
      }
    }
  }
  }
  // at most 64 loaded values live per thread: rows with more than 64 / QPT
  // terms sweep the tile in two halves
  constexpr int QH = QPT > 1 ? QPT / 2 : 1;
  for (int32_t r = 0; r < nr; r++) {
    const QuadDesc Q = spine_row_desc(quads, sr[r]);
    if (u0 >= Q.W) continue;
    AccT* dst = ((sr[r].flags & SPINE_INNER) ? inner : out) + sr[r].dst;
    switch (sr[r].term_count) {
#define FHT_SPINE_CASE(N)                                                   \
  case N:                                                                   \
    if constexpr (N * QPT <= 64) {                                          \
      spine_tile<kC, N, BS, QPT, AccT>(st[r], Q, ws, dst, u0);              \
    } else {                                                                \
      spine_tile<kC, N, BS, QH, AccT>(st[r], Q, ws, dst, u0);               \
      if (u0 + BS * QH < Q.W) spine_tile<kC, N, BS, QH, AccT>(st[r], Q, ws, dst, u0 + BS * QH); \
    }                                                                       \
    break;
      FHT_SPINE_CASE(1) FHT_SPINE_CASE(2) FHT_SPINE_CASE(3) FHT_SPINE_CASE(4) FHT_SPINE_CASE(5) FHT_SPINE_CASE(6)
      FHT_SPINE_CASE(7) FHT_SPINE_CASE(8) FHT_SPINE_CASE(9) FHT_SPINE_CASE(10) FHT_SPINE_CASE(11)
      FHT_SPINE_CASE(12) FHT_SPINE_CASE(13) FHT_SPINE_CASE(14) FHT_SPINE_CASE(15) FHT_SPINE_CASE(16)
#undef FHT_SPINE_CASE
      default:
        break;
    }
  }
}

}  // namespace fht
