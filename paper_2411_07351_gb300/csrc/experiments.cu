// The paper's accuracy experiment (Sections 4-5) on the GPU: the maximum
// orthotropic error of the generating patterns,
//   E(n) = max over t in [0, n), x in [0, n) of |x t/(n-1) - pat(n,t)(x)|,
// for every n of a range, under either split rule.  Returned as the exact
// integer numerator max |x t - pat(n,t)(x) (n - 1)|.
//
// One thread per (n, t): the pattern of Algorithm 2 is produced leaf by leaf
// by a depth-first walk of the split tree with an explicit stack (each node
// carries its size, its slope and the offset its leaves add); child slopes are
// [t (m_i - 1)/(m - 1)] rounded half to even in integers.  Block maximum, then
// one 64-bit atomicMax per block.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/fht.h"

namespace {

__device__ __forceinline__ int32_t round_half_even_u(uint32_t a, uint32_t d) {
  const uint32_t q = a / d, r = a - q * d;
  if (2 * r > d) return (int32_t)q + 1;
  if (2 * r < d) return (int32_t)q;
  return (int32_t)(q + (q & 1));
}

__device__ __forceinline__ void split_sizes(int32_t m, int32_t rule, int32_t& m0, int32_t& m1) {
  if (rule == 0) {
    // Split_T: the largest power of two below m (m itself halves when it is one)
    m0 = 1 << (31 - __clz(m - 1));
  } else {
    m0 = m / 2;  // Split_S
  }
  m1 = m - m0;
}

__global__ void pattern_error_kernel(int32_t n_lo, int32_t n_hi, int32_t rule, unsigned long long* out) {
  const int32_t n = n_lo + blockIdx.y;
  if (n > n_hi) return;
  unsigned long long best = 0;
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    // stack entries: size, slope, offset, first x
    int32_t sm[32], st[32], so[32], sx[32];
    int32_t top = 0;
    sm[0] = n;
    st[0] = t;
    so[0] = 0;
    sx[0] = 0;
    top = 1;
    while (top > 0) {
      top--;
      int32_t m = sm[top], tt = st[top], off = so[top], x = sx[top];
      // descend along left children, pushing right children
      while (m > 1) {
        int32_t m0, m1;
        split_sizes(m, rule, m0, m1);
        const uint32_t d = (uint32_t)(m - 1);
        const int32_t t1 = round_half_even_u((uint32_t)tt * (uint32_t)(m0 - 1), d);
        const int32_t t2 = round_half_even_u((uint32_t)tt * (uint32_t)(m1 - 1), d);
        sm[top] = m1;
        st[top] = t2;
        so[top] = off + (tt - t2);
        sx[top] = x + m0;
        top++;
        m = m0;
        tt = t1;
      }
      // leaf: pattern value `off` at position x
      const long long e = (long long)x * t - (long long)off * (n - 1);
      const unsigned long long a = (unsigned long long)(e < 0 ? -e : e);
      best = a > best ? a : best;
    }
  }
  // block maximum
  __shared__ unsigned long long red[32];
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_down_sync(0xffffffffu, best, o);
      best = v > best ? v : best;
    }
    if (threadIdx.x == 0) atomicMax(&out[n - n_lo], best);
  }
}

}  // namespace

fht_status fht_capi_fail(fht_status st, const std::string& msg);

extern "C" fht_status fht_pattern_errors(int32_t n_lo, int32_t n_hi, fht_split split, int64_t* d_num,
                                         void* stream) {
  if (n_lo < 1 || n_hi < n_lo || n_hi > 65535 || !d_num)
    return fht_capi_fail(FHT_ERR_INVALID, "fht_pattern_errors: need 1 <= n_lo <= n_hi <= 65535 and an output");
  if ((int)split != 0 && (int)split != 1) return fht_capi_fail(FHT_ERR_INVALID, "fht_pattern_errors: split rule");
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t count = n_hi - n_lo + 1;
  cudaError_t e = cudaMemsetAsync(d_num, 0, sizeof(int64_t) * count, st);
  if (e != cudaSuccess) return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_pattern_errors: ") + cudaGetErrorString(e));
  const int32_t threads = 128;
  const int32_t xblocks = (n_hi + threads - 1) / threads;
  for (int32_t base = 0; base < count; base += 65535) {
    const int32_t c = count - base < 65535 ? count - base : 65535;
    dim3 grid(xblocks, c);
    pattern_error_kernel<<<grid, threads, 0, st>>>(n_lo + base, n_hi, (int32_t)split,
                                                   reinterpret_cast<unsigned long long*>(d_num) + base);
    e = cudaGetLastError();
    if (e != cudaSuccess)
      return fht_capi_fail(FHT_ERR_CUDA, std::string("fht_pattern_errors: ") + cudaGetErrorString(e));
  }
  return FHT_OK;
}
