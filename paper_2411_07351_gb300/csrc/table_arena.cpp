// Device memory for plan tables, sub-allocated from large chunks.
//
// A serving process builds a plan for nearly every request (image sizes
// rarely repeat), thousands per second on builder threads.  One cudaMalloc
// per plan made those threads call into the CUDA driver's allocator that often,
// and the calls slowed down as allocations accumulated until they held up
// the serving thread's own CUDA calls for tens of milliseconds.  Plans now
// take their tables from chunks of kChunk bytes allocated once per device
// (first fit over a free list with coalescing; tables above kChunk / 4 get an
// allocation of their own).  Chunks are kept until the process exits; freed
// ranges are reused.  The paper has no counterpart: this is runtime of this
// library.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>
#include <mutex>
#include <vector>

#include "table_arena.hpp"

namespace fht {
namespace {

constexpr size_t kChunk = size_t(64) << 20;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

struct Chunk {
  unsigned char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free;  // offset -> length of each free range, coalesced
  size_t largest = 0;             // longest free range (chunks that cannot fit are skipped)
};

struct Arena {
  std::mutex mu;
  std::vector<Chunk> chunks;
  std::map<uintptr_t, size_t> by_base;  // chunk base address -> index in chunks
};

void recompute_largest(Chunk& c) {
  c.largest = 0;
  for (const auto& f : c.free) c.largest = std::max(c.largest, f.second);
}

Arena g_arena[kMaxDevices];

bool take(Chunk& c, size_t bytes, void** out) {
  if (c.largest < bytes) return false;
  for (auto it = c.free.begin(); it != c.free.end(); ++it) {
    if (it->second < bytes) continue;
    const size_t off = it->first, len = it->second;
    c.free.erase(it);
    if (len > bytes) c.free.emplace(off + bytes, len - bytes);
    if (len == c.largest) recompute_largest(c);
    *out = c.base + off;
    return true;
  }
  return false;
}

void give_back(Chunk& c, size_t off, size_t bytes) {
  auto next = c.free.lower_bound(off);
  if (next != c.free.end() && off + bytes == next->first) {  // merge with the range after
    bytes += next->second;
    next = c.free.erase(next);
  }
  if (next != c.free.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {  // merge with the range before
      prev->second += bytes;
      c.largest = std::max(c.largest, prev->second);
      return;
    }
  }
  c.free.emplace(off, bytes);
  c.largest = std::max(c.largest, bytes);
}

}  // namespace

size_t table_arena_round(size_t bytes) { return (std::max<size_t>(bytes, 1) + kAlign - 1) / kAlign * kAlign; }

cudaError_t table_arena_alloc(int device, size_t bytes, void** out) {
  *out = nullptr;
  bytes = table_arena_round(bytes);
  if (device < 0 || device >= kMaxDevices || bytes > kChunk / 4) return cudaMalloc(out, bytes);
  Arena& a = g_arena[device];
  std::lock_guard<std::mutex> lock(a.mu);
  for (Chunk& c : a.chunks)
    if (take(c, bytes, out)) return cudaSuccess;
  Chunk c;
  void* base = nullptr;
  const cudaError_t e = cudaMalloc(&base, kChunk);
  if (e != cudaSuccess) return e;
  c.base = static_cast<unsigned char*>(base);
  c.size = kChunk;
  c.free.emplace(0, kChunk);
  c.largest = kChunk;
  a.by_base.emplace(reinterpret_cast<uintptr_t>(base), a.chunks.size());
  a.chunks.push_back(std::move(c));
  take(a.chunks.back(), bytes, out);
  return cudaSuccess;
}

void table_arena_free(int device, void* p, size_t bytes) {
  if (!p) return;
  bytes = table_arena_round(bytes);
  if (device < 0 || device >= kMaxDevices || bytes > kChunk / 4) {
    cudaFree(p);
    return;
  }
  Arena& a = g_arena[device];
  std::lock_guard<std::mutex> lock(a.mu);
  const uintptr_t q = reinterpret_cast<uintptr_t>(p);
  auto it = a.by_base.upper_bound(q);  // the chunk with the highest base <= q
  if (it == a.by_base.begin()) return;
  --it;
  Chunk& c = a.chunks[it->second];
  if (q < it->first + c.size) give_back(c, (size_t)(q - it->first), bytes);
}

}  // namespace fht
