"""The device-table arena's range bookkeeping (CPU only).

Plans take their device tables from ranges of large per-device chunks
(csrc/table_arena.cpp).  Here that file is compiled with g++ against a stand-in
for cudaMalloc / cudaFree backed by host memory, and a random mix of
allocations and frees checks that:
  * every range is 256-byte aligned and no two live ranges overlap (each
    live range carries its own byte pattern, verified before it is freed);
  * ranges above a quarter chunk get an allocation of their own, returned on
    free;
  * freed neighbours coalesce: once everything is freed, the chunks hold
    quarter-chunk ranges back to back without a new chunk;
  * a free range with both neighbours held is handed out again.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2411_07351_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>
#include "table_arena.hpp"

static int g_mallocs = 0, g_frees = 0;
extern "C" cudaError_t cudaMalloc(void** p, size_t n) {
  *p = aligned_alloc(256, (n + 255) / 256 * 256);
  g_mallocs++;
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
extern "C" cudaError_t cudaFree(void* p) {
  free(p);
  g_frees++;
  return cudaSuccess;
}

struct Live { unsigned char* p; size_t n; unsigned char tag; };

static bool intact(const Live& l) {
  for (size_t i = 0; i < l.n; i++)
    if (l.p[i] != l.tag) return false;
  return true;
}

int main() {
  const size_t kChunk = size_t(64) << 20;
  std::mt19937_64 g(7);
  std::vector<Live> live;
  int tag = 0, dedicated = 0;
  for (int op = 0; op < 4000; op++) {
    const bool alloc = live.empty() || (g() % 100) < 55;
    if (alloc) {
      size_t n;
      const int kind = (int)(g() % 100);
      if (kind < 2) { n = kChunk / 4 + 1 + g() % (8 << 20); dedicated++; }   // own allocation
      else if (kind < 10) n = (size_t)(1 + g() % (kChunk / 4));               // up to a quarter chunk
      else n = (size_t)(1 + g() % (512 << 10));                               // typical tables
      void* p = nullptr;
      if (fht::table_arena_alloc(0, n, &p) != cudaSuccess || !p) { printf("FAIL alloc %zu\n", n); return 1; }
      if ((uintptr_t)p % 256) { printf("FAIL alignment\n"); return 1; }
      Live l{(unsigned char*)p, n, (unsigned char)(++tag & 0xff)};
      memset(l.p, l.tag, l.n);
      live.push_back(l);
    } else {
      const size_t k = (size_t)(g() % live.size());
      if (!intact(live[k])) { printf("FAIL overlap: a live range was overwritten\n"); return 1; }
      fht::table_arena_free(0, live[k].p, live[k].n);
      live[k] = live.back();
      live.pop_back();
    }
  }
  for (const Live& l : live) {
    if (!intact(l)) { printf("FAIL overlap at the end\n"); return 1; }
    fht::table_arena_free(0, l.p, l.n);
  }
  live.clear();
  // every dedicated range was returned through cudaFree, nothing else was
  const int chunks = g_mallocs - dedicated;
  if (g_frees != dedicated) { printf("FAIL frees %d dedicated %d\n", g_frees, dedicated); return 1; }
  // all free again: each chunk holds four quarter-chunk ranges with no new allocation
  const int before = g_mallocs;
  std::vector<void*> q;
  for (int i = 0; i < 4 * chunks; i++) {
    void* p = nullptr;
    if (fht::table_arena_alloc(0, kChunk / 4, &p) != cudaSuccess) { printf("FAIL quarter alloc\n"); return 1; }
    q.push_back(p);
  }
  if (g_mallocs != before) { printf("FAIL not coalesced: %d new chunks\n", g_mallocs - before); return 1; }
  // every chunk is full: an isolated free range (both neighbours held) is found again
  fht::table_arena_free(0, q[1], kChunk / 4);
  void* again = nullptr;
  if (fht::table_arena_alloc(0, kChunk / 4, &again) != cudaSuccess || again != q[1] || g_mallocs != before) {
    printf("FAIL isolated free range not reused\n");
    return 1;
  }
  for (void* p : q) fht::table_arena_free(0, p, kChunk / 4);
  printf("OK chunks %d dedicated %d\n", chunks, dedicated);
  return 0;
}
"""


def test_arena_ranges_disjoint_aligned_and_coalesced(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "arena_harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "arena_harness"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CUDA_INC, "-I", CSRC, str(src),
                    os.path.join(CSRC, "table_arena.cpp"), "-o", str(exe)], check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
    chunks = int(r.stdout.split()[2])
    assert chunks >= 1
