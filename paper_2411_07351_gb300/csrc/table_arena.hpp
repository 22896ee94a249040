// Device memory for plan tables: sub-allocated from large per-device chunks
// (no driver allocation per plan).  Thread-safe.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace fht {

// Bytes a request of `bytes` occupies (rounded up to 256).
size_t table_arena_round(size_t bytes);
// `bytes` of device memory on `device` (the current device), 256-byte aligned.
cudaError_t table_arena_alloc(int device, size_t bytes, void** out);
// Returns a range from table_arena_alloc (same device and bytes).  The caller
// has made sure that no launch still reads it: the range may be handed out
// again at once.
void table_arena_free(int device, void* p, size_t bytes);

}  // namespace fht
