// Device primitives for regrouping points by grid cell: a stable least-significant-digit
// radix sort of (32-bit key, 32-bit value) pairs and an exclusive scan of ints.  All counts
// are integers and every output position is a function of the input order alone, so the
// results are deterministic (no float atomics anywhere).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int SORT_THREADS = 256;                  // threads per sort block (8 warps)
constexpr int SORT_ITEMS = 8;                      // keys per thread
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_TILE = 2 * SCAN_THREADS;

// bytes of device workspace that sort_pairs needs for n pairs
size_t sort_workspace_bytes(long long n);

// Stable sort of n pairs by the low `bits` bits of the keys (1 <= bits <= 32; higher bits
// must be zero).  keys/vals are sorted in place; tmp_keys/tmp_vals hold n entries each;
// work holds sort_workspace_bytes(n) bytes.  n < 2^31.
cudaError_t sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys, uint32_t *tmp_vals, long long n,
                       int bits, void *work, cudaStream_t st);

// bytes of device workspace that exclusive_scan needs for n ints
size_t scan_workspace_bytes(long long n);

// out[i] = sum_{j < i} in[j] (in == out allowed)
cudaError_t exclusive_scan(const int *in, int *out, long long n, void *work, cudaStream_t st);

}  // namespace lbm
