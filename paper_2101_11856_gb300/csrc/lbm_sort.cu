// Stable radix sort and exclusive scan (see lbm_sort.cuh).
#include "lbm_sort.cuh"

namespace lbm {

namespace {

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }
inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// ---- exclusive scan ------------------------------------------------------------------------

// inclusive scan of v over the warp
__device__ __forceinline__ int warp_inclusive(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// each block scans SCAN_TILE consecutive entries (two per thread) and writes its total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const int *in, int *out, long long n, int *sums) {
    __shared__ int wsum[SCAN_THREADS / 32];
    const long long i0 = (long long)blockIdx.x * SCAN_TILE + 2 * threadIdx.x;
    const int a = i0 < n ? in[i0] : 0;
    const int b = i0 + 1 < n ? in[i0 + 1] : 0;
    const int s = a + b;
    const int incl = warp_inclusive(s);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
        const int vi = warp_inclusive(v);
        if (lane < SCAN_THREADS / 32) wsum[lane] = vi - v;   // exclusive prefix of the warps
        if (lane == SCAN_THREADS / 32 - 1 && sums) sums[blockIdx.x] = vi;
    }
    __syncthreads();
    const int excl = wsum[warp] + incl - s;
    if (i0 < n) out[i0] = excl;
    if (i0 + 1 < n) out[i0 + 1] = excl + a;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(int *out, long long n, const int *sums) {
    const int add = sums[blockIdx.x];
    const long long i0 = (long long)blockIdx.x * SCAN_TILE + 2 * threadIdx.x;
    if (i0 < n) out[i0] += add;
    if (i0 + 1 < n) out[i0 + 1] += add;
}

// ---- radix sort ------------------------------------------------------------------------------

// per-block histogram of one 8-bit digit; hist is digit-major: hist[digit * nblocks + block]
__global__ void __launch_bounds__(SORT_THREADS) k_digit_hist(const uint32_t *keys, long long n, int shift, int *hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * SORT_TILE;
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const long long e = base + it * SORT_THREADS + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// stable scatter: element order within a tile is (warp, item, lane); the rank of a key among
// equal digits is counted per warp with __match_any_sync, then offset by the warps before it
// and by the digit's global start for this block (scanned histogram)
__global__ void __launch_bounds__(SORT_THREADS) k_digit_scatter(const uint32_t *keys, const uint32_t *vals,
                                                                uint32_t *okeys, uint32_t *ovals, long long n,
                                                                int shift, const int *start) {
    constexpr int WARPS = SORT_THREADS / 32;
    __shared__ int wcnt[WARPS][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < WARPS * 256; k += SORT_THREADS) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * SORT_TILE + (long long)warp * 32 * SORT_ITEMS;
    uint32_t key[SORT_ITEMS], val[SORT_ITEMS];
    int rank[SORT_ITEMS];
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const long long e = base + it * 32 + lane;
        const bool valid = e < n;
        key[it] = valid ? keys[e] : 0u;
        val[it] = valid ? vals[e] : 0u;
        const uint32_t digit = valid ? (key[it] >> shift) & 255u : 256u;   // 256: past the end
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const int before = valid ? wcnt[warp][digit] : 0;
        rank[it] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][digit] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;   // one thread per digit
        int run = start[(long long)d * gridDim.x + blockIdx.x];
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const long long e = base + it * 32 + lane;
        if (e < n) {
            const int pos = wcnt[warp][(key[it] >> shift) & 255u] + rank[it];
            okeys[pos] = key[it];
            ovals[pos] = val[it];
        }
    }
}

}  // namespace

size_t scan_workspace_bytes(long long n) {
    size_t b = 0;
    for (long long m = ceil_div(n, SCAN_TILE); m > 1; m = ceil_div(m, SCAN_TILE)) b += align256((size_t)m * sizeof(int));
    return b + 256;
}

cudaError_t exclusive_scan(const int *in, int *out, long long n, void *work, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const long long nb = ceil_div(n, SCAN_TILE);
    int *sums = nb > 1 ? static_cast<int *>(work) : nullptr;
    k_scan_tile<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, sums);
    if (nb == 1) return cudaGetLastError();
    void *rest = static_cast<char *>(work) + align256((size_t)nb * sizeof(int));
    cudaError_t e = exclusive_scan(sums, sums, nb, rest, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(out, n, sums);
    return cudaGetLastError();
}

size_t sort_workspace_bytes(long long n) {
    const long long nb = ceil_div(n > 0 ? n : 1, SORT_TILE);
    return align256((size_t)256 * nb * sizeof(int)) + scan_workspace_bytes(256 * nb);
}

cudaError_t sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys, uint32_t *tmp_vals, long long n,
                       int bits, void *work, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const long long nb = ceil_div(n, SORT_TILE);
    int *hist = static_cast<int *>(work);
    void *scan_work = static_cast<char *>(work) + align256((size_t)256 * nb * sizeof(int));
    uint32_t *ka = keys, *va = vals, *kb = tmp_keys, *vb = tmp_vals;
    for (int shift = 0; shift < bits; shift += 8) {
        k_digit_hist<<<(unsigned)nb, SORT_THREADS, 0, st>>>(ka, n, shift, hist);
        cudaError_t e = exclusive_scan(hist, hist, 256 * nb, scan_work, st);
        if (e != cudaSuccess) return e;
        k_digit_scatter<<<(unsigned)nb, SORT_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (ka != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, ka, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        return e;
    }
    return cudaSuccess;
}

}  // namespace lbm
