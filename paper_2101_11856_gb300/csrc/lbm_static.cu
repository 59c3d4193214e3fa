// Allocation-free FP64 sum of per-sample immersed-boundary forces (lbm_sum_forces_static).
//
// The context-based lbm_reductions keeps its partial sums in scratch that lbm_create /
// the first reduction allocates with cudaMalloc.  Some callers cannot call cudaMalloc at
// the point where they need the sum: code that runs while a memory pool is locked or
// allocation is forbidden (real-time loops, allocator-less embeddings, regions where a
// surrounding framework owns every allocation).  This entry point takes the caller's
// forces and output and keeps its partial sums in the fixed device array below, so it
// allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// its 48 KiB until the process exits.  All calls on a device share it and it keeps the
// last call's contents; every slot a call reads is written by that same call first, so
// nothing has to start at zero.  Calls whose work overlaps on the GPU (different streams,
// no ordering between them) race on the array and must be serialised by the caller.  The
// array's device address is looked up once per device and cached, so a cudaDeviceReset after
// the first call in the same process is not supported (the cached address would be stale).
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kStaticBlocks = 2048;      // partial sums per component
constexpr int kStaticThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_force_partial[3 * kStaticBlocks];

double *g_partial_addr[kMaxDevices] = {};
std::mutex g_partial_mutex;

// device address of g_force_partial on the current device (looked up once per device)
cudaError_t static_partial(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_partial_mutex);
    if (!g_partial_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_force_partial);
        if (e != cudaSuccess) return e;
        g_partial_addr[dev] = static_cast<double *>(p);
    }
    *out = g_partial_addr[dev];
    return cudaSuccess;
}

// per-block FP64 sums of g[3 s + a] (caller's interleaved layout), grid-stride over samples
__global__ void __launch_bounds__(kStaticThreads) k_sum_forces_aos(long long S, const float *__restrict__ g,
                                                                   double *__restrict__ partial) {
    __shared__ double s[3][kStaticThreads];
    double a[3] = {0.0, 0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
        a[0] += g[3 * i];
        a[1] += g[3 * i + 1];
        a[2] += g[3 * i + 2];
    }
    for (int k = 0; k < 3; ++k) s[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partial[(long long)k * gridDim.x + blockIdx.x] = s[k][0];
}

}  // namespace

extern "C" int lbm_sum_forces_static(const float *g, long long count, double *out, void *cuda_stream) {
    if (count < 0 || count > LBM_STATIC_MAX_SAMPLES || !out || (count > 0 && !g)) return LBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // an error left pending by earlier work on this thread is not this call's: report it
    // without launching and leave it pending, so the launch checks below see only this call
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
    double *partial = nullptr;
    if (static_partial(&partial) != cudaSuccess) return LBM_ECUDA;
    long long blocks = (count + kStaticThreads - 1) / kStaticThreads;
    if (blocks > kStaticBlocks) blocks = kStaticBlocks;
    if (blocks > 0) k_sum_forces_aos<<<(unsigned)blocks, kStaticThreads, 0, st>>>(count, g, partial);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (lbm::launch_finalize(partial, blocks, 3, out, st) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}
