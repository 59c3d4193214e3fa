// Smoke tracers (Sec. 6, rendering paragraph): advection by the explicit midpoint rule in the
// trilinear lattice velocity with seeded re-injection, and the cloud-in-cell density on a
// volume grid.  The readings are stated in lbm.h.
//
// Storage: the tracers are kept in 4x4x4-cell brick order (a stable radix sort by brick
// after every advection, carrying the caller's index of each tracer), so the eight-corner
// velocity gathers of a warp fall on a few cache lines.  Density: the tracers are sorted
// by base voxel, the first entry of every run is recorded in a dense table, and each voxel
// gathers the runs of its eight lower neighbours in a fixed order (FP64): a segmented
// reduction without float atomics, so the result is bit-reproducible.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbm_ctx.h"
#include "lbm_sort.cuh"

using namespace lbm_host;

namespace lbm {
namespace {

struct TracerGrid {
    int n[3];           // nodes (advection) or voxels (density) per axis
    int periodic[3];
};

// lower / upper index and upper weight along one axis (see lbm_set_tracers)
__device__ __forceinline__ void axis_stencil(float x, int n, int periodic, int &i0, int &i1, float &w) {
    if (periodic) {
        const float b = floorf(x);
        w = x - b;
        int i = (int)b % n;
        if (i < 0) i += n;
        i0 = i;
        i1 = i + 1 == n ? 0 : i + 1;
    } else {
        const float b = fminf(floorf(x), (float)(n - 2));
        w = x - b;
        i0 = (int)b;
        i1 = i0 + 1;
    }
}

__device__ __forceinline__ void interp_u(const float *__restrict__ u, long long ncell, const TracerGrid &g, float x,
                                         float y, float z, float &ux, float &uy, float &uz) {
    int x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
    axis_stencil(x, g.n[0], g.periodic[0], x0, x1, wx);
    axis_stencil(y, g.n[1], g.periodic[1], y0, y1, wy);
    axis_stencil(z, g.n[2], g.periodic[2], z0, z1, wz);
    ux = uy = uz = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int ix = c & 1 ? x1 : x0, iy = c & 2 ? y1 : y0, iz = c & 4 ? z1 : z0;
        const float k = (c & 1 ? wx : 1.0f - wx) * (c & 2 ? wy : 1.0f - wy) * (c & 4 ? wz : 1.0f - wz);
        const long long cell = ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
        ux = fmaf(k, __ldg(u + cell), ux);
        uy = fmaf(k, __ldg(u + ncell + cell), uy);
        uz = fmaf(k, __ldg(u + 2 * ncell + cell), uz);
    }
}

__device__ __forceinline__ float wrap_axis(float x, int n, int periodic) {
    if (periodic) {
        if (x < 0.0f) x += (float)n;
        if (x >= (float)n) x -= (float)n;
    }
    return x;
}

__device__ __forceinline__ bool inside(const TracerGrid &g, float x, float y, float z) {
    const float c[3] = {x, y, z};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (!g.periodic[a]) ok = ok && c[a] >= 0.0f && c[a] <= (float)(g.n[a] - 1);
    return ok;
}

struct Emitter {
    float lo[3], ext[3];
    unsigned long long seed;
};

// brick (4x4x4 cells) of a position: the storage order of the tracers
constexpr int BRICK = 4;
__device__ __forceinline__ uint32_t brick_key(const TracerGrid &g, float x, float y, float z) {
    const int bx = (g.n[0] + BRICK - 1) / BRICK, by = (g.n[1] + BRICK - 1) / BRICK;
    const int ix = min(max((int)x, 0), g.n[0] - 1) / BRICK, iy = min(max((int)y, 0), g.n[1] - 1) / BRICK,
              iz = min(max((int)z, 0), g.n[2] - 1) / BRICK;
    return (uint32_t)(ix + bx * (iy + by * iz));
}

// one stored tracer per thread; positions SoA [3][count], id = the caller's index (the
// counter of its re-injection draws); writes the new position and its brick key and slot
__global__ void __launch_bounds__(256) k_advect(float *__restrict__ X, const uint32_t *__restrict__ id, long long count,
                                                const float *__restrict__ u, long long ncell, TracerGrid g, Emitter em,
                                                long long t, uint32_t *__restrict__ key, uint32_t *__restrict__ slot) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float x = X[i], y = X[count + i], z = X[2 * count + i];
    float ux, uy, uz;
    interp_u(u, ncell, g, x, y, z, ux, uy, uz);
    const float xm = wrap_axis(fmaf(0.5f, ux, x), g.n[0], g.periodic[0]);
    const float ym = wrap_axis(fmaf(0.5f, uy, y), g.n[1], g.periodic[1]);
    const float zm = wrap_axis(fmaf(0.5f, uz, z), g.n[2], g.periodic[2]);
    float xn = x, yn = y, zn = z;
    bool ok = inside(g, xm, ym, zm);
    if (ok) {
        interp_u(u, ncell, g, xm, ym, zm, ux, uy, uz);
        xn = wrap_axis(x + ux, g.n[0], g.periodic[0]);
        yn = wrap_axis(y + uy, g.n[1], g.periodic[1]);
        zn = wrap_axis(z + uz, g.n[2], g.periodic[2]);
        ok = inside(g, xn, yn, zn);
    }
    if (!ok) {
        float p[3];
        const unsigned long long me = id[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long ctr =
                ((unsigned long long)(t - 1) * (unsigned long long)count + me) * 3ull + (unsigned long long)a;
            const float U = (float)(splitmix64(em.seed, ctr) >> 40) * 0x1p-24f;
            p[a] = fmaf(em.ext[a], U, em.lo[a]);
        }
        xn = p[0]; yn = p[1]; zn = p[2];
    }
    X[i] = xn;
    X[count + i] = yn;
    X[2 * count + i] = zn;
    key[i] = brick_key(g, xn, yn, zn);
    slot[i] = (uint32_t)i;
}

// gather the stored tracers into the sorted order: slot j of the output takes slot perm[j]
__global__ void __launch_bounds__(256) k_permute(const float *__restrict__ X, const uint32_t *__restrict__ id,
                                                 const uint32_t *__restrict__ perm, long long count,
                                                 float *__restrict__ Xo, uint32_t *__restrict__ ido) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const long long i = perm[j];
    Xo[j] = X[i];
    Xo[count + j] = X[count + i];
    Xo[2 * count + j] = X[2 * count + i];
    ido[j] = id[i];
}

// base voxel of every stored tracer on the density grid (spacing s)
__global__ void __launch_bounds__(256) k_density_keys(const float *__restrict__ X, long long count, TracerGrid g,
                                                      float s, uint32_t *__restrict__ key, uint32_t *__restrict__ slot) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int x0, x1, y0, y1, z0, z1;
    float w;
    axis_stencil(X[i] / s, g.n[0], g.periodic[0], x0, x1, w);
    axis_stencil(X[count + i] / s, g.n[1], g.periodic[1], y0, y1, w);
    axis_stencil(X[2 * count + i] / s, g.n[2], g.periodic[2], z0, z1, w);
    key[i] = (uint32_t)(x0 + g.n[0] * (y0 + g.n[1] * z0));
    slot[i] = (uint32_t)i;
}

// first sorted entry of every run of equal base voxels (start[] preset to -1)
__global__ void __launch_bounds__(256) k_run_heads(const uint32_t *__restrict__ key, long long count,
                                                   int *__restrict__ start) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    if (j == 0 || key[j - 1] != key[j]) start[key[j]] = (int)j;
}

// density of voxel v: the runs of the base voxels v - o, o in {0,1}^3 (wrapped on periodic
// axes), each tracer weighted for its corner o; FP64 in the fixed order (o, sorted entry)
__global__ void __launch_bounds__(256) k_density_gather(const float *__restrict__ X, long long count, TracerGrid g,
                                                        float s, const uint32_t *__restrict__ key,
                                                        const uint32_t *__restrict__ slot, const int *__restrict__ start,
                                                        float *__restrict__ out) {
    const long long G = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G) return;
    const int vx = (int)(v % g.n[0]), vy = (int)((v / g.n[0]) % g.n[1]), vz = (int)(v / ((long long)g.n[0] * g.n[1]));
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int dx = o & 1, dy = (o >> 1) & 1, dz = o >> 2;
        int bx = vx - dx, by = vy - dy, bz = vz - dz;
        if (bx < 0) { if (!g.periodic[0]) continue; bx += g.n[0]; }
        if (by < 0) { if (!g.periodic[1]) continue; by += g.n[1]; }
        if (bz < 0) { if (!g.periodic[2]) continue; bz += g.n[2]; }
        const uint32_t b = (uint32_t)(bx + g.n[0] * (by + g.n[1] * bz));
        for (long long j = start[b]; j >= 0 && j < count && key[j] == b; ++j) {
            const long long i = slot[j];
            int i0, i1;
            float wx, wy, wz;
            axis_stencil(X[i] / s, g.n[0], g.periodic[0], i0, i1, wx);
            axis_stencil(X[count + i] / s, g.n[1], g.periodic[1], i0, i1, wy);
            axis_stencil(X[2 * count + i] / s, g.n[2], g.periodic[2], i0, i1, wz);
            acc += (double)((dx ? wx : 1.0f - wx) * (dy ? wy : 1.0f - wy) * (dz ? wz : 1.0f - wz));
        }
    }
    out[v] = (float)acc;
}

// AoS (x, y, z per tracer) -> SoA [3][count]
__global__ void k_aos_to_soa(const float *__restrict__ in, float *__restrict__ out, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int a = 0; a < 3; ++a) out[a * count + i] = in[3 * i + a];
}
// stored order -> the caller's order (AoS)
__global__ void k_soa_to_aos(const float *__restrict__ in, const uint32_t *__restrict__ id, float *__restrict__ out,
                             long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const long long k = id[i];
    for (int a = 0; a < 3; ++a) out[3 * k + a] = in[a * count + i];
}
__global__ void k_iota(uint32_t *__restrict__ out, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (uint32_t)i;
}

inline unsigned blocks_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }
inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

TracerGrid lattice_grid(const lbm_ctx *h) {
    TracerGrid g{};
    g.n[0] = h->nx; g.n[1] = h->ny; g.n[2] = h->nz;
    for (int a = 0; a < 3; ++a) g.periodic[a] = h->cfg.face_type[2 * a] == LBM_FACE_PERIODIC;
    return g;
}

// density grid of spacing s; false if a periodic axis is not divisible by s
bool density_grid(const lbm_ctx *h, int s, TracerGrid &g) {
    g = lattice_grid(h);
    for (int a = 0; a < 3; ++a) {
        const int n = g.n[a];
        if (g.periodic[a]) {
            if (n % s) return false;
            g.n[a] = n / s;
        } else {
            g.n[a] = (n - 1 + s - 1) / s + 1;
        }
    }
    return true;
}

int bits_for(long long values) {
    int bits = 1;
    while (bits < 32 && (1LL << bits) < values) ++bits;
    return bits;
}

// the tracer workspace: key, slot and their sort copies (P words each), the sort workspace,
// then `extra` bytes (density tables)
struct TracerWs {
    uint32_t *key, *slot, *tkey, *tslot;
    void *sort;
    char *extra;
};

int tracer_ws(lbm_ctx *h, size_t extra, TracerWs &w) {
    const long long P = h->ntracer;
    const size_t pw = al256((size_t)4 * P), sb = al256(sort_workspace_bytes(P));
    const size_t need = 4 * pw + sb + extra;
    if (need > h->tracer_ws_bytes) {
        if (h->tracer_ws) cudaFree(h->tracer_ws);
        h->tracer_ws = nullptr;
        h->tracer_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&h->tracer_ws, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->tracer_ws = nullptr;
            return fail(h, LBM_ENOMEM, "cannot allocate the tracer workspace (" + std::to_string(need) + " bytes)");
        }
        h->tracer_ws_bytes = need;
    }
    char *p = static_cast<char *>(h->tracer_ws);
    w.key = reinterpret_cast<uint32_t *>(p);
    w.slot = reinterpret_cast<uint32_t *>(p + pw);
    w.tkey = reinterpret_cast<uint32_t *>(p + 2 * pw);
    w.tslot = reinterpret_cast<uint32_t *>(p + 3 * pw);
    w.sort = p + 4 * pw;
    w.extra = p + 4 * pw + sb;
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

namespace lbm_host {

int advect_tracers(lbm_ctx *h, long long t) {
    const long long P = h->ntracer;
    if (P == 0) return LBM_OK;
    lbm::TracerWs w;
    int rc = lbm::tracer_ws(h, 0, w);
    if (rc) return rc;
    const lbm::TracerGrid g = lbm::lattice_grid(h);
    lbm::Emitter em{};
    for (int a = 0; a < 3; ++a) {
        em.lo[a] = (float)h->emitter.lo[a];
        em.ext[a] = (float)(h->emitter.hi[a] - h->emitter.lo[a]);
    }
    em.seed = h->emitter.seed;
    {
        Timed tm(h, LBM_KERNEL_TRACER);
        lbm::k_advect<<<lbm::blocks_of(P, 256), 256, 0, h->stream>>>(h->tx, h->tid, P, h->tracer_u, h->N, g, em, t,
                                                                     w.key, w.slot);
        CK(cudaGetLastError());
    }
    {
        // keep the brick order for the next step's gathers
        Timed tm(h, LBM_KERNEL_OTHER);
        const long long bricks = (long long)((h->nx + 3) / 4) * ((h->ny + 3) / 4) * ((h->nz + 3) / 4);
        CK(lbm::sort_pairs(w.key, w.slot, w.tkey, w.tslot, P, lbm::bits_for(bricks), w.sort, h->stream));
        lbm::k_permute<<<lbm::blocks_of(P, 256), 256, 0, h->stream>>>(h->tx, h->tid, w.slot, P, h->tx_alt, h->tid_alt);
        CK(cudaGetLastError());
        std::swap(h->tx, h->tx_alt);
        std::swap(h->tid, h->tid_alt);
    }
    return LBM_OK;
}

}  // namespace lbm_host

extern "C" {

int lbm_set_tracers(lbm_ctx *h, const float *X, long long count, const lbm_emitter *em) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (count < 0 || count >= (1LL << 28)) return fail(h, LBM_EINVAL, "tracer count must be in [0, 2^28)");
    if (count > 0 && !X) return fail(h, LBM_EINVAL, "X is NULL");
    const lbm::TracerGrid g = lbm::lattice_grid(h);
    const int n[3] = {h->nx, h->ny, h->nz};
    bool all_periodic = true;
    for (int a = 0; a < 3; ++a) {
        if (!g.periodic[a]) {
            all_periodic = false;
            if (count > 0 && n[a] < 2) return fail(h, LBM_EINVAL, "tracers need >= 2 nodes along non-periodic axes");
        }
    }
    if (count > 0 && !all_periodic && !em) return fail(h, LBM_EINVAL, "an emitter is required with non-periodic faces");
    if (em && count > 0) {
        for (int a = 0; a < 3; ++a) {
            const double top = g.periodic[a] ? (double)n[a] : (double)(n[a] - 1);
            if (!(em->lo[a] >= 0.0 && em->lo[a] <= em->hi[a] && em->hi[a] <= top))
                return fail(h, LBM_EINVAL, "emitter box outside the domain or lo > hi");
        }
    }
    std::vector<float> pos;
    if (count > 0) {
        pos.resize((size_t)3 * count);
        if (is_device_ptr(X)) {
            CK(cudaMemcpyAsync(pos.data(), X, pos.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        } else {
            std::memcpy(pos.data(), X, pos.size() * sizeof(float));
        }
        for (long long i = 0; i < count; ++i)
            for (int a = 0; a < 3; ++a) {
                const float v = pos[3 * i + a];
                const bool ok = g.periodic[a] ? (v >= 0.0f && v < (float)n[a]) : (v >= 0.0f && v <= (float)(n[a] - 1));
                if (!ok) return fail(h, LBM_EINVAL, "tracer " + std::to_string(i) + " outside the domain");
            }
    }
    free_tracers(h);
    if (count == 0) return LBM_OK;
    int rc;
    if ((rc = dev_alloc(h, &h->tx, (size_t)3 * count)) || (rc = dev_alloc(h, &h->tx_alt, (size_t)3 * count)) ||
        (rc = dev_alloc(h, &h->tid, (size_t)count)) || (rc = dev_alloc(h, &h->tid_alt, (size_t)count)) ||
        (rc = dev_alloc(h, &h->tracer_u, (size_t)3 * h->N))) {
        free_tracers(h);
        return rc;
    }
    h->ntracer = count;
    if (em) h->emitter = *em;
    else std::memset(&h->emitter, 0, sizeof(h->emitter));
    // stage the AoS positions in the spare position buffer, then transpose
    cudaError_t e = cudaMemcpyAsync(h->tx_alt, pos.data(), pos.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        lbm::k_aos_to_soa<<<lbm::blocks_of(count, 256), 256, 0, h->stream>>>(h->tx_alt, h->tx, count);
        lbm::k_iota<<<lbm::blocks_of(count, 256), 256, 0, h->stream>>>(h->tid, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        free_tracers(h);
        return fail(h, LBM_ECUDA, std::string("tracer upload: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

long long lbm_tracer_count(const lbm_ctx *h) { return h ? h->ntracer : 0; }

int lbm_tracers(lbm_ctx *h, float *X) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (h->ntracer == 0) return LBM_OK;
    if (!X) return fail(h, LBM_EINVAL, "X is NULL");
    const size_t bytes = (size_t)12 * h->ntracer;
    const bool dev = is_device_ptr(X);
    float *out = X;
    int rc;
    if (!dev && (rc = dev_alloc(h, &out, (size_t)3 * h->ntracer))) return rc;
    lbm::k_soa_to_aos<<<lbm::blocks_of(h->ntracer, 256), 256, 0, h->stream>>>(h->tx, h->tid, out, h->ntracer);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(X, out, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (!dev) cudaFree(out);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, std::string("lbm_tracers: ") + cudaGetErrorString(e));
    return LBM_OK;
}

int lbm_tracer_dims(const lbm_ctx *h, int s, int dims[3]) {
    if (!h || !dims) return fail(const_cast<lbm_ctx *>(h), LBM_EINVAL, "null argument");
    if (s < 1) return fail(const_cast<lbm_ctx *>(h), LBM_EINVAL, "s must be >= 1");
    lbm::TracerGrid g;
    if (!lbm::density_grid(h, s, g)) return fail(const_cast<lbm_ctx *>(h), LBM_EINVAL, "periodic axis not divisible by s");
    for (int a = 0; a < 3; ++a) dims[a] = g.n[a];
    return LBM_OK;
}

int lbm_tracer_density(lbm_ctx *h, int s, float *out) {
    int dims[3];
    int rc = lbm_tracer_dims(h, s, dims);
    if (rc) return rc;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    const long long G = (long long)dims[0] * dims[1] * dims[2];
    if (G >= (1LL << 31)) return fail(h, LBM_EINVAL, "density grid of 2^31 voxels or more");
    lbm::TracerGrid g;
    lbm::density_grid(h, s, g);
    const long long P = h->ntracer;
    const bool dev = is_device_ptr(out);
    // extra workspace: run starts (G ints), then the grid when out is on the host
    const size_t start_b = lbm::al256((size_t)4 * G);
    lbm::TracerWs w;
    if ((rc = lbm::tracer_ws(h, start_b + (dev ? 0 : (size_t)4 * G), w))) return rc;
    int *start = reinterpret_cast<int *>(w.extra);
    float *grid = dev ? out : reinterpret_cast<float *>(w.extra + start_b);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        if (P == 0) {
            CK(cudaMemsetAsync(grid, 0, (size_t)4 * G, h->stream));
        } else {
            lbm::k_density_keys<<<lbm::blocks_of(P, 256), 256, 0, h->stream>>>(h->tx, P, g, (float)s, w.key, w.slot);
            CK(cudaGetLastError());
            CK(lbm::sort_pairs(w.key, w.slot, w.tkey, w.tslot, P, lbm::bits_for(G), w.sort, h->stream));
            CK(cudaMemsetAsync(start, 0xff, (size_t)4 * G, h->stream));
            lbm::k_run_heads<<<lbm::blocks_of(P, 256), 256, 0, h->stream>>>(w.key, P, start);
            lbm::k_density_gather<<<lbm::blocks_of(G, 256), 256, 0, h->stream>>>(h->tx, P, g, (float)s, w.key, w.slot,
                                                                                  start, grid);
            CK(cudaGetLastError());
        }
    }
    if (!dev) CK(cudaMemcpyAsync(out, grid, (size_t)4 * G, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // extern "C"
