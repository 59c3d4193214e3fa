// Smoke tracers (Sec. 6, rendering paragraph): advection by the explicit midpoint rule in the
// trilinear lattice velocity with seeded re-injection, and the cloud-in-cell density on a
// volume grid computed as a stable sort of the contributions by voxel followed by a
// segmented sum (deterministic, no float atomics).  The readings are stated in lbm.h.
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

// one tracer per thread; positions are SoA [3][count]
__global__ void __launch_bounds__(256) k_advect(float *__restrict__ X, long long count, const float *__restrict__ u,
                                                long long ncell, TracerGrid g, Emitter em, long long t) {
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
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long ctr = ((unsigned long long)(t - 1) * (unsigned long long)count +
                                            (unsigned long long)i) * 3ull + (unsigned long long)a;
            const float U = (float)(splitmix64(em.seed, ctr) >> 40) * 0x1p-24f;
            p[a] = fmaf(em.ext[a], U, em.lo[a]);
        }
        xn = p[0]; yn = p[1]; zn = p[2];
    }
    X[i] = xn;
    X[count + i] = yn;
    X[2 * count + i] = zn;
}

// the 8 (voxel, weight) contributions of every tracer: entry 8 i + c, c = dx + 2 dy + 4 dz
__global__ void __launch_bounds__(256) k_splat_pairs(const float *__restrict__ X, long long count, TracerGrid g,
                                                     float s, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int x0, x1, y0, y1, z0, z1;
    float wx, wy, wz;
    axis_stencil(X[i] / s, g.n[0], g.periodic[0], x0, x1, wx);
    axis_stencil(X[count + i] / s, g.n[1], g.periodic[1], y0, y1, wy);
    axis_stencil(X[2 * count + i] / s, g.n[2], g.periodic[2], z0, z1, wz);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int ix = c & 1 ? x1 : x0, iy = c & 2 ? y1 : y0, iz = c & 4 ? z1 : z0;
        const float k = (c & 1 ? wx : 1.0f - wx) * (c & 2 ? wy : 1.0f - wy) * (c & 4 ? wz : 1.0f - wz);
        keys[8 * i + c] = (uint32_t)(ix + g.n[0] * (iy + g.n[1] * iz));
        vals[8 * i + c] = __float_as_uint(k);
    }
}

// AoS (x, y, z per tracer) <-> SoA [3][count]
__global__ void k_aos_to_soa(const float *__restrict__ in, float *__restrict__ out, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int a = 0; a < 3; ++a) out[a * count + i] = in[3 * i + a];
}
__global__ void k_soa_to_aos(const float *__restrict__ in, float *__restrict__ out, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int a = 0; a < 3; ++a) out[3 * i + a] = in[a * count + i];
}

inline unsigned blocks_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }

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

}  // namespace
}  // namespace lbm

namespace lbm_host {

int advect_tracers(lbm_ctx *h, long long t) {
    if (h->ntracer == 0) return LBM_OK;
    Timed tm(h, LBM_KERNEL_TRACER);
    lbm::Emitter em{};
    for (int a = 0; a < 3; ++a) {
        em.lo[a] = (float)h->emitter.lo[a];
        em.ext[a] = (float)(h->emitter.hi[a] - h->emitter.lo[a]);
    }
    em.seed = h->emitter.seed;
    lbm::k_advect<<<lbm::blocks_of(h->ntracer, 256), 256, 0, h->stream>>>(h->tx, h->ntracer, h->tracer_u, h->N,
                                                                          lbm::lattice_grid(h), em, t);
    CK(cudaGetLastError());
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
    float *staging = nullptr;
    if ((rc = dev_alloc(h, &h->tx, (size_t)3 * count)) || (rc = dev_alloc(h, &h->tracer_u, (size_t)3 * h->N)) ||
        (rc = dev_alloc(h, &staging, (size_t)3 * count))) {
        dev_free(staging);
        free_tracers(h);
        return rc;
    }
    h->ntracer = count;
    if (em) h->emitter = *em;
    else std::memset(&h->emitter, 0, sizeof(h->emitter));
    cudaError_t e = cudaMemcpyAsync(staging, pos.data(), pos.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        lbm::k_aos_to_soa<<<lbm::blocks_of(count, 256), 256, 0, h->stream>>>(staging, h->tx, count);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(staging);
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
    lbm::k_soa_to_aos<<<lbm::blocks_of(h->ntracer, 256), 256, 0, h->stream>>>(h->tx, out, h->ntracer);
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
    const long long M = 8 * h->ntracer;   // contributions
    const bool dev = is_device_ptr(out);
    // workspace: [grid if out is on the host][4 arrays of M words][sort workspace]
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t grid_b = dev ? 0 : al((size_t)4 * G), pair_b = al((size_t)4 * M);
    const size_t need = grid_b + 4 * pair_b + lbm::sort_workspace_bytes(M);
    if (need > h->tracer_ws_bytes) {
        if (h->tracer_ws) cudaFree(h->tracer_ws);
        h->tracer_ws = nullptr;
        h->tracer_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&h->tracer_ws, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->tracer_ws = nullptr;
            return fail(h, LBM_ENOMEM, "cannot allocate the density workspace (" + std::to_string(need) + " bytes)");
        }
        h->tracer_ws_bytes = need;
    }
    char *w = static_cast<char *>(h->tracer_ws);
    float *grid = dev ? out : reinterpret_cast<float *>(w);
    w += grid_b;
    uint32_t *keys = reinterpret_cast<uint32_t *>(w), *vals = reinterpret_cast<uint32_t *>(w + pair_b);
    uint32_t *tk = reinterpret_cast<uint32_t *>(w + 2 * pair_b), *tv = reinterpret_cast<uint32_t *>(w + 3 * pair_b);
    void *sort_ws = w + 4 * pair_b;
    int bits = 1;
    while (bits < 32 && (1LL << bits) < G) ++bits;
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(cudaMemsetAsync(grid, 0, (size_t)4 * G, h->stream));
        if (M > 0) {
            lbm::k_splat_pairs<<<lbm::blocks_of(h->ntracer, 256), 256, 0, h->stream>>>(h->tx, h->ntracer, g, (float)s,
                                                                                       keys, vals);
            CK(cudaGetLastError());
            CK(lbm::sort_pairs(keys, vals, tk, tv, M, bits, sort_ws, h->stream));
            CK(lbm::segmented_sum(keys, reinterpret_cast<const float *>(vals), M, grid, h->stream));
        }
    }
    if (!dev) CK(cudaMemcpyAsync(out, grid, (size_t)4 * G, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // extern "C"
