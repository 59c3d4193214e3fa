// Moving and rotating solids (Algorithm 2 (c): the sample update after the IB stage, and the
// torque reduction).  At the start of every step the samples are placed at the pose of the
// previous time in FP64, re-sorted by base cell with the stable radix sort, and the band
// (bitmap + tile offsets), the corner band indices and the spreading lists are rebuilt on the
// device, the same structures lbm_set_solids builds on the host for a static solid.  The
// band arrays have the fixed stride nband = 8 S (or N) and the band size is a device count,
// so the host never waits for the rebuild.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lbm_ctx.h"
#include "lbm_sort.cuh"

using namespace lbm_host;

namespace lbm {
namespace {

struct Pose {
    double c0[3];        // rotation centre of the reference pose
    double c[3];         // centre now
    double R[9];         // rotation now (row-major)
    double V[3];         // translation per step
    double Om[3];        // angular velocity vector
};

struct Lattice {
    int nx, ny, nz;
    long long nxy;
};

__device__ __forceinline__ void pose_point(const Pose &p, const float *__restrict__ rel, long long S, long long i,
                                           double (&X)[3]) {
    const double r[3] = {(double)rel[i], (double)rel[S + i], (double)rel[2 * S + i]};
#pragma unroll
    for (int a = 0; a < 3; ++a) X[a] = p.c[a] + p.R[3 * a] * r[0] + p.R[3 * a + 1] * r[1] + p.R[3 * a + 2] * r[2];
}

// base cell of a position (kept inside [0, n-2] per axis; the host checks the pose first)
__device__ __forceinline__ long long base_cell(const Lattice &L, float x, float y, float z) {
    const int bx = min(max((int)floorf(x), 0), L.nx - 2), by = min(max((int)floorf(y), 0), L.ny - 2),
              bz = min(max((int)floorf(z), 0), L.nz - 2);
    return bx + (long long)L.nx * by + L.nxy * bz;
}

// positions of the reference samples (in their current order) at the new pose, with keys
__global__ void __launch_bounds__(256) k_pose(long long S, const float *__restrict__ rel, Pose p, Lattice L,
                                              float *__restrict__ Xtmp, uint32_t *__restrict__ key,
                                              uint32_t *__restrict__ slot) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    double X[3];
    pose_point(p, rel, S, i, X);
    const float x = (float)X[0], y = (float)X[1], z = (float)X[2];
    Xtmp[i] = x;
    Xtmp[S + i] = y;
    Xtmp[2 * S + i] = z;
    key[i] = (uint32_t)base_cell(L, x, y, z);
    slot[i] = (uint32_t)i;
}

// the samples in sorted order: positions, reference coordinates, area, caller index and the
// rigid-body boundary velocity V + Om x (X - c) (FP64)
__global__ void __launch_bounds__(256) k_gather_samples(long long S, const uint32_t *__restrict__ slot,
                                                        const float *__restrict__ Xtmp, const float *__restrict__ rel,
                                                        const float *__restrict__ area, const int *__restrict__ sid,
                                                        Pose p, float *__restrict__ X, float *__restrict__ rel_o,
                                                        float *__restrict__ area_o, int *__restrict__ sid_o,
                                                        float *__restrict__ ub) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    const long long i = slot[j];
    double P[3];
    pose_point(p, rel, S, i, P);
    const double d[3] = {P[0] - p.c[0], P[1] - p.c[1], P[2] - p.c[2]};
    const double u[3] = {p.V[0] + p.Om[1] * d[2] - p.Om[2] * d[1], p.V[1] + p.Om[2] * d[0] - p.Om[0] * d[2],
                         p.V[2] + p.Om[0] * d[1] - p.Om[1] * d[0]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        X[a * S + j] = Xtmp[a * S + i];
        rel_o[a * S + j] = rel[a * S + i];
        ub[a * S + j] = (float)u[a];
    }
    area_o[j] = area[i];
    sid_o[j] = sid[i];
}

__device__ __forceinline__ long long corner_cell(const Lattice &L, long long base, int c) {
    return base + (c & 1) + ((c >> 1) & 1) * (long long)L.nx + ((c >> 2) & 1) * L.nxy;
}

// band bitmap: the 8 stencil nodes of every sample
__global__ void __launch_bounds__(256) k_mark_band(long long S, const float *__restrict__ X, Lattice L,
                                                   uint32_t *__restrict__ mask) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    const long long b = base_cell(L, X[j], X[S + j], X[2 * S + j]);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long cell = corner_cell(L, b, c);
        atomicOr(&mask[cell >> 5], 1u << (cell & 31));
    }
}

__global__ void __launch_bounds__(256) k_popc(long long ntiles, const uint32_t *__restrict__ mask, int *__restrict__ off) {
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < ntiles) off[w] = __popc(mask[w]);
}

__global__ void k_band_total(long long ntiles, const uint32_t *__restrict__ mask, const int *__restrict__ off,
                             int *__restrict__ count) {
    *count = off[ntiles - 1] + __popc(mask[ntiles - 1]);
}

__device__ __forceinline__ int band_index(const uint32_t *__restrict__ mask, const int *__restrict__ off, long long cell) {
    const uint32_t m = mask[cell >> 5];
    const int l = (int)(cell & 31);
    if (!((m >> l) & 1u)) return -1;
    return off[cell >> 5] + __popc(m & ((1u << l) - 1u));
}

// band index of the 8 corners of every sample, and the cell of every band node
__global__ void __launch_bounds__(256) k_corner_band(long long S, const float *__restrict__ X, Lattice L,
                                                     const uint32_t *__restrict__ mask, const int *__restrict__ off,
                                                     int *__restrict__ corner_band, int *__restrict__ band_cell) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    const long long b = base_cell(L, X[j], X[S + j], X[2 * S + j]);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long cell = corner_cell(L, b, c);
        const int bi = band_index(mask, off, cell);
        corner_band[c * S + j] = bi;
        band_cell[bi] = (int)cell;   // equal values from every sample sharing the node
    }
}

// the run of samples based at each band node: first sorted index, then its length
__global__ void __launch_bounds__(256) k_run_start(long long S, const uint32_t *__restrict__ key,
                                                   const int *__restrict__ corner_band, int *__restrict__ cstart) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    if (j == 0 || key[j - 1] != key[j]) cstart[corner_band[j]] = (int)j;
}
__global__ void __launch_bounds__(256) k_run_count(long long S, const uint32_t *__restrict__ key,
                                                   const int *__restrict__ corner_band, const int *__restrict__ cstart,
                                                   int *__restrict__ ccount) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    if (j == S - 1 || key[j + 1] != key[j]) {
        const int bi = corner_band[j];
        ccount[bi] = (int)(j - cstart[bi] + 1);
    }
}

// for every band node, the band node of each of its 8 lower neighbours that is the base of
// at least one sample (-1 otherwise); stride = the band array stride
__global__ void __launch_bounds__(256) k_base_nbr(long long stride, const int *__restrict__ count,
                                                  const int *__restrict__ band_cell, Lattice L,
                                                  const uint32_t *__restrict__ mask, const int *__restrict__ off,
                                                  const int *__restrict__ ccount, int *__restrict__ base_nbr) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *count) return;
    const long long cell = band_cell[k];
    const int x = (int)(cell % L.nx), y = (int)((cell / L.nx) % L.ny), z = (int)(cell / L.nxy);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int bx = x - (c & 1), by = y - ((c >> 1) & 1), bz = z - ((c >> 2) & 1);
        int v = -1;
        if (bx >= 0 && by >= 0 && bz >= 0) {
            const int bi = band_index(mask, off, bx + (long long)L.nx * by + L.nxy * bz);
            if (bi >= 0 && ccount[bi] > 0) v = bi;
        }
        base_nbr[c * stride + k] = v;
    }
}

// FP64 block partial sums of the torque sum (X - c) x (-g)
__global__ void __launch_bounds__(256) k_sum_torque(long long S, const float *__restrict__ X, const float *__restrict__ g,
                                                   double cx, double cy, double cz, double *__restrict__ partial) {
    __shared__ double s[3][256];
    double a[3] = {0.0, 0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
        const double dx = (double)X[i] - cx, dy = (double)X[S + i] - cy, dz = (double)X[2 * S + i] - cz;
        const double fx = -(double)g[i], fy = -(double)g[S + i], fz = -(double)g[2 * S + i];
        a[0] += dy * fz - dz * fy;
        a[1] += dz * fx - dx * fz;
        a[2] += dx * fy - dy * fx;
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

__global__ void __launch_bounds__(256) k_rel(long long S, const float *__restrict__ X, double cx, double cy, double cz,
                                             float *__restrict__ rel) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    rel[i] = (float)((double)X[i] - cx);
    rel[S + i] = (float)((double)X[S + i] - cy);
    rel[2 * S + i] = (float)((double)X[2 * S + i] - cz);
}

inline unsigned blocks_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }
inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

int bits_for(long long values) {
    int bits = 1;
    while (bits < 32 && (1LL << bits) < values) ++bits;
    return bits;
}

// pose of the motion at tau steps after lbm_set_motion
Pose make_pose(const lbm_motion &m, double tau) {
    Pose p{};
    double k[3] = {m.axis[0], m.axis[1], m.axis[2]};
    const double n = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    const double w = n > 0.0 ? m.omega : 0.0;
    if (n > 0.0)
        for (double &v : k) v /= n;
    const double th = w * tau, c = std::cos(th), s = std::sin(th), C = 1.0 - c;
    const double R[9] = {c + k[0] * k[0] * C,        k[0] * k[1] * C - k[2] * s, k[0] * k[2] * C + k[1] * s,
                         k[1] * k[0] * C + k[2] * s, c + k[1] * k[1] * C,        k[1] * k[2] * C - k[0] * s,
                         k[2] * k[0] * C - k[1] * s, k[2] * k[1] * C + k[0] * s, c + k[2] * k[2] * C};
    for (int i = 0; i < 9; ++i) p.R[i] = R[i];
    for (int a = 0; a < 3; ++a) {
        p.c0[a] = m.center[a];
        p.c[a] = m.center[a] + m.velocity[a] * tau;
        p.V[a] = m.velocity[a];
        p.Om[a] = w * k[a];
    }
    return p;
}

Lattice lattice(const lbm_ctx *h) { return Lattice{h->nx, h->ny, h->nz, (long long)h->nx * h->ny}; }

}  // namespace
}  // namespace lbm

namespace lbm_host {

namespace {

// key, slot and their sort copies (S words each) and the sort workspace
struct MotionWs {
    uint32_t *key, *slot, *tkey, *tslot;
    void *sort;
};

int motion_ws(lbm_ctx *h, MotionWs &w) {
    const long long S = h->S;
    const size_t pw = lbm::al256((size_t)4 * S);
    const size_t need = 4 * pw + lbm::al256(std::max(lbm::sort_workspace_bytes(S), lbm::scan_workspace_bytes(h->ntiles)));
    if (need > h->motion_ws_bytes) {
        if (h->motion_ws) cudaFree(h->motion_ws);
        h->motion_ws = nullptr;
        h->motion_ws_bytes = 0;
        if (cudaMalloc(&h->motion_ws, need) != cudaSuccess) {
            cudaGetLastError();
            h->motion_ws = nullptr;
            return fail(h, LBM_ENOMEM, "cannot allocate the motion workspace");
        }
        h->motion_ws_bytes = need;
    }
    char *p = static_cast<char *>(h->motion_ws);
    w.key = reinterpret_cast<uint32_t *>(p);
    w.slot = reinterpret_cast<uint32_t *>(p + pw);
    w.tkey = reinterpret_cast<uint32_t *>(p + 2 * pw);
    w.tslot = reinterpret_cast<uint32_t *>(p + 3 * pw);
    w.sort = p + 4 * pw;
    return LBM_OK;
}

// the samples at the pose of time `abs_t` (absolute step count); rebuilds every IB structure
int rebuild(lbm_ctx *h, long long abs_t) {
    const long long S = h->S;
    const double tau = (double)(abs_t - h->posed_tau0);
    const lbm::Pose p = lbm::make_pose(h->motion, tau);
    // the sphere of radius r_max about the centre must stay inside [0, n - 1) with a margin
    const int n[3] = {h->nx, h->ny, h->nz};
    for (int a = 0; a < 3; ++a)
        if (!(p.c[a] - h->r_max >= 1e-3 && p.c[a] + h->r_max <= n[a] - 1 - 1e-3))
            return fail(h, LBM_EINVAL, "the moving solid leaves the domain at step " + std::to_string(abs_t + 1));
    MotionWs w;
    int rc = motion_ws(h, w);
    if (rc) return rc;
    const lbm::Lattice L = lbm::lattice(h);
    const unsigned bs = lbm::blocks_of(S, 256);
    Timed tm(h, LBM_KERNEL_MOTION);
    lbm::k_pose<<<bs, 256, 0, h->stream>>>(S, h->X0, p, L, h->Xtmp, w.key, w.slot);
    CK(cudaGetLastError());
    CK(lbm::sort_pairs(w.key, w.slot, w.tkey, w.tslot, S, lbm::bits_for(h->N), w.sort, h->stream));
    lbm::k_gather_samples<<<bs, 256, 0, h->stream>>>(S, w.slot, h->Xtmp, h->X0, h->area, h->sid, p, h->X, h->X0_alt,
                                                     h->area_alt, h->sid_alt, h->ub);
    CK(cudaGetLastError());
    std::swap(h->X0, h->X0_alt);
    std::swap(h->area, h->area_alt);
    std::swap(h->sid, h->sid_alt);
    CK(cudaMemsetAsync(h->tile_mask, 0, (size_t)4 * h->ntiles, h->stream));
    lbm::k_mark_band<<<bs, 256, 0, h->stream>>>(S, h->X, L, h->tile_mask);
    lbm::k_popc<<<lbm::blocks_of(h->ntiles, 256), 256, 0, h->stream>>>(h->ntiles, h->tile_mask, h->tile_off);
    CK(cudaGetLastError());
    CK(lbm::exclusive_scan(h->tile_off, h->tile_off, h->ntiles, w.sort, h->stream));
    lbm::k_band_total<<<1, 1, 0, h->stream>>>(h->ntiles, h->tile_mask, h->tile_off, h->band_count_dev);
    lbm::k_corner_band<<<bs, 256, 0, h->stream>>>(S, h->X, L, h->tile_mask, h->tile_off, h->corner_band, h->band_cell);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(h->ccount, 0, (size_t)4 * h->nband, h->stream));
    lbm::k_run_start<<<bs, 256, 0, h->stream>>>(S, w.key, h->corner_band, h->cstart);
    lbm::k_run_count<<<bs, 256, 0, h->stream>>>(S, w.key, h->corner_band, h->cstart, h->ccount);
    lbm::k_base_nbr<<<lbm::blocks_of(h->nband, 256), 256, 0, h->stream>>>(h->nband, h->band_count_dev, h->band_cell, L,
                                                                          h->tile_mask, h->tile_off, h->ccount,
                                                                          h->base_nbr);
    CK(cudaGetLastError());
    h->posed_tau = abs_t;
    return LBM_OK;
}

}  // namespace

int motion_before_step(lbm_ctx *h, long long t) {
    if (!h->moving || h->S == 0 || h->posed_tau == t - 1) return LBM_OK;
    return rebuild(h, t - 1);
}

int sync_order(lbm_ctx *h) {
    if (!h->sid || h->S == 0) return LBM_OK;
    std::vector<int> sid((size_t)h->S);
    CK(cudaMemcpyAsync(sid.data(), h->sid, sid.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < sid.size(); ++i) h->order[i] = sid[i];
    return LBM_OK;
}

}  // namespace lbm_host

extern "C" {

int lbm_set_motion(lbm_ctx *h, const lbm_motion *m) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (h->S == 0) return fail(h, LBM_ESTATE, "lbm_set_solids has not been called");
    if (!m) {
        h->moving = false;
        return LBM_OK;
    }
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(m->center[a]) || !std::isfinite(m->velocity[a]) || !std::isfinite(m->axis[a]))
            return fail(h, LBM_EINVAL, "non-finite motion");
    if (!std::isfinite(m->omega)) return fail(h, LBM_EINVAL, "non-finite motion");
    const long long S = h->S;
    int rc;
    if (!h->band_count_dev) {
        // first motion of this solid: switch the band arrays to the fixed stride and set up
        // the reference samples (the current positions, relative to the centre)
        const long long cap = std::min<long long>(8 * S, h->N);
        CK(cudaStreamSynchronize(h->stream));
        dev_free(h->band_cell); dev_free(h->cstart); dev_free(h->ccount); dev_free(h->base_nbr);
        dev_free(h->band_rho); dev_free(h->band_u); dev_free(h->bandF);
        if ((rc = dev_alloc(h, &h->band_cell, (size_t)cap)) || (rc = dev_alloc(h, &h->cstart, (size_t)cap)) ||
            (rc = dev_alloc(h, &h->ccount, (size_t)cap)) || (rc = dev_alloc(h, &h->base_nbr, (size_t)8 * cap)) ||
            (rc = dev_alloc(h, &h->band_rho, (size_t)cap)) || (rc = dev_alloc(h, &h->band_u, (size_t)3 * cap)) ||
            (rc = dev_alloc(h, &h->bandF, (size_t)3 * cap)) || (rc = dev_alloc(h, &h->band_count_dev, 1)) ||
            (rc = dev_alloc(h, &h->X0, (size_t)3 * S)) || (rc = dev_alloc(h, &h->X0_alt, (size_t)3 * S)) ||
            (rc = dev_alloc(h, &h->area_alt, (size_t)S)) || (rc = dev_alloc(h, &h->Xtmp, (size_t)3 * S)) ||
            (rc = dev_alloc(h, &h->sid, (size_t)S)) || (rc = dev_alloc(h, &h->sid_alt, (size_t)S))) {
            free_solid(h);
            return rc;
        }
        h->nband = cap;
        CK(cudaMemsetAsync(h->bandF, 0, (size_t)12 * cap, h->stream));
        std::vector<int> sid((size_t)S);
        for (long long i = 0; i < S; ++i) sid[i] = (int)h->order[i];
        CK(cudaMemcpyAsync(h->sid, sid.data(), sid.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    // reference pose = the samples now, about the given centre
    std::vector<float> X((size_t)3 * S);
    CK(cudaMemcpyAsync(X.data(), h->X, X.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double r2 = 0.0;
    for (long long i = 0; i < S; ++i) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double d = (double)X[a * S + i] - m->center[a];
            d2 += d * d;
        }
        r2 = std::max(r2, d2);
    }
    lbm::k_rel<<<lbm::blocks_of(S, 256), 256, 0, h->stream>>>(S, h->X, m->center[0], m->center[1], m->center[2], h->X0);
    CK(cudaGetLastError());
    h->motion = *m;
    h->r_max = std::sqrt(r2);
    h->moving = true;
    h->ub_zero = false;             // the rigid-body velocities are written at every pose
    h->posed_tau0 = h->t;
    h->posed_tau = -1;
    if ((rc = rebuild(h, h->t))) {
        h->moving = false;
        return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_solid_samples(lbm_ctx *h, float *X) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (h->S == 0) return LBM_OK;
    if (!X) return fail(h, LBM_EINVAL, "X is NULL");
    int rc = sync_order(h);
    if (rc) return rc;
    const size_t S = (size_t)h->S;
    std::vector<float> sorted(3 * S), out(3 * S);
    CK(cudaMemcpyAsync(sorted.data(), h->X, 3 * S * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < S; ++i)
        for (int a = 0; a < 3; ++a) out[3 * h->order[i] + a] = sorted[a * S + i];
    CK(cudaMemcpyAsync(X, out.data(), 3 * S * sizeof(float), cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_solid_torque(lbm_ctx *h, const double center[3], double torque[3]) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!torque) return fail(h, LBM_EINVAL, "torque is NULL");
    double c[3] = {0.0, 0.0, 0.0};
    if (center) {
        for (int a = 0; a < 3; ++a) c[a] = center[a];
    } else if (h->band_count_dev) {
        const lbm::Pose p = lbm::make_pose(h->motion, (double)(h->posed_tau - h->posed_tau0));
        for (int a = 0; a < 3; ++a) c[a] = p.c[a];
    }
    if (h->S == 0 || h->t == 0) {
        for (int a = 0; a < 3; ++a) torque[a] = 0.0;
        return LBM_OK;
    }
    const int blocks = lbm::force_sum_blocks();
    int rc = ensure_partial(h, (size_t)3 * blocks);
    if (rc) return rc;
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        lbm::k_sum_torque<<<blocks, 256, 0, h->stream>>>(h->S, h->X, h->g, c[0], c[1], c[2], h->partial);
        CK(cudaGetLastError());
        CK(lbm::launch_finalize(h->partial, blocks, 3, h->red, h->stream));
    }
    CK(cudaMemcpyAsync(torque, h->red, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // extern "C"
