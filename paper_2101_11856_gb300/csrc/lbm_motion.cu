// Moving and rotating solids (Algorithm 2 (c): the sample update after the IB stage, and the
// torque reduction).  At the start of every step one cooperative launch (k_rebuild) places the
// samples at the pose of the previous time in FP64, re-sorts them by base cell with a stable
// radix sort, and rebuilds the band (bitmap + tile offsets), the corner band indices and the
// spreading lists on the device, the same structures lbm_set_solids builds on the host for a
// static solid.  The band arrays have the fixed stride nband = 8 S (or N) and the band size is
// a device count, so the host never waits for the rebuild.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cooperative_groups.h>

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

__device__ __forceinline__ long long corner_cell(const Lattice &L, long long base, int c) {
    return base + (c & 1) + ((c >> 1) & 1) * (long long)L.nx + ((c >> 2) & 1) * L.nxy;
}

__device__ __forceinline__ int band_index(const uint32_t *__restrict__ mask, const int *__restrict__ off, long long cell) {
    const uint32_t m = mask[cell >> 5];
    const int l = (int)(cell & 31);
    if (!((m >> l) & 1u)) return -1;
    return off[cell >> 5] + __popc(m & ((1u << l) - 1u));
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

// ---- the whole rebuild in one cooperative launch ----------------------------------------------
// Phases of one kernel whose blocks are all resident (cooperative launch) and meet at grid-wide
// barriers between the phases: pose and
// keys (with the bitmap and run counters cleared), a stable LSD radix sort of the keys (8-bit
// digits; the first REBUILD_SORT_BLOCKS blocks sort contiguous chunks, so the order within a
// digit is the input order, as in sort_pairs), the samples gathered in sorted order, the band
// bitmap, its prefix offsets and the band count, the corner band indices, band cells and the runs
// of samples per base cell, and the spreading lists (the structures lbm_set_solids builds on the
// host for a static solid).
constexpr int REBUILD_THREADS = 256;   // also the largest grid (one block scans the block sums)
constexpr int REBUILD_SORT_BLOCKS = 32;   // blocks that sort (at most the grid; 16, 64 and all measured slower)

struct RebuildArgs {
    long long S, ntiles, stride;   // samples, bitmap words, band array stride
    long long clr0, clr1;          // bitmap words cleared: those the last rebuild or this one can set
    long long scan0, scan1;        // bitmap words this rebuild can set (offsets and band count)
    int bits;                      // significant bits of the keys
    int klo[3], kdim[3];           // box of the base cells the solid can reach: origin, sizes
    Pose p;
    Lattice L;
    const float *rel, *area_in;
    const int *sid_in;
    float *Xtmp, *X, *rel_o, *area_o, *ub;
    int *sid_o;
    uint32_t *key, *slot, *tkey, *tslot;
    int *hist;                     // [gridDim.x][256] digit counts of each block's chunk
    int *bsum;                     // [gridDim.x]
    uint32_t *mask;
    int *off, *count, *corner_band, *band_cell, *cstart, *ccount, *base_nbr;
};

// exclusive scan of one value per thread over the block (REBUILD_THREADS threads); returns the
// block total through *total (all threads)
__device__ __forceinline__ long long block_exclusive(long long v, long long *total) {
    __shared__ long long warp_tot[REBUILD_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < REBUILD_THREADS / 32; ++w) {
        if (w < warp) before += warp_tot[w];
        all += warp_tot[w];
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(REBUILD_THREADS) k_rebuild(RebuildArgs a) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long S = a.S;
    // pose, keys; clear the bitmap and the run counters
    for (long long i = tid; i < S; i += nthr) {
        double X[3];
        pose_point(a.p, a.rel, S, i, X);
        const float x = (float)X[0], y = (float)X[1], z = (float)X[2];
        a.Xtmp[i] = x;
        a.Xtmp[S + i] = y;
        a.Xtmp[2 * S + i] = z;
        // sort key: the base cell's index within the solid's box (the same order as the cell
        // index of the grid, on fewer bits)
        const int bx = min(max((int)floorf(x), 0), a.L.nx - 2), by = min(max((int)floorf(y), 0), a.L.ny - 2),
                  bz = min(max((int)floorf(z), 0), a.L.nz - 2);
        const int kx = min(max(bx - a.klo[0], 0), a.kdim[0] - 1), ky = min(max(by - a.klo[1], 0), a.kdim[1] - 1),
                  kz = min(max(bz - a.klo[2], 0), a.kdim[2] - 1);
        a.key[i] = (uint32_t)(kx + a.kdim[0] * (ky + a.kdim[1] * kz));
        a.slot[i] = (uint32_t)i;
    }
    for (long long w = a.clr0 + tid; w < a.clr1; w += nthr) a.mask[w] = 0u;
    for (long long k = tid; k < a.stride; k += nthr) a.ccount[k] = 0;
    grid.sync();

    // The band bitmap's marks (from the unsorted positions) and its offset scan (an exclusive
    // scan of the words' popcounts over contiguous chunks of the words this rebuild can set; the
    // others are zero and their offsets are never read) ride along the sort's phases: marks in
    // the first histogram phase, then one scan stage per phase; grid-wide barriers separate the
    // stages.  Stages: 0 = block partial sums, 1 = block 0 scans them (and the band count), 2 =
    // offsets written.
    const long long nw = a.scan1 - a.scan0;
    const long long wchunk = (nw + gridDim.x - 1) / gridDim.x;
    const long long w0 = a.scan0 + (blockIdx.x * wchunk < nw ? blockIdx.x * wchunk : nw);
    const long long w1 = w0 + wchunk < a.scan1 ? w0 + wchunk : a.scan1;
    const long long per = (wchunk + blockDim.x - 1) / blockDim.x;
    const long long t0w = w0 + threadIdx.x * per, t1w = t0w + per < w1 ? t0w + per : w1;
    long long sbefore = 0;   // this thread's words' offset within the block
    int scan_stage = 0;
    auto scan_step = [&]() {
        if (scan_stage == 0) {
            long long local = 0;
            for (long long w = t0w; w < t1w; ++w) local += __popc(a.mask[w]);
            long long total;
            sbefore = block_exclusive(local, &total);
            if (threadIdx.x == 0) a.bsum[blockIdx.x] = (int)total;
        } else if (scan_stage == 1) {
            if (blockIdx.x == 0) {
                const long long v = threadIdx.x < gridDim.x ? a.bsum[threadIdx.x] : 0;
                long long all;
                // gridDim.x <= REBUILD_THREADS (checked on the host)
                const long long ex = block_exclusive(v, &all);
                __syncthreads();
                if (threadIdx.x < gridDim.x) a.bsum[threadIdx.x] = (int)ex;
                if (threadIdx.x == 0) *a.count = (int)all;
            }
        } else if (scan_stage == 2) {
            long long run = a.bsum[blockIdx.x] + sbefore;
            for (long long w = t0w; w < t1w; ++w) {
                a.off[w] = (int)run;
                run += __popc(a.mask[w]);
            }
        }
        ++scan_stage;
    };

    // stable radix sort of (key, slot) by 8-bit digits
    __shared__ int cnt[256];
    __shared__ int wcnt[REBUILD_THREADS / 32][256];
    const int SB = (int)gridDim.x < REBUILD_SORT_BLOCKS ? (int)gridDim.x : REBUILD_SORT_BLOCKS;
    const bool sorter = (int)blockIdx.x < SB;
    const long long chunk = (S + SB - 1) / SB;
    uint32_t *ka = a.key, *va = a.slot, *kb = a.tkey, *vb = a.tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int shift = 0; shift < a.bits; shift += 8) {
        const long long c0 = sorter && blockIdx.x * chunk < S ? blockIdx.x * chunk : S;
        const long long c1 = c0 + chunk < S ? c0 + chunk : S;
        if (sorter) {
            cnt[threadIdx.x] = 0;
            __syncthreads();
            for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) atomicAdd(&cnt[(ka[e] >> shift) & 255u], 1);
            __syncthreads();
            a.hist[(long long)blockIdx.x * 256 + threadIdx.x] = cnt[threadIdx.x];
        }
        if (shift == 0) {
            // band bitmap: the 8 corner cells of every sample's base cell
            for (long long j = tid; j < S; j += nthr) {
                const long long b = base_cell(a.L, a.Xtmp[j], a.Xtmp[S + j], a.Xtmp[2 * S + j]);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const long long cell = corner_cell(a.L, b, c);
                    atomicOr(&a.mask[cell >> 5], 1u << (cell & 31));
                }
            }
        } else if (scan_stage == 1) {
            scan_step();
        }
        grid.sync();
        if (sorter) {
            // start of digit d in this chunk: all keys of smaller digits, plus digit d's keys of
            // the chunks before this one (thread d reads every chunk's count of digit d)
            long long before = 0, tot = 0;
            for (int g = 0; g < SB; ++g) {
                const int c = a.hist[(long long)g * 256 + threadIdx.x];
                if (g < (int)blockIdx.x) before += c;
                tot += c;
            }
            long long all;
            const long long start = block_exclusive(tot, &all);
            cnt[threadIdx.x] = (int)(start + before);
            __syncthreads();
        }
        if (sorter) {
            // running start of each digit for this chunk, tile by tile in (warp, item, lane) order
            const uint32_t lt = (1u << lane) - 1u;
            for (long long t0 = c0; t0 < c1; t0 += SORT_TILE) {
                for (int k = threadIdx.x; k < (REBUILD_THREADS / 32) * 256; k += blockDim.x) (&wcnt[0][0])[k] = 0;
                __syncthreads();
                const long long base = t0 + (long long)warp * 32 * SORT_ITEMS;
                uint32_t key[SORT_ITEMS], val[SORT_ITEMS];
                int rank[SORT_ITEMS];
#pragma unroll
                for (int it = 0; it < SORT_ITEMS; ++it) {
                    const long long e = base + it * 32 + lane;
                    const bool valid = e < c1;
                    key[it] = valid ? ka[e] : 0u;
                    val[it] = valid ? va[e] : 0u;
                    const uint32_t digit = valid ? (key[it] >> shift) & 255u : 256u;
                    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
                    const int before = valid ? wcnt[warp][digit] : 0;
                    rank[it] = before + __popc(peers & lt);
                    __syncwarp();
                    if (valid && lane == __ffs(peers) - 1) wcnt[warp][digit] = before + __popc(peers);
                    __syncwarp();
                }
                __syncthreads();
                {
                    const int d = threadIdx.x;
                    int run = cnt[d];
#pragma unroll
                    for (int w = 0; w < REBUILD_THREADS / 32; ++w) {
                        const int c = wcnt[w][d];
                        wcnt[w][d] = run;
                        run += c;
                    }
                    cnt[d] = run;
                }
                __syncthreads();
#pragma unroll
                for (int it = 0; it < SORT_ITEMS; ++it) {
                    const long long e = base + it * 32 + lane;
                    if (e < c1) {
                        const int pos = wcnt[warp][(key[it] >> shift) & 255u] + rank[it];
                        kb[pos] = key[it];
                        vb[pos] = val[it];
                    }
                }
                __syncthreads();
            }
        }
        if (scan_stage == 0 || scan_stage == 2) scan_step();
        grid.sync();
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    while (scan_stage < 3) {   // fewer than two sort passes
        scan_step();
        grid.sync();
    }

    // samples in sorted order, rigid-body boundary velocities; then (the same thread, the same
    // sample) the corner band indices
    for (long long j = tid; j < S; j += nthr) {
        const long long i = va[j];
        double P[3];
        pose_point(a.p, a.rel, S, i, P);
        const double d[3] = {P[0] - a.p.c[0], P[1] - a.p.c[1], P[2] - a.p.c[2]};
        const double u[3] = {a.p.V[0] + a.p.Om[1] * d[2] - a.p.Om[2] * d[1],
                             a.p.V[1] + a.p.Om[2] * d[0] - a.p.Om[0] * d[2],
                             a.p.V[2] + a.p.Om[0] * d[1] - a.p.Om[1] * d[0]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.X[c * S + j] = a.Xtmp[c * S + i];
            a.rel_o[c * S + j] = a.rel[c * S + i];
            a.ub[c * S + j] = (float)u[c];
        }
        a.area_o[j] = a.area_in[i];
        a.sid_o[j] = a.sid_in[i];
    }
    // corner band indices and band cells; the first sample of each run of equal base cells (sorted
    // keys) records the run's start and length at its base cell's band node
    for (long long j = tid; j < S; j += nthr) {
        const long long b = base_cell(a.L, a.X[j], a.X[S + j], a.X[2 * S + j]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const long long cell = corner_cell(a.L, b, c);
            const int bi = band_index(a.mask, a.off, cell);
            a.corner_band[c * S + j] = bi;
            a.band_cell[bi] = (int)cell;
            if (c == 0 && (j == 0 || ka[j - 1] != ka[j])) {
                long long k = j;
                while (k + 1 < S && ka[k + 1] == ka[j]) ++k;
                a.cstart[bi] = (int)j;
                a.ccount[bi] = (int)(k - j + 1);
            }
        }
    }
    grid.sync();
    // spreading lists: for every band node, the band node of each of its 8 lower neighbours that
    // is the base of at least one sample
    const long long nb = *a.count;
    for (long long k = tid; k < nb; k += nthr) {
        const long long cell = a.band_cell[k];
        const int x = (int)(cell % a.L.nx), y = (int)((cell / a.L.nx) % a.L.ny), z = (int)(cell / a.L.nxy);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int bx = x - (c & 1), by = y - ((c >> 1) & 1), bz = z - ((c >> 2) & 1);
            int v = -1;
            if (bx >= 0 && by >= 0 && bz >= 0) {
                const int bi = band_index(a.mask, a.off, bx + (long long)a.L.nx * by + a.L.nxy * bz);
                if (bi >= 0 && a.ccount[bi] > 0) v = bi;
            }
            a.base_nbr[c * a.stride + k] = v;
        }
    }
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
    const size_t need = 4 * pw + lbm::al256(sizeof(int) * ((size_t)256 * lbm::REBUILD_THREADS + lbm::REBUILD_THREADS));
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

// blocks of the cooperative rebuild (one per SM, at most REBUILD_THREADS so that one block scans
// the per-block sums), or 0 when the device cannot run it (no cooperative launch)
int rebuild_grid() {
    static int grid = -1;
    if (grid < 0) {
        int dev = 0, coop = 0, sms = 0, per_sm = 0;
        grid = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm::k_rebuild, lbm::REBUILD_THREADS, 0) ==
                cudaSuccess &&
            per_sm >= 1)
            grid = std::min(sms, lbm::REBUILD_THREADS);
        cudaGetLastError();
    }
    return grid;
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
    const int coop_grid = rebuild_grid();
    if (coop_grid <= 0) return fail(h, LBM_ECUDA, "the device cannot run the cooperative rebuild of a moving solid");
    Timed tm(h, LBM_KERNEL_MOTION);
    {
        lbm::RebuildArgs a{};
        a.S = S;
        a.ntiles = h->ntiles;
        a.stride = h->nband;
        // base cells within r_max of the centre, one cell of margin (the samples are FP32 roundings)
        long long box = 1;
        for (int k = 0; k < 3; ++k) {
            const int lo = std::max(0, (int)std::floor(p.c[k] - h->r_max) - 1);
            const int hi = std::min(n[k] - 2, (int)std::floor(p.c[k] + h->r_max) + 1);
            a.klo[k] = lo;
            a.kdim[k] = std::max(1, hi - lo + 1);
            box *= a.kdim[k];
        }
        a.bits = lbm::bits_for(box);
        // bitmap words of the box's band cells (base cells and their +1 corners)
        const long long c0 = a.klo[0] + (long long)h->nx * (a.klo[1] + (long long)h->ny * a.klo[2]);
        const long long c1 = (a.klo[0] + a.kdim[0]) + (long long)h->nx * ((a.klo[1] + a.kdim[1]) +
                                                                          (long long)h->ny * (a.klo[2] + a.kdim[2]));
        a.scan0 = c0 >> 5;
        a.scan1 = std::min(h->ntiles, (c1 >> 5) + 1);
        a.clr0 = h->mask_w1 < 0 ? 0 : std::min(h->mask_w0, a.scan0);
        a.clr1 = h->mask_w1 < 0 ? h->ntiles : std::max(h->mask_w1, a.scan1);
        a.p = p;
        a.L = L;
        a.rel = h->X0;
        a.area_in = h->area;
        a.sid_in = h->sid;
        a.Xtmp = h->Xtmp;
        a.X = h->X;
        a.rel_o = h->X0_alt;
        a.area_o = h->area_alt;
        a.ub = h->ub;
        a.sid_o = h->sid_alt;
        a.key = w.key;
        a.slot = w.slot;
        a.tkey = w.tkey;
        a.tslot = w.tslot;
        a.hist = static_cast<int *>(w.sort);
        a.bsum = a.hist + 256 * lbm::REBUILD_THREADS;
        a.mask = h->tile_mask;
        a.off = h->tile_off;
        a.count = h->band_count_dev;
        a.corner_band = h->corner_band;
        a.band_cell = h->band_cell;
        a.cstart = h->cstart;
        a.ccount = h->ccount;
        a.base_nbr = h->base_nbr;
        void *args[] = {&a};
        CK(cudaLaunchCooperativeKernel((const void *)lbm::k_rebuild, dim3(coop_grid), dim3(lbm::REBUILD_THREADS), args,
                                       0, h->stream));
        std::swap(h->X0, h->X0_alt);
        std::swap(h->area, h->area_alt);
        std::swap(h->sid, h->sid_alt);
        h->mask_w0 = a.scan0;
        h->mask_w1 = a.scan1;
    }
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
    h->ib_overlap = false;          // the band moves
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
    const int blocks = lbm::force_sum_blocks(h->S);
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
