// CUDA kernels of the GB300 path: the fused D3Q27 step (main and edge-strip kernels), its
// initialisation, the immersed-boundary band / interpolation / spreading kernels, and the
// diagnostics.  The AA-pattern addressing lives in lbm_step.cuh.
#include <algorithm>

#include "lbm_step.cuh"

namespace lbm {


// ---- initialisation: f = f_eq(rho, u), stored as the post-collision state of t = 0 ------

__device__ __forceinline__ float phi1(int c, float u) {
    return c == 0 ? (2.0f / 3.0f - u * u) : 0.5f * ((1.0f / 3.0f) + u * u + (float)c * u);
}
// deviation of the product-form equilibrium from w rho0, expanded to keep precision
__device__ __forceinline__ float phi_dev(int c, float u) {
    // phi(c, u) - w1(c)
    return c == 0 ? -u * u : 0.5f * (u * u + (float)c * u);
}

template <typename St>
__global__ void k_init(StepParams P, const float *__restrict__ rho, const float *__restrict__ u) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= P.g.ncell) return;
    const float r = rho[cell];
    const float ux = u[cell], uy = u[P.g.ncell + cell], uz = u[2 * P.g.ncell + cell];
    St *A = static_cast<St *>(P.f);
    int x, y, z;
    decompose(P.g, cell, x, y, z);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        // f = r prod phi = r prod (w1 + dphi); h = f - rho0 w
        const float wx = w1(cx(d)), wy = w1(cy(d)), wz = w1(cz(d));
        const float px = phi_dev(cx(d), ux), py = phi_dev(cy(d), uy), pz = phi_dev(cz(d), uz);
        // prod(w + p) - prod(w) expanded
        const float dprod = px * wy * wz + wx * py * wz + wx * wy * pz + px * py * wz + px * wy * pz +
                            wx * py * pz + px * py * pz;
        const float hv = (r - P.rho0) * wgt(d) + r * dprod;
        Store<St>::st(A + opp(d) * P.g.plane + cell, hv);
        if (x == P.g.nx - 1 && P.g.face[1] == FACE_OUTLET && cx(d) == -1) {
            St *B = static_cast<St *>(P.outlet);
            Store<St>::st(B + ((long long)(d / 3) * P.g.nyz + y + P.g.ny * z), hv);
        }
    }
}

// ---- post-collision populations of the current time (canonical layout) ----------------

template <typename St, bool AFTER_NB>
__device__ __forceinline__ void load_post(const StepParams &P, int x, int y, int z, int cell, float (&h)[27]) {
    const St *A = static_cast<const St *>(P.f);
    const long long pl = P.g.plane;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (AFTER_NB) {
            // pushed to x + c_d; across free-slip faces only, to the tangential neighbour's slot
            // of the mirrored direction; across any other face, to the node's own slot
            const Nbr n = neighbour<+1>(P.g, d, x, y, z);
            if (n.kind == 0) h[d] = Store<St>::ld(A + d * pl + n.idx);
            else if (n.kind == CROSS_FREESLIP) h[d] = Store<St>::ld(A + mirror_dir(d, n.mir) * pl + n.idx);
            else h[d] = Store<St>::ld(A + opp(d) * pl + cell);
        } else {
            h[d] = Store<St>::ld(A + opp(d) * pl + cell);
        }
    }
}

// per-cell rho and Guo-shifted u of the last collision, optional field output and FP64
// block partial sums for the deterministic global reductions: mass, momentum (3) and the
// kinetic energy 1/2 rho |u|^2 of the slab ke_x0 <= x < ke_x1 (grid-stride over the cells)
template <typename St, bool AFTER_NB, bool BAND>
__global__ void __launch_bounds__(256) k_macro(StepParams P, int force_on, float *__restrict__ rho_out,
                                               float *__restrict__ u_out, float *__restrict__ f_out,
                                               double *__restrict__ partial, int *__restrict__ nonfinite,
                                               int ke_x0, int ke_x1) {
    double acc[MACRO_SUMS] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < P.g.ncell; cell += gridDim.x * blockDim.x) {
        int x, y, z;
        decompose(P.g, cell, x, y, z);
        float h[27];
        load_post<St, AFTER_NB>(P, x, y, z, cell, h);
        if (f_out) {
            const float r0 = P.rho0;
#pragma unroll
            for (int d = 0; d < 27; ++d) f_out[(long long)d * P.g.ncell + cell] = h[d] + wgt(d) * r0;
        }
        float rp = 0.0f, px = 0.0f, py = 0.0f, pz = 0.0f;
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            rp += h[d];
            if (cx(d)) px += cx(d) * h[d];
            if (cy(d)) py += cy(d) * h[d];
            if (cz(d)) pz += cz(d) * h[d];
        }
        float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
        if (force_on) band_force<BAND>(P, cell, Fx, Fy, Fz);
        // post-collision momentum is j + F, so rho u = sum c f_post - F/2
        const float rho = P.rho0 + rp;
        const float jxs = px - 0.5f * Fx, jys = py - 0.5f * Fy, jzs = pz - 0.5f * Fz;
        const float inv = 1.0f / rho;
        if (rho_out) rho_out[cell] = rho;
        if (u_out) {
            u_out[cell] = jxs * inv;
            u_out[P.g.ncell + cell] = jys * inv;
            u_out[2 * P.g.ncell + cell] = jzs * inv;
        }
        if (nonfinite && !(isfinite(rho) && isfinite(jxs * inv) && isfinite(jys * inv) && isfinite(jzs * inv)))
            atomicOr(nonfinite, 1);
        acc[0] += (double)rho;
        acc[1] += (double)jxs;
        acc[2] += (double)jys;
        acc[3] += (double)jzs;
        if (x >= ke_x0 && x < ke_x1)
            acc[4] += 0.5 * ((double)jxs * jxs + (double)jys * jys + (double)jzs * jzs) / (double)rho;
    }
    if (partial) {
        // fixed-order block tree reduction in FP64
        __shared__ double s[MACRO_SUMS][256];
#pragma unroll
        for (int k = 0; k < MACRO_SUMS; ++k) s[k][threadIdx.x] = acc[k];
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
#pragma unroll
                for (int k = 0; k < MACRO_SUMS; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < MACRO_SUMS; ++k) partial[(long long)k * gridDim.x + blockIdx.x] = s[k][0];
        }
    }
}

// sum `count` rows of `n` doubles each (row k at partial + k * n) in a fixed order
__global__ void k_finalize(const double *__restrict__ partial, long long n, int count, double *__restrict__ out) {
    __shared__ double s[256];
    for (int k = 0; k < count; ++k) {
        double acc = 0.0;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) acc += partial[(long long)k * n + i];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = s[0];
        __syncthreads();
    }
}

// ---- immersed boundary ---------------------------------------------------------------

// band moments: rho* and the pre-IB velocity (j + F_body/2)/rho* at every band node
template <typename St, bool NB>
__global__ void __launch_bounds__(256) k_band_moments(StepParams P, const int *__restrict__ band_cell,
                                                      float *__restrict__ band_rho, float *__restrict__ band_u) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (P.band_count ? (long long)*P.band_count : P.nband)) return;
    const int cell = band_cell[k];
    int x, y, z;
    decompose(P.g, cell, x, y, z);
    float h[27];
    // nodes away from every face pull with constant offsets; the rest apply the face rules
    if (x >= 1 && x <= P.g.nx - 2 && y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2)
        load_interior<St, NB>(P, cell, h);
    else
        load_general<St, NB>(P, x, y, z, cell, h);
    float rp = 0.0f, px = 0.0f, py = 0.0f, pz = 0.0f;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        rp += h[d];
        if (cx(d)) px += cx(d) * h[d];
        if (cy(d)) py += cy(d) * h[d];
        if (cz(d)) pz += cz(d) * h[d];
    }
    const float rho = P.rho0 + rp;
    const float inv = 1.0f / rho;
    band_rho[k] = rho;
    band_u[k] = (px + 0.5f * P.Fx) * inv;
    band_u[P.nband + k] = (py + 0.5f * P.Fy) * inv;
    band_u[2 * P.nband + k] = (pz + 0.5f * P.Fz) * inv;
}

// trilinear weight of corner c (bit 0: x, bit 1: y, bit 2: z) for fractions (wx, wy, wz)
__device__ __forceinline__ float corner_weight(int c, float wx, float wy, float wz) {
    return ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
}

// band index of a node known to be in the band, from the band bitmap (one mask and one offset
// word per 32 cells)
__device__ __forceinline__ int band_of(const StepParams &P, long long cell) {
    const uint32_t mask = P.tile_mask[cell >> 5];
    return P.tile_off[cell >> 5] + __popc(mask & ((1u << (cell & 31)) - 1u));
}

// interpolation (Eq. 6) and penalty force (Eq. 7) per sample; the 8 stencil nodes' band indices
// come from the bitmap (cached words, shared by the neighbouring samples of the cell-sorted
// order) instead of a stored table; ub = nullptr: boundary velocity 0
__global__ void __launch_bounds__(256) k_ib_interp(StepParams P, long long S, const float *__restrict__ X,
                                                   const float *__restrict__ area, const float *__restrict__ ub,
                                                   const float *__restrict__ band_rho, const float *__restrict__ band_u,
                                                   float *__restrict__ g) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const long long nband = P.nband;
    const float x = X[s], y = X[S + s], z = X[2 * S + s];
    const float fx = floorf(x), fy = floorf(y), fz = floorf(z);
    const float wx = x - fx, wy = y - fy, wz = z - fz;
    const long long base = (long long)fx + P.g.nx * ((long long)fy + (long long)P.g.ny * (long long)fz);
    float rs = 0.0f, us = 0.0f, vs = 0.0f, ws = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long cell = base + (c & 1) + ((c & 2) ? P.g.nx : 0) + ((c & 4) ? (long long)P.g.nxy : 0);
        const int b = band_of(P, cell);
        const float K = corner_weight(c, wx, wy, wz);
        rs = fmaf(K, band_rho[b], rs);
        us = fmaf(K, band_u[b], us);
        vs = fmaf(K, band_u[nband + b], vs);
        ws = fmaf(K, band_u[2 * nband + b], ws);
    }
    const float a = rs * area[s];
    const float bx = ub ? ub[s] : 0.0f, by = ub ? ub[S + s] : 0.0f, bz = ub ? ub[2 * S + s] : 0.0f;
    g[s] = a * (bx - us);
    g[S + s] = a * (by - vs);
    g[2 * S + s] = a * (bz - ws);
}

// spreading (Eq. 8) as a deterministic gather: band node k sums K g over the samples whose
// base cell is x_k - c for the 8 corners c, in sample order (samples sorted by base cell)
__global__ void __launch_bounds__(256) k_ib_spread(long long S, long long nband, const int *__restrict__ count,
                                                   const float *__restrict__ X, const float *__restrict__ g,
                                                   const int *__restrict__ base_nbr, const int *__restrict__ cstart,
                                                   const int *__restrict__ ccount, float *__restrict__ bandF) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (count ? (long long)*count : nband)) return;
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        const int b = base_nbr[(long long)c * nband + k];
        if (b < 0) continue;
        const int s0 = cstart[b], s1 = s0 + ccount[b];
        for (int s = s0; s < s1; ++s) {
            const float x = X[s], y = X[S + s], z = X[2 * S + s];
            const float K = corner_weight(c, x - floorf(x), y - floorf(y), z - floorf(z));
            fx = fmaf(K, g[s], fx);
            fy = fmaf(K, g[S + s], fy);
            fz = fmaf(K, g[2 * S + s], fz);
        }
    }
    bandF[k] = fx;
    bandF[nband + k] = fy;
    bandF[2 * nband + k] = fz;
}

// Two-phase immersed boundary of a static solid (Eqs. 6-8 in Algorithm 2's order).
// Phase 1, one thread per occupied base cell i (band index occ_bi[i]): the cell's samples share
// their 8 stencil nodes, so the thread reads those nodes' moments once, interpolates and forms the
// penalty force of each sample with the arithmetic of k_ib_interp (the same g_s bit for bit), and
// sums K_c g_s over its samples per corner c into cellS[3 c + a][i] (each sample's weights once).
__global__ void __launch_bounds__(256) k_ib_cells(StepParams P, long long S, long long nocc, const int *__restrict__ occ_bi,
                                                  const int *__restrict__ band_cell, const int *__restrict__ cstart,
                                                  const int *__restrict__ ccount, const float *__restrict__ X,
                                                  const float *__restrict__ area, const float *__restrict__ ub,
                                                  const float *__restrict__ band_rho, const float *__restrict__ band_u,
                                                  float *__restrict__ g, float *__restrict__ cellS) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nocc) return;
    const long long nband = P.nband;
    const int bi = occ_bi[i];
    const long long base = band_cell[bi];
    const int s0 = cstart[bi], s1 = s0 + ccount[bi];
    float r[8], vx[8], vy[8], vz[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long cell = base + (c & 1) + ((c & 2) ? P.g.nx : 0) + ((c & 4) ? (long long)P.g.nxy : 0);
        const int b = band_of(P, cell);
        r[c] = band_rho[b];
        vx[c] = band_u[b];
        vy[c] = band_u[nband + b];
        vz[c] = band_u[2 * nband + b];
    }
    float acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0.0f;
    for (int s = s0; s < s1; ++s) {
        const float x = X[s], y = X[S + s], z = X[2 * S + s];
        const float wx = x - floorf(x), wy = y - floorf(y), wz = z - floorf(z);
        float rs = 0.0f, us = 0.0f, vs = 0.0f, ws = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float K = corner_weight(c, wx, wy, wz);
            rs = fmaf(K, r[c], rs);
            us = fmaf(K, vx[c], us);
            vs = fmaf(K, vy[c], vs);
            ws = fmaf(K, vz[c], ws);
        }
        const float a = rs * area[s];
        const float bx = ub ? ub[s] : 0.0f, by = ub ? ub[S + s] : 0.0f, bz = ub ? ub[2 * S + s] : 0.0f;
        const float gx = a * (bx - us), gy = a * (by - vs), gz = a * (bz - ws);
        g[s] = gx;
        g[S + s] = gy;
        g[2 * S + s] = gz;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float K = corner_weight(c, wx, wy, wz);
            acc[3 * c] = fmaf(K, gx, acc[3 * c]);
            acc[3 * c + 1] = fmaf(K, gy, acc[3 * c + 1]);
            acc[3 * c + 2] = fmaf(K, gz, acc[3 * c + 2]);
        }
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) cellS[k * nocc + i] = acc[k];
}

// Phase 2, one thread per band node k: the spread force (Eq. 8) is the sum over the 8 base cells
// x_k - c (corner c of that cell is node k; occ_nbr[c][k] = its occupied-cell index or -1) of the
// cells' corner-c sums, in corner order: a fixed order, no atomics.
__global__ void __launch_bounds__(256) k_ib_gather(long long nband, long long nocc, const int *__restrict__ occ_nbr,
                                                   const float *__restrict__ cellS, float *__restrict__ bandF) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nband) return;
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int o = occ_nbr[(long long)c * nband + k];
        if (o < 0) continue;
        fx += cellS[(long long)(3 * c) * nocc + o];
        fy += cellS[(long long)(3 * c + 1) * nocc + o];
        fz += cellS[(long long)(3 * c + 2) * nocc + o];
    }
    bandF[k] = fx;
    bandF[nband + k] = fy;
    bandF[2 * nband + k] = fz;
}

// FP64 block partial sums of the penalty forces (drag = -sum g)
// per-block FP64 sums of the three force components; component k of block b at
// partial[k * stride + b]
__global__ void __launch_bounds__(256) k_sum_forces(long long S, const float *__restrict__ g, double *__restrict__ partial,
                                                    long long stride) {
    __shared__ double s[3][256];
    double a[3] = {0.0, 0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
        a[0] += g[i];
        a[1] += g[S + i];
        a[2] += g[2 * S + i];
    }
    for (int k = 0; k < 3; ++k) s[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partial[(long long)k * stride + blockIdx.x] = s[k][0];
}

// ---- host launchers ------------------------------------------------------------------

static inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

long long boundary_count(const Geometry &g) { return (long long)edge_per_row(g) * g.ny * g.nz; }

template <typename F>
static cudaError_t dispatch_storage(int storage, F &&fn) {
    switch (storage) {
        case 0: return fn(float{});
        case 1: return fn(__half{});
        default: return fn(__nv_bfloat16{});
    }
}

// The free-slip variants (FS) serve the grids with a free-slip face.  They run over the rows on a
// y/z face only, in the boundary part (edge strips and main range of those rows), and the kernels
// without FS over the other rows (inner_rows): the mirror logic is compiled out of the kernel
// that updates nearly every node, which keeps its register count.  Grids without a main range
// run the FS rows kernel on every row.
namespace {
bool has_freeslip(const Geometry &g) {
    bool fs = false;
    for (int k = 2; k < 6; ++k) fs = fs || g.face[k] == FACE_FREESLIP;
    return fs;
}

template <bool FS>
cudaError_t launch_step_fs(int storage, const StepParams &P, bool band, int part, int collision, cudaStream_t st) {
    switch (collision) {
        case COLL_BGK: return launch_step_coll<COLL_BGK, FS>(storage, P, band, part, st);
        case COLL_RAW: return launch_step_coll<COLL_RAW, FS>(storage, P, band, part, st);
        default: return launch_step_coll<COLL_ACM, FS>(storage, P, band, part, st);
    }
}
}  // namespace

int step_launches(const StepParams &P, int part) {
    if (part == STEP_INTERIOR) return has_interior(P.g) ? 1 : 0;
    const bool split = has_freeslip(P.g) && has_interior(P.g);
    if (part == STEP_STRIPS) return 1;
    if (part == STEP_FACE_ROWS) return split ? 2 : 0;
    return split ? 3 : 1;
}

cudaError_t launch_step(int storage, const StepParams &P, bool band, int part, int collision, cudaStream_t st) {
    if (!has_freeslip(P.g)) {
        if (part == STEP_FACE_ROWS) return cudaSuccess;
        return launch_step_fs<false>(storage, P, band, part == STEP_STRIPS ? STEP_BOUNDARY : part, collision, st);
    }
    StepParams Pi = P;
    Pi.inner_rows = 1;
    if (part == STEP_INTERIOR)
        return has_interior(P.g) ? launch_step_fs<false>(storage, Pi, band, part, collision, st) : cudaSuccess;
    if (part != STEP_FACE_ROWS && has_interior(P.g)) {
        const cudaError_t e = launch_step_fs<false>(storage, Pi, band, STEP_BOUNDARY, collision, st);
        if (e != cudaSuccess) return e;
    }
    if (part == STEP_STRIPS && has_interior(P.g)) return cudaSuccess;
    return launch_step_fs<true>(storage, P, band, STEP_BOUNDARY, collision, st);
}

cudaError_t launch_init(int storage, const StepParams &P, const float *rho, const float *u, cudaStream_t st) {
    return dispatch_storage(storage, [&](auto tag) {
        k_init<decltype(tag)><<<blocks_for(P.g.ncell, 256), 256, 0, st>>>(P, rho, u);
        return cudaGetLastError();
    });
}

long long macro_blocks(const StepParams &P) { return std::min<long long>(blocks_for(P.g.ncell, 256), 2432); }

cudaError_t launch_macro(int storage, const StepParams &P, bool band, int force_on, float *rho, float *u, float *f,
                         double *partial, int *nonfinite, cudaStream_t st, int ke_x0, int ke_x1) {
    // the state after step t was written by a neighbour step when t is odd
    const bool after_nb = (P.t & 1) != 0;
    return dispatch_storage(storage, [&](auto tag) {
        using St = decltype(tag);
        const unsigned grid = (unsigned)macro_blocks(P);
        if (after_nb) {
            if (band) k_macro<St, true, true><<<grid, 256, 0, st>>>(P, force_on, rho, u, f, partial, nonfinite, ke_x0, ke_x1);
            else k_macro<St, true, false><<<grid, 256, 0, st>>>(P, force_on, rho, u, f, partial, nonfinite, ke_x0, ke_x1);
        } else {
            if (band) k_macro<St, false, true><<<grid, 256, 0, st>>>(P, force_on, rho, u, f, partial, nonfinite, ke_x0, ke_x1);
            else k_macro<St, false, false><<<grid, 256, 0, st>>>(P, force_on, rho, u, f, partial, nonfinite, ke_x0, ke_x1);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_finalize(const double *partial, long long n, int count, double *out, cudaStream_t st) {
    k_finalize<<<1, 256, 0, st>>>(partial, n, count, out);
    return cudaGetLastError();
}

cudaError_t launch_band_moments(int storage, const StepParams &P, const int *band_cell, float *band_rho, float *band_u,
                                cudaStream_t st) {
    const bool nb = (P.t & 1) != 0;
    return dispatch_storage(storage, [&](auto tag) {
        using St = decltype(tag);
        const unsigned grid = blocks_for(P.nband, 256);
        if (nb) k_band_moments<St, true><<<grid, 256, 0, st>>>(P, band_cell, band_rho, band_u);
        else k_band_moments<St, false><<<grid, 256, 0, st>>>(P, band_cell, band_rho, band_u);
        return cudaGetLastError();
    });
}

cudaError_t launch_ib_interp(const StepParams &P, long long S, const float *X, const float *area, const float *ub,
                             const float *band_rho, const float *band_u, float *g, cudaStream_t st) {
    k_ib_interp<<<blocks_for(S, 256), 256, 0, st>>>(P, S, X, area, ub, band_rho, band_u, g);
    return cudaGetLastError();
}

cudaError_t launch_ib_spread(long long S, long long nband, const int *count, const float *X, const float *g,
                             const int *base_nbr, const int *cstart, const int *ccount, float *bandF, cudaStream_t st) {
    k_ib_spread<<<blocks_for(nband, 256), 256, 0, st>>>(S, nband, count, X, g, base_nbr, cstart, ccount, bandF);
    return cudaGetLastError();
}

cudaError_t launch_ib_cells(const StepParams &P, long long S, long long nocc, const int *occ_bi, const int *band_cell,
                            const int *cstart, const int *ccount, const float *X, const float *area, const float *ub,
                            const float *band_rho, const float *band_u, float *g, float *cellS, cudaStream_t st) {
    k_ib_cells<<<blocks_for(nocc, 256), 256, 0, st>>>(P, S, nocc, occ_bi, band_cell, cstart, ccount, X, area, ub, band_rho,
                                                      band_u, g, cellS);
    return cudaGetLastError();
}

cudaError_t launch_ib_gather(long long nband, long long nocc, const int *occ_nbr, const float *cellS, float *bandF,
                             cudaStream_t st) {
    k_ib_gather<<<blocks_for(nband, 256), 256, 0, st>>>(nband, nocc, occ_nbr, cellS, bandF);
    return cudaGetLastError();
}

// blocks of the per-sample sums: at least 2048 samples per block (small solids take one block,
// so the per-step drag of the adjoint's forward pass costs no idle blocks), at most 1024
int force_sum_blocks(long long S) {
    const long long b = (S + 2047) / 2048;
    return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t launch_sum_forces(long long S, const float *g, double *partial, cudaStream_t st, long long stride) {
    const int nb = force_sum_blocks(S);
    k_sum_forces<<<nb, 256, 0, st>>>(S, g, partial, stride > 0 ? stride : nb);
    return cudaGetLastError();
}

}  // namespace lbm
