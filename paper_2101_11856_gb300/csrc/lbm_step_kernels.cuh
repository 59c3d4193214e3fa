// The fused step kernels (main range and edge strips) and their launchers, templated on the
// storage type, the AA parity, the immersed-boundary force, the collision model and the
// presence of a free-slip face.  Each collision model is instantiated in its own translation
// units (lbm_step_acm.cu and lbm_step_acm_fs.cu, likewise bgk and raw) so that they compile in
// parallel.
#pragma once

#include <type_traits>

#include "lbm_models.cuh"
#include "lbm_step.cuh"
#include "lbm_step_tma.cuh"

namespace lbm {

inline unsigned step_blocks(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }
// grid of gx x n blocks with n folded into (y, z) (y at most 65535)
inline dim3 face_grid(unsigned gx, long long n) {
    const long long gy = n < 65535 ? (n > 0 ? n : 1) : 65535;
    return dim3(gx, (unsigned)gy, (unsigned)((n + gy - 1) / gy > 0 ? (n + gy - 1) / gy : 1));
}

// the velocity field output of a step (for the smoke tracers; kernels with VOUT only)
__device__ __forceinline__ void store_velocity(const StepParams &P, int cell, float ux, float uy, float uz) {
    {
        const long long n = P.g.ncell;
        P.u_out[cell] = ux;
        P.u_out[n + cell] = uy;
        P.u_out[2 * n + cell] = uz;
    }
}

// ---- the fused step ---------------------------------------------------------------------
// Pull the 27 streamed populations, add the body force and the band's immersed-boundary
// force, collide in registers, store in place.  k_step_main updates the nodes
// XEDGE <= x < nx - XEDGE (two per thread for FP32): one block row per (y, z), so a block's y/z face status is
// uniform (interior rows use constant offsets; face rows of odd steps use wrapped or bounced
// rows; even steps address only the node's own slots).  k_step_edges updates the two edge
// strips of each row with the general face rules (inlet, outlet, x wrap) in whole warps.
// Every node is updated by exactly one of the two, and the two touch disjoint slots.
// nodes per thread of the main kernel: two for FP32 storage (memory bound: the shared
// addresses and the doubled bytes in flight pay), one for FP16 / BF16 (issue bound: the
// lower register count keeps twice the warps resident)
template <typename St> __host__ __device__ constexpr int main_nodes() { return sizeof(St) == 4 ? 2 : 1; }

// Without FS a block row is (blockIdx.y, blockIdx.z) = (y, z); the FS kernels (a grid with a
// free-slip face) run over the face rows only (face_row of blockIdx.y + gridDim.y blockIdx.z),
// while the kernels without FS skip those rows (inner_rows): the mirror logic costs registers,
// which would otherwise slow every row.
template <typename St, bool NB, bool BAND, int COLL, bool VOUT, bool FS>
__global__ void __launch_bounds__(STEP_BX) k_step_main(StepParams P) {
    int y, z;
    bool inner;   // uniform per block
    if constexpr (FS) {
        const long long r = blockIdx.y + (long long)gridDim.y * blockIdx.z;
        if (r >= face_rows(P.g)) return;
        face_row(P.g, r, y, z);
        inner = false;
    } else {
        y = blockIdx.y;
        z = blockIdx.z;
        inner = y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2;
        if (P.inner_rows && !inner) return;
    }
    const int xend = P.g.nx - XEDGE;
    float Fx, Fy, Fz, rho, ux, uy, uz;
    if constexpr (main_nodes<St>() == 2) {
        // a block covers 2 blockDim.x nodes of a row; warp w, lane l: nodes 64 w + l and 64 w + l + 32
        const int x = blockIdx.x * (2 * blockDim.x) + (threadIdx.x >> 5) * 64 + (threadIdx.x & 31) + XEDGE;
        if (x >= xend) return;
        const bool two = x + 32 < xend;
        const int cell = x + P.g.nx * (y + P.g.ny * z);
        float h0[27], h1[27];
        if (!NB || inner) load_interior2<St, NB>(P, cell, two, h0, h1);
        else load_yzface2<St, FS>(P, y, z, cell, two, h0, h1);
        band_force<BAND>(P, cell, Fx, Fy, Fz);
        collide_model<COLL>(h0, Fx, Fy, Fz, P, rho, ux, uy, uz);
        if (VOUT) store_velocity(P, cell, ux, uy, uz);
        if (two) {
            band_force<BAND>(P, cell + 32, Fx, Fy, Fz);
            collide_model<COLL>(h1, Fx, Fy, Fz, P, rho, ux, uy, uz);
            if (VOUT) store_velocity(P, cell + 32, ux, uy, uz);
        }
        if (!NB || inner) store_interior2<St, NB>(P, cell, two, h0, h1);
        else store_yzface2<St, FS>(P, y, z, cell, two, h0, h1);
    } else {
        const int x = blockIdx.x * blockDim.x + threadIdx.x + XEDGE;
        if (x >= xend) return;
        const int cell = x + P.g.nx * (y + P.g.ny * z);
        float h[27];
        if (!NB || inner) load_interior<St, NB>(P, cell, h);
        else load_yzface<St, FS>(P, y, z, cell, h);
        band_force<BAND>(P, cell, Fx, Fy, Fz);
        collide_model<COLL>(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
        if (!NB || inner) store_interior<St, NB>(P, cell, h);
        else store_yzface<St, FS>(P, y, z, cell, h);
        if (VOUT) store_velocity(P, cell, ux, uy, uz);
    }
}

// Main range with 16-bit storage and the method's collision on a grid with nx even: node pairs
// (x, x + 1), x = XEDGE + 2 i, the packed FP32 collision (collide_v<F2>: bit for bit the same
// arithmetic as one node at a time) and 32-bit accesses for both nodes wherever the AA addressing
// keeps the pair aligned (load_pair / store_pair).  Rows as k_step_main without FS.
// FP16: at most 80 registers (24 resident one-warp blocks per SM instead of 21 at 94-96, a few
// spilled values); BF16: at most 96 (its conversions need the registers; with no bound at all the
// compiler takes 140-160 and halves the resident warps)
template <typename St> constexpr int pair_min_blocks() { return std::is_same<St, __half>::value ? 12 : 10; }
template <typename St, bool NB, bool BAND, bool VOUT>
__global__ void __launch_bounds__(STEP_BX, pair_min_blocks<St>()) k_step_pair(StepParams P) {
    const int y = blockIdx.y, z = blockIdx.z;
    const bool inner = y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2;   // uniform per block
    if (P.inner_rows && !inner) return;
    const int x = XEDGE + 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= P.g.nx - XEDGE) return;
    const int cell = x + P.g.nx * (y + P.g.ny * z);
    int off[9], mir[9];
    bool bb[9];
    F2 h[27];
    if (!NB || inner) {
        row_offsets<-1, true, false>(P.g, y, z, off, bb, mir);
        load_pair<St, NB>(P, cell, off, bb, h);
    } else {
        row_offsets<-1, false, false>(P.g, y, z, off, bb, mir);
        load_pair<St, NB>(P, cell, off, bb, h);
    }
    F2 Fx, Fy, Fz, rho, ux, uy, uz;
    band_force_pair<BAND>(P, cell, Fx, Fy, Fz);
    collide_v<F2>(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
    if (VOUT) {
        const long long n = P.g.ncell;
        *reinterpret_cast<float2 *>(P.u_out + cell) = ux.v;
        *reinterpret_cast<float2 *>(P.u_out + n + cell) = uy.v;
        *reinterpret_cast<float2 *>(P.u_out + 2 * n + cell) = uz.v;
    }
    if (!NB || inner) {
        row_offsets<+1, true, false>(P.g, y, z, off, bb, mir);
        store_pair<St, NB>(P, cell, off, bb, h);
    } else {
        row_offsets<+1, false, false>(P.g, y, z, off, bb, mir);
        store_pair<St, NB>(P, cell, off, bb, h);
    }
}

// the main range runs in node pairs: 16-bit storage, the method's collision, nx even
template <typename St, int COLL> __host__ __device__ constexpr bool pair_storage() {
    return sizeof(St) == 2 && COLL == COLL_ACM;
}
inline bool pair_grid(const Geometry &g) { return g.nx % 2 == 0; }

// one warp per edge strip of one row, EDGE_ROWS rows (y) per block: blockIdx.y * EDGE_ROWS +
// threadIdx.y = y, blockIdx.z = z.  With a main range, blockIdx.x picks the left (0) or right
// (1) strip (one launch for both: measured faster than a launch per side); short rows run the
// SIDE = 2 kernel over consecutive warps.
template <typename St, bool NB, bool BAND, int SIDE, int COLL, bool VOUT, bool FS>
__device__ __forceinline__ void edge_node(const StepParams &P, int y, int z) {
    const int x = edge_x<SIDE>(P.g);
    if (x >= P.g.nx) return;
    const int cell = x + P.g.nx * (y + P.g.ny * z);
    float h[27];
    load_edge<St, NB, SIDE, FS>(P, x, y, z, cell, h);
    float Fx, Fy, Fz;
    band_force<BAND>(P, cell, Fx, Fy, Fz);
    float rho, ux, uy, uz;
    collide_model<COLL>(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
    store_edge<St, NB, SIDE, FS>(P, x, y, z, cell, h);
    if (VOUT) store_velocity(P, cell, ux, uy, uz);
}

template <typename St, bool NB, bool BAND, int COLL, bool VOUT, bool FS>
__global__ void __launch_bounds__(XEDGE * EDGE_ROWS) k_step_edges(StepParams P) {
    int y, z;
    if constexpr (FS) {   // face rows only (as k_step_main)
        const long long r = (blockIdx.y + (long long)gridDim.y * blockIdx.z) * EDGE_ROWS + threadIdx.y;
        if (r >= face_rows(P.g)) return;
        face_row(P.g, r, y, z);
    } else {
        y = blockIdx.y * EDGE_ROWS + threadIdx.y;
        z = blockIdx.z;
        if (y >= P.g.ny) return;
        if (P.inner_rows && !(y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2)) return;
    }
    if (blockIdx.x == 0) edge_node<St, NB, BAND, 0, COLL, VOUT, FS>(P, y, z);
    else edge_node<St, NB, BAND, 1, COLL, VOUT, FS>(P, y, z);
}

template <typename St, bool NB, bool BAND, int COLL, bool VOUT, bool FS>
__global__ void __launch_bounds__(XEDGE * EDGE_ROWS) k_step_rows(StepParams P) {
    const int y = blockIdx.y * EDGE_ROWS + threadIdx.y, z = blockIdx.z;
    if (y >= P.g.ny) return;
    edge_node<St, NB, BAND, 2, COLL, VOUT, FS>(P, y, z);
}

// FS (face rows of a grid with a free-slip face): the boundary part launches the edge strips and
// the main range of those rows; there is no FS interior part
template <typename St, bool NB, bool BAND, int COLL, bool VOUT, bool FS>
cudaError_t launch_step_tt(const StepParams &P, int part, cudaStream_t st) {
    const Geometry &g = P.g;
    // one warp per block when a row's main range fits in one warp's nodes (short rows would
    // leave the second warp idle)
    const int range = g.nx - 2 * XEDGE, per_warp = 32 * main_nodes<St>();
    const int threads = range <= per_warp ? 32 : STEP_BX;
    const unsigned xb = step_blocks(range, main_nodes<St>() * threads);
    if (part == STEP_BOUNDARY) {
        const dim3 block(XEDGE, EDGE_ROWS);
        if (has_interior(g)) {
            const dim3 grid = FS ? face_grid(2, (face_rows(g) + EDGE_ROWS - 1) / EDGE_ROWS)
                                 : dim3(2, step_blocks(g.ny, EDGE_ROWS), g.nz);
            k_step_edges<St, NB, BAND, COLL, VOUT, FS><<<grid, block, 0, st>>>(P);
            if (FS) k_step_main<St, NB, BAND, COLL, VOUT, FS><<<face_grid(xb, face_rows(g)), threads, 0, st>>>(P);
        } else {
            const dim3 grid(step_blocks(g.nx, XEDGE), step_blocks(g.ny, EDGE_ROWS), g.nz);
            k_step_rows<St, NB, BAND, COLL, VOUT, FS><<<grid, block, 0, st>>>(P);
        }
    } else if (has_interior(g)) {
        if constexpr (FS) {
            return cudaErrorInvalidValue;
        } else if constexpr (pair_storage<St, COLL>()) {
            CUtensorMap m27, m3;
            if (pair_grid(g) && P.pair_bulk && g.nx % 8 == 0) {
                // requested explicitly: a layout the tensor-map encoder refuses is an error, not a fallback
                if (!encode_population_map(&m27, P.fp[0], g, 27) || !encode_population_map(&m3, P.fp[0], g, 3))
                    return cudaErrorNotSupported;
                // persistent, fed by tensor copies: as many CTAs as fit on the GPU at once
                static int grid_max = 0;
                if (!grid_max) {
                    int dev = 0, sms = 0, per_sm = 0;
                    cudaGetDevice(&dev);
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_pair_tma<St, NB, BAND, VOUT>, TMA_THREADS,
                                                                  TMA_SMEM);
                    grid_max = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
                }
                const long long tiles = tma_tiles(g, P.inner_rows).count;
                if (tiles > 0) {
                    const unsigned grid = (unsigned)(tiles < grid_max ? tiles : grid_max);
                    // pair_bulk 2: the wait-limit self-test (every barrier waits for 16 bytes no copy delivers)
                    k_step_pair_tma<St, NB, BAND, VOUT><<<grid, TMA_THREADS, TMA_SMEM, st>>>(m27, m3, P, P.err,
                                                                                          P.pair_bulk == 2 ? 16 : 0);
                }
            } else if (pair_grid(g)) {
                // one-warp blocks: at 94-96 registers a 64-thread block leaves part of the SM's
                // registers unused (10 blocks, 20 warps), one-warp blocks fit 21 (measured 0.7 % faster)
                const int pairs = range / 2, pthreads = 32;
                k_step_pair<St, NB, BAND, VOUT><<<dim3(step_blocks(pairs, pthreads), g.ny, g.nz), pthreads, 0, st>>>(P);
            } else {
                k_step_main<St, NB, BAND, COLL, VOUT, FS><<<dim3(xb, g.ny, g.nz), threads, 0, st>>>(P);
            }
        } else {
            k_step_main<St, NB, BAND, COLL, VOUT, FS><<<dim3(xb, g.ny, g.nz), threads, 0, st>>>(P);
        }
    }
    return cudaGetLastError();
}

template <typename St, int COLL, bool VOUT, bool FS>
cudaError_t launch_step_v(const StepParams &P, bool band, int part, cudaStream_t st) {
    const bool nb = (P.t & 1) != 0;
    if (nb) return band ? launch_step_tt<St, true, true, COLL, VOUT, FS>(P, part, st)
                        : launch_step_tt<St, true, false, COLL, VOUT, FS>(P, part, st);
    return band ? launch_step_tt<St, false, true, COLL, VOUT, FS>(P, part, st)
                : launch_step_tt<St, false, false, COLL, VOUT, FS>(P, part, st);
}

template <typename St, int COLL, bool FS>
cudaError_t launch_step_t(const StepParams &P, bool band, int part, cudaStream_t st) {
    return P.u_out ? launch_step_v<St, COLL, true, FS>(P, band, part, st)
                   : launch_step_v<St, COLL, false, FS>(P, band, part, st);
}

// one part of one step for the collision model COLL, on a grid with (FS) or without a free-slip
// face; instantiated in lbm_step_<model>.cu and lbm_step_<model>_fs.cu
template <int COLL, bool FS>
cudaError_t launch_step_coll(int storage, const StepParams &P, bool band, int part, cudaStream_t st) {
    switch (storage) {
        case 0: return launch_step_t<float, COLL, FS>(P, band, part, st);
        case 1: return launch_step_t<__half, COLL, FS>(P, band, part, st);
        default: return launch_step_t<__nv_bfloat16, COLL, FS>(P, band, part, st);
    }
}

}  // namespace lbm
