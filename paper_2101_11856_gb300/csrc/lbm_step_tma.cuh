// Main range of the fused step for 16-bit storage with the method's collision, fed by the tensor
// memory accelerator: a persistent kernel whose CTAs walk tiles of TMA_W consecutive nodes of one
// row.  Thread 0 issues, TMA_STAGES - 1 tiles ahead of the compute, the tiled tensor copies
// (cp.async.bulk.tensor over a 4-D map (x, y, z, direction plane) of the population array,
// completion counted in bytes on an mbarrier) of the tile's 27 source segments into one stage of
// a shared-memory ring: an even step reads every node's own slots, one box of 27 planes; an odd
// step pulls from the 9 (c_y, c_z) neighbour rows, one box of the 3 adjacent planes of each row.
// The consumer threads take one node pair (x, x + 1) each, read its 27 pair values from shared
// memory and run the same packed-FP32 collision and stores as k_step_pair.  The populations in
// flight sit in shared memory instead of registers, so the kernel keeps more bytes in flight per
// SM than the register-bound k_step_pair.  Requires nx % 8 == 0 (16-byte aligned rows).
#pragma once

#include <cuda.h>

#include "lbm_step.cuh"

namespace lbm {

constexpr int TMA_C = 128;                 // threads per CTA: consumers of one node pair each
constexpr int TMA_W = 240;                 // nodes per tile (TMA_W / 2 consumers busy)
constexpr int TMA_SEG = 256;               // elements per plane segment: box of TMA_W + 16 along x
constexpr int TMA_STAGES = 3;
constexpr int TMA_THREADS = TMA_C;         // thread 0 also issues the copies
constexpr int TMA_STAGE_BYTES = 27 * TMA_SEG * 2;
// dynamic shared memory: 128 bytes of alignment slack, the stages, then the mbarriers
constexpr size_t TMA_SMEM = 128 + (size_t)TMA_STAGES * TMA_STAGE_BYTES + TMA_STAGES * 8;
// a bounded wait gives up after this many SM clocks (about a second)
constexpr long long TMA_WAIT_CLOCKS = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for phase `parity` of the barrier, at most TMA_WAIT_CLOCKS; false when the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > TMA_WAIT_CLOCKS) return false;
    return true;
}
// tiled 4-D tensor copy of the box at (x, y, z, plane) into shared memory at dst
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int d, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(d), "r"(bar)
        : "memory");
}

struct TmaTiles {
    int per_row;      // tiles per row
    int rows_y, y0;   // rows y0 <= y < y0 + rows_y, z0 <= z < z0 + rows_z
    int z0;
    long long count;  // tiles
};

__host__ __device__ inline TmaTiles tma_tiles(const Geometry &g, int inner_rows) {
    TmaTiles T;
    const int range = g.nx - 2 * XEDGE;
    T.per_row = (range + TMA_W - 1) / TMA_W;
    T.y0 = inner_rows ? 1 : 0;
    T.z0 = inner_rows ? 1 : 0;
    T.rows_y = inner_rows ? (g.ny > 2 ? g.ny - 2 : 0) : g.ny;
    const int rows_z = inner_rows ? (g.nz > 2 ? g.nz - 2 : 0) : g.nz;
    T.count = (long long)T.per_row * T.rows_y * rows_z;
    return T;
}

// tile k: row (y, z), first node x0, nodes wt (a multiple of 8: nx % 8 == 0)
__host__ __device__ inline void tma_tile(const Geometry &g, const TmaTiles &T, long long k, int &y, int &z, int &x0, int &wt) {
    const int c = (int)(k % T.per_row);
    const long long r = k / T.per_row;
    y = T.y0 + (int)(r % T.rows_y);
    z = T.z0 + (int)(r / T.rows_y);
    x0 = XEDGE + c * TMA_W;
    const int xend = g.nx - XEDGE;
    wt = xend - x0 < TMA_W ? xend - x0 : TMA_W;
}

// Issue the copies of tile k into the stage at shared address buf (thread 0).  Segment q of the
// stage holds elements [x0 - 8, x0 + TMA_W + 8) of one plane (boxes reaching past the row end are
// filled with zeros by the copy and not read): even steps, planes 0..26 of the node's own row;
// odd steps, for each (c_y, c_z) row j, planes 24 - 3j .. 26 - 3j (the opposite directions of
// d = 3j + 2 .. 3j) of the source row into segments 3j .. 3j + 2, or the node's own planes
// 3j .. 3j + 2 when the source row lies across a no-slip face (bounce-back reads the own slot).
// tx_extra: bytes the barrier waits for beyond the copies (0; 16 in the wait-limit self-test,
// where no tile's data ever counts as complete)
template <bool NB>
__device__ __forceinline__ void tma_issue(const CUtensorMap *m27, const CUtensorMap *m3, const Geometry &g,
                                          const TmaTiles &T, long long k, uint32_t buf, uint32_t bar, int tx_extra) {
    int y, z, x0, wt;
    tma_tile(g, T, k, y, z, x0, wt);
    mbar_expect_tx(bar, (uint32_t)(TMA_STAGE_BYTES + tx_extra));
    if constexpr (!NB) {
        tma_load4(buf, m27, x0 - 8, y, z, 0, bar);
    } else {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            int yy = y - (j % 3 - 1), zz = z - (j / 3 - 1);
            bool bb = false;
            if (yy < 0 || yy >= g.ny) {
                if (g.periodic[1]) yy += yy < 0 ? g.ny : -g.ny;
                else bb = true;
            }
            if (zz < 0 || zz >= g.nz) {
                if (g.periodic[2]) zz += zz < 0 ? g.nz : -g.nz;
                else bb = true;
            }
            const uint32_t dst = buf + (uint32_t)(3 * j * TMA_SEG * 2);
            if (bb) tma_load4(dst, m3, x0 - 8, y, z, 3 * j, bar);
            else tma_load4(dst, m3, x0 - 8, yy, zz, 24 - 3 * j, bar);
        }
    }
}

template <typename St, bool NB, bool BAND, bool VOUT>
__global__ void __launch_bounds__(TMA_THREADS, 5) k_step_pair_tma(const __grid_constant__ CUtensorMap m27,
                                                                  const __grid_constant__ CUtensorMap m3, StepParams P,
                                                                  int *err, int tx_extra) {
    extern __shared__ unsigned char tma_smem_raw[];
    // 128-byte aligned stages (the copies' destinations), then the barriers
    const uint32_t base = (smem_addr(tma_smem_raw) + 127u) & ~127u;
    const St *stage = reinterpret_cast<const St *>(tma_smem_raw + (base - smem_addr(tma_smem_raw)));
    const uint32_t bars = base + (uint32_t)(TMA_STAGES * TMA_STAGE_BYTES);
    const TmaTiles T = tma_tiles(P.g, P.inner_rows);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < TMA_STAGES; ++s) mbar_init(bars + 8u * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m27)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m3)) : "memory");
    }
    __syncthreads();
    // prologue: the first TMA_STAGES tiles of this CTA
    if (tid == 0)
        for (int s = 0; s < TMA_STAGES; ++s) {
            const long long k = blockIdx.x + (long long)s * gridDim.x;
            if (k < T.count)
                tma_issue<NB>(&m27, &m3, P.g, T, k, base + (uint32_t)(s * TMA_STAGE_BYTES), bars + 8u * s, tx_extra);
        }
    for (long long i = 0;; ++i) {
        const long long k = blockIdx.x + i * gridDim.x;
        if (k >= T.count) break;
        const int s = (int)(i % TMA_STAGES);
        int y, z, x0, wt;
        tma_tile(P.g, T, k, y, z, x0, wt);
        const int cell = x0 + 2 * tid + P.g.nx * (y + P.g.ny * z);
        const bool active = 2 * tid < wt;
        // the pair's band-bitmap word, loaded before the wait so that its latency overlaps it
        uint32_t bmask = 0u;
        if (BAND && active) bmask = P.tile_mask[cell >> 5];
        const bool ok = __syncthreads_and(mbar_wait_bounded(bars + 8u * s, (uint32_t)((i / TMA_STAGES) & 1)));
        if (!ok) {
            // record the failure, give the copies still in flight for the other stages a bounded
            // wait (they write this CTA's shared memory), and leave
            if (tid == 0) {
                atomicExch(err, 1);
                for (int q = 1; q < TMA_STAGES; ++q) {
                    const long long iq = i + q;
                    if (blockIdx.x + iq * gridDim.x < T.count)
                        mbar_wait_bounded(bars + 8u * (uint32_t)(iq % TMA_STAGES), (uint32_t)((iq / TMA_STAGES) & 1));
                }
            }
            return;
        }
        if (active) {
            int off[9], mir[9];
            bool bb[9];
            const bool inner = y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2;
            if (inner) row_offsets<-1, true, false>(P.g, y, z, off, bb, mir);
            else row_offsets<-1, false, false>(P.g, y, z, off, bb, mir);
            const St *buf = stage + (size_t)s * 27 * TMA_SEG + 8 + 2 * tid;
            F2 h[27];
#pragma unroll
            for (int d = 0; d < 27; ++d) {
                const int j = d / 3, c = d % 3;
                if (!NB) {
                    h[d] = ld_pair<St, false>(buf + d * TMA_SEG, 0);
                } else if (bb[j]) {
                    h[d] = ld_pair<St, false>(buf + d * TMA_SEG, 0);
                } else {
                    // plane opp(d) of source row j sits in segment 3j + 2 - c, shifted by -c_x
                    const St *seg = buf + (3 * j + 2 - c) * TMA_SEG;
                    if (cx(d) == 0) h[d] = ld_pair<St, false>(seg, 0);
                    else h[d] = ld_pair<St, true>(seg, -cx(d));
                }
            }
            F2 Fx, Fy, Fz, rho, ux, uy, uz;
            Fx = {make_float2(P.Fx, P.Fx)};
            Fy = {make_float2(P.Fy, P.Fy)};
            Fz = {make_float2(P.Fz, P.Fz)};
            if (BAND) {
                const int lane = cell & 31;
                const uint32_t two = (bmask >> lane) & 3u;
                if (two) {
                    const long long b = P.tile_off[cell >> 5] + __popc(bmask & ((1u << lane) - 1u));
                    if (two & 1u) {
                        Fx.v.x += P.bandF[b];
                        Fy.v.x += P.bandF[P.nband + b];
                        Fz.v.x += P.bandF[2 * P.nband + b];
                    }
                    if (two & 2u) {
                        const long long b1 = b + (two & 1u);
                        Fx.v.y += P.bandF[b1];
                        Fy.v.y += P.bandF[P.nband + b1];
                        Fz.v.y += P.bandF[2 * P.nband + b1];
                    }
                }
            }
            collide_v<F2>(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
            if (VOUT) {
                const long long n = P.g.ncell;
                *reinterpret_cast<float2 *>(P.u_out + cell) = ux.v;
                *reinterpret_cast<float2 *>(P.u_out + n + cell) = uy.v;
                *reinterpret_cast<float2 *>(P.u_out + 2 * n + cell) = uz.v;
            }
            if (inner) row_offsets<+1, true, false>(P.g, y, z, off, bb, mir);
            else row_offsets<+1, false, false>(P.g, y, z, off, bb, mir);
            store_pair<St, NB>(P, cell, off, bb, h);
        }
        // every consumer has read stage s: refill it with the tile TMA_STAGES ahead
        __syncthreads();
        if (tid == 0) {
            const long long kn = k + (long long)TMA_STAGES * gridDim.x;
            if (kn < T.count) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_issue<NB>(&m27, &m3, P.g, T, kn, base + (uint32_t)(s * TMA_STAGE_BYTES), bars + 8u * s, tx_extra);
            }
        }
    }
}

// 4-D tensor map (x, y, z, direction plane) of a population array of 16-bit values whose 27
// planes start at `base` with a stride of `plane` elements; boxes of TMA_SEG x 1 x 1 x planes.
// False when the driver's encoder is unavailable or rejects the layout.
inline bool encode_population_map(CUtensorMap *m, const void *base, const Geometry &g, int planes) {
    typedef CUresult (*Encode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                               const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<Encode>(fn);
        else
            cudaGetLastError();
    }
    if (!encode) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 27};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 2, (cuuint64_t)g.nxy * 2, (cuuint64_t)g.plane * 2};
    const cuuint32_t box[4] = {(cuuint32_t)TMA_SEG, 1, 1, (cuuint32_t)planes};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void *>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbm
