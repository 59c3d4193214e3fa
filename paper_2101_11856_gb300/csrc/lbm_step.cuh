// Pull (load) and push (store) addressing of the fused step for the AA pattern, shared by
// the forward kernels (lbm_kernels.cu) and the adjoint kernels (lbm_adjoint.cu).
//
// AA pattern (in-place streaming, one population array): with A[d][cell] the storage,
//  * after an even step (and at t = 0) A[opp(d)][x] holds the post-collision f_d(x);
//  * an odd step t ("neighbour" step) pulls f*_d(x) = A[opp(d)][x - c_d] and writes the
//    new f_d(x) to A[d][x + c_d];
//  * an even step ("local" step) reads f*_d(x) = A[d][x] and writes f_d(x) to A[opp(d)][x].
// Each node reads and writes the same 27 slots, so one array suffices and no two threads
// touch a slot.  A population whose source lies behind a non-periodic face is found in
// the node's own slot A[d][x] (the previous step wrote the reflected value there), which
// gives half-way bounce-back (the paper's Algorithm 1) and the moving-wall inlet; the
// outlet reads a ping-pong copy of the outlet plane's previous post-collision values.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// ---- loads of the streamed populations f*(x) ------------------------------------------

// interior node: every neighbour exists, constant offsets; one base pointer per plane
template <typename St, bool NB>
__device__ __forceinline__ void load_interior(const StepParams &P, int cell, float (&h)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (NB) {
            const St *p = static_cast<const St *>(P.fp[opp(d)]) + (cell - (cy(d) * P.g.nx + cz(d) * P.g.nxy));
            h[d] = Store<St>::ld(p - cx(d));
        } else {
            h[d] = Store<St>::ld(static_cast<const St *>(P.fp[d]) + cell);
        }
    }
}

template <typename St, bool NB>
__device__ __forceinline__ void load_general(const StepParams &P, int x, int y, int z, int cell, float (&h)[27]) {
    const St *A = static_cast<const St *>(P.f);
    const St *B = static_cast<const St *>(P.outlet);
    const long long pl = P.g.plane;
    const int rpar = (int)((P.t - 1) & 1);
    const bool inlet_node = (x == 0) && P.g.face[0] == FACE_INLET;
    const float uw = inlet_node ? inlet_velocity(P, y, z) : 0.0f;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        const Nbr n = neighbour<-1>(P.g, d, x, y, z);
        float v;
        if (n.kind == 0) {
            v = NB ? Store<St>::ld(A + opp(d) * pl + n.idx) : Store<St>::ld(A + d * pl + cell);
        } else if (n.kind & CROSS_NOSLIP) {
            v = Store<St>::ld(A + d * pl + cell);
        } else if (n.kind & CROSS_INLET) {
            // moving wall: f*_d = f_opp(d) + 2 w_d rho0 (c_d . u_w) / c_s^2
            v = Store<St>::ld(A + d * pl + cell) + 6.0f * wgt(d) * P.rho0 * (float)cx(d) * uw;
        } else if (n.kind & CROSS_OUTLET) {
            // outlet ghost: post-collision f_d of (nx-1, y - c_dy, z - c_dz) of the previous step
            // (across a free-slip face: the mirrored source and direction)
            const int md = mirror_dir(d, n.mir);
            v = Store<St>::ld(B + ((long long)(rpar * 9 + md / 3) * P.g.nyz + n.y + P.g.ny * n.z));
        } else {
            // free-slip faces only: the specular image from the tangential neighbour (odd steps);
            // even steps find it in the node's own slot
            v = NB ? Store<St>::ld(A + opp(mirror_dir(d, n.mir)) * pl + n.idx) : Store<St>::ld(A + d * pl + cell);
        }
        h[d] = v;
    }
}

// ---- stores of the post-collision populations ------------------------------------------

template <typename St, bool NB>
__device__ __forceinline__ void store_interior(const StepParams &P, int cell, const float (&h)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (NB) {
            St *p = static_cast<St *>(P.fpo[d]) + (cell + (cy(d) * P.g.nx + cz(d) * P.g.nxy));
            Store<St>::st(p + cx(d), h[d]);
        } else {
            Store<St>::st(static_cast<St *>(P.fpo[opp(d)]) + cell, h[d]);
        }
    }
}

__device__ __forceinline__ void decompose(const Geometry &g, int cell, int &x, int &y, int &z) {
    z = cell / g.nxy;
    const int r = cell - z * g.nxy;
    y = r / g.nx;
    x = r - y * g.nx;
}

// immersed-boundary force of the band node at `cell` (zero off the band)
template <bool BAND>
__device__ __forceinline__ void band_force(const StepParams &P, int cell, float &Fx, float &Fy, float &Fz) {
    Fx = P.Fx; Fy = P.Fy; Fz = P.Fz;
    if (BAND) {
        const uint32_t mask = P.tile_mask[cell >> 5];
        const int lane = cell & 31;
        if ((mask >> lane) & 1u) {
            const long long b = P.tile_off[cell >> 5] + __popc(mask & ((1u << lane) - 1u));
            Fx += P.bandF[b];
            Fy += P.bandF[P.nband + b];
            Fz += P.bandF[2 * P.nband + b];
        }
    }
}

// ---- rows of a block's y/z neighbours ----------------------------------------------------
// The y and z faces are periodic, no-slip or free-slip.  For the node rows y + S c_y,
// z + S c_z (S = -1: pull source, S = +1: push target) give the cell offset of the row (with
// periodic wrap), or mark it as crossing a no-slip face (bounce-back to the node's own slot),
// or as crossing free-slip faces: mir bit 0 (y) / bit 1 (z), the row offset of that axis is 0
// and the population is the specular image (mirror_dir).  No-slip wins over free-slip.
// Row j of direction d is j = d / 3 = (c_y + 1) + 3 (c_z + 1).  FS: the grid has a free-slip face
// (without it the mirror flags are the constant 0 and every mirrored direction folds to d).
template <int S, bool FS>
__device__ __forceinline__ void yz_rows(const Geometry &g, int y, int z, int (&off)[9], bool (&bb)[9], int (&mir)[9]) {
    int oy[3], oz[3];
    bool by[3], bz[3], my[3], mz[3];
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
        int yy = y + S * c, zz = z + S * c;
        by[c + 1] = bz[c + 1] = my[c + 1] = mz[c + 1] = false;
        if (yy < 0) {
            if (g.periodic[1]) yy += g.ny;
            else if (FS && g.face[2] == FACE_FREESLIP) { my[c + 1] = true; yy = y; }
            else by[c + 1] = true;
        } else if (yy >= g.ny) {
            if (g.periodic[1]) yy -= g.ny;
            else if (FS && g.face[3] == FACE_FREESLIP) { my[c + 1] = true; yy = y; }
            else by[c + 1] = true;
        }
        if (zz < 0) {
            if (g.periodic[2]) zz += g.nz;
            else if (FS && g.face[4] == FACE_FREESLIP) { mz[c + 1] = true; zz = z; }
            else bz[c + 1] = true;
        } else if (zz >= g.nz) {
            if (g.periodic[2]) zz -= g.nz;
            else if (FS && g.face[5] == FACE_FREESLIP) { mz[c + 1] = true; zz = z; }
            else bz[c + 1] = true;
        }
        oy[c + 1] = (yy - y) * g.nx;
        oz[c + 1] = (zz - z) * g.nxy;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        off[j] = oy[j % 3] + oz[j / 3];
        bb[j] = by[j % 3] || bz[j / 3];
        mir[j] = FS ? (my[j % 3] ? 1 : 0) | (mz[j / 3] ? 2 : 0) : 0;
    }
}

// direction D of a row with free-slip mirror flags m (warp-uniform): its specular image for
// the mirrored axes in which D has a nonzero component (constant D after unrolling); D itself
// without a free-slip face (spelled out: the flags 0 alone do not fold the table index)
template <bool FS>
__device__ __forceinline__ int mdir(int D, int m) {
    if (!FS) return D;
    const int my = cy(D) != 0 ? (m & 1) : 0, mz = cz(D) != 0 ? (m & 2) : 0;
    return mirror_dir(D, my | mz);
}

// odd-step loads/stores of a node with 1 <= x <= nx-2 on a y or z face
template <typename St, bool FS>
__device__ __forceinline__ void load_yzface(const StepParams &P, int y, int z, int cell, float (&h)[27]) {
    int off[9], mir[9];
    bool bb[9];
    yz_rows<-1, FS>(P.g, y, z, off, bb, mir);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (bb[d / 3]) h[d] = Store<St>::ld(static_cast<const St *>(P.fp[d]) + cell);
        else h[d] = Store<St>::ld(static_cast<const St *>(P.fp[opp(mdir<FS>(d, mir[d / 3]))]) + (cell + off[d / 3]) - cx(d));
    }
}

template <typename St, bool FS>
__device__ __forceinline__ void store_yzface(const StepParams &P, int y, int z, int cell, const float (&h)[27]) {
    int off[9], mir[9];
    bool bb[9];
    yz_rows<+1, FS>(P.g, y, z, off, bb, mir);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (bb[d / 3]) Store<St>::st(static_cast<St *>(P.fpo[opp(d)]) + cell, h[d]);
        else Store<St>::st(static_cast<St *>(P.fpo[mdir<FS>(d, mir[d / 3])]) + (cell + off[d / 3]) + cx(d), h[d]);
    }
}

// ---- two nodes per thread (x and x + 32) for the main kernel -------------------------------
// The address of each direction is formed once and serves both nodes through an immediate
// offset of 32 elements, so a warp's accesses stay coalesced (32 consecutive nodes each).
template <typename St, bool NB>
__device__ __forceinline__ void load_interior2(const StepParams &P, int cell, bool two, float (&h0)[27],
                                               float (&h1)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        const St *p = NB ? static_cast<const St *>(P.fp[opp(d)]) + (cell - (cy(d) * P.g.nx + cz(d) * P.g.nxy)) - cx(d)
                         : static_cast<const St *>(P.fp[d]) + cell;
        h0[d] = Store<St>::ld(p);
        h1[d] = two ? Store<St>::ld(p + 32) : 0.0f;
    }
}

template <typename St, bool NB>
__device__ __forceinline__ void store_interior2(const StepParams &P, int cell, bool two, const float (&h0)[27],
                                                const float (&h1)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        St *p = NB ? static_cast<St *>(P.fpo[d]) + (cell + (cy(d) * P.g.nx + cz(d) * P.g.nxy)) + cx(d)
                   : static_cast<St *>(P.fpo[opp(d)]) + cell;
        Store<St>::st(p, h0[d]);
        if (two) Store<St>::st(p + 32, h1[d]);
    }
}

template <typename St, bool FS>
__device__ __forceinline__ void load_yzface2(const StepParams &P, int y, int z, int cell, bool two, float (&h0)[27],
                                             float (&h1)[27]) {
    int off[9], mir[9];
    bool bb[9];
    yz_rows<-1, FS>(P.g, y, z, off, bb, mir);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        const St *p = bb[d / 3] ? static_cast<const St *>(P.fp[d]) + cell
                                : static_cast<const St *>(P.fp[opp(mdir<FS>(d, mir[d / 3]))]) + (cell + off[d / 3]) - cx(d);
        h0[d] = Store<St>::ld(p);
        h1[d] = two ? Store<St>::ld(p + 32) : 0.0f;
    }
}

template <typename St, bool FS>
__device__ __forceinline__ void store_yzface2(const StepParams &P, int y, int z, int cell, bool two,
                                              const float (&h0)[27], const float (&h1)[27]) {
    int off[9], mir[9];
    bool bb[9];
    yz_rows<+1, FS>(P.g, y, z, off, bb, mir);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        St *p = bb[d / 3] ? static_cast<St *>(P.fpo[opp(d)]) + cell
                          : static_cast<St *>(P.fpo[mdir<FS>(d, mir[d / 3])]) + (cell + off[d / 3]) + cx(d);
        Store<St>::st(p, h0[d]);
        if (two) Store<St>::st(p + 32, h1[d]);
    }
}

// ---- node pairs (x, x + 1) with x even, 16-bit storage ---------------------------------------
// With nx even every pair starts on an even cell index, so one aligned 32-bit word holds both
// nodes' values of a direction wherever the access is not shifted along x: every access of an
// even step and the c_x = 0 directions of an odd step.  The c_x = +-1 directions of an odd step
// are shifted by one element: their two values are the high half of the aligned word before and
// the low half of the aligned word after (the neighbouring threads read the same words, so the
// second read is served by L1), and they are written as two 16-bit halves.
template <typename St> struct Half2Of;
template <> struct Half2Of<__half> {
    static __device__ __forceinline__ F2 unpack(uint32_t w) { return {__half22float2(*reinterpret_cast<const __half2 *>(&w))}; }
    static __device__ __forceinline__ uint32_t pack(F2 v) {
        const __half2 p = __float22half2_rn(v.v);
        return *reinterpret_cast<const uint32_t *>(&p);
    }
};
template <> struct Half2Of<__nv_bfloat16> {
    static __device__ __forceinline__ F2 unpack(uint32_t w) {
        return {__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w))};
    }
    static __device__ __forceinline__ uint32_t pack(F2 v) {
        const __nv_bfloat162 p = __float22bfloat162_rn(v.v);
        return *reinterpret_cast<const uint32_t *>(&p);
    }
};
// the values of elements e, e + 1 of a plane; SHIFTED: e is odd
template <typename St, bool SHIFTED> __device__ __forceinline__ F2 ld_pair(const St *plane, long long e) {
    if (!SHIFTED) return Half2Of<St>::unpack(*reinterpret_cast<const uint32_t *>(plane + e));
    const uint32_t lo = *reinterpret_cast<const uint32_t *>(plane + (e - 1));
    const uint32_t hi = *reinterpret_cast<const uint32_t *>(plane + (e + 1));
    return Half2Of<St>::unpack(__byte_perm(lo, hi, 0x5432));
}
template <typename St, bool SHIFTED> __device__ __forceinline__ void st_pair(St *plane, long long e, F2 v) {
    const uint32_t w = Half2Of<St>::pack(v);
    if (!SHIFTED) {
        *reinterpret_cast<uint32_t *>(plane + e) = w;
    } else {
        *reinterpret_cast<uint16_t *>(plane + e) = (uint16_t)(w & 0xffffu);
        *reinterpret_cast<uint16_t *>(plane + (e + 1)) = (uint16_t)(w >> 16);
    }
}

// streamed populations of the pair at `cell` (x even, 1 <= x, x + 1 <= nx - 2); row offsets off
// and bounce-back flags bb of the 9 (c_y, c_z) source rows (odd steps)
template <typename St, bool NB>
__device__ __forceinline__ void load_pair(const StepParams &P, int cell, const int (&off)[9], const bool (&bb)[9],
                                          F2 (&h)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (!NB || bb[d / 3]) {
            h[d] = ld_pair<St, false>(static_cast<const St *>(P.fp[d]), cell);
        } else {
            const St *pl = static_cast<const St *>(P.fp[opp(d)]);
            const long long e = (long long)cell + off[d / 3] - cx(d);
            h[d] = cx(d) == 0 ? ld_pair<St, false>(pl, e) : ld_pair<St, true>(pl, e);
        }
    }
}

template <typename St, bool NB>
__device__ __forceinline__ void store_pair(const StepParams &P, int cell, const int (&off)[9], const bool (&bb)[9],
                                           const F2 (&h)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        if (!NB || bb[d / 3]) {
            st_pair<St, false>(static_cast<St *>(P.fpo[opp(d)]), cell, h[d]);
        } else {
            St *pl = static_cast<St *>(P.fpo[d]);
            const long long e = (long long)cell + off[d / 3] + cx(d);
            if (cx(d) == 0) st_pair<St, false>(pl, e, h[d]);
            else st_pair<St, true>(pl, e, h[d]);
        }
    }
}

// body force plus the band's immersed-boundary force of the pair (cell, cell + 1), cell even:
// both nodes lie in the same 32-cell word of the band bitmap
template <bool BAND>
__device__ __forceinline__ void band_force_pair(const StepParams &P, int cell, F2 &Fx, F2 &Fy, F2 &Fz) {
    Fx = {make_float2(P.Fx, P.Fx)};
    Fy = {make_float2(P.Fy, P.Fy)};
    Fz = {make_float2(P.Fz, P.Fz)};
    if (BAND) {
        const uint32_t mask = P.tile_mask[cell >> 5];
        const int lane = cell & 31;
        const uint32_t two = (mask >> lane) & 3u;
        if (two) {
            const long long b = P.tile_off[cell >> 5] + __popc(mask & ((1u << lane) - 1u));
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
}

// ---- the edge strips: y/z faces per block, x faces per lane --------------------------------
// The pull rules of load_general and the matching push rules, arranged for a block that covers one
// strip of one (y, z) row: the y/z rows come from yz_rows (uniform), and only the lanes at
// x = 0 or x = nx-1 take the x-face rule for the directions whose source (pull) or target
// (push) lies across that face.  Priority at edges: no-slip > inlet > outlet.
// Row offsets of the 9 (c_y, c_z) neighbour rows, pull (S = -1) or push (S = +1): constant
// offsets for a row away from the y/z faces (INNER), else yz_rows (wrap / no-slip flags).
template <int S, bool INNER, bool FS>
__device__ __forceinline__ void row_offsets(const Geometry &g, int y, int z, int (&off)[9], bool (&bb)[9],
                                            int (&mir)[9]) {
    if (INNER) {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            off[j] = S * ((j % 3 - 1) * g.nx + (j / 3 - 1) * g.nxy);
            bb[j] = false;
            mir[j] = 0;
        }
    } else {
        yz_rows<S, FS>(g, y, z, off, bb, mir);
    }
}

// SIDE: 0 = left strip (only x = 0 can be a face lane), 1 = right strip (only x = nx-1),
// 2 = a whole short row (both)
template <typename St, bool NB, bool INNER, int SIDE, bool FS>
__device__ __forceinline__ void load_edge_t(const StepParams &P, int x, int y, int z, int cell, float (&h)[27]) {
    int off[9], mir[9];
    bool bb[9];
    row_offsets<-1, INNER, FS>(P.g, y, z, off, bb, mir);
    const bool xlo = SIDE != 1 && x == 0, xhi = SIDE != 0 && x == P.g.nx - 1;
    // every lane pulls as an interior node; the lanes at x = 0 / nx-1 read their own slot for
    // the directions whose source lies across the x face, and are fixed up below
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        const int j = d / 3;
        if (!NB) {
            h[d] = Store<St>::ld(static_cast<const St *>(P.fp[d]) + cell);
            continue;
        }
        bool own = bb[j];
        if (cx(d) == 1) own = own || xlo;
        if (cx(d) == -1) own = own || xhi;
        const St *base = static_cast<const St *>(own ? P.fp[d] : P.fp[opp(mdir<FS>(d, mir[j]))]);
        h[d] = Store<St>::ld(base + (own ? cell : cell + off[j] - cx(d)));
    }
    // x-face rules of the face lanes (one per warp), once per side
    if (xlo) {
        const int ft = P.g.face[0];
        const float uw = ft == FACE_INLET ? inlet_velocity(P, y, z) : 0.0f;
#pragma unroll
        for (int d = 2; d < 27; d += 3) {   // c_x = +1: sources across the -x face
            if (bb[d / 3]) continue;         // no-slip wins at edges
            if (ft == FACE_PERIODIC && NB)
                h[d] = Store<St>::ld(static_cast<const St *>(P.fp[opp(mdir<FS>(d, mir[d / 3]))]) +
                                     (cell + off[d / 3] + (P.g.nx - 1)));
            else if (ft == FACE_INLET)
                h[d] += 6.0f * wgt(d) * P.rho0 * uw;
        }
    }
    if (xhi) {
        const int ft = P.g.face[1];
        const St *B = static_cast<const St *>(P.outlet) + (long long)(((P.t - 1) & 1) * 9) * P.g.nyz;
#pragma unroll
        for (int d = 0; d < 27; d += 3) {   // c_x = -1: sources across the +x face
            if (bb[d / 3]) continue;
            if (ft == FACE_PERIODIC && NB) {
                h[d] = Store<St>::ld(static_cast<const St *>(P.fp[opp(mdir<FS>(d, mir[d / 3]))]) +
                                     (cell + off[d / 3] - (P.g.nx - 1)));
            } else if (ft == FACE_OUTLET) {
                // outlet ghost: post-collision f_d of (nx-1, y - c_dy, z - c_dz) of the previous
                // step; across a free-slip face the source keeps y (z) and the direction mirrors
                const int m = mir[d / 3], dd = mdir<FS>(d, m);
                int ys = y - cy(d), zs = z - cz(d);
                ys += ys < 0 ? P.g.ny : (ys >= P.g.ny ? -P.g.ny : 0);
                zs += zs < 0 ? P.g.nz : (zs >= P.g.nz ? -P.g.nz : 0);
                if (m & 1) ys = y;
                if (m & 2) zs = z;
                h[d] = Store<St>::ld(B + (long long)(dd / 3) * P.g.nyz + ys + P.g.ny * zs);
            }
        }
    }
}

template <typename St, bool NB, bool INNER, int SIDE, bool FS>
__device__ __forceinline__ void store_edge_t(const StepParams &P, int x, int y, int z, int cell, const float (&h)[27]) {
    const bool xlo = SIDE != 1 && x == 0, xhi = SIDE != 0 && x == P.g.nx - 1, per = P.g.periodic[0];
    if (NB) {
        int off[9], mir[9];
        bool bb[9];
        row_offsets<+1, INNER, FS>(P.g, y, z, off, bb, mir);
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            const int j = d / 3;
            bool xc = false;
            if (cx(d) == 1) xc = xhi;
            if (cx(d) == -1) xc = xlo;
            // target across a no-slip face (or a non-periodic x face): the node's own slot
            const bool own = bb[j] || (xc && !per);
            const int idx = own ? cell : cell + off[j] + (xc ? -cx(d) * (P.g.nx - 1) : cx(d));
            St *base = static_cast<St *>(own ? P.fpo[opp(d)] : P.fpo[mdir<FS>(d, mir[j])]);
            Store<St>::st(base + idx, h[d]);
        }
    } else {
#pragma unroll
        for (int d = 0; d < 27; ++d) Store<St>::st(static_cast<St *>(P.fpo[opp(d)]) + cell, h[d]);
    }
    if (xhi && P.g.face[1] == FACE_OUTLET) {
        St *B = static_cast<St *>(P.outlet_o) + (long long)((P.t & 1) * 9) * P.g.nyz + y + P.g.ny * z;
#pragma unroll
        for (int d = 0; d < 27; d += 3)   // the nine directions with c_x = -1
            Store<St>::st(B + (long long)(d / 3) * P.g.nyz, h[d]);
    }
}

// edge-strip node of a warp row: INNER when the row is away from the y/z faces (warp-uniform)
template <typename St, bool NB, int SIDE, bool FS>
__device__ __forceinline__ void load_edge(const StepParams &P, int x, int y, int z, int cell, float (&h)[27]) {
    // (the FS kernels see face rows, or every row of a grid without a main range: yz_rows serves both)
    if (!FS && y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2) load_edge_t<St, NB, true, SIDE, FS>(P, x, y, z, cell, h);
    else load_edge_t<St, NB, false, SIDE, FS>(P, x, y, z, cell, h);
}

template <typename St, bool NB, int SIDE, bool FS>
__device__ __forceinline__ void store_edge(const StepParams &P, int x, int y, int z, int cell, const float (&h)[27]) {
    if (!FS && y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2) store_edge_t<St, NB, true, SIDE, FS>(P, x, y, z, cell, h);
    else store_edge_t<St, NB, false, SIDE, FS>(P, x, y, z, cell, h);
}

// x of an edge-strip thread: SIDE 0 / 1 = left / right strip of a row with a main range,
// SIDE 2 = consecutive warps over a row too short for the main kernel
template <int SIDE> __device__ __forceinline__ int edge_x(const Geometry &g) {
    return SIDE == 0 ? (int)threadIdx.x : SIDE == 1 ? g.nx - XEDGE + (int)threadIdx.x : (int)(blockIdx.x * XEDGE + threadIdx.x);
}
constexpr int EDGE_ROWS = 4;   // rows (y) per edge-kernel block, one warp each

}  // namespace lbm
