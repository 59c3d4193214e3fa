// Hand-written adjoint of the time step: gradients of a drag + kinetic-energy loss with
// respect to the inflow-profile coefficients and the immersed-boundary sample positions.
//
// Forward step t (Algorithm 2): f*_t = S(f_{t-1}; a) (streaming with the faces; the inlet
// adds 2 w_i rho0 c_i.u_w with u_w linear in the inflow coefficients a), IB force
// F_t = spread(g(f*_t; X); X), f_t = C(f*_t, F_b + F_t) (central-moment collision).
// With lambda_t = dL/df_t the backward step computes, per node, the vector-Jacobian product
// of the collision (recomputed in registers from the stored f_{t-1}), the IB terms (the
// transposes of spreading and interpolation, and the trilinear weights' derivatives for the
// positions), and pushes mu = dL/df* back along the streaming (its transpose):
// lambda_{t-1}[i](x - c_i) = mu_i(x), bounce-back slots get mu of the reflected direction,
// the slots the outlet ghost copied take its second use on top.  States f_{t-1} come from
// segment recomputation between checkpoints taken every K steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lbm_ctx.h"
#include "lbm_step.cuh"

using namespace lbm;
using namespace lbm_host;

namespace lbm {

// ---- 3-point maps of the adjoint (transposes of the forward per-axis maps) -------------
// forward raw R: (a, b, c) -> (a + b + c, c - a, c + a); its transpose
__device__ __forceinline__ void rawT3(float &a, float &b, float &c) {
    const float l0 = a, l1 = b, l2 = c;
    a = l0 - l1 + l2;
    b = l0;
    c = l0 + l1 + l2;
}
// forward inverse raw R^-1: (r0, r1, r2) -> ((r2 - r1)/2, r0 - r2, (r2 + r1)/2); its transpose
__device__ __forceinline__ void invrawT3(float &a, float &b, float &c) {
    const float la = a, lb = b, lc = c;
    a = lb;
    b = 0.5f * (lc - la);
    c = 0.5f * (la + lc) - lb;
}
// central shift Sh(u) = [[1,0,0],[-u,1,0],[u^2,-2u,1]]; its transpose
__device__ __forceinline__ void shiftT3(float &a, float &b, float &c, float u) {
    const float l1 = b, l2 = c;
    a = fmaf(u * u, l2, fmaf(-u, l1, a));
    b = fmaf(-2.0f * u, l2, l1);
}
// transpose of the inverse shift Sh(u)^-1 = [[1,0,0],[u,1,0],[u^2,2u,1]]
__device__ __forceinline__ void invshiftT3(float &a, float &b, float &c, float u) {
    a = fmaf(u * u, c, fmaf(u, b, a));
    b = fmaf(2.0f * u, c, b);
}

template <int S, typename Op> __device__ __forceinline__ void sweep(float (&h)[27], Op op) {
#pragma unroll
    for (int k = 0; k < 9; ++k) op(h[tri_base<S>(k)], h[tri_base<S>(k) + S], h[tri_base<S>(k) + 2 * S]);
}

// sum over the triplets of axis S of l[1] v[0] + 2 l[2] v[1]: the contraction with the
// generator A of the shift (dSh/du = -A Sh, d(Sh^-1)/du = A Sh^-1)
template <int S> __device__ __forceinline__ float gen_contract(const float (&l)[27], const float (&v)[27]) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int b = tri_base<S>(k);
        acc = fmaf(l[b + S], v[b], acc);
        acc = fmaf(2.0f * l[b + 2 * S], v[b + S], acc);
    }
    return acc;
}

struct AdjExtra {
    float drho, djx, djy, djz;   // direct dL/d rho*, dL/d j at this node (IB terms)
    float wke;                   // weight of 1/2 rho |u|^2 at this node (last step, slab), else 0
};

// Vector-Jacobian product of the collision f_post = C(f*, F) (Eqs. 4-5, same operator as
// collide() in lbm_device.cuh): in lam = dL/df_post, out lam = dL/df*, dF += dL/dF.
__device__ __forceinline__ void collide_vjp(const float (&fs)[27], float Fx, float Fy, float Fz, const StepParams &P,
                                            const AdjExtra &ex, float (&lam)[27], float &dFx, float &dFy, float &dFz) {
    // forward recompute in full populations
    float k[27];
#pragma unroll
    for (int d = 0; d < 27; ++d) k[d] = fs[d];
    sweep<1>(k, [](float &a, float &b, float &c) { raw3(a, b, c); });
    sweep<3>(k, [](float &a, float &b, float &c) { raw3(a, b, c); });
    sweep<9>(k, [](float &a, float &b, float &c) { raw3(a, b, c); });
    const float rho = k[K(0, 0, 0)];
    const float inv = 1.0f / rho;
    const float ux = (k[K(1, 0, 0)] + 0.5f * Fx) * inv;
    const float uy = (k[K(0, 1, 0)] + 0.5f * Fy) * inv;
    const float uz = (k[K(0, 0, 1)] + 0.5f * Fz) * inv;
    sweep<1>(k, [ux](float &a, float &b, float &c) { shift3(a, b, c, ux); });
    sweep<3>(k, [uy](float &a, float &b, float &c) { shift3(a, b, c, uy); });
    sweep<9>(k, [uz](float &a, float &b, float &c) { shift3(a, b, c, uz); });
    const float wb = 1.0f - P.rb, w4 = 1.0f - P.r4, w6 = 1.0f - P.r6;
    const float third = 1.0f / 3.0f, ninth = 1.0f / 9.0f;

    // backward: populations -> post-collision raw moments -> post-collision central moments
    sweep<1>(lam, [](float &a, float &b, float &c) { invrawT3(a, b, c); });
    sweep<3>(lam, [](float &a, float &b, float &c) { invrawT3(a, b, c); });
    sweep<9>(lam, [](float &a, float &b, float &c) { invrawT3(a, b, c); });
    sweep<1>(lam, [ux](float &a, float &b, float &c) { invshiftT3(a, b, c, ux); });
    sweep<3>(lam, [uy](float &a, float &b, float &c) { invshiftT3(a, b, c, uy); });
    sweep<9>(lam, [uz](float &a, float &b, float &c) { invshiftT3(a, b, c, uz); });
    // u through the inverse shift: d/du_a (Sh^-1 kappa') = A_a Sh^-1 kappa' = Sh^-1 A_a kappa'
    // (A_a generates the shifts and commutes with them), so the contraction pairs dL/dkappa'
    // with the post-collision central moments kappa', formed here from kappa (k)
    float dux, duy, duz;
    {
        float kp[27];
#pragma unroll
        for (int d = 0; d < 27; ++d) kp[d] = k[d];
        kp[K(1, 0, 0)] += Fx;
        kp[K(0, 1, 0)] += Fy;
        kp[K(0, 0, 1)] += Fz;
        kp[K(1, 1, 0)] *= P.rs;
        kp[K(1, 0, 1)] *= P.rs;
        kp[K(0, 1, 1)] *= P.rs;
        {
            const float a = k[K(2, 0, 0)] - rho * third, b = k[K(0, 2, 0)] - rho * third, c = k[K(0, 0, 2)] - rho * third;
            const float s3 = (a + b + c) * third;
            kp[K(2, 0, 0)] = rho * third + P.rb * s3 + P.rs * (a - s3);
            kp[K(0, 2, 0)] = rho * third + P.rb * s3 + P.rs * (b - s3);
            kp[K(0, 0, 2)] = rho * third + P.rb * s3 + P.rs * (c - s3);
        }
        kp[K(2, 1, 0)] = fmaf(P.r3, k[K(2, 1, 0)], P.q3 * third * Fy);
        kp[K(2, 0, 1)] = fmaf(P.r3, k[K(2, 0, 1)], P.q3 * third * Fz);
        kp[K(1, 2, 0)] = fmaf(P.r3, k[K(1, 2, 0)], P.q3 * third * Fx);
        kp[K(0, 2, 1)] = fmaf(P.r3, k[K(0, 2, 1)], P.q3 * third * Fz);
        kp[K(1, 0, 2)] = fmaf(P.r3, k[K(1, 0, 2)], P.q3 * third * Fx);
        kp[K(0, 1, 2)] = fmaf(P.r3, k[K(0, 1, 2)], P.q3 * third * Fy);
        kp[K(1, 1, 1)] = P.r3 * k[K(1, 1, 1)];
        kp[K(2, 2, 0)] = fmaf(P.r4, k[K(2, 2, 0)], w4 * ninth * rho);
        kp[K(2, 0, 2)] = fmaf(P.r4, k[K(2, 0, 2)], w4 * ninth * rho);
        kp[K(0, 2, 2)] = fmaf(P.r4, k[K(0, 2, 2)], w4 * ninth * rho);
        kp[K(2, 1, 1)] = P.r4 * k[K(2, 1, 1)];
        kp[K(1, 2, 1)] = P.r4 * k[K(1, 2, 1)];
        kp[K(1, 1, 2)] = P.r4 * k[K(1, 1, 2)];
        kp[K(2, 2, 1)] = fmaf(P.r5, k[K(2, 2, 1)], P.q5 * ninth * Fz);
        kp[K(2, 1, 2)] = fmaf(P.r5, k[K(2, 1, 2)], P.q5 * ninth * Fy);
        kp[K(1, 2, 2)] = fmaf(P.r5, k[K(1, 2, 2)], P.q5 * ninth * Fx);
        dux = gen_contract<1>(lam, kp);
        duy = gen_contract<3>(lam, kp);
        duz = gen_contract<9>(lam, kp);
    }
    // relaxation: lam = dL/d kappa'
    float drho = 0.0f;
    dFx += lam[K(1, 0, 0)] + P.q3 * third * (lam[K(1, 2, 0)] + lam[K(1, 0, 2)]) + P.q5 * ninth * lam[K(1, 2, 2)];
    dFy += lam[K(0, 1, 0)] + P.q3 * third * (lam[K(2, 1, 0)] + lam[K(0, 1, 2)]) + P.q5 * ninth * lam[K(2, 1, 2)];
    dFz += lam[K(0, 0, 1)] + P.q3 * third * (lam[K(2, 0, 1)] + lam[K(0, 2, 1)]) + P.q5 * ninth * lam[K(2, 2, 1)];
    drho += wb * third * (lam[K(2, 0, 0)] + lam[K(0, 2, 0)] + lam[K(0, 0, 2)]);
    drho += w4 * ninth * (lam[K(2, 2, 0)] + lam[K(2, 0, 2)] + lam[K(0, 2, 2)]);
    drho += w6 * (1.0f / 27.0f) * lam[K(2, 2, 2)];
    lam[K(1, 1, 0)] *= P.rs;
    lam[K(1, 0, 1)] *= P.rs;
    lam[K(0, 1, 1)] *= P.rs;
    {
        // the diagonal block (rb/3) J + (rs/3)(3 I - J) is symmetric
        const float a = lam[K(2, 0, 0)], b = lam[K(0, 2, 0)], c = lam[K(0, 0, 2)];
        const float s3 = (a + b + c) * third;
        lam[K(2, 0, 0)] = P.rb * s3 + P.rs * (a - s3);
        lam[K(0, 2, 0)] = P.rb * s3 + P.rs * (b - s3);
        lam[K(0, 0, 2)] = P.rb * s3 + P.rs * (c - s3);
    }
    lam[K(2, 1, 0)] *= P.r3; lam[K(2, 0, 1)] *= P.r3; lam[K(1, 2, 0)] *= P.r3;
    lam[K(0, 2, 1)] *= P.r3; lam[K(1, 0, 2)] *= P.r3; lam[K(0, 1, 2)] *= P.r3; lam[K(1, 1, 1)] *= P.r3;
    lam[K(2, 2, 0)] *= P.r4; lam[K(2, 0, 2)] *= P.r4; lam[K(0, 2, 2)] *= P.r4;
    lam[K(2, 1, 1)] *= P.r4; lam[K(1, 2, 1)] *= P.r4; lam[K(1, 1, 2)] *= P.r4;
    lam[K(2, 2, 1)] *= P.r5; lam[K(2, 1, 2)] *= P.r5; lam[K(1, 2, 2)] *= P.r5;
    lam[K(2, 2, 2)] *= P.r6;
    // u through the forward shift: d/du_a (Sh r) = -A_a kappa
    dux -= gen_contract<1>(lam, k);
    duy -= gen_contract<3>(lam, k);
    duz -= gen_contract<9>(lam, k);
    sweep<1>(lam, [ux](float &a, float &b, float &c) { shiftT3(a, b, c, ux); });
    sweep<3>(lam, [uy](float &a, float &b, float &c) { shiftT3(a, b, c, uy); });
    sweep<9>(lam, [uz](float &a, float &b, float &c) { shiftT3(a, b, c, uz); });
    // kinetic-energy term 1/2 rho |u|^2 of the loss
    if (ex.wke != 0.0f) {
        dux = fmaf(ex.wke * rho, ux, dux);
        duy = fmaf(ex.wke * rho, uy, duy);
        duz = fmaf(ex.wke * rho, uz, duz);
        drho = fmaf(0.5f * ex.wke, ux * ux + uy * uy + uz * uz, drho);
    }
    // u = (j + F/2) / rho
    dFx += 0.5f * dux * inv;
    dFy += 0.5f * duy * inv;
    dFz += 0.5f * duz * inv;
    drho -= (dux * ux + duy * uy + duz * uz) * inv;
    lam[K(0, 0, 0)] += drho + ex.drho;
    lam[K(1, 0, 0)] += dux * inv + ex.djx;
    lam[K(0, 1, 0)] += duy * inv + ex.djy;
    lam[K(0, 0, 1)] += duz * inv + ex.djz;
    sweep<1>(lam, [](float &a, float &b, float &c) { rawT3(a, b, c); });
    sweep<3>(lam, [](float &a, float &b, float &c) { rawT3(a, b, c); });
    sweep<9>(lam, [](float &a, float &b, float &c) { rawT3(a, b, c); });
}

}  // namespace lbm

namespace {

// full streamed populations f* of node (x, y, z) at step P.t from the stored f_{t-1}, with
// the general per-direction face classification (band nodes: few, anywhere in the domain)
template <typename St, bool NB>
__device__ __forceinline__ void adj_load_fstar(const StepParams &P, int x, int y, int z, int cell, float (&h)[27]) {
    load_general<St, NB>(P, x, y, z, cell, h);
#pragma unroll
    for (int d = 0; d < 27; ++d) h[d] += wgt(d) * P.rho0;
}

__device__ __forceinline__ bool band_index(const StepParams &P, int cell, long long &b) {
    const uint32_t mask = P.tile_mask[cell >> 5];
    const int lane = cell & 31;
    if (!((mask >> lane) & 1u)) return false;
    b = P.tile_off[cell >> 5] + __popc(mask & ((1u << lane) - 1u));
    return true;
}

struct AdjParams {
    const float *lam_cur;        // [27][N] dL/df_t (canonical, library direction order)
    float *lam_prev;             // [27][N] dL/df_{t-1}
    double *s_inlet;             // [nyz] accumulated sum_i mu_i 6 w_i rho0 c_ix per inlet node
    const float *adj_band;       // [4][nband] dL/d rho*, dL/d j of the band nodes
    float *dF_band;              // [3][nband] dL/dF of the band nodes
    float wke;                   // w_ke on the last step, else 0
    int ke_x0, ke_x1;
    const float *ghost_in;       // [9][nyz] outlet ghost uses of step t + 1 (x-face kernel)
    float *ghost_out;            // [9][nyz] outlet ghost uses of this step
    int row_y0, row_z0;          // k_adj_main covers the rows (row_y0 + blockIdx.y, row_z0 + blockIdx.z)
};

// lambda_t of node (x, y, z) as its own backward step uses it: at x = nx - 1 next to an outlet the
// slots the outlet ghost copied take the ghost's use of step t + 1 (ghost_in; the slot itself
// holds the push of (nx-2, y, z)), and the slots of populations that left through the outlet
// (no use) read as zero
__device__ __forceinline__ void read_lambda(const StepParams &P, const AdjParams &A, int x, int y, int z, int cell,
                                            float (&lam)[27]) {
    const long long N = P.g.ncell;
    const bool outlet = x == P.g.nx - 1 && P.g.face[1] == FACE_OUTLET;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        lam[d] = A.lam_cur[d * N + cell];
        if (outlet && cx(d) == 1 && neighbour<+1>(P.g, d, x, y, z).kind == CROSS_OUTLET) lam[d] = 0.0f;
        if (outlet && cx(d) == -1) {
            // the ghost of (nx-1, y + c_y, z + c_z) copied this slot for its f*_d
            int yy = y + cy(d), zz = z + cz(d);
            bool src = true;
            if (yy < 0 || yy >= P.g.ny) { if (P.g.periodic[1]) yy += yy < 0 ? P.g.ny : -P.g.ny; else src = false; }
            if (zz < 0 || zz >= P.g.nz) { if (P.g.periodic[2]) zz += zz < 0 ? P.g.nz : -P.g.nz; else src = false; }
            if (src) lam[d] += A.ghost_in[(long long)(d / 3) * P.g.nyz + yy + P.g.ny * zz];
        }
    }
}

// dL/dF at the band nodes (collision VJP with respect to the force)
template <typename St, bool NB>
__global__ void __launch_bounds__(128) k_adj_band_force(StepParams P, AdjParams A, const int *__restrict__ band_cell) {
    const long long kb = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (kb >= P.nband) return;
    const int cell = band_cell[kb];
    int x, y, z;
    decompose(P.g, cell, x, y, z);
    float fs[27], lam[27];
    adj_load_fstar<St, NB>(P, x, y, z, cell, fs);
    read_lambda(P, A, x, y, z, cell, lam);
    const float Fx = P.Fx + P.bandF[kb], Fy = P.Fy + P.bandF[P.nband + kb], Fz = P.Fz + P.bandF[2 * P.nband + kb];
    AdjExtra ex{0.0f, 0.0f, 0.0f, 0.0f, (x >= A.ke_x0 && x < A.ke_x1) ? A.wke : 0.0f};
    float dFx = 0.0f, dFy = 0.0f, dFz = 0.0f;
    collide_vjp(fs, Fx, Fy, Fz, P, ex, lam, dFx, dFy, dFz);
    A.dF_band[kb] = dFx;
    A.dF_band[P.nband + kb] = dFy;
    A.dF_band[2 * P.nband + kb] = dFz;
}

__device__ __forceinline__ float cw(int c, float wx, float wy, float wz) {
    return ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
}

// per sample: dL/dg = interpolated dL/dF + drag weight; dL/d rho_s, dL/du_s (Eq. 7 transposed);
// position gradient from the spreading and interpolation weights (Eqs. 6 and 8)
__global__ void __launch_bounds__(256) k_adj_samples(long long S, long long nband, const float *__restrict__ X,
                                                     const float *__restrict__ area, const float *__restrict__ ub,
                                                     const int *__restrict__ corner_band,
                                                     const float *__restrict__ band_rho, const float *__restrict__ band_u,
                                                     const float *__restrict__ g, const float *__restrict__ dF,
                                                     float drag_w, float *__restrict__ adj_samp, double *__restrict__ dX) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const float wx = X[s] - floorf(X[s]), wy = X[S + s] - floorf(X[S + s]), wz = X[2 * S + s] - floorf(X[2 * S + s]);
    float dgx = drag_w, dgy = 0.0f, dgz = 0.0f, rs = 0.0f, us = 0.0f, vs = 0.0f, ws = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int b = corner_band[(long long)c * S + s];
        const float Kc = cw(c, wx, wy, wz);
        dgx = fmaf(Kc, dF[b], dgx);
        dgy = fmaf(Kc, dF[nband + b], dgy);
        dgz = fmaf(Kc, dF[2 * nband + b], dgz);
        rs = fmaf(Kc, band_rho[b], rs);
        us = fmaf(Kc, band_u[b], us);
        vs = fmaf(Kc, band_u[nband + b], vs);
        ws = fmaf(Kc, band_u[2 * nband + b], ws);
    }
    const float a = area[s];
    const float drs = a * ((ub[s] - us) * dgx + (ub[S + s] - vs) * dgy + (ub[2 * S + s] - ws) * dgz);
    const float dus = -rs * a * dgx, dvs = -rs * a * dgy, dws = -rs * a * dgz;
    adj_samp[s] = drs;
    adj_samp[S + s] = dus;
    adj_samp[2 * S + s] = dvs;
    adj_samp[3 * S + s] = dws;
    const float gx = g[s], gy = g[S + s], gz = g[2 * S + s];
    float px = 0.0f, py = 0.0f, pz = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int b = corner_band[(long long)c * S + s];
        const float kx = (c & 1) ? wx : 1.0f - wx, ky = (c & 2) ? wy : 1.0f - wy, kz = (c & 4) ? wz : 1.0f - wz;
        const float sx = (c & 1) ? 1.0f : -1.0f, sy = (c & 2) ? 1.0f : -1.0f, sz = (c & 4) ? 1.0f : -1.0f;
        // value the corner weight multiplies: spreading (dF . g) and interpolation (rho*, u_IB)
        const float v = dF[b] * gx + dF[nband + b] * gy + dF[2 * nband + b] * gz + drs * band_rho[b] +
                        dus * band_u[b] + dvs * band_u[nband + b] + dws * band_u[2 * nband + b];
        px = fmaf(sx * ky * kz, v, px);
        py = fmaf(sy * kx * kz, v, py);
        pz = fmaf(sz * kx * ky, v, pz);
    }
    dX[s] += px;
    dX[S + s] += py;
    dX[2 * S + s] += pz;
}

// per band node: gather dL/d rho*, dL/du_IB from the samples (transpose of Eq. 6), then
// through u_IB = (j + F_body/2)/rho* to dL/d rho*, dL/dj (returned as x, y, z, w = rho*, j_x,
// j_y, j_z)
__device__ __forceinline__ float4 band_gather(long long k, long long S, long long nband, const float *__restrict__ X,
                                              const int *__restrict__ base_nbr, const int *__restrict__ cstart,
                                              const int *__restrict__ ccount, const float *__restrict__ adj_samp,
                                              const float *__restrict__ band_rho, const float *__restrict__ band_u) {
    float dr = 0.0f, du = 0.0f, dv = 0.0f, dw = 0.0f;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        const int b = base_nbr[(long long)c * nband + k];
        if (b < 0) continue;
        const int s0 = cstart[b], s1 = s0 + ccount[b];
        for (int s = s0; s < s1; ++s) {
            const float Kc = cw(c, X[s] - floorf(X[s]), X[S + s] - floorf(X[S + s]), X[2 * S + s] - floorf(X[2 * S + s]));
            dr = fmaf(Kc, adj_samp[s], dr);
            du = fmaf(Kc, adj_samp[S + s], du);
            dv = fmaf(Kc, adj_samp[2 * S + s], dv);
            dw = fmaf(Kc, adj_samp[3 * S + s], dw);
        }
    }
    const float rho = band_rho[k], inv = 1.0f / rho;
    const float u = band_u[k], v = band_u[nband + k], w = band_u[2 * nband + k];
    return make_float4(dr - (du * u + dv * v + dw * w) * inv, du * inv, dv * inv, dw * inv);
}

__global__ void __launch_bounds__(256) k_adj_band_gather(long long S, long long nband, const float *__restrict__ X,
                                                         const int *__restrict__ base_nbr, const int *__restrict__ cstart,
                                                         const int *__restrict__ ccount, const float *__restrict__ adj_samp,
                                                         const float *__restrict__ band_rho,
                                                         const float *__restrict__ band_u, float *__restrict__ adj_band) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nband) return;
    const float4 a = band_gather(k, S, nband, X, base_nbr, cstart, ccount, adj_samp, band_rho, band_u);
    adj_band[k] = a.x;
    adj_band[nband + k] = a.y;
    adj_band[2 * nband + k] = a.z;
    adj_band[3 * nband + k] = a.w;
}

// dL/df* of a node: collision VJP with the band's IB terms and the loss's kinetic-energy term
// (lam holds the incoming lambda_t of the node on entry)
template <bool BAND>
__device__ __forceinline__ void node_vjp_in(const StepParams &P, const AdjParams &A, int x, int cell, float (&fs)[27],
                                            float (&lam)[27]) {
#pragma unroll
    for (int d = 0; d < 27; ++d) fs[d] += wgt(d) * P.rho0;
    float Fx = P.Fx, Fy = P.Fy, Fz = P.Fz;
    AdjExtra ex{0.0f, 0.0f, 0.0f, 0.0f, (x >= A.ke_x0 && x < A.ke_x1) ? A.wke : 0.0f};
    long long b;
    if (BAND && band_index(P, cell, b)) {
        Fx += P.bandF[b];
        Fy += P.bandF[P.nband + b];
        Fz += P.bandF[2 * P.nband + b];
        ex.drho = A.adj_band[b];
        ex.djx = A.adj_band[P.nband + b];
        ex.djy = A.adj_band[2 * P.nband + b];
        ex.djz = A.adj_band[3 * P.nband + b];
    }
    float dFx = 0.0f, dFy = 0.0f, dFz = 0.0f;
    collide_vjp(fs, Fx, Fy, Fz, P, ex, lam, dFx, dFy, dFz);
}

template <bool BAND>
__device__ __forceinline__ void node_vjp(const StepParams &P, const AdjParams &A, int x, int cell, float (&fs)[27],
                                         float (&lam)[27]) {
    const long long N = P.g.ncell;
#pragma unroll
    for (int d = 0; d < 27; ++d) lam[d] = A.lam_cur[d * N + cell];
    node_vjp_in<BAND>(P, A, x, cell, fs, lam);
}

// push of mu from a node 1 <= x <= nx - 2 of row (y, z)
__device__ __forceinline__ void adj_push_main(const StepParams &P, const AdjParams &A, int y, int z, int cell, bool inner,
                                              const float (&lam)[27]) {
    const long long N = P.g.ncell;
    if (inner) {
#pragma unroll
        for (int d = 0; d < 27; ++d)
            A.lam_prev[d * N + cell - (cx(d) + cy(d) * P.g.nx + cz(d) * P.g.nxy)] = lam[d];
    } else {
        int off[9], mir[9];
        bool bb[9];
        yz_rows<-1, false>(P.g, y, z, off, bb, mir);   // free-slip faces are rejected by lbm_adjoint
#pragma unroll
        for (int d = 0; d < 27; ++d) {
            if (bb[d / 3]) A.lam_prev[opp(d) * N + cell] = lam[d];
            else A.lam_prev[d * N + cell + off[d / 3] - cx(d)] = lam[d];
        }
    }
}

// Backward step of the nodes 1 <= x <= nx - 2 (one block row per (y, z); the lanes of x = 0 and
// x >= nx - 1 idle): mu = dL/df* pushed along the transposed streaming,
// lambda_{t-1}[d](x - c_d) = mu_d(x), or to the bounce-back slot lambda_{t-1}[opp(d)](x) where
// the source lies across a no-slip y/z face.  No lane crosses an x face, so every lane of a
// warp runs the same addressing.  12 resident blocks per SM (80 registers, a few spilled values)
// measured faster than the 96 registers the compiler picks alone (21 warps per SM).
template <typename St, bool NB, bool BAND>
__global__ void __launch_bounds__(STEP_BX, 12) k_adj_main(StepParams P, AdjParams A) {
    const int x = blockIdx.x * STEP_BX + threadIdx.x;
    if (x < 1 || x > P.g.nx - 2) return;
    const int y = blockIdx.y + A.row_y0, z = blockIdx.z + A.row_z0;
    const int cell = x + P.g.nx * (y + P.g.ny * z);
    const bool inner = y >= 1 && y <= P.g.ny - 2 && z >= 1 && z <= P.g.nz - 2;   // uniform per block
    float fs[27], lam[27];
    if (!NB || inner) load_interior<St, NB>(P, cell, fs);
    else load_yzface<St, false>(P, y, z, cell, fs);
    node_vjp<BAND>(P, A, x, cell, fs, lam);
    adj_push_main(P, A, y, z, cell, inner, lam);
}

// Backward step of the x-face nodes x = 0 (blockIdx.y = 0) and x = nx - 1 (blockIdx.y = 1), one
// thread per node (nx >= 3).  Each mu_d goes back to the slot its streamed value came from, by
// the pull's own per-direction rules: the wrapped neighbour (periodic x), the node's reflected
// slot (no-slip; the inlet also feeds the inflow-coefficient gradient), or, through the outlet
// ghost, the previous post-collision value of (nx-1, y - c_y, z - c_z) that the ghost copied.
// That slot (c_x = -1) also takes the push of (nx-2, y, z) from k_adj_main, so the ghost's use
// goes to ghost_out and the next backward step adds it where it reads the slot (read_lambda), so
// no slot is written by both kernels and none is read back and written again.
template <typename St, bool NB, bool BAND>
__global__ void __launch_bounds__(128) k_adj_xface(StepParams P, AdjParams A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.g.nyz) return;
    const int z = i / P.g.ny, y = i - z * P.g.ny;
    const int x = blockIdx.y ? P.g.nx - 1 : 0;
    const int cell = x + P.g.nx * (y + P.g.ny * z);
    const long long N = P.g.ncell;
    float fs[27], lam[27];
    load_general<St, NB>(P, x, y, z, cell, fs);
    read_lambda(P, A, x, y, z, cell, lam);
    node_vjp_in<BAND>(P, A, x, cell, fs, lam);
    float sth = 0.0f;   // this node's inflow sensitivity (accumulated over steps in FP64)
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        const Nbr n = neighbour<-1>(P.g, d, x, y, z);
        const float mu = lam[d];
        if (n.kind == 0) {
            A.lam_prev[d * N + n.idx] = mu;
        } else if (n.kind & (CROSS_NOSLIP | CROSS_INLET)) {
            A.lam_prev[opp(d) * N + cell] = mu;
            if (!(n.kind & CROSS_NOSLIP)) sth = fmaf(mu, 6.0f * wgt(d) * P.rho0, sth);   // inlet: c_x = +1
        } else {
            A.ghost_out[(long long)(d / 3) * P.g.nyz + y + P.g.ny * z] = mu;   // outlet ghost
        }
    }
    if (!blockIdx.y && P.g.face[0] == FACE_INLET) A.s_inlet[y + P.g.ny * z] += (double)sth;
}

__global__ void k_finalize_add(const double *__restrict__ partial, long long n, int count, double *__restrict__ out) {
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
        if (threadIdx.x == 0) out[k] += s[0];
        __syncthreads();
    }
}

unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename F> cudaError_t with_storage(int storage, F &&fn) {
    switch (storage) {
        case 0: return fn(float{});
        case 1: return fn(__half{});
        default: return fn(__nv_bfloat16{});
    }
}

// the adjoint's device workspace, kept by the context between calls: the k-th request of a
// call reuses the k-th buffer when it is large enough (calls with the same sizes allocate
// nothing after the first)
// the context's IB arrays (band moments, penalty forces, spread forces) pointed at other storage
// for a while: the recompute of a segment keeps each step's values, which the backward step then
// reads instead of computing them again; the context's own arrays come back on every exit
struct IBArrays {
    lbm_ctx *h;
    float *rho, *u, *g, *F;
    explicit IBArrays(lbm_ctx *h_) : h(h_), rho(h_->band_rho), u(h_->band_u), g(h_->g), F(h_->bandF) {}
    void point(float *r, float *uu, float *gg, float *ff) {
        h->band_rho = r;
        h->band_u = uu;
        h->g = gg;
        h->bandF = ff;
    }
    void restore() { point(rho, u, g, F); }
    ~IBArrays() { restore(); }
};

// one forward step as lbm_step takes it (moving solids excluded by lbm_adjoint), reading the
// state buffer src and writing the state buffer dst, or the context's own state for dst = NULL
int adj_forward_step(lbm_ctx *h, void *src, void *dst) {
    const long long t = h->t + 1;
    int rc;
    StepParams P = make_params(h, t);
    if (h->ntracer) P.u_out = h->tracer_u;
    if (dst) {
        point_states(P, h, src, dst);
    } else {
        const size_t pb = (size_t)h->plane * h->esize;
        P.f = src;
        for (int d = 0; d < 27; ++d) P.fp[d] = static_cast<char *>(src) + d * pb;
        P.outlet = h->outlet ? static_cast<char *>(src) + 27 * pb : nullptr;
    }
    if ((rc = step_with(h, P))) return rc;
    if ((rc = advect_tracers(h, t))) return rc;
    h->t = t;
    return LBM_OK;
}

// the backward pass runs on a stream of the highest priority beside the segment recompute
constexpr bool kBackwardPriority = true;

struct AdjBuffers {
    lbm_ctx *h;
    size_t next = 0;
    explicit AdjBuffers(lbm_ctx *h_) : h(h_) {}
    // quiet: a failed allocation returns LBM_ENOMEM without recording an error message
    template <typename T> int get(lbm_ctx *, T **p, size_t n, bool quiet = false) {
        const size_t bytes = n * sizeof(T);
        if (next == h->adj_ws.size()) h->adj_ws.push_back({nullptr, 0});
        auto &slot = h->adj_ws[next++];
        if (slot.second < bytes) {
            if (slot.first) cudaFree(slot.first);
            slot = {nullptr, 0};
            void *q = nullptr;
            if (cudaMalloc(&q, bytes) != cudaSuccess) {
                cudaGetLastError();
                if (quiet) return LBM_ENOMEM;
                return fail(h, LBM_ENOMEM, "cannot allocate the adjoint workspace (" + std::to_string(bytes) + " bytes)");
            }
            slot = {q, bytes};
        }
        *p = static_cast<T *>(slot.first);
        return LBM_OK;
    }
};

// the main backward kernel over the rows of box r (nothing for an empty box), then (xface) the
// x-face kernel
template <typename St, bool NB, bool BAND>
cudaError_t launch_adj_step_tt(const StepParams &P, AdjParams A, const RowBox &r, bool xface, cudaStream_t st) {
    const Geometry &g = P.g;
    if (r.ny > 0 && r.nz > 0) {
        A.row_y0 = r.y0;
        A.row_z0 = r.z0;
        k_adj_main<St, NB, BAND><<<dim3(nblocks(g.nx - 1, STEP_BX), r.ny, r.nz), STEP_BX, 0, st>>>(P, A);
    }
    if (xface) k_adj_xface<St, NB, BAND><<<dim3(nblocks(g.nyz, 128), 2), 128, 0, st>>>(P, A);
    return cudaGetLastError();
}

template <typename St>
cudaError_t launch_adj_step(const StepParams &P, const AdjParams &A, bool nb, bool band, const RowBox &r, bool xface,
                            cudaStream_t st) {
    if (nb) return band ? launch_adj_step_tt<St, true, true>(P, A, r, xface, st)
                        : launch_adj_step_tt<St, true, false>(P, A, r, xface, st);
    return band ? launch_adj_step_tt<St, false, true>(P, A, r, xface, st)
                : launch_adj_step_tt<St, false, false>(P, A, r, xface, st);
}

}  // namespace

extern "C" int lbm_adjoint(lbm_ctx *h, int n, int K, const lbm_loss *loss, double *dL_dinflow, double *dL_dpos,
                           double *L) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!h->has_state) return fail(h, LBM_ESTATE, "lbm_set_state (or lbm_load) has not been called");
    if (n < 1 || !loss) return fail(h, LBM_EINVAL, "n must be >= 1 and loss given");
    if (h->cfg.collision != LBM_COLL_ACM) return fail(h, LBM_EINVAL, "the adjoint exists for the ACM-MRT collision only");
    if (h->nx < 3) return fail(h, LBM_EINVAL, "the adjoint needs nx >= 3");
    if (h->band_count_dev) return fail(h, LBM_EINVAL, "the adjoint exists for static solids only (lbm_set_motion was called)");
    for (int k = 2; k < 6; ++k)
        if (h->cfg.face_type[k] == LBM_FACE_FREESLIP) return fail(h, LBM_EINVAL, "the adjoint does not cover free-slip faces");
    if (loss->ke_x0 < 0 || loss->ke_x1 > h->nx || loss->ke_x0 > loss->ke_x1) return fail(h, LBM_EINVAL, "bad slab");
    K = std::max(1, std::min(K, n));
    const long long N = h->N, S = h->S, nb = h->nband;
    const int nyz = h->ny * h->nz;
    const size_t pop_bytes = (size_t)27 * h->plane * h->esize;
    const size_t out_bytes = h->outlet ? (size_t)2 * 9 * nyz * h->esize : 0;
    const size_t state_bytes = pop_bytes + out_bytes;
    const int nck = (n + K - 1) / K;
    AdjBuffers B(h);
    int rc;
    float *lamA, *lamB, *dF_band = nullptr, *adj_band = nullptr, *adj_samp = nullptr;
    double *s_inlet, *dX = nullptr, *acc;
    const int fblk = force_sum_blocks(S);
    double *step_sums = nullptr;   // [3][n * fblk] per-step, per-block sums of the penalty forces
    float *ghost = nullptr;   // [2][9][nyz] outlet ghost uses of alternate steps
    if ((rc = B.get(h, &lamA, (size_t)27 * N)) || (rc = B.get(h, &lamB, (size_t)27 * N)) ||
        (rc = B.get(h, &s_inlet, (size_t)nyz)) || (rc = B.get(h, &acc, 8)) || (rc = B.get(h, &ghost, (size_t)18 * nyz)))
        return rc;
    if (S > 0 && (rc = B.get(h, &step_sums, (size_t)3 * n * fblk))) return rc;
    if (S > 0 && ((rc = B.get(h, &dX, (size_t)3 * S)) || (rc = B.get(h, &dF_band, (size_t)3 * nb)) ||
                  (rc = B.get(h, &adj_band, (size_t)4 * nb)) || (rc = B.get(h, &adj_samp, (size_t)4 * S))))
        return rc;
    float *g_last = nullptr, *F_last = nullptr;     // IB diagnostics of the last step, restored at the end
    if (S > 0 && ((rc = B.get(h, &g_last, (size_t)3 * S)) || (rc = B.get(h, &F_last, (size_t)3 * nb)))) return rc;
    // cell sums of the IB stages the backward stream runs, apart from those of the recompute beside it
    float *cellS_b = nullptr;
    if (h->nocc > 0 && (rc = B.get(h, &cellS_b, (size_t)24 * h->nocc))) return rc;
    // Segment sets: the states f_{t0 + k} of a segment and the IB values of its recomputed steps
    // (slot j: the step from state t0 + j; the last step of a segment keeps none).  With two or
    // more sets the recompute of segment s - 1 runs on a second stream beside the backward pass of
    // segment s, into the set of the segment nset - 1 after s; a second set that does not fit in
    // device memory leaves one, and the recompute and the backward pass alternate.
    struct SegSet {
        std::vector<char *> f;
        float *rho = nullptr, *u = nullptr, *g = nullptr, *F = nullptr;
    };
    const size_t nslot = (size_t)(K - 1);
    auto get_set = [&](SegSet &q, bool quiet) -> int {
        q.f.assign(K, nullptr);
        for (int i = 0; i < K; ++i) if ((rc = B.get(h, &q.f[i], state_bytes, quiet))) return rc;
        if (S > 0 && nslot > 0 &&
            ((rc = B.get(h, &q.rho, nslot * nb, quiet)) || (rc = B.get(h, &q.u, nslot * 3 * nb, quiet)) ||
             (rc = B.get(h, &q.g, nslot * 3 * S, quiet)) || (rc = B.get(h, &q.F, nslot * 3 * nb, quiet))))
            return rc;
        return LBM_OK;
    };
    // Up to kMaxSets sets: the forward pass keeps the last nset segments in them (no recompute);
    // an extra set replaces a checkpoint, so a set is added only while the device memory free now
    // (plus this context's unclaimed workspace) holds it with the checkpoints still needed and a
    // margin; a set that does not fit after all ends the list.
    constexpr int kMaxSets = 4;
    SegSet sets[kMaxSets];
    if ((rc = get_set(sets[0], false))) return rc;
    int want = 1;
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = total_b = 0;
        }
        size_t held = 0;   // workspace slots this call has not claimed yet
        for (size_t i = B.next; i < h->adj_ws.size(); ++i) held += h->adj_ws[i].second;
        const size_t avail = free_b + held, margin = ((size_t)1 << 30) + total_b / 20;
        const size_t set_bytes = (size_t)K * state_bytes + (S > 0 ? nslot * (7 * (size_t)nb + 3 * (size_t)S) * 4 : 0);
        for (int m = 2; m <= std::min(kMaxSets, nck); ++m) {
            // sets 1..m-1 and the checkpoints of the other nck - m segments (set 0 is held)
            const size_t need = (size_t)(m - 1) * set_bytes + (size_t)(nck - m) * state_bytes;
            if (need + margin <= avail) want = m;
        }
        if (nck > 1 && want < 2) want = 2;   // the second set is always tried (the recompute beside the backward)
    }
    int nset = 1;
    while (nset < want && get_set(sets[nset], true) == LBM_OK) ++nset;
    // checkpoints of the segments whose states the forward pass does not keep in a set (all but
    // the last nset)
    const int nstored = nset;
    std::vector<char *> ckpt(nck, nullptr);
    for (int i = 0; i + nstored < nck; ++i) if ((rc = B.get(h, &ckpt[i], state_bytes))) return rc;
    IBArrays ib(h);
    // the forward pass asks each step for its drag sums (h->fsum); no request outlives this call
    struct FsumClear {
        lbm_ctx *h;
        ~FsumClear() { h->fsum = nullptr; }
    } fsum_clear{h};
    auto point_slot = [&](const SegSet &q, long long j) {
        ib.point(q.rho + j * nb, q.u + j * 3 * nb, q.g + j * 3 * S, q.F + j * 3 * nb);
    };
    StepParams P0 = make_params(h, h->t);
    const long long mblk = macro_blocks(P0);
    if ((rc = ensure_partial(h, (size_t)MACRO_SUMS * mblk))) return rc;
    cudaStream_t st = h->stream;
    // with two sets: the recompute stream, the backward pass on a stream of the highest priority
    // (the block scheduler serves its launches first, the recompute fills the rest), and the
    // events between them and the context's stream
    struct SideStreams {
        cudaStream_t s = nullptr, b = nullptr;
        cudaEvent_t done[kMaxSets] = {}, free_[kMaxSets] = {}, fork = nullptr, join = nullptr;
        ~SideStreams() {
            for (cudaStream_t q : {s, b})
                if (q) cudaStreamSynchronize(q);
            for (int k = 0; k < kMaxSets; ++k)
                for (cudaEvent_t e : {done[k], free_[k]})
                    if (e) cudaEventDestroy(e);
            for (cudaEvent_t e : {fork, join})
                if (e) cudaEventDestroy(e);
            for (cudaStream_t q : {s, b})
                if (q) cudaStreamDestroy(q);
        }
    } side;
    if (nset >= 2) {
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&side.s, cudaStreamNonBlocking, lo));
        CK(cudaStreamCreateWithPriority(&side.b, cudaStreamNonBlocking, kBackwardPriority ? hi : lo));
        for (int k = 0; k < nset; ++k) {
            CK(cudaEventCreateWithFlags(&side.done[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&side.free_[k], cudaEventDisableTiming));
        }
        for (cudaEvent_t *e : {&side.fork, &side.join}) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    CK(cudaMemsetAsync(s_inlet, 0, nyz * sizeof(double), st));
    CK(cudaMemsetAsync(acc, 0, 8 * sizeof(double), st));
    if (dX) CK(cudaMemsetAsync(dX, 0, 3 * S * sizeof(double), st));
    CK(cudaMemsetAsync(lamA, 0, (size_t)27 * N * sizeof(float), st));
    CK(cudaMemsetAsync(ghost, 0, (size_t)18 * nyz * sizeof(float), st));

    // forward pass: checkpoints, drag accumulation, final kinetic energy.  The last nstored
    // segments run out of place through their sets and keep their IB values, as their recompute
    // would (the backward pass then starts without one); the last step writes the context's state.
    const long long t_start = h->t;
    const int first_kept = nck - nstored;   // first segment kept in a set
    auto set_of = [&](int sgi) -> SegSet & { return sets[(nck - 1 - sgi) % nset]; };
    for (int i = 0; i < n; ++i) {
        const int sgi = i / K, k = i % K;
        const int len = std::min(K, n - sgi * K);
        if (S > 0) {
            // this step's per-block drag sums, launched right after its IB stage on that stage's stream
            h->fsum = step_sums + (size_t)i * fblk;
            h->fsum_stride = (long long)n * fblk;
        }
        if (sgi < first_kept) {
            if (k == 0) {
                CK(cudaMemcpyAsync(ckpt[sgi], h->f, pop_bytes, cudaMemcpyDeviceToDevice, st));
                if (out_bytes) CK(cudaMemcpyAsync(ckpt[sgi] + pop_bytes, h->outlet, out_bytes, cudaMemcpyDeviceToDevice, st));
            }
            if ((rc = lbm_step(h, 1))) return rc;
        } else {
            SegSet &q = set_of(sgi);
            if (i == first_kept * K) {   // the context's state enters the first kept segment
                CK(cudaMemcpyAsync(q.f[0], h->f, pop_bytes, cudaMemcpyDeviceToDevice, st));
                if (out_bytes) CK(cudaMemcpyAsync(q.f[0] + pop_bytes, h->outlet, out_bytes, cudaMemcpyDeviceToDevice, st));
            }
            const bool inner = k + 1 < len;
            if (S > 0) {
                if (inner) point_slot(q, k);
                else ib.restore();
            }
            // the segment's last step writes the next segment's first state, or the context's
            char *dst = inner ? q.f[k + 1] : (sgi + 1 < nck ? set_of(sgi + 1).f[0] : nullptr);
            if ((rc = adj_forward_step(h, q.f[k], dst))) return rc;
        }
    }
    if (S > 0) {
        k_finalize_add<<<1, 256, 0, st>>>(step_sums, (long long)n * fblk, 3, acc);
        CK(cudaGetLastError());
    }
    {
        StepParams P = make_params(h, h->t);
        CK(launch_macro(h->storage, P, S > 0, 1, nullptr, nullptr, nullptr, h->partial, nullptr, st, loss->ke_x0,
                        loss->ke_x1));
        k_finalize_add<<<1, 256, 0, st>>>(h->partial + 4 * mblk, mblk, 1, acc + 3);
        CK(cudaGetLastError());
    }
    if (S > 0) {
        CK(cudaMemcpyAsync(g_last, h->g, 3 * S * sizeof(float), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(F_last, h->bandF, 3 * nb * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }

    // recompute segment sgi's states out of place into set q on stream rs: f[k] = f_{t0 + k}
    auto recompute = [&](int sgi, const SegSet &q, cudaStream_t rs) -> int {
        const long long t0 = t_start + (long long)sgi * K;
        const int len = (int)std::min<long long>(K, t_start + n - t0);
        CK(cudaMemcpyAsync(q.f[0], ckpt[sgi], state_bytes, cudaMemcpyDeviceToDevice, rs));
        struct StreamSwap {   // step_with launches on the context's stream
            lbm_ctx *h;
            cudaStream_t old;
            StreamSwap(lbm_ctx *h_, cudaStream_t s) : h(h_), old(h_->stream) { h->stream = s; }
            ~StreamSwap() { h->stream = old; }
        } swap_(h, rs);
        for (int k = 0; k + 1 < len; ++k) {
            if (S > 0) point_slot(q, k);
            StepParams Pf = make_params(h, t0 + k + 1);
            point_states(Pf, h, q.f[k], q.f[k + 1]);
            int r = step_with(h, Pf);
            if (r) return r;
        }
        return LBM_OK;
    };

    // The rows of the main backward kernel: the box of rows holding band nodes, which waits for the
    // IB chain of each backward step (band forces, samples, band gather), and up to four boxes of
    // rows around it, which run beside that chain on a stream of the highest priority.
    RowBox band_box{0, h->ny, 0, h->nz}, free_box[4];
    int nfree = 0;
    // With no band node on an x face the x-face kernel needs no IB term either: it runs on a third
    // stream of the highest priority beside both (xs), its blocks placed first as SMs free up.
    struct FreeStream {
        cudaStream_t s = nullptr, xs = nullptr;
        cudaEvent_t fork = nullptr, joined = nullptr, xjoined = nullptr;
        ~FreeStream() {
            for (cudaStream_t q : {s, xs})
                if (q) cudaStreamSynchronize(q);
            for (cudaEvent_t e : {fork, joined, xjoined})
                if (e) cudaEventDestroy(e);
            for (cudaStream_t q : {s, xs})
                if (q) cudaStreamDestroy(q);
        }
    } bfree;
    if (S > 0 && h->band_y1 >= h->band_y0) {
        nfree = band_row_boxes(h->ny, h->nz, h->band_y0, h->band_y1, h->band_z0, h->band_z1, band_box, free_box);
        if (nfree > 0) {
            int lo = 0, hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(cudaStreamCreateWithPriority(&bfree.s, cudaStreamNonBlocking, hi));
            CK(cudaEventCreateWithFlags(&bfree.fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&bfree.joined, cudaEventDisableTiming));
            if (h->band_x0 > 0 && h->band_x1 < h->nx - 1) {
                CK(cudaStreamCreateWithPriority(&bfree.xs, cudaStreamNonBlocking, hi));
                CK(cudaEventCreateWithFlags(&bfree.xjoined, cudaEventDisableTiming));
            }
        }
    }
    const RowBox no_rows{0, 0, 0, 0};

    // backward pass over the segments, last first; segment sgi uses set (nck - 1 - sgi) % nset
    float *lam_cur = lamA, *lam_prev = lamB;
    const float drag_w = (float)(-loss->w_drag / n);
    cudaStream_t bs = st;   // stream of the backward pass
    if (nset >= 2) {
        for (int k = 1; k < nset; ++k) CK(cudaEventRecord(side.free_[k], st));   // checkpoints written
        CK(cudaEventRecord(side.fork, st));
        CK(cudaStreamWaitEvent(side.b, side.fork, 0));
        bs = side.b;
    }
    for (int sgi = nck - 1; sgi >= 0; --sgi) {
        const long long t0 = t_start + (long long)sgi * K;
        const int len = (int)std::min<long long>(K, t_start + n - t0);
        const int cur = (nck - 1 - sgi) % nset;
        const SegSet &q = sets[cur];
        if (nset >= 2) {
            if (sgi < first_kept) CK(cudaStreamWaitEvent(bs, side.done[cur], 0));
            if (sgi >= 1 && sgi - 1 < first_kept) {
                // the set of segment sgi - 1 last held segment sgi + nset - 1, whose backward is done
                const int nxt = (cur + 1) % nset;
                CK(cudaStreamWaitEvent(side.s, side.free_[nxt], 0));
                if ((rc = recompute(sgi - 1, sets[nxt], side.s))) return rc;
                CK(cudaEventRecord(side.done[nxt], side.s));
            }
        } else if (sgi < first_kept) {
            if ((rc = recompute(sgi, q, st))) return rc;
        }
        for (long long t = t0 + len; t > t0; --t) {
            const long long j = t - 1 - t0;
            const bool kept = S > 0 && j + 1 < len;   // the recompute left this step's IB values
            if (kept) point_slot(q, j);
            else ib.restore();
            StepParams P = make_params(h, t);
            point_states(P, h, q.f[j], q.f[j]);
            AdjParams A{};
            A.lam_cur = lam_cur;
            A.lam_prev = lam_prev;
            A.s_inlet = s_inlet;
            A.adj_band = adj_band;
            A.dF_band = dF_band;
            A.wke = (t == t_start + n) ? (float)loss->w_ke : 0.0f;
            A.ke_x0 = loss->ke_x0;
            A.ke_x1 = loss->ke_x1;
            A.ghost_in = ghost + (size_t)((t + 1) & 1) * 9 * nyz;
            A.ghost_out = ghost + (size_t)(t & 1) * 9 * nyz;
            const bool nbp = (t & 1) != 0;
            if (nfree > 0) {
                // rows without band nodes: their backward step needs no IB term, so it starts at once
                CK(cudaEventRecord(bfree.fork, bs));
                if (bfree.xs) {
                    CK(cudaStreamWaitEvent(bfree.xs, bfree.fork, 0));
                    CK(with_storage(h->storage, [&](auto tag) {
                        using St = decltype(tag);
                        return launch_adj_step<St>(P, A, nbp, false, no_rows, true, bfree.xs);
                    }));
                    CK(cudaEventRecord(bfree.xjoined, bfree.xs));
                }
                CK(cudaStreamWaitEvent(bfree.s, bfree.fork, 0));
                for (int r = 0; r < nfree; ++r)
                    CK(with_storage(h->storage, [&](auto tag) {
                        using St = decltype(tag);
                        return launch_adj_step<St>(P, A, nbp, false, free_box[r], false, bfree.s);
                    }));
            }
            if (S > 0) {
                if (!kept) {
                    // the forward step's IB values, recomputed by the same kernels
                    const int r = ib_stage(h, P, bs, cellS_b);
                    if (r) return r;
                }
                CK(with_storage(h->storage, [&](auto tag) {
                    using St = decltype(tag);
                    if (nbp) k_adj_band_force<St, true><<<nblocks(nb, 128), 128, 0, bs>>>(P, A, h->band_cell);
                    else k_adj_band_force<St, false><<<nblocks(nb, 128), 128, 0, bs>>>(P, A, h->band_cell);
                    return cudaGetLastError();
                }));
                k_adj_samples<<<nblocks(S, 256), 256, 0, bs>>>(S, nb, h->X, h->area, h->ub, h->corner_band, h->band_rho,
                                                               h->band_u, h->g, dF_band, drag_w, adj_samp, dX);
                k_adj_band_gather<<<nblocks(nb, 256), 256, 0, bs>>>(S, nb, h->X, h->base_nbr, h->cstart, h->ccount,
                                                                    adj_samp, h->band_rho, h->band_u, adj_band);
                CK(cudaGetLastError());
            }
            if (nfree > 0) {
                // the band's rows read the IB chain's terms; the other rows run beside it (launched
                // above on the band-free streams, which join before the next step reads lambda)
                CK(with_storage(h->storage, [&](auto tag) {
                    using St = decltype(tag);
                    return launch_adj_step<St>(P, A, nbp, true, band_box, !bfree.xs, bs);
                }));
                CK(cudaEventRecord(bfree.joined, bfree.s));
                CK(cudaStreamWaitEvent(bs, bfree.joined, 0));
                if (bfree.xs) CK(cudaStreamWaitEvent(bs, bfree.xjoined, 0));
            } else {
                CK(with_storage(h->storage, [&](auto tag) {
                    using St = decltype(tag);
                    return launch_adj_step<St>(P, A, nbp, S > 0, RowBox{0, h->ny, 0, h->nz}, true, bs);
                }));
            }
            std::swap(lam_cur, lam_prev);
        }
        if (nset >= 2) CK(cudaEventRecord(side.free_[cur], bs));
    }
    if (nset >= 2) {
        CK(cudaEventRecord(side.join, bs));
        CK(cudaStreamWaitEvent(st, side.join, 0));
    }
    ib.restore();
    // the forward pass left the state at t_start + n; restore its IB diagnostics
    if (S > 0) {
        CK(cudaMemcpyAsync(h->g, g_last, 3 * S * sizeof(float), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(h->bandF, F_last, 3 * nb * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    h->t = t_start + n;

    double hacc[8];
    std::vector<double> sin_(nyz);
    CK(cudaMemcpyAsync(hacc, acc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(sin_.data(), s_inlet, nyz * sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> dxs(S > 0 ? 3 * S : 0);
    if (S > 0) CK(cudaMemcpyAsync(dxs.data(), dX, 3 * S * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (L) *L = loss->w_drag * (-hacc[0]) / n + loss->w_ke * hacc[3];
    if (dL_dinflow) {
        // dL/da_mq = sum_z sin(q pi (z + 1/2) / nz) sum_y sin(m pi (y + 1/2) / ny) s(y, z)
        std::vector<double> sy(4 * (size_t)h->ny), sz(4 * (size_t)h->nz), row(4 * (size_t)h->nz, 0.0);
        for (int m = 1; m <= 4; ++m) {
            for (int y = 0; y < h->ny; ++y) sy[(m - 1) * (size_t)h->ny + y] = std::sin(m * M_PI * (y + 0.5) / h->ny);
            for (int z = 0; z < h->nz; ++z) sz[(m - 1) * (size_t)h->nz + z] = std::sin(m * M_PI * (z + 0.5) / h->nz);
        }
        for (int m = 0; m < 4; ++m)
            for (int z = 0; z < h->nz; ++z) {
                double v = 0.0;
                for (int y = 0; y < h->ny; ++y) v += sin_[y + (size_t)h->ny * z] * sy[m * (size_t)h->ny + y];
                row[m * (size_t)h->nz + z] = v;
            }
        for (int m = 0; m < 4; ++m)
            for (int q = 0; q < 4; ++q) {
                double v = 0.0;
                for (int z = 0; z < h->nz; ++z) v += row[m * (size_t)h->nz + z] * sz[q * (size_t)h->nz + z];
                dL_dinflow[m * 4 + q] = h->cfg.face_type[0] == LBM_FACE_INLET ? v : 0.0;
            }
    }
    if (dL_dpos && S > 0) {
        for (long long i = 0; i < S; ++i)
            for (int a = 0; a < 3; ++a) dL_dpos[3 * h->order[i] + a] = dxs[a * S + i];
    }
    return LBM_OK;
}
