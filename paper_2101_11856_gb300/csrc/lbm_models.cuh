// Collision models of the fused step: ACM-MRT (central moments, the method) and the two
// comparison models of the paper's Sec. 6.1 results, D3Q27 BGK and raw-moment MRT, under
// the same streaming, forcing (Guo) and faces.  All three act on the deviations
// h = f - w rho0 in registers and return the density and Guo-shifted velocity.
#pragma once

#include "lbm_internal.h"

namespace lbm {

// per-axis factors of the product forms at velocity u, indexed by c + 1:
// w = rest weights, dp = phi - w (phi: 1-D equilibrium, central moments 1, 0, 1/3),
// p = phi, g = 1-D force factor (central moments 0, 1, 0)
struct AxisFactors {
    float dp[3], p[3], g[3];
    __device__ __forceinline__ explicit AxisFactors(float u) {
        const float u2 = u * u;
        dp[0] = 0.5f * (u2 - u); dp[1] = -u2; dp[2] = 0.5f * (u2 + u);
        p[0] = w1(-1) + dp[0]; p[1] = w1(0) + dp[1]; p[2] = w1(1) + dp[2];
        g[0] = u - 0.5f; g[1] = -2.0f * u; g[2] = u + 0.5f;
    }
};

// BGK: h' = h - omega (h - h_eq) + (1 - omega/2) G with omega the shear rate, the product
// equilibrium f_eq = rho prod phi and the force distribution G = sum_a F_a g_a prod_{b != a} phi_b
__device__ __forceinline__ void collide_bgk(float (&h)[27], float Fx, float Fy, float Fz, const StepParams &P,
                                            float &rho, float &ux, float &uy, float &uz) {
    float rp = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        rp += h[d];
        if (cx(d)) jx += cx(d) * h[d];
        if (cy(d)) jy += cy(d) * h[d];
        if (cz(d)) jz += cz(d) * h[d];
    }
    rho = P.rho0 + rp;
    const float inv = __frcp_rn(rho);
    ux = fmaf(0.5f, Fx, jx) * inv;
    uy = fmaf(0.5f, Fy, jy) * inv;
    uz = fmaf(0.5f, Fz, jz) * inv;
    const AxisFactors ax(ux), ay(uy), az(uz);
    const float om = 1.0f - P.rs, q = 0.5f * (1.0f + P.rs);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
        const int a = cx(d) + 1, b = cy(d) + 1, c = cz(d) + 1;
        const float wx = w1(a - 1), wy = w1(b - 1), wz = w1(c - 1);
        const float pyz = ay.p[b] * az.p[c];
        // prod phi - prod w, telescoped so that no O(1) terms cancel
        const float dprod = ax.dp[a] * pyz + wx * (ay.dp[b] * az.p[c] + wy * az.dp[c]);
        const float heq = fmaf(rp, wgt(d), rho * dprod);
        const float G = Fx * ax.g[a] * pyz + ax.p[a] * (Fy * ay.g[b] * az.p[c] + Fz * ay.p[b] * az.g[c]);
        h[d] = fmaf(q, G, fmaf(-om, h[d] - heq, h[d]));
    }
}

// inverse of raw3: raw moments (sum v, sum c v, sum c^2 v) -> populations
__device__ __forceinline__ void rawinv3(float &a, float &b, float &c) {
    const float r0 = a, r1 = b, r2 = c;
    a = 0.5f * (r2 - r1);
    b = r0 - r2;
    c = 0.5f * (r2 + r1);
}

// Raw-moment MRT: Eq. 5 with the u-independent raw moments c_x^p c_y^q c_z^r, the same rate
// groups as ACM-MRT (trace / deviators at second order), equilibrium moments rho prod e_p
// (e = 1, u, 1/3 + u^2) and force moments sum_a F_a gr_p(a) prod e (gr = 0, 1, 2u).
__device__ __forceinline__ void collide_raw(float (&h)[27], float Fx, float Fy, float Fz, const StepParams &P,
                                            float &rho, float &ux, float &uy, float &uz) {
    sweep_raw<1>(h);
    sweep_raw<3>(h);
    sweep_raw<9>(h);
    const float rp = h[K(0, 0, 0)];
    rho = P.rho0 + rp;
    const float inv = __frcp_rn(rho);
    ux = fmaf(0.5f, Fx, h[K(1, 0, 0)]) * inv;
    uy = fmaf(0.5f, Fy, h[K(0, 1, 0)]) * inv;
    uz = fmaf(0.5f, Fz, h[K(0, 0, 1)]) * inv;
    const float third = 1.0f / 3.0f;
    const float ex[3] = {1.0f, ux, fmaf(ux, ux, third)}, ey[3] = {1.0f, uy, fmaf(uy, uy, third)},
                ez[3] = {1.0f, uz, fmaf(uz, uz, third)};
    const float dx[3] = {0.0f, ux, ux * ux}, dy[3] = {0.0f, uy, uy * uy}, dz[3] = {0.0f, uz, uz * uz};
    const float gx[3] = {0.0f, 1.0f, 2.0f * ux}, gy[3] = {0.0f, 1.0f, 2.0f * uy}, gz[3] = {0.0f, 1.0f, 2.0f * uz};
    const float m[3] = {1.0f, 0.0f, third};
    const float r0 = P.rho0;
    float e[27], rg[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) {
        const int p = k % 3, q = (k / 3) % 3, r = k / 9;
        // rho prod e - rho0 prod m, telescoped
        const float dE = dx[p] * ey[q] * ez[r] + m[p] * (dy[q] * ez[r] + m[q] * dz[r]);
        e[k] = fmaf(rp, ex[p] * ey[q] * ez[r], r0 * dE);
        rg[k] = Fx * gx[p] * ey[q] * ez[r] + ex[p] * (Fy * gy[q] * ez[r] + Fz * ey[q] * gz[r]);
    }
    const float rate_r[7] = {0.0f, 0.0f, P.rs, P.r3, P.r4, P.r5, P.r6};   // 1 - omega by order
#pragma unroll
    for (int k = 0; k < 27; ++k) {
        const int p = k % 3, q = (k / 3) % 3, r = k / 9, o = p + q + r;
        if (o == 0) continue;
        if (o == 1) {
            h[k] += rg[k];          // conserved: kappa' = kappa + F
            continue;
        }
        if (o == 2 && (p == 2 || q == 2 || r == 2)) continue;   // diagonal: below
        const float rr = rate_r[o], qq = 0.5f * (1.0f + rr);
        h[k] = fmaf(qq, rg[k], fmaf(rr, h[k] - e[k], e[k]));
    }
    {
        const int i200 = K(2, 0, 0), i020 = K(0, 2, 0), i002 = K(0, 0, 2);
        const float a = h[i200] - e[i200], b = h[i020] - e[i020], c = h[i002] - e[i002];
        const float qb = 0.5f * (1.0f + P.rb), qs = 0.5f * (1.0f + P.rs);
        const float tr = P.rb * (a + b + c) + qb * (rg[i200] + rg[i020] + rg[i002]);
        const float d1 = P.rs * (a - b) + qs * (rg[i200] - rg[i020]);
        const float d2 = P.rs * (a - c) + qs * (rg[i200] - rg[i002]);
        h[i200] = e[i200] + third * (tr + d1 + d2);
        h[i020] = e[i020] + third * (tr - 2.0f * d1 + d2);
        h[i002] = e[i002] + third * (tr + d1 - 2.0f * d2);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) rawinv3(h[tri_base<9>(k)], h[tri_base<9>(k) + 9], h[tri_base<9>(k) + 18]);
#pragma unroll
    for (int k = 0; k < 9; ++k) rawinv3(h[tri_base<3>(k)], h[tri_base<3>(k) + 3], h[tri_base<3>(k) + 6]);
#pragma unroll
    for (int k = 0; k < 9; ++k) rawinv3(h[tri_base<1>(k)], h[tri_base<1>(k) + 1], h[tri_base<1>(k) + 2]);
}

template <int COLL>
__device__ __forceinline__ void collide_model(float (&h)[27], float Fx, float Fy, float Fz, const StepParams &P,
                                              float &rho, float &ux, float &uy, float &uz) {
    if (COLL == COLL_BGK) collide_bgk(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
    else if (COLL == COLL_RAW) collide_raw(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
    else collide(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
}

}  // namespace lbm
