// Device-side building blocks of the fused D3Q27 step: lattice tables, population
// storage types, the AA-pattern addressing with the domain faces, and the
// central-moment MRT collision with Guo forcing computed in registers.
//
// Direction order (this library's own): d = (cx+1) + 3 (cy+1) + 9 (cz+1), so the 27
// populations of a node form a 3x3x3 tensor and the central-moment transform of Eq. 5
// factorises into three sweeps of nine 3-point transforms.  opp(d) = 26 - d.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

__host__ __device__ constexpr int cx(int d) { return d % 3 - 1; }
__host__ __device__ constexpr int cy(int d) { return (d / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int d) { return d / 9 - 1; }
__host__ __device__ constexpr int opp(int d) { return 26 - d; }
__host__ __device__ constexpr float w1(int c) { return c == 0 ? 2.0f / 3.0f : 1.0f / 6.0f; }
// lattice weight of direction d (8/27, 2/27, 1/54, 1/216)
__host__ __device__ constexpr float wgt(int d) { return w1(cx(d)) * w1(cy(d)) * w1(cz(d)); }
// index of central moment kappa_pqr in the in-place moment tensor
__host__ __device__ constexpr int K(int p, int q, int r) { return p + 3 * q + 9 * r; }

enum FaceType { FACE_PERIODIC = 0, FACE_NOSLIP = 1, FACE_INLET = 2, FACE_OUTLET = 3, FACE_FREESLIP = 4 };
// bits of a crossing classification
enum { CROSS_NOSLIP = 1, CROSS_INLET = 2, CROSS_OUTLET = 4, CROSS_FREESLIP = 8 };

__host__ __device__ constexpr int face_bit(int t) {
    return t == FACE_NOSLIP ? CROSS_NOSLIP : t == FACE_INLET ? CROSS_INLET : t == FACE_OUTLET ? CROSS_OUTLET
         : t == FACE_FREESLIP ? CROSS_FREESLIP : 0;
}

// direction d with its y (bit 0 of mir) and / or z (bit 1) component reversed: the specular
// image at a free-slip face
__host__ __device__ constexpr int mirror_dir(int d, int mir) {
    return d + ((mir & 1) ? -6 * cy(d) : 0) + ((mir & 2) ? -18 * cz(d) : 0);
}

// ---- population storage: deviations h_i = f_i - w_i rho0 ---------------------------

template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// ---- launch parameters -----------------------------------------------------------------

struct Geometry {
    int nx, ny, nz;
    int nxy;             // nx * ny
    int ncell;           // nx * ny * nz
    int nyz;             // ny * nz (outlet plane)
    long long plane;     // elements between consecutive direction planes (>= ncell)
    int periodic[3];
    int face[6];         // FaceType of -x, +x, -y, +y, -z, +z
};

struct StepParams {
    void *f;                     // populations, 27 planes (AA in place)
    void *fp[27];                // start of the plane of each direction (read)
    void *fpo[27];               // planes written by the step (= fp in place; another state out of place)
    void *outlet;                // outlet ghost plane, [2][9][nyz] (ping-pong by step parity), read
    void *outlet_o;              // outlet ghost plane written by the step
    Geometry g;
    float rho0;
    float Fx, Fy, Fz;            // body force
    float rs, rb, r3, r4, r5, r6;   // 1 - omega of shear, bulk, orders 3..6
    float q3, q5;                // 1 - omega/2 of orders 3 and 5 (their force moments)
    float u_in, noise;           // inlet velocity and relative noise amplitude
    // relaxation coefficients of the central-moment collision in the form
    // sigma (rr h + (1 - rr) e + force), sigma = 2^-(number of nonzero indices): see collide_v
    float a2, b2;                // shear off-diagonal: sigma 1/4, e = -rho0 u_a u_b
    float tb6, ts6, r0h;         // trace / deviators: rb / 6, rs / 6; rho0 / 2
    float a3, b3, f3;            // order 3 with force: sigma 1/4, e = rho0 u t; force q3 / 3
    float a3e, b3e;              // kappa_111: sigma 1/8
    float a4, b4r, b4u;          // kappa_220-type: sigma 1/4, e = rhop / 9 - rho0 / 3 (3 u2 v2 + u2 + v2)
    float a4m, b4m;              // kappa_211-type: sigma 1/8, e = -rho0 t_a u_b u_c
    float a5, b5, f5;            // order 5: sigma 1/8, e = rho0 u_c t_a t_b; force q5 / 9
    float a6, b6r, b6u;          // kappa_222: sigma 1/8, e = rhop / 27 - rho0 (s1 / 9 + s2 / 3 + s3)
    unsigned long long seed;
    long long t;                 // index of the step being computed (1-based)
    const float *inlet_profile;  // [nyz] Fourier part of the inflow, or nullptr
    const uint32_t *tile_mask;   // bit l of word w: cell 32 w + l is a band node
    const int *tile_off;         // band index of the first band node of word w
    const float *bandF;          // [3][nband] immersed-boundary force of the band nodes
    long long nband;             // band nodes, or the stride of the band arrays when band_count is set
    const int *band_count;       // device count of band nodes (moving solids), or nullptr
    float *u_out;                // [3][ncell] Guo-shifted velocity of the step, or nullptr
    int inner_rows;              // 1: the step kernels skip the rows on a y/z face (run by the
                                 // free-slip kernels of the same step)
};

// ---- inlet noise: counter-based SplitMix64 (Steele, Lea, Flood 2014) ------------------

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long n) {
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// inlet wall velocity u_in (1 + noise xi) + profile at inlet node (y, z) and step t
__device__ __forceinline__ float inlet_velocity(const StepParams &P, int y, int z) {
    double u = P.u_in;
    if (P.noise != 0.0f) {
        unsigned long long n = ((unsigned long long)P.t * P.g.ny + y) * P.g.nz + z;
        double xi = 2.0 * ((double)(splitmix64(P.seed, n) >> 11) * 0x1.0p-53) - 1.0;
        u = (double)P.u_in * (1.0 + (double)P.noise * xi);
    }
    float uw = (float)u;
    if (P.inlet_profile) uw += P.inlet_profile[y + P.g.ny * z];
    return uw;
}

// ---- neighbour classification with the domain faces ----------------------------------

struct Nbr {
    int idx;    // flat index of the (wrapped) node, valid when kind == 0 or for lateral wraps;
                // across a free-slip face the coordinate of that axis is the node's own
    int y, z;   // wrapped (or free-slip mirrored) lateral coordinates
    int kind;   // CROSS_* bits of the non-periodic faces crossed
    int mir;    // free-slip axes crossed: bit 0 y, bit 1 z
};

// node x + S c_D (S = -1: pull source, S = +1: push target); D is a constant after unrolling
template <int S>
__device__ __forceinline__ Nbr neighbour(const Geometry &g, int D, int x, int y, int z) {
    int sx = x + S * cx(D), sy = y + S * cy(D), sz = z + S * cz(D);
    int kind = 0;
    if (cx(D) != 0) {
        if (sx < 0) { if (g.periodic[0]) sx += g.nx; else kind |= face_bit(g.face[0]); }
        else if (sx >= g.nx) { if (g.periodic[0]) sx -= g.nx; else kind |= face_bit(g.face[1]); }
    }
    int mir = 0;
    if (cy(D) != 0) {
        const int fy = sy < 0 ? g.face[2] : g.face[3];
        if (sy < 0 || sy >= g.ny) {
            if (g.periodic[1]) sy += sy < 0 ? g.ny : -g.ny;
            else { kind |= face_bit(fy); if (fy == FACE_FREESLIP) { mir |= 1; sy = y; } }
        }
    }
    if (cz(D) != 0) {
        const int fz = sz < 0 ? g.face[4] : g.face[5];
        if (sz < 0 || sz >= g.nz) {
            if (g.periodic[2]) sz += sz < 0 ? g.nz : -g.nz;
            else { kind |= face_bit(fz); if (fz == FACE_FREESLIP) { mir |= 2; sz = z; } }
        }
    }
    Nbr n;
    n.idx = sx + g.nx * (sy + g.ny * sz);
    n.y = sy;
    n.z = sz;
    n.kind = kind;
    n.mir = mir;
    return n;
}

// ---- scalar helpers of the templated arithmetic ---------------------------------------
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
template <typename V> __device__ __forceinline__ V vconst(float s) { return V(s); }

// ---- the 3-point transforms of the factorised central-moment basis -------------------
// A triplet holds (v(c=-1), v(c=0), v(c=+1)) of one axis; after a forward transform the
// same slots hold the moments of order 0, 1, 2 along that axis.

// populations -> raw moments (sum v, sum c v, sum c^2 v)
template <typename V> __device__ __forceinline__ void raw3(V &a, V &b, V &c) {
    const V s = a + c, d = c - a;
    a = s + b;
    b = d;
    c = s;
}
// raw -> central moments about u
template <typename V> __device__ __forceinline__ void shift3(V &m0, V &m1, V &m2, V u) {
    const V u2 = u * u, m2u = -2.0f * u;   // shared by the nine triplets of a sweep
    m2 = vfma(u2, m0, vfma(m2u, m1, m2));
    m1 = vfma(-u, m0, m1);
}
// central moments about u -> populations, with the order-1 and order-2 moments given halved
// (k0, k1 / 2, k2 / 2); hu = u / 2, tu = 2 u, u2h = u^2 / 2
__device__ __forceinline__ void inv3h(float &m0, float &m1, float &m2, float hu, float tu, float u2h) {
    const float r1h = fmaf(hu, m0, m1);                 // (k1 + u k0) / 2
    const float R2 = fmaf(u2h, m0, fmaf(tu, m1, m2));   // (k2 + 2 u k1 + u^2 k0) / 2
    const float k0 = m0;
    m0 = R2 - r1h;
    m2 = R2 + r1h;
    m1 = fmaf(-2.0f, R2, k0);
}

// base index of the k-th triplet along the axis with stride S (1: x, 3: y, 9: z)
template <int S> __host__ __device__ constexpr int tri_base(int k) {
    return S == 1 ? 3 * k : S == 3 ? (k % 3) + 9 * (k / 3) : k;
}

template <int S, typename V> __device__ __forceinline__ void sweep_raw(V (&h)[27]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) raw3(h[tri_base<S>(k)], h[tri_base<S>(k) + S], h[tri_base<S>(k) + 2 * S]);
}
template <int S, typename V> __device__ __forceinline__ void sweep_shift(V (&h)[27], V u) {
#pragma unroll
    for (int k = 0; k < 9; ++k) shift3(h[tri_base<S>(k)], h[tri_base<S>(k) + S], h[tri_base<S>(k) + 2 * S], u);
}
template <int S> __device__ __forceinline__ void sweep_invh(float (&h)[27], float u, float u2) {
    const float hu = 0.5f * u, tu = u + u, u2h = 0.5f * u2;
#pragma unroll
    for (int k = 0; k < 9; ++k) inv3h(h[tri_base<S>(k)], h[tri_base<S>(k) + S], h[tri_base<S>(k) + 2 * S], hu, tu, u2h);
}

// ---- collision (Eqs. 4-5) ---------------------------------------------------------------
// In: h = streamed deviations f*_i - w_i rho0 (tensor order), F = total force.
// Out: h = post-collision deviations; rho, u = density and Guo-shifted velocity.
//
// With kappa the central moments of f about u, kappa_eq = rho m_p m_q m_r (m = 1, 0, 1/3)
// and R^F the force moments, every moment is relaxed as
//     kappa' = kappa - omega (kappa - kappa_eq) + (1 - omega/2) R^F,
// the diagonal second-order moments through their trace (omega_b) and two deviators
// (omega_s).  The transform acts on the deviations h; the rest-weight part w rho0 has the
// central moments rho0 t_p(u_x) t_q(u_y) t_r(u_z), t = (1, -u, 1/3 + u^2), so with
// e = kappa_eq - rho0 t t t the update reads h' = rr h + (1 - rr) e + (1 - omega/2) R^F in
// moment space (rr = 1 - omega), every term small; the e are expanded to avoid cancellation.
// Each relaxed moment is stored multiplied by sigma = 2^-(number of nonzero indices), which the
// inverse sweeps (inv3h) expect; the products of sigma with the rates come precomputed in the
// launch parameters (make_params), so they cost no instructions here.
template <typename V>
__device__ __forceinline__ void collide_v(V (&h)[27], V Fx, V Fy, V Fz, const StepParams &P, V &rho, V &ux, V &uy,
                                          V &uz) {
    sweep_raw<1>(h);
    sweep_raw<3>(h);
    sweep_raw<9>(h);
    const V rhop = h[K(0, 0, 0)];            // rho - rho0
    rho = P.rho0 + rhop;
    const V inv = vrcp(rho);
    ux = vfma(0.5f, Fx, h[K(1, 0, 0)]) * inv;
    uy = vfma(0.5f, Fy, h[K(0, 1, 0)]) * inv;
    uz = vfma(0.5f, Fz, h[K(0, 0, 1)]) * inv;
    sweep_shift<1>(h, ux);
    sweep_shift<3>(h, uy);
    sweep_shift<9>(h, uz);

    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const float third = 1.0f / 3.0f;
    const V tx = third + ux2, ty = third + uy2, tz = third + uz2;
    const V uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;

    // order 1: conserved, kappa'_100 = F_x / 2 (stored as deviation moment rho0 u_x + F_x/2), times 1/2
    h[K(1, 0, 0)] = vfma(P.r0h, ux, 0.25f * Fx);
    h[K(0, 1, 0)] = vfma(P.r0h, uy, 0.25f * Fy);
    h[K(0, 0, 1)] = vfma(P.r0h, uz, 0.25f * Fz);

    // sigma (rr h + (1 - rr) e + f) with A = sigma rr and B e_term = sigma (1 - rr) e
#define RELAX(idx, A, Be) h[idx] = vfma(vconst<V>(A), h[idx], (Be))
    // order 2, off-diagonal (shear)
    RELAX(K(1, 1, 0), P.a2, P.b2 * uxy);
    RELAX(K(1, 0, 1), P.a2, P.b2 * uxz);
    RELAX(K(0, 1, 1), P.a2, P.b2 * uyz);
    // order 2, diagonal: trace (bulk) and two deviators (shear), times 1/2
    {
        const V a = vfma(P.rho0, ux2, vfma(-third, rhop, h[K(2, 0, 0)]));   // kappa - e, e = rhop/3 - rho0 u^2
        const V b = vfma(P.rho0, uy2, vfma(-third, rhop, h[K(0, 2, 0)]));
        const V c = vfma(P.rho0, uz2, vfma(-third, rhop, h[K(0, 0, 2)]));
        const V sixth_rhop = (0.5f * third) * rhop;
        const V T = P.tb6 * (a + b + c);
        const V D1 = P.ts6 * (a - b);
        const V D2 = P.ts6 * (a - c);
        const V TD1 = T + D1;
        h[K(2, 0, 0)] = (TD1 + D2) + vfma(-P.r0h, ux2, sixth_rhop);
        h[K(0, 2, 0)] = vfma(-2.0f, D1, T + D2) + vfma(-P.r0h, uy2, sixth_rhop);
        h[K(0, 0, 2)] = vfma(-2.0f, D2, TD1) + vfma(-P.r0h, uz2, sixth_rhop);
    }
    // order 3 (force moments F/3 on 210, 201, 120, 021, 102, 012)
    const V gx3 = P.f3 * Fx, gy3 = P.f3 * Fy, gz3 = P.f3 * Fz;
    RELAX(K(2, 1, 0), P.a3, vfma(P.b3, uy * tx, gy3));
    RELAX(K(2, 0, 1), P.a3, vfma(P.b3, uz * tx, gz3));
    RELAX(K(1, 2, 0), P.a3, vfma(P.b3, ux * ty, gx3));
    RELAX(K(0, 2, 1), P.a3, vfma(P.b3, uz * ty, gz3));
    RELAX(K(1, 0, 2), P.a3, vfma(P.b3, ux * tz, gx3));
    RELAX(K(0, 1, 2), P.a3, vfma(P.b3, uy * tz, gy3));
    RELAX(K(1, 1, 1), P.a3e, P.b3e * (uxy * uz));
    // order 4
    {
        const V x3 = 3.0f * ux2, y3 = 3.0f * uy2;
        const V r4 = P.b4r * rhop;
        RELAX(K(2, 2, 0), P.a4, vfma(P.b4u, vfma(x3, uy2, ux2 + uy2), r4));
        RELAX(K(2, 0, 2), P.a4, vfma(P.b4u, vfma(x3, uz2, ux2 + uz2), r4));
        RELAX(K(0, 2, 2), P.a4, vfma(P.b4u, vfma(y3, uz2, uy2 + uz2), r4));
    }
    RELAX(K(2, 1, 1), P.a4m, P.b4m * (tx * uyz));
    RELAX(K(1, 2, 1), P.a4m, P.b4m * (ty * uxz));
    RELAX(K(1, 1, 2), P.a4m, P.b4m * (tz * uxy));
    // order 5 (force moments F/9 on 221, 212, 122)
    RELAX(K(2, 2, 1), P.a5, vfma(P.b5, uz * (tx * ty), P.f5 * Fz));
    RELAX(K(2, 1, 2), P.a5, vfma(P.b5, uy * (tx * tz), P.f5 * Fy));
    RELAX(K(1, 2, 2), P.a5, vfma(P.b5, ux * (ty * tz), P.f5 * Fx));
    // order 6
    {
        const V s1 = ux2 + uy2 + uz2;
        const V s2 = vfma(ux2, uy2 + uz2, uy2 * uz2);
        const V s3 = ux2 * uy2 * uz2;
        RELAX(K(2, 2, 2), P.a6, vfma(P.b6u, vfma(1.0f / 9.0f, s1, vfma(third, s2, s3)), P.b6r * rhop));
    }
#undef RELAX
    sweep_invh<9>(h, uz, uz2);
    sweep_invh<3>(h, uy, uy2);
    sweep_invh<1>(h, ux, ux2);
}

__device__ __forceinline__ void collide(float (&h)[27], float Fx, float Fy, float Fz, const StepParams &P,
                                        float &rho, float &ux, float &uy, float &uz) {
    collide_v<float>(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
}

}  // namespace lbm
