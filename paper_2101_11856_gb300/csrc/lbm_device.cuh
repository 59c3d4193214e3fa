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

// Coefficients of the central-moment collision (collide_v), for one node (S = float) or for a
// node pair in the packed FP32 instructions (S = float2, the same value in both halves).  The
// relaxation products sigma rr and sigma (1 - rr) e of every moment group are precomputed on the
// host (make_params) with sigma = 2^-(number of nonzero indices); the remaining members are the
// fixed constants of the transform, held here so that a node pair reads them as operand pairs.
template <typename S> struct CollCoef {
    S rho0, r0h, mr0h;           // rho0, rho0 / 2, -rho0 / 2
    S a2, b2;                    // shear off-diagonal: sigma 1/4, e = -rho0 u_a u_b
    S tb6, ts6;                  // trace / deviators: rb / 6, rs / 6
    S a3, b3, f3;                // order 3 with force: sigma 1/4, e = rho0 u t; force q3 / 3
    S a3e, b3e;                  // kappa_111: sigma 1/8
    S a4, b4r, b4u;              // kappa_220-type: sigma 1/4, e = rhop / 9 - rho0 / 3 (3 u2 v2 + u2 + v2)
    S a4m, b4m;                  // kappa_211-type: sigma 1/8, e = -rho0 t_a u_b u_c
    S a5, b5, f5;                // order 5: sigma 1/8, e = rho0 u_c t_a t_b; force q5 / 9
    S a6, b6r, b6u;              // kappa_222: sigma 1/8, e = rhop / 27 - rho0 (s1 / 9 + s2 / 3 + s3)
    S half, quarter, third, mthird, sixth, ninth, three, mtwo, mone;
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
    CollCoef<float> cc;          // the collision's coefficients (one node)
    CollCoef<float2> cc2;        // the same, for node pairs (packed FP32)
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
    int pair_bulk;               // 16-bit storage, node pairs: 1 = the tensor-copy fed main kernel
                                 // (k_step_pair_tma, nx % 8 == 0), 0 = k_step_pair, 2 = the former's
                                 // wait-limit self-test
    int *err;                    // device flag set by a kernel whose bounded wait ran out
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

// ---- arithmetic of the templated collision: one node (float) or a node pair (F2) --------
// F2 holds the values of two nodes and maps every operation to the packed FP32 instructions of
// sm_100+ (one f32x2 add / multiply / fma for both nodes): each half is the IEEE FP32 result
// with round-to-nearest, so a node pair computes bit for bit what two single nodes compute.
struct F2 {
    float2 v;
};
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b), rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2 *>(&rd);
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {f2sub(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator+(float2 a, F2 b) { return {__fadd2_rn(a, b.v)}; }
__device__ __forceinline__ F2 operator*(float2 a, F2 b) { return {__fmul2_rn(a, b.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 vfma(float2 a, F2 b, F2 c) { return {__ffma2_rn(a, b.v, c.v)}; }
__device__ __forceinline__ F2 vrcp(F2 a) { return {make_float2(__frcp_rn(a.v.x), __frcp_rn(a.v.y))}; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
// a coefficient as an operand of V's arithmetic (float for one node, float2 for a pair)
template <typename V> struct CoefOf { using T = float; };
template <> struct CoefOf<F2> { using T = float2; };
template <typename V> __device__ __forceinline__ const CollCoef<typename CoefOf<V>::T> &coefs(const StepParams &P);
template <> __device__ __forceinline__ const CollCoef<float> &coefs<float>(const StepParams &P) { return P.cc; }
template <> __device__ __forceinline__ const CollCoef<float2> &coefs<F2>(const StepParams &P) { return P.cc2; }

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
// raw -> central moments about u; u2 = u^2, m2u = -2 u, mu = -u (shared by the nine triplets
// of a sweep)
template <typename V> __device__ __forceinline__ void shift3(V &m0, V &m1, V &m2, V u2, V m2u, V mu) {
    m2 = vfma(u2, m0, vfma(m2u, m1, m2));
    m1 = vfma(mu, m0, m1);
}
// the same for one triplet, forming u^2, -2 u and -u itself (the adjoint's recompute)
__device__ __forceinline__ void shift3(float &m0, float &m1, float &m2, float u) {
    shift3(m0, m1, m2, u * u, -2.0f * u, -u);
}
// central moments about u -> populations, with the order-1 and order-2 moments given halved
// (k0, k1 / 2, k2 / 2); hu = u / 2, tu = 2 u, u2h = u^2 / 2, mtwo = -2
template <typename V, typename C>
__device__ __forceinline__ void inv3h(V &m0, V &m1, V &m2, V hu, V tu, V u2h, C mtwo) {
    const V r1h = vfma(hu, m0, m1);                 // (k1 + u k0) / 2
    const V R2 = vfma(u2h, m0, vfma(tu, m1, m2));   // (k2 + 2 u k1 + u^2 k0) / 2
    const V k0 = m0;
    m0 = R2 - r1h;
    m2 = R2 + r1h;
    m1 = vfma(mtwo, R2, k0);
}

// base index of the k-th triplet along the axis with stride S (1: x, 3: y, 9: z)
template <int S> __host__ __device__ constexpr int tri_base(int k) {
    return S == 1 ? 3 * k : S == 3 ? (k % 3) + 9 * (k / 3) : k;
}

template <int S, typename V> __device__ __forceinline__ void sweep_raw(V (&h)[27]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) raw3(h[tri_base<S>(k)], h[tri_base<S>(k) + S], h[tri_base<S>(k) + 2 * S]);
}
template <int S, typename V, typename C> __device__ __forceinline__ void sweep_shift(V (&h)[27], V u, const C &k) {
    const V u2 = u * u, m2u = k.mtwo * u, mu = k.mone * u;
#pragma unroll
    for (int j = 0; j < 9; ++j)
        shift3(h[tri_base<S>(j)], h[tri_base<S>(j) + S], h[tri_base<S>(j) + 2 * S], u2, m2u, mu);
}
template <int S, typename V, typename C> __device__ __forceinline__ void sweep_invh(V (&h)[27], V u, V u2, const C &k) {
    const V hu = k.half * u, tu = u + u, u2h = k.half * u2;
#pragma unroll
    for (int j = 0; j < 9; ++j)
        inv3h(h[tri_base<S>(j)], h[tri_base<S>(j) + S], h[tri_base<S>(j) + 2 * S], hu, tu, u2h, k.mtwo);
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
    const auto &k = coefs<V>(P);
    sweep_raw<1>(h);
    sweep_raw<3>(h);
    sweep_raw<9>(h);
    const V rhop = h[K(0, 0, 0)];            // rho - rho0
    rho = k.rho0 + rhop;
    const V inv = vrcp(rho);
    ux = vfma(k.half, Fx, h[K(1, 0, 0)]) * inv;
    uy = vfma(k.half, Fy, h[K(0, 1, 0)]) * inv;
    uz = vfma(k.half, Fz, h[K(0, 0, 1)]) * inv;
    sweep_shift<1>(h, ux, k);
    sweep_shift<3>(h, uy, k);
    sweep_shift<9>(h, uz, k);

    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V tx = k.third + ux2, ty = k.third + uy2, tz = k.third + uz2;
    const V uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;

    // order 1: conserved, kappa'_100 = F_x / 2 (stored as deviation moment rho0 u_x + F_x/2), times 1/2
    h[K(1, 0, 0)] = vfma(k.r0h, ux, k.quarter * Fx);
    h[K(0, 1, 0)] = vfma(k.r0h, uy, k.quarter * Fy);
    h[K(0, 0, 1)] = vfma(k.r0h, uz, k.quarter * Fz);

    // sigma (rr h + (1 - rr) e + f) with A = sigma rr and B e_term = sigma (1 - rr) e
#define RELAX(idx, A, Be) h[idx] = vfma((A), h[idx], (Be))
    // order 2, off-diagonal (shear)
    RELAX(K(1, 1, 0), k.a2, k.b2 * uxy);
    RELAX(K(1, 0, 1), k.a2, k.b2 * uxz);
    RELAX(K(0, 1, 1), k.a2, k.b2 * uyz);
    // order 2, diagonal: trace (bulk) and two deviators (shear), times 1/2
    {
        const V a = vfma(k.rho0, ux2, vfma(k.mthird, rhop, h[K(2, 0, 0)]));   // kappa - e, e = rhop/3 - rho0 u^2
        const V b = vfma(k.rho0, uy2, vfma(k.mthird, rhop, h[K(0, 2, 0)]));
        const V c = vfma(k.rho0, uz2, vfma(k.mthird, rhop, h[K(0, 0, 2)]));
        const V sixth_rhop = k.sixth * rhop;
        const V T = k.tb6 * (a + b + c);
        const V D1 = k.ts6 * (a - b);
        const V D2 = k.ts6 * (a - c);
        const V TD1 = T + D1;
        h[K(2, 0, 0)] = (TD1 + D2) + vfma(k.mr0h, ux2, sixth_rhop);
        h[K(0, 2, 0)] = vfma(k.mtwo, D1, T + D2) + vfma(k.mr0h, uy2, sixth_rhop);
        h[K(0, 0, 2)] = vfma(k.mtwo, D2, TD1) + vfma(k.mr0h, uz2, sixth_rhop);
    }
    // order 3 (force moments F/3 on 210, 201, 120, 021, 102, 012)
    const V gx3 = k.f3 * Fx, gy3 = k.f3 * Fy, gz3 = k.f3 * Fz;
    RELAX(K(2, 1, 0), k.a3, vfma(k.b3, uy * tx, gy3));
    RELAX(K(2, 0, 1), k.a3, vfma(k.b3, uz * tx, gz3));
    RELAX(K(1, 2, 0), k.a3, vfma(k.b3, ux * ty, gx3));
    RELAX(K(0, 2, 1), k.a3, vfma(k.b3, uz * ty, gz3));
    RELAX(K(1, 0, 2), k.a3, vfma(k.b3, ux * tz, gx3));
    RELAX(K(0, 1, 2), k.a3, vfma(k.b3, uy * tz, gy3));
    RELAX(K(1, 1, 1), k.a3e, k.b3e * (uxy * uz));
    // order 4
    {
        const V x3 = k.three * ux2, y3 = k.three * uy2;
        const V r4 = k.b4r * rhop;
        RELAX(K(2, 2, 0), k.a4, vfma(k.b4u, vfma(x3, uy2, ux2 + uy2), r4));
        RELAX(K(2, 0, 2), k.a4, vfma(k.b4u, vfma(x3, uz2, ux2 + uz2), r4));
        RELAX(K(0, 2, 2), k.a4, vfma(k.b4u, vfma(y3, uz2, uy2 + uz2), r4));
    }
    RELAX(K(2, 1, 1), k.a4m, k.b4m * (tx * uyz));
    RELAX(K(1, 2, 1), k.a4m, k.b4m * (ty * uxz));
    RELAX(K(1, 1, 2), k.a4m, k.b4m * (tz * uxy));
    // order 5 (force moments F/9 on 221, 212, 122)
    RELAX(K(2, 2, 1), k.a5, vfma(k.b5, uz * (tx * ty), k.f5 * Fz));
    RELAX(K(2, 1, 2), k.a5, vfma(k.b5, uy * (tx * tz), k.f5 * Fy));
    RELAX(K(1, 2, 2), k.a5, vfma(k.b5, ux * (ty * tz), k.f5 * Fx));
    // order 6
    {
        const V s1 = ux2 + uy2 + uz2;
        const V s2 = vfma(ux2, uy2 + uz2, uy2 * uz2);
        const V s3 = ux2 * uy2 * uz2;
        RELAX(K(2, 2, 2), k.a6, vfma(k.b6u, vfma(k.ninth, s1, vfma(k.third, s2, s3)), k.b6r * rhop));
    }
#undef RELAX
    sweep_invh<9>(h, uz, uz2, k);
    sweep_invh<3>(h, uy, uy2, k);
    sweep_invh<1>(h, ux, ux2, k);
}

__device__ __forceinline__ void collide(float (&h)[27], float Fx, float Fy, float Fz, const StepParams &P,
                                        float &rho, float &ux, float &uy, float &uz) {
    collide_v<float>(h, Fx, Fy, Fz, P, rho, ux, uy, uz);
}

}  // namespace lbm
