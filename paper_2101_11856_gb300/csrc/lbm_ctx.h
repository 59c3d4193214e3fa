// The solver context shared by the C-ABI translation units (lbm_api.cu, lbm_adjoint.cu)
// and the host helpers they use.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

struct lbm_adjoint_buffers;

struct EventRec {
    int kind;
    cudaEvent_t a, b;
};

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0;
    long long N = 0, plane = 0;
    int storage = 0;
    size_t esize = 4;
    double nu = 0, forcing[3] = {0, 0, 0};
    lbm_config cfg{};
    cudaStream_t stream = nullptr;

    void *f = nullptr;          // 27 * plane elements of the storage type
    void *outlet = nullptr;     // 2 * 9 * ny * nz elements
    float *inlet_profile = nullptr;
    long long t = 0;
    bool has_state = false;

    // immersed solid (samples sorted by base cell)
    long long S = 0, nband = 0, ntiles = 0;
    float *X = nullptr, *area = nullptr, *ub = nullptr, *g = nullptr;
    int *corner_band = nullptr, *band_cell = nullptr, *base_nbr = nullptr, *cstart = nullptr, *ccount = nullptr;
    float *band_rho = nullptr, *band_u = nullptr, *bandF = nullptr;
    bool ub_zero = false;           // every boundary velocity is 0 (the interpolation skips ub)
    // two-phase IB of a static solid: the occupied base cells (band index of each, ascending),
    // the occupied-cell index of the base cell x_k - c of every band node ([8][nband], -1 if
    // none) and the cells' per-corner force sums ([24][nocc])
    long long nocc = 0;
    int *occ_bi = nullptr, *occ_nbr = nullptr;
    float *cellS = nullptr;
    uint32_t *tile_mask = nullptr;
    int *tile_off = nullptr;
    std::vector<long long> order;   // sorted position -> caller's sample index

    // moving solids (lbm_set_motion): the band arrays use the fixed stride nband = 8 S (or
    // N) and the device count band_count_dev; the samples are re-posed, re-sorted and the
    // band rebuilt on the device at the start of every step
    bool moving = false;
    lbm_motion motion{};
    double r_max = 0.0;             // largest |X0 - c0| of the reference samples
    long long posed_tau0 = 0;       // step count at lbm_set_motion (the reference pose's time)
    long long posed_tau = -1;       // time of the pose the band was last built for
    // bitmap words [mask_w0, mask_w1) that can hold band bits of the last rebuild (all words
    // until the first one)
    long long mask_w0 = 0, mask_w1 = -1;
    int *band_count_dev = nullptr;
    float *X0 = nullptr, *X0_alt = nullptr, *area_alt = nullptr, *Xtmp = nullptr;
    int *sid = nullptr, *sid_alt = nullptr;
    void *motion_ws = nullptr;
    size_t motion_ws_bytes = 0;

    // smoke tracers, stored in 4x4x4-cell brick order (re-sorted after every advection):
    // positions [3][ntracer] (SoA) and the caller's index of each stored tracer, a second
    // copy of both for the reordering, the velocity field [3][N] written by each step while
    // tracers exist, the emitter of re-injected tracers, and the sort / density workspace
    long long ntracer = 0;
    float *tx = nullptr, *tx_alt = nullptr, *tracer_u = nullptr;
    uint32_t *tid = nullptr, *tid_alt = nullptr;
    lbm_emitter emitter{};
    void *tracer_ws = nullptr;
    size_t tracer_ws_bytes = 0;

    // device staging of host-pointer fields (lbm_set_state / lbm_macroscopic), kept between calls
    float *stage = nullptr;
    size_t stage_cap = 0;           // floats

    // scratch of the reductions
    double *partial = nullptr;
    size_t partial_cap = 0;         // doubles
    double *red = nullptr;          // 8 doubles
    int *flag = nullptr;
    // set by a step kernel whose bounded wait for its asynchronous copies ran out
    int *wait_err = nullptr;
    // 16-bit storage: the main range in the tensor-copy fed kernel (lbm_set_pair_kernel; off by
    // default: measured slower than the register-fed pair kernel on GB300)
    int pair_bulk = 0;

    // profiling
    bool prof = false;
    std::vector<EventRec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[LBM_NUM_KERNEL_KINDS] = {};
    long long launches[LBM_NUM_KERNEL_KINDS] = {};

    // device workspace of lbm_adjoint (pointer, bytes), reused by later calls
    std::vector<std::pair<void *, size_t>> adj_ws;

    // asynchronous host transfers (lbm_set_state_async, lbm_macroscopic_async), made on first
    // use: a host-to-device and a device-to-host copy stream, two input staging buffers taken
    // in turn (rho | u, 4 N floats each) and one output staging buffer; in_ready[k] = copy into
    // buffer k done, in_free[k] = the initialisation that read it done, out_ready = moments
    // written, out_free = copy out done
    cudaStream_t h2d = nullptr, d2h = nullptr;
    float *stage_in[2] = {nullptr, nullptr};
    int stage_in_next = 0;
    cudaEvent_t in_ready[2] = {nullptr, nullptr}, in_free[2] = {nullptr, nullptr};
    float *stage_out = nullptr;
    cudaEvent_t out_ready = nullptr, out_free = nullptr;

    // the immersed-boundary stage on its own stream, overlapping the edge strips (static solids
    // with no band node in the strips: ib_overlap): ib_in = the step's inputs are ready, ib_done =
    // band forces written; made on first use
    bool ib_overlap = false;
    // rows (y, z) holding band nodes of a static solid: y in [band_y0, band_y1], z in [band_z0,
    // band_z1] (the adjoint's backward step runs the other rows beside its IB chain)
    int band_y0 = 0, band_y1 = -1, band_z0 = 0, band_z1 = -1;
    int band_x0 = 0, band_x1 = -1;   // x range of the band nodes
    cudaStream_t ibs = nullptr;
    cudaEvent_t ib_in = nullptr, ib_done = nullptr;
    // per-block FP64 sums of the next step's penalty forces, written by that step right after its
    // IB stage on the IB stage's stream (component k of block b at fsum[k * fsum_stride + b]);
    // nullptr: none.  Consumed by the step.
    double *fsum = nullptr;
    long long fsum_stride = 0;

    std::string err;
};

namespace lbm_host {

int fail(lbm_ctx *h, int code, const std::string &msg);

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(h, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

inline bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
inline int dev_alloc(lbm_ctx *h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return LBM_OK;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(h, LBM_ENOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return LBM_OK;
}

template <typename T> inline void dev_free(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

inline cudaEvent_t pool_event(lbm_ctx *h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// event pair around the launches of one kernel kind on stream st (the context's stream by default)
struct Timed {
    lbm_ctx *h;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Timed(lbm_ctx *h_, int k, int nlaunch = 1, cudaStream_t s = nullptr) : h(h_), kind(k), st(s ? s : h_->stream) {
        h->launches[kind] += nlaunch;
        if (h->prof) {
            a = pool_event(h);
            cudaEventRecord(a, st);
        }
    }
    ~Timed() {
        if (h->prof) {
            cudaEvent_t b = pool_event(h);
            cudaEventRecord(b, st);
            h->recs.push_back({kind, a, b});
        }
    }
};

inline lbm::StepParams make_params(const lbm_ctx *h, long long t) {
    lbm::StepParams P{};
    P.f = h->f;
    for (int d = 0; d < 27; ++d) P.fp[d] = P.fpo[d] = static_cast<char *>(h->f) + (size_t)d * h->plane * h->esize;
    P.outlet = P.outlet_o = h->outlet;
    lbm::Geometry &g = P.g;
    g.nx = h->nx; g.ny = h->ny; g.nz = h->nz;
    g.nxy = h->nx * h->ny;
    g.ncell = (int)h->N;
    g.nyz = h->ny * h->nz;
    g.plane = h->plane;
    for (int a = 0; a < 3; ++a) g.periodic[a] = h->cfg.face_type[2 * a] == LBM_FACE_PERIODIC;
    for (int k = 0; k < 6; ++k) g.face[k] = h->cfg.face_type[k];
    P.rho0 = (float)h->cfg.rho0;
    P.Fx = (float)h->forcing[0];
    P.Fy = (float)h->forcing[1];
    P.Fz = (float)h->forcing[2];
    const double ws = 1.0 / (3.0 * h->nu + 0.5);
    P.rs = (float)(1.0 - ws);
    P.rb = (float)(1.0 - h->cfg.omega_bulk);
    P.r3 = (float)(1.0 - h->cfg.omega_hi[0]);
    P.r4 = (float)(1.0 - h->cfg.omega_hi[1]);
    P.r5 = (float)(1.0 - h->cfg.omega_hi[2]);
    P.r6 = (float)(1.0 - h->cfg.omega_hi[3]);
    P.q3 = (float)(1.0 - 0.5 * h->cfg.omega_hi[0]);
    P.q5 = (float)(1.0 - 0.5 * h->cfg.omega_hi[2]);
    {
        // coefficients of the scaled relaxation in collide_v (FP64 products, rounded once)
        const double r0 = h->cfg.rho0, rs = 1.0 - ws, rb = 1.0 - h->cfg.omega_bulk;
        const double r3 = 1.0 - h->cfg.omega_hi[0], r4 = 1.0 - h->cfg.omega_hi[1];
        const double r5 = 1.0 - h->cfg.omega_hi[2], r6 = 1.0 - h->cfg.omega_hi[3];
        const double q3 = 1.0 - 0.5 * h->cfg.omega_hi[0], q5 = 1.0 - 0.5 * h->cfg.omega_hi[2];
        lbm::CollCoef<float> &k = P.cc;
        k.rho0 = (float)r0; k.r0h = (float)(r0 / 2); k.mr0h = -k.r0h;
        k.a2 = (float)(rs / 4); k.b2 = (float)(-(1 - rs) / 4 * r0);
        k.tb6 = (float)(rb / 6); k.ts6 = (float)(rs / 6);
        k.a3 = (float)(r3 / 4); k.b3 = (float)((1 - r3) / 4 * r0); k.f3 = (float)(q3 / 3 / 4);
        k.a3e = (float)(r3 / 8); k.b3e = (float)((1 - r3) / 8 * r0);
        k.a4 = (float)(r4 / 4); k.b4r = (float)((1 - r4) / 4 / 9); k.b4u = (float)(-(1 - r4) / 4 * r0 / 3);
        k.a4m = (float)(r4 / 8); k.b4m = (float)(-(1 - r4) / 8 * r0);
        k.a5 = (float)(r5 / 8); k.b5 = (float)((1 - r5) / 8 * r0); k.f5 = (float)(q5 / 9 / 8);
        k.a6 = (float)(r6 / 8); k.b6r = (float)((1 - r6) / 8 / 27); k.b6u = (float)(-(1 - r6) / 8 * r0);
        // the transform's fixed constants: FP32 values (third and ninth rounded once from 1/3
        // and 1/9, sixth = third / 2 exactly)
        k.half = 0.5f; k.quarter = 0.25f; k.third = 1.0f / 3.0f; k.mthird = -k.third; k.sixth = 0.5f * k.third;
        k.ninth = 1.0f / 9.0f; k.three = 3.0f; k.mtwo = -2.0f; k.mone = -1.0f;
        // node pairs: every coefficient twice
        const float *src = reinterpret_cast<const float *>(&k);
        float2 *dst = reinterpret_cast<float2 *>(&P.cc2);
        static_assert(sizeof(lbm::CollCoef<float2>) == 2 * sizeof(lbm::CollCoef<float>), "coefficient layout");
        for (size_t i = 0; i < sizeof(lbm::CollCoef<float>) / sizeof(float); ++i) dst[i] = make_float2(src[i], src[i]);
    }
    P.u_in = (float)h->cfg.u_in;
    P.noise = (float)h->cfg.inlet_noise;
    P.seed = h->cfg.seed;
    P.t = t;
    P.inlet_profile = h->inlet_profile;
    P.tile_mask = h->tile_mask;
    P.tile_off = h->tile_off;
    P.bandF = h->bandF;
    P.nband = h->nband;
    P.band_count = h->band_count_dev;
    P.pair_bulk = h->pair_bulk;
    P.err = h->wait_err;
    return P;
}

// point the reads (src) and writes (dst) of a step at two stored states; a stored state is
// the 27 population planes followed by the outlet ghost plane (when the grid has an outlet)
inline void point_states(lbm::StepParams &P, const lbm_ctx *h, void *src, void *dst) {
    P.f = src;
    const size_t pb = (size_t)h->plane * h->esize;
    for (int d = 0; d < 27; ++d) {
        P.fp[d] = static_cast<char *>(src) + d * pb;
        P.fpo[d] = static_cast<char *>(dst) + d * pb;
    }
    P.outlet = h->outlet ? static_cast<char *>(src) + 27 * pb : nullptr;
    P.outlet_o = h->outlet ? static_cast<char *>(dst) + 27 * pb : nullptr;
}

// one full time step t (IB stage + fused step kernels) reading P's source and writing its
// destination; defined in lbm_api.cu
int step_with(lbm_ctx *h, const lbm::StepParams &P);

// the immersed-boundary stage of step P.t (band moments, interpolation and penalty, spreading)
// on stream st, with the per-corner cell sums in cellS ([24][nocc] floats; NULL: the context's
// buffer); defined in lbm_api.cu
int ib_stage(lbm_ctx *h, const lbm::StepParams &P, cudaStream_t st, float *cellS = nullptr);

// move the smoke tracers by one step in the velocity field the step wrote (lbm_tracers.cu)
int advect_tracers(lbm_ctx *h, long long t);

// moving solids (lbm_motion.cu): pose the samples for step t (the pose of time t - 1) and
// rebuild the band; refresh the host copy of the samples' caller order
int motion_before_step(lbm_ctx *h, long long t);
int sync_order(lbm_ctx *h);

inline int ensure_stage(lbm_ctx *h, size_t floats) {
    if (floats <= h->stage_cap) return LBM_OK;
    dev_free(h->stage);
    h->stage_cap = 0;
    int rc = dev_alloc(h, &h->stage, floats);
    if (rc) return rc;
    h->stage_cap = floats;
    return LBM_OK;
}

// the copy streams and events of the asynchronous host transfers, all or none
inline int ensure_async(lbm_ctx *h) {
    if (h->h2d) return LBM_OK;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev[6] = {};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
        for (auto x : st)
            if (x) cudaStreamDestroy(x);
        return fail(h, LBM_ECUDA, std::string("copy streams: ") + cudaGetErrorString(e));
    }
    h->h2d = st[0];
    h->d2h = st[1];
    h->in_ready[0] = ev[0];
    h->in_ready[1] = ev[1];
    h->in_free[0] = ev[2];
    h->in_free[1] = ev[3];
    h->out_ready = ev[4];
    h->out_free = ev[5];
    return LBM_OK;
}

// the stream and events of the overlapped IB stage, all or none (higher priority than the
// context's stream: the main kernel waits for the stage)
inline int ensure_ib_stream(lbm_ctx *h) {
    if (h->ibs) return LBM_OK;
    int lo = 0, hi = 0;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        return fail(h, LBM_ECUDA, std::string("IB stream: ") + cudaGetErrorString(e));
    }
    h->ibs = s;
    h->ib_in = e0;
    h->ib_done = e1;
    return LBM_OK;
}

inline void free_ib_stream(lbm_ctx *h) {
    if (!h->ibs) return;
    cudaStreamSynchronize(h->ibs);
    cudaEventDestroy(h->ib_in);
    cudaEventDestroy(h->ib_done);
    cudaStreamDestroy(h->ibs);
    h->ibs = nullptr;
}

inline void free_async(lbm_ctx *h) {
    if (!h->h2d) return;
    cudaStreamSynchronize(h->h2d);
    cudaStreamSynchronize(h->d2h);
    for (int k = 0; k < 2; ++k) {
        dev_free(h->stage_in[k]);
        cudaEventDestroy(h->in_ready[k]);
        cudaEventDestroy(h->in_free[k]);
    }
    dev_free(h->stage_out);
    cudaEventDestroy(h->out_ready);
    cudaEventDestroy(h->out_free);
    cudaStreamDestroy(h->h2d);
    cudaStreamDestroy(h->d2h);
    h->h2d = h->d2h = nullptr;
}

inline int ensure_partial(lbm_ctx *h, size_t doubles) {
    if (doubles <= h->partial_cap) return LBM_OK;
    dev_free(h->partial);
    h->partial_cap = 0;
    int rc = dev_alloc(h, &h->partial, doubles);
    if (rc) return rc;
    h->partial_cap = doubles;
    return LBM_OK;
}

inline void free_tracers(lbm_ctx *h) {
    dev_free(h->tx);
    dev_free(h->tx_alt);
    dev_free(h->tid);
    dev_free(h->tid_alt);
    dev_free(h->tracer_u);
    if (h->tracer_ws) cudaFree(h->tracer_ws);
    h->tracer_ws = nullptr;
    h->tracer_ws_bytes = 0;
    h->ntracer = 0;
}

inline void free_solid(lbm_ctx *h) {
    dev_free(h->X); dev_free(h->area); dev_free(h->ub); dev_free(h->g);
    dev_free(h->corner_band); dev_free(h->band_cell); dev_free(h->base_nbr);
    dev_free(h->cstart); dev_free(h->ccount);
    dev_free(h->band_rho); dev_free(h->band_u); dev_free(h->bandF);
    dev_free(h->tile_mask); dev_free(h->tile_off);
    dev_free(h->occ_bi); dev_free(h->occ_nbr); dev_free(h->cellS);
    h->nocc = 0;
    dev_free(h->band_count_dev);
    dev_free(h->X0); dev_free(h->X0_alt); dev_free(h->area_alt); dev_free(h->Xtmp);
    dev_free(h->sid); dev_free(h->sid_alt);
    if (h->motion_ws) cudaFree(h->motion_ws);
    h->motion_ws = nullptr;
    h->motion_ws_bytes = 0;
    h->moving = false;
    h->ub_zero = false;
    h->ib_overlap = false;
    h->posed_tau = -1;
    h->S = h->nband = h->ntiles = 0;
    h->band_y0 = 0; h->band_y1 = -1; h->band_z0 = 0; h->band_z1 = -1;
    h->band_x0 = 0; h->band_x1 = -1;
    h->mask_w0 = 0;
    h->mask_w1 = -1;
    h->order.clear();
}


}  // namespace lbm_host
