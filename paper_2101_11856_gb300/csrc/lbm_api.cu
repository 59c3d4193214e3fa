// C ABI of the solver (include/lbm.h): context, device buffers, the immersed-boundary
// set-up on the host, the per-step launch sequence, diagnostics and checkpoints.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "lbm_ctx.h"

using namespace lbm;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace lbm_host {
int fail(lbm_ctx *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

// the three immersed-boundary kernels of step P.t on stream st: band moments, then for a static
// solid the two-phase interpolation / spreading over the occupied base cells and the band nodes
// (cellS: the cells' per-corner sums, the context's buffer when NULL; work queued on two streams
// at once needs one buffer each), for a moving one (band rebuilt on the device every step) per
// sample and per band node
int ib_stage(lbm_ctx *h, const StepParams &P, cudaStream_t st, float *cellS) {
    if (!cellS) cellS = h->cellS;
    { Timed tm(h, LBM_KERNEL_BAND, 1, st); CK(launch_band_moments(h->storage, P, h->band_cell, h->band_rho, h->band_u, st)); }
    const float *ub = h->ub_zero ? nullptr : h->ub;
    if (h->nocc > 0 && !h->band_count_dev) {
        { Timed tm(h, LBM_KERNEL_INTERP, 1, st); CK(launch_ib_cells(P, h->S, h->nocc, h->occ_bi, h->band_cell, h->cstart, h->ccount, h->X, h->area, ub, h->band_rho, h->band_u, h->g, cellS, st)); }
        { Timed tm(h, LBM_KERNEL_SPREAD, 1, st); CK(launch_ib_gather(h->nband, h->nocc, h->occ_nbr, cellS, h->bandF, st)); }
        return LBM_OK;
    }
    { Timed tm(h, LBM_KERNEL_INTERP, 1, st); CK(launch_ib_interp(P, h->S, h->X, h->area, ub, h->band_rho, h->band_u, h->g, st)); }
    { Timed tm(h, LBM_KERNEL_SPREAD, 1, st); CK(launch_ib_spread(h->S, h->nband, h->band_count_dev, h->X, h->g, h->base_nbr, h->cstart, h->ccount, h->bandF, st)); }
    return LBM_OK;
}

// the per-block force sums a caller asked of this step (h->fsum), on the IB stage's stream
static int step_force_sum(lbm_ctx *h, cudaStream_t st) {
    if (!h->fsum) return LBM_OK;
    double *out = h->fsum;
    h->fsum = nullptr;
    CK(launch_sum_forces(h->S, h->g, out, st, h->fsum_stride));
    return LBM_OK;
}

int step_with(lbm_ctx *h, const StepParams &P) {
    const bool band = h->S > 0;
    int rc;
    if (band && h->ib_overlap && has_interior(P.g)) {
        // No band node lies in the edge strips, so the strips neither read the band forces nor
        // write a slot the band pass reads (AA: every slot is read and written by its own node):
        // the IB stage runs on its own stream beside the strips, and the face rows and the main
        // range wait for it.
        if ((rc = ensure_ib_stream(h))) return rc;
        CK(cudaEventRecord(h->ib_in, h->stream));
        CK(cudaStreamWaitEvent(h->ibs, h->ib_in, 0));
        if ((rc = ib_stage(h, P, h->ibs))) return rc;
        if ((rc = step_force_sum(h, h->ibs))) return rc;
        CK(cudaEventRecord(h->ib_done, h->ibs));
        {
            Timed tm(h, LBM_KERNEL_BOUNDARY, step_launches(P, STEP_STRIPS));
            CK(launch_step(h->storage, P, band, STEP_STRIPS, h->cfg.collision, h->stream));
        }
        CK(cudaStreamWaitEvent(h->stream, h->ib_done, 0));
        if (step_launches(P, STEP_FACE_ROWS) > 0) {
            Timed tm(h, LBM_KERNEL_BOUNDARY, step_launches(P, STEP_FACE_ROWS));
            CK(launch_step(h->storage, P, band, STEP_FACE_ROWS, h->cfg.collision, h->stream));
        }
    } else {
        if (band && (rc = ib_stage(h, P, h->stream))) return rc;
        if (band && (rc = step_force_sum(h, h->stream))) return rc;
        Timed tm(h, LBM_KERNEL_BOUNDARY, step_launches(P, STEP_BOUNDARY));
        CK(launch_step(h->storage, P, band, STEP_BOUNDARY, h->cfg.collision, h->stream));
    }
    if (has_interior(P.g)) {
        Timed tm(h, LBM_KERNEL_STEP, step_launches(P, STEP_INTERIOR));
        CK(launch_step(h->storage, P, band, STEP_INTERIOR, h->cfg.collision, h->stream));
    }
    return LBM_OK;
}
}  // namespace lbm_host

using namespace lbm_host;

namespace {

// copy n floats from a host or device pointer into a host vector
int fetch_floats(lbm_ctx *h, const float *src, size_t n, std::vector<float> &dst) {
    dst.resize(n);
    if (n == 0) return LBM_OK;
    if (is_device_ptr(src)) {
        CK(cudaMemcpyAsync(dst.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    } else {
        std::memcpy(dst.data(), src, n * sizeof(float));
    }
    return LBM_OK;
}

template <typename T> int upload(lbm_ctx *h, T **dst, const std::vector<T> &src) {
    int rc = dev_alloc(h, dst, src.size());
    if (rc) return rc;
    if (!src.empty()) CK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return LBM_OK;
}

// the Fourier part of the inflow profile on the inlet nodes, from h->cfg.inflow_coef (freed
// when every coefficient is zero or there is no inlet)
int upload_inflow(lbm_ctx *h) {
    const lbm_config &c = h->cfg;
    bool any_coef = false;
    for (int k = 0; k < 16; ++k) any_coef |= c.inflow_coef[k] != 0.0;
    if (h->f) cudaStreamSynchronize(h->stream);
    dev_free(h->inlet_profile);
    if (!any_coef || c.face_type[0] != LBM_FACE_INLET) return LBM_OK;
    const int ny = h->ny, nz = h->nz;
    std::vector<float> prof((size_t)ny * nz);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            double v = 0.0;
            for (int m = 1; m <= 4; ++m)
                for (int n = 1; n <= 4; ++n)
                    v += c.inflow_coef[(m - 1) * 4 + (n - 1)] * std::sin(m * M_PI * (y + 0.5) / ny) *
                         std::sin(n * M_PI * (z + 0.5) / nz);
            prof[y + (size_t)ny * z] = (float)v;
        }
    return upload(h, &h->inlet_profile, prof);
}

int require_state(lbm_ctx *h) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!h->has_state) return fail(h, LBM_ESTATE, "lbm_set_state (or lbm_load) has not been called");
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_config_default(lbm_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->storage = LBM_STORE_F32;
    for (int k = 0; k < 6; ++k) cfg->face_type[k] = LBM_FACE_PERIODIC;
    cfg->rho0 = 1.0;
    cfg->seed = 2101ull;
    cfg->omega_bulk = 1.0;
    for (int k = 0; k < 4; ++k) cfg->omega_hi[k] = 1.0;
    cfg->cuda_stream = nullptr;
    cfg->collision = LBM_COLL_ACM;
}

int lbm_create(lbm_ctx **out, int nx, int ny, int nz, double nu, const double forcing[3], const lbm_config *cfg) {
    lbm_ctx *h = nullptr;
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "dimensions must be >= 1");
    const long long N = (long long)nx * ny * nz;
    if (N > 2000000000LL) return fail(nullptr, LBM_EINVAL, "more than 2e9 cells");
    if (ny > 65535 || nz > 65535) return fail(nullptr, LBM_EINVAL, "ny and nz must be <= 65535");
    if (!(nu > 0.0) || !std::isfinite(nu)) return fail(nullptr, LBM_EINVAL, "nu must be positive and finite");
    lbm_config c;
    if (cfg) c = *cfg;
    else lbm_config_default(&c);
    if (c.storage < 0 || c.storage > 2) return fail(nullptr, LBM_EINVAL, "unknown storage type");
    if (c.collision < LBM_COLL_ACM || c.collision > LBM_COLL_RAW) return fail(nullptr, LBM_EINVAL, "unknown collision model");
    for (int k = 0; k < 6; ++k)
        if (c.face_type[k] < 0 || c.face_type[k] > 4) return fail(nullptr, LBM_EINVAL, "unknown face type");
    for (int a = 0; a < 3; ++a)
        if ((c.face_type[2 * a] == LBM_FACE_PERIODIC) != (c.face_type[2 * a + 1] == LBM_FACE_PERIODIC))
            return fail(nullptr, LBM_EINVAL, "periodic faces must come in pairs");
    for (int k = 0; k < 6; ++k) {
        if (c.face_type[k] == LBM_FACE_INLET && k != 0) return fail(nullptr, LBM_EINVAL, "the inlet must be the -x face");
        if (c.face_type[k] == LBM_FACE_OUTLET && k != 1) return fail(nullptr, LBM_EINVAL, "the outlet must be the +x face");
        if (c.face_type[k] == LBM_FACE_FREESLIP && k < 2) return fail(nullptr, LBM_EINVAL, "free-slip faces are y or z faces");
    }
    if (!(c.rho0 > 0.0)) return fail(nullptr, LBM_EINVAL, "rho0 must be positive");

    h = new (std::nothrow) lbm_ctx();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    h->nx = nx; h->ny = ny; h->nz = nz;
    h->N = N;
    h->plane = (N + 63) / 64 * 64;
    h->storage = c.storage;
    h->esize = c.storage == LBM_STORE_F32 ? 4 : 2;
    h->nu = nu;
    if (forcing) for (int a = 0; a < 3; ++a) h->forcing[a] = forcing[a];
    h->cfg = c;
    h->stream = (cudaStream_t)c.cuda_stream;

    auto bail = [&](int rc) {
        std::string msg = h->err;
        lbm_destroy(h);
        g_create_error = msg;
        return rc;
    };
    cudaError_t e = cudaMalloc(&h->f, (size_t)27 * h->plane * h->esize);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->f = nullptr;
        h->err = "cannot allocate the population array (" + std::to_string((size_t)27 * h->plane * h->esize) + " bytes)";
        return bail(LBM_ENOMEM);
    }
    if (cudaMemsetAsync(h->f, 0, (size_t)27 * h->plane * h->esize, h->stream) != cudaSuccess) {
        h->err = "cudaMemsetAsync failed";
        return bail(LBM_ECUDA);
    }
    if (c.face_type[1] == LBM_FACE_OUTLET) {
        if (cudaMalloc(&h->outlet, (size_t)2 * 9 * ny * nz * h->esize) != cudaSuccess) {
            cudaGetLastError();
            h->outlet = nullptr;
            h->err = "cannot allocate the outlet plane";
            return bail(LBM_ENOMEM);
        }
    }
    if (upload_inflow(h) != LBM_OK) return bail(LBM_ENOMEM);
    if (dev_alloc(h, &h->red, 8) != LBM_OK || dev_alloc(h, &h->flag, 1) != LBM_OK ||
        dev_alloc(h, &h->wait_err, 1) != LBM_OK)
        return bail(LBM_ENOMEM);
    if (cudaMemsetAsync(h->wait_err, 0, sizeof(int), h->stream) != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->err = "cudaMemsetAsync failed";
        return bail(LBM_ECUDA);
    }
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx *h) {
    if (!h) return LBM_OK;
    if (h->f) cudaStreamSynchronize(h->stream);
    free_async(h);
    free_ib_stream(h);
    free_solid(h);
    free_tracers(h);
    dev_free(h->stage);
    dev_free(h->f);
    dev_free(h->outlet);
    dev_free(h->inlet_profile);
    dev_free(h->partial);
    dev_free(h->red);
    dev_free(h->flag);
    dev_free(h->wait_err);
    for (auto &r : h->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    for (auto &w : h->adj_ws)
        if (w.first) cudaFree(w.first);
    delete h;
    return LBM_OK;
}

int lbm_set_state(lbm_ctx *h, const float *rho, const float *u) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!rho || !u) return fail(h, LBM_EINVAL, "rho and u are required");
    const float *drho = rho, *du = u;
    const bool dev = is_device_ptr(rho) && is_device_ptr(u);
    if (!dev) {
        int rc = ensure_stage(h, (size_t)4 * h->N);
        if (rc) return rc;
        CK(cudaMemcpyAsync(h->stage, rho, (size_t)h->N * sizeof(float), cudaMemcpyDefault, h->stream));
        CK(cudaMemcpyAsync(h->stage + h->N, u, (size_t)3 * h->N * sizeof(float), cudaMemcpyDefault, h->stream));
        drho = h->stage;
        du = h->stage + h->N;
    }
    StepParams P = make_params(h, 0);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_init(h->storage, P, drho, du, h->stream));
    }
    if (!dev) CK(cudaStreamSynchronize(h->stream));   // the caller may reuse its host buffers
    h->t = 0;
    h->has_state = true;
    return LBM_OK;
}

int lbm_set_state_async(lbm_ctx *h, const float *rho, const float *u) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!rho || !u) return fail(h, LBM_EINVAL, "rho and u are required");
    const float *drho = rho, *du = u;
    const bool dev = is_device_ptr(rho) && is_device_ptr(u);
    const int k = h->stage_in_next;
    if (!dev) {
        int rc = ensure_async(h);
        if (rc) return rc;
        if (!h->stage_in[k] && (rc = dev_alloc(h, &h->stage_in[k], (size_t)4 * h->N))) return rc;
        // the copy waits until the initialisation that last read this buffer is done, and the
        // initialisation below waits for the copy
        CK(cudaStreamWaitEvent(h->h2d, h->in_free[k], 0));
        CK(cudaMemcpyAsync(h->stage_in[k], rho, (size_t)h->N * sizeof(float), cudaMemcpyDefault, h->h2d));
        CK(cudaMemcpyAsync(h->stage_in[k] + h->N, u, (size_t)3 * h->N * sizeof(float), cudaMemcpyDefault, h->h2d));
        CK(cudaEventRecord(h->in_ready[k], h->h2d));
        CK(cudaStreamWaitEvent(h->stream, h->in_ready[k], 0));
        drho = h->stage_in[k];
        du = h->stage_in[k] + h->N;
    }
    StepParams P = make_params(h, 0);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_init(h->storage, P, drho, du, h->stream));
    }
    if (!dev) {
        CK(cudaEventRecord(h->in_free[k], h->stream));
        h->stage_in_next = k ^ 1;
    }
    h->t = 0;
    h->has_state = true;
    return LBM_OK;
}

int lbm_set_solids(lbm_ctx *h, const float *samples, long long count, const float *area, const float *u_b) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (count < 0) return fail(h, LBM_EINVAL, "negative sample count");
    if (count == 0) {
        CK(cudaStreamSynchronize(h->stream));
        free_solid(h);
        return LBM_OK;
    }
    if (!samples) return fail(h, LBM_EINVAL, "samples is NULL");
    if (count > 1000000000LL) return fail(h, LBM_EINVAL, "more than 1e9 samples");
    const size_t S = (size_t)count;
    std::vector<float> pos, ar, vb;
    int rc;
    if ((rc = fetch_floats(h, samples, 3 * S, pos))) return rc;
    if (area) { if ((rc = fetch_floats(h, area, S, ar))) return rc; }
    else ar.assign(S, 1.0f);
    if (u_b) { if ((rc = fetch_floats(h, u_b, 3 * S, vb))) return rc; }
    else vb.assign(3 * S, 0.0f);

    const int n[3] = {h->nx, h->ny, h->nz};
    std::vector<long long> key(S);
    for (size_t s = 0; s < S; ++s) {
        int b[3];
        for (int a = 0; a < 3; ++a) {
            const float v = pos[3 * s + a];
            if (!std::isfinite(v) || !(v >= 0.0f) || !(v < (float)(n[a] - 1)))
                return fail(h, LBM_EINVAL, "sample " + std::to_string(s) + " outside [0, n-1) or not finite");
            b[a] = (int)std::floor(v);
        }
        if (!std::isfinite(ar[s]) || !std::isfinite(vb[3 * s]) || !std::isfinite(vb[3 * s + 1]) || !std::isfinite(vb[3 * s + 2]))
            return fail(h, LBM_EINVAL, "non-finite area or boundary velocity");
        key[s] = b[0] + (long long)h->nx * (b[1] + (long long)h->ny * b[2]);
    }
    std::vector<long long> ord(S);
    std::iota(ord.begin(), ord.end(), 0LL);
    std::stable_sort(ord.begin(), ord.end(), [&](long long a, long long b) { return key[a] < key[b]; });

    // band: every node within the 2x2x2 stencil of a sample, as a bitmap over the cells
    const long long ntiles = (h->N + 31) / 32;
    std::vector<uint32_t> mask(ntiles, 0u);
    const long long cstep[8] = {0, 1, h->nx, (long long)h->nx + 1, (long long)h->nx * h->ny,
                                (long long)h->nx * h->ny + 1, (long long)h->nx * h->ny + h->nx,
                                (long long)h->nx * h->ny + h->nx + 1};
    for (size_t s = 0; s < S; ++s)
        for (int c = 0; c < 8; ++c) {
            const long long cell = key[s] + cstep[c];
            mask[cell >> 5] |= 1u << (cell & 31);
        }
    std::vector<int> toff(ntiles);
    long long nb = 0;
    for (long long w = 0; w < ntiles; ++w) {
        toff[w] = (int)nb;
        nb += __builtin_popcount(mask[w]);
    }
    if (nb > 2000000000LL) return fail(h, LBM_EINVAL, "band too large");
    auto band_index = [&](long long cell) -> int {
        const uint32_t m = mask[cell >> 5];
        const int l = (int)(cell & 31);
        if (!((m >> l) & 1u)) return -1;
        return toff[cell >> 5] + __builtin_popcount(m & ((1u << l) - 1u));
    };
    std::vector<int> bcell(nb);
    for (long long w = 0, k = 0; w < ntiles; ++w)
        for (int l = 0; l < 32; ++l)
            if ((mask[w] >> l) & 1u) bcell[k++] = (int)(w * 32 + l);
    std::vector<int> cst(nb, 0), ccnt(nb, 0);
    for (size_t i = 0; i < S; ++i) {
        const int bi = band_index(key[ord[i]]);
        if (ccnt[bi] == 0) cst[bi] = (int)i;
        ccnt[bi]++;
    }
    std::vector<int> bnbr((size_t)8 * nb);
    for (long long k = 0; k < nb; ++k) {
        const long long cell = bcell[k];
        const int x = (int)(cell % h->nx), y = (int)((cell / h->nx) % h->ny), z = (int)(cell / ((long long)h->nx * h->ny));
        for (int c = 0; c < 8; ++c) {
            const int bx = x - (c & 1), by = y - ((c >> 1) & 1), bz = z - ((c >> 2) & 1);
            int v = -1;
            if (bx >= 0 && by >= 0 && bz >= 0) {
                const int bi = band_index(bx + (long long)h->nx * (by + (long long)h->ny * bz));
                if (bi >= 0 && ccnt[bi] > 0) v = bi;
            }
            bnbr[(size_t)c * nb + k] = v;
        }
    }
    // occupied base cells (ascending band index = sample order) and their index per band node corner
    std::vector<int> obi, onbr((size_t)8 * nb, -1), occ_of(nb, -1);
    for (long long k = 0; k < nb; ++k)
        if (ccnt[k] > 0) {
            occ_of[k] = (int)obi.size();
            obi.push_back((int)k);
        }
    for (size_t e = 0; e < (size_t)8 * nb; ++e)
        if (bnbr[e] >= 0) onbr[e] = occ_of[bnbr[e]];
    std::vector<int> cb((size_t)8 * S);
    std::vector<float> Xs(3 * S), As(S), Us(3 * S);
    for (size_t i = 0; i < S; ++i) {
        const long long s = ord[i];
        for (int c = 0; c < 8; ++c) cb[(size_t)c * S + i] = band_index(key[s] + cstep[c]);
        for (int a = 0; a < 3; ++a) {
            Xs[a * S + i] = pos[3 * s + a];
            Us[a * S + i] = vb[3 * s + a];
        }
        As[i] = ar[s];
    }

    CK(cudaStreamSynchronize(h->stream));
    free_solid(h);
    h->S = (long long)S;
    h->nband = nb;
    h->ub_zero = std::all_of(vb.begin(), vb.end(), [](float v) { return v == 0.0f; });
    // the IB stage may overlap the edge strips when no band node lies in them
    h->ib_overlap = h->nx >= 2 * XEDGE + 1 && std::all_of(bcell.begin(), bcell.end(), [&](int c) {
        const int x = c % h->nx;
        return x >= XEDGE && x < h->nx - XEDGE;
    });
    h->band_y0 = h->ny; h->band_y1 = -1; h->band_z0 = h->nz; h->band_z1 = -1;
    h->band_x0 = h->nx; h->band_x1 = -1;
    for (const int c : bcell) {
        const int y = (int)((c / h->nx) % h->ny), z = (int)(c / ((long long)h->nx * h->ny));
        h->band_x0 = std::min(h->band_x0, c % h->nx); h->band_x1 = std::max(h->band_x1, c % h->nx);
        h->band_y0 = std::min(h->band_y0, y); h->band_y1 = std::max(h->band_y1, y);
        h->band_z0 = std::min(h->band_z0, z); h->band_z1 = std::max(h->band_z1, z);
    }
    h->ntiles = ntiles;
    h->nocc = (long long)obi.size();
    h->order = ord;
    if ((rc = upload(h, &h->X, Xs)) || (rc = upload(h, &h->area, As)) || (rc = upload(h, &h->ub, Us)) ||
        (rc = upload(h, &h->corner_band, cb)) || (rc = upload(h, &h->band_cell, bcell)) ||
        (rc = upload(h, &h->base_nbr, bnbr)) || (rc = upload(h, &h->cstart, cst)) || (rc = upload(h, &h->ccount, ccnt)) ||
        (rc = upload(h, &h->tile_mask, mask)) || (rc = upload(h, &h->tile_off, toff)) ||
        (rc = upload(h, &h->occ_bi, obi)) || (rc = upload(h, &h->occ_nbr, onbr))) {
        free_solid(h);
        return rc;
    }
    if ((rc = dev_alloc(h, &h->g, 3 * S)) || (rc = dev_alloc(h, &h->band_rho, (size_t)nb)) ||
        (rc = dev_alloc(h, &h->band_u, (size_t)3 * nb)) || (rc = dev_alloc(h, &h->bandF, (size_t)3 * nb)) ||
        (rc = dev_alloc(h, &h->cellS, (size_t)24 * obi.size()))) {
        free_solid(h);
        return rc;
    }
    CK(cudaMemsetAsync(h->g, 0, 3 * S * sizeof(float), h->stream));
    CK(cudaMemsetAsync(h->bandF, 0, (size_t)3 * nb * sizeof(float), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_step(lbm_ctx *h, int n) {
    int rc = require_state(h);
    if (rc) return rc;
    if (n < 0) return fail(h, LBM_EINVAL, "negative step count");
    for (int k = 0; k < n; ++k) {
        const long long t = h->t + 1;
        if ((rc = motion_before_step(h, t))) return rc;
        lbm::StepParams P = make_params(h, t);
        if (h->ntracer) P.u_out = h->tracer_u;   // the tracers move in this step's velocity
        if ((rc = step_with(h, P))) return rc;
        if ((rc = advect_tracers(h, t))) return rc;
        h->t = t;
    }
    return LBM_OK;
}

int lbm_macroscopic(lbm_ctx *h, float *rho, float *u) {
    int rc = require_state(h);
    if (rc) return rc;
    if (!rho && !u) return LBM_OK;
    const bool dr = !rho || is_device_ptr(rho), du = !u || is_device_ptr(u);
    float *drho = rho, *duu = u;
    if (!dr || !du) {
        if ((rc = ensure_stage(h, (size_t)4 * h->N))) return rc;
        if (!dr) drho = h->stage;
        if (!du) duu = h->stage + h->N;
    }
    StepParams P = make_params(h, h->t);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_macro(h->storage, P, h->S > 0, h->t > 0, drho, duu, nullptr, nullptr, nullptr, h->stream));
    }
    if (!dr) CK(cudaMemcpyAsync(rho, drho, (size_t)h->N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (!du) CK(cudaMemcpyAsync(u, duu, (size_t)3 * h->N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (!dr || !du) CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_macroscopic_async(lbm_ctx *h, float *rho, float *u) {
    int rc = require_state(h);
    if (rc) return rc;
    if (!rho && !u) return LBM_OK;
    const bool dr = !rho || is_device_ptr(rho), du = !u || is_device_ptr(u);
    float *drho = rho, *duu = u;
    const bool host = !dr || !du;
    if (host) {
        if ((rc = ensure_async(h))) return rc;
        if (!h->stage_out && (rc = dev_alloc(h, &h->stage_out, (size_t)4 * h->N))) return rc;
        // the moments wait until the previous copy out of the staging buffer is done
        CK(cudaStreamWaitEvent(h->stream, h->out_free, 0));
        if (!dr) drho = h->stage_out;
        if (!du) duu = h->stage_out + h->N;
    }
    StepParams P = make_params(h, h->t);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_macro(h->storage, P, h->S > 0, h->t > 0, drho, duu, nullptr, nullptr, nullptr, h->stream));
    }
    if (host) {
        CK(cudaEventRecord(h->out_ready, h->stream));
        CK(cudaStreamWaitEvent(h->d2h, h->out_ready, 0));
        if (!dr) CK(cudaMemcpyAsync(rho, drho, (size_t)h->N * sizeof(float), cudaMemcpyDefault, h->d2h));
        if (!du) CK(cudaMemcpyAsync(u, duu, (size_t)3 * h->N * sizeof(float), cudaMemcpyDefault, h->d2h));
        CK(cudaEventRecord(h->out_free, h->d2h));
    }
    return LBM_OK;
}

int lbm_reductions(lbm_ctx *h, double *mass, double mom[3], double drag[3]) {
    int rc = require_state(h);
    if (rc) return rc;
    StepParams P = make_params(h, h->t);
    const long long nblk = macro_blocks(P);
    const int fblk = force_sum_blocks(h->S);
    if ((rc = ensure_partial(h, (size_t)std::max<long long>(MACRO_SUMS * nblk, 3 * fblk)))) return rc;
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_macro(h->storage, P, h->S > 0, h->t > 0, nullptr, nullptr, nullptr, h->partial, nullptr, h->stream));
        CK(launch_finalize(h->partial, nblk, 4, h->red, h->stream));   // the first 4 rows
    }
    if (h->S > 0 && h->t > 0) {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_sum_forces(h->S, h->g, h->partial, h->stream));
        CK(launch_finalize(h->partial, fblk, 3, h->red + 4, h->stream));
    } else {
        CK(cudaMemsetAsync(h->red + 4, 0, 3 * sizeof(double), h->stream));
    }
    double r[7];
    CK(cudaMemcpyAsync(r, h->red, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (mass) *mass = r[0];
    if (mom) for (int a = 0; a < 3; ++a) mom[a] = r[1 + a];
    if (drag) for (int a = 0; a < 3; ++a) drag[a] = -r[4 + a];
    return LBM_OK;
}

int lbm_ib_forces(lbm_ctx *h, float *g) {
    int rc = require_state(h);
    if (rc) return rc;
    if (!g) return fail(h, LBM_EINVAL, "g is NULL");
    const size_t S = (size_t)h->S;
    if (S == 0) return LBM_OK;
    if ((rc = sync_order(h))) return rc;
    std::vector<float> sorted(3 * S), out(3 * S);
    CK(cudaMemcpyAsync(sorted.data(), h->g, 3 * S * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < S; ++i)
        for (int a = 0; a < 3; ++a) out[3 * h->order[i] + a] = sorted[a * S + i];
    CK(cudaMemcpyAsync(g, out.data(), 3 * S * sizeof(float), cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

int lbm_populations(lbm_ctx *h, float *f) {
    int rc = require_state(h);
    if (rc) return rc;
    if (!f) return fail(h, LBM_EINVAL, "f is NULL");
    float *df = f, *tmp = nullptr;
    const bool dev = is_device_ptr(f);
    if (!dev) {
        if ((rc = dev_alloc(h, &tmp, (size_t)27 * h->N))) return rc;
        df = tmp;
    }
    StepParams P = make_params(h, h->t);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_macro(h->storage, P, h->S > 0, h->t > 0, nullptr, nullptr, df, nullptr, nullptr, h->stream));
    }
    if (!dev) {
        CK(cudaMemcpyAsync(f, tmp, (size_t)27 * h->N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        dev_free(tmp);
    }
    return LBM_OK;
}

int lbm_velocity(int i, int c[3]) {
    if (i < 0 || i >= 27 || !c) return LBM_EINVAL;
    c[0] = cx(i);
    c[1] = cy(i);
    c[2] = cz(i);
    return LBM_OK;
}

long long lbm_time(const lbm_ctx *h) { return h ? h->t : -1; }

int lbm_set_pair_kernel(lbm_ctx *h, int bulk) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (bulk < 0 || bulk > 2) return fail(h, LBM_EINVAL, "lbm_set_pair_kernel takes 0, 1 or 2");
    h->pair_bulk = bulk;
    return LBM_OK;
}

int lbm_set_inflow(lbm_ctx *h, const double coef[16]) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!coef) return fail(h, LBM_EINVAL, "coef is NULL");
    if (h->cfg.face_type[0] != LBM_FACE_INLET) return fail(h, LBM_EINVAL, "the -x face is not an inlet");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(coef[k])) return fail(h, LBM_EINVAL, "non-finite inflow coefficient");
    for (int k = 0; k < 16; ++k) h->cfg.inflow_coef[k] = coef[k];
    int rc = upload_inflow(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

long long lbm_solid_count(const lbm_ctx *h) { return h ? h->S : -1; }

int lbm_dims(const lbm_ctx *h, int dims[3]) {
    if (!h || !dims) return LBM_EINVAL;
    dims[0] = h->nx;
    dims[1] = h->ny;
    dims[2] = h->nz;
    return LBM_OK;
}

long long lbm_band_size(const lbm_ctx *h) {
    if (!h) return -1;
    if (!h->band_count_dev) return h->nband;
    int n = 0;   // moving solids: the count of the last rebuild
    if (cudaMemcpyAsync(&n, h->band_count_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return n;
}

// LBM_ETIMEOUT when a step kernel's bounded device-side wait ran out since the last check (the
// flag is cleared); call after the context's stream finished
static int wait_error(lbm_ctx *h) {
    int w = 0;
    CK(cudaMemcpy(&w, h->wait_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!w) return LBM_OK;
    CK(cudaMemset(h->wait_err, 0, sizeof(int)));
    return fail(h, LBM_ETIMEOUT, "a step kernel's wait for its asynchronous copies ran out; the state is invalid");
}

int lbm_check(lbm_ctx *h) {
    int rc = require_state(h);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    StepParams P = make_params(h, h->t);
    {
        Timed tm(h, LBM_KERNEL_OTHER);
        CK(launch_macro(h->storage, P, h->S > 0, h->t > 0, nullptr, nullptr, nullptr, nullptr, h->flag, h->stream));
    }
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if ((rc = wait_error(h))) return rc;
    if (bad) return fail(h, LBM_EUNSTABLE, "non-finite density or velocity at step " + std::to_string(h->t));
    return LBM_OK;
}

int lbm_synchronize(lbm_ctx *h, double timeout_s) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    // the context's stream and, once made, the copy streams of the asynchronous transfers
    cudaStream_t streams[3] = {h->stream, h->h2d, h->d2h};
    const int ns = h->h2d ? 3 : 1;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    auto destroy = [&]() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    };
    for (int i = 0; i < ns; ++i) {
        cudaError_t c = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (c == cudaSuccess) c = cudaEventRecord(ev[i], streams[i]);
        if (c != cudaSuccess) {
            destroy();
            return fail(h, LBM_ECUDA, std::string("event record failed: ") + cudaGetErrorString(c));
        }
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < ns;) {
        cudaError_t q = cudaEventQuery(ev[i]);
        if (q == cudaSuccess) {
            ++i;
            continue;
        }
        if (q != cudaErrorNotReady) {
            destroy();
            return fail(h, LBM_ECUDA, std::string("stream failed: ") + cudaGetErrorString(q));
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s > 0 && el > timeout_s) {
            destroy();
            return fail(h, LBM_ETIMEOUT, "stream did not finish within the time limit");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    destroy();
    return wait_error(h);
}

// checkpoint layout: header (8 int64) | populations (27 planes of N elements) | outlet plane;
// header = magic, nx, ny, nz, storage, t, outlet bytes, configuration hash
static const long long kMagic = 0x4c424d4741413032LL;   // "LBMGAA02"

// FNV-1a (64 bit) over the configuration that a restored state is only valid under: nu, the
// body force, the face types, the collision model and its rates, rho0 and the inlet
// parameters (velocity, noise amplitude and seed, inflow coefficients)
static long long config_hash(const lbm_ctx *h) {
    unsigned long long x = 0xcbf29ce484222325ull;
    auto mix = [&x](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            x ^= b[i];
            x *= 0x100000001b3ull;
        }
    };
    const lbm_config &c = h->cfg;
    mix(&h->nu, sizeof(double));
    mix(h->forcing, sizeof(h->forcing));
    mix(c.face_type, sizeof(c.face_type));
    mix(&c.collision, sizeof(int));
    mix(&c.rho0, sizeof(double));
    mix(&c.omega_bulk, sizeof(double));
    mix(c.omega_hi, sizeof(c.omega_hi));
    mix(&c.u_in, sizeof(double));
    mix(&c.inlet_noise, sizeof(double));
    mix(&c.seed, sizeof(c.seed));
    mix(c.inflow_coef, sizeof(c.inflow_coef));
    return (long long)x;
}

int lbm_save(lbm_ctx *h, void *buf, size_t *bytes) {
    int rc = require_state(h);
    if (rc) return rc;
    if (!bytes) return fail(h, LBM_EINVAL, "bytes is NULL");
    const size_t pop = (size_t)27 * h->N * h->esize;
    const size_t outl = h->outlet ? (size_t)2 * 9 * h->ny * h->nz * h->esize : 0;
    const size_t need = 8 * sizeof(long long) + pop + outl;
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (*bytes < need) return fail(h, LBM_EINVAL, "buffer too small");
    long long hdr[8] = {kMagic, h->nx, h->ny, h->nz, h->storage, h->t, (long long)outl, config_hash(h)};
    char *p = static_cast<char *>(buf);
    std::memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    for (int d = 0; d < 27; ++d)
        CK(cudaMemcpyAsync(p + (size_t)d * h->N * h->esize, static_cast<char *>(h->f) + (size_t)d * h->plane * h->esize,
                           (size_t)h->N * h->esize, cudaMemcpyDefault, h->stream));
    if (outl) CK(cudaMemcpyAsync(p + pop, h->outlet, outl, cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *bytes = need;
    return LBM_OK;
}

int lbm_load(lbm_ctx *h, const void *buf, size_t bytes) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    if (!buf || bytes < 8 * sizeof(long long)) return fail(h, LBM_EINVAL, "bad checkpoint buffer");
    long long hdr[8];
    std::memcpy(hdr, buf, sizeof(hdr));
    const size_t pop = (size_t)27 * h->N * h->esize;
    const size_t outl = h->outlet ? (size_t)2 * 9 * h->ny * h->nz * h->esize : 0;
    if (hdr[0] != kMagic || hdr[1] != h->nx || hdr[2] != h->ny || hdr[3] != h->nz || hdr[4] != h->storage ||
        hdr[6] != (long long)outl || bytes < sizeof(hdr) + pop + outl)
        return fail(h, LBM_EINVAL, "checkpoint does not match this context");
    if (hdr[7] != config_hash(h))
        return fail(h, LBM_EINVAL, "checkpoint was written under another configuration (nu, force, faces, collision, "
                                   "rates, rho0 or inlet parameters)");
    const char *p = static_cast<const char *>(buf) + sizeof(hdr);
    for (int d = 0; d < 27; ++d)
        CK(cudaMemcpyAsync(static_cast<char *>(h->f) + (size_t)d * h->plane * h->esize, p + (size_t)d * h->N * h->esize,
                           (size_t)h->N * h->esize, cudaMemcpyDefault, h->stream));
    if (outl) CK(cudaMemcpyAsync(h->outlet, p + pop, outl, cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->t = hdr[5];
    h->has_state = true;
    return LBM_OK;
}

int lbm_profile(lbm_ctx *h, int enable) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    CK(cudaStreamSynchronize(h->stream));
    for (auto &r : h->recs) {
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->recs.clear();
    for (int k = 0; k < LBM_NUM_KERNEL_KINDS; ++k) {
        h->ms[k] = 0.0;
        h->launches[k] = 0;
    }
    h->prof = enable != 0;
    return LBM_OK;
}

int lbm_kernel_times(lbm_ctx *h, double ms[LBM_NUM_KERNEL_KINDS], long long launches[LBM_NUM_KERNEL_KINDS]) {
    if (!h) return fail(nullptr, LBM_EINVAL, "null context");
    CK(cudaStreamSynchronize(h->stream));
    for (auto &r : h->recs) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        h->ms[r.kind] += t;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->recs.clear();
    for (int k = 0; k < LBM_NUM_KERNEL_KINDS; ++k) {
        if (ms) ms[k] = h->ms[k];
        if (launches) launches[k] = h->launches[k];
    }
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
