// Launchers of the CUDA kernels (lbm_kernels.cu), used by the C-ABI host code (lbm_api.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// parts of a step: STEP_BOUNDARY = the edge strips and (grids with a free-slip face) the face
// rows; STEP_INTERIOR = the main range; STEP_STRIPS / STEP_FACE_ROWS = the two halves of
// STEP_BOUNDARY (the strips of the rows the main kernel runs, and the face-row kernels), launched
// apart when the immersed-boundary stage overlaps the strips
enum { STEP_BOUNDARY = 0, STEP_INTERIOR = 1, STEP_STRIPS = 2, STEP_FACE_ROWS = 3 };
// collision models, numbered as LBM_COLL_* of the C ABI
enum CollisionModel { COLL_ACM = 0, COLL_BGK = 1, COLL_RAW = 2 };
// The x range is split into two edge strips of XEDGE nodes per row, run by the general face
// kernel (STEP_BOUNDARY; a warp takes the strips of 32 / XEDGE rows, coalesced per row), and the
// nodes XEDGE <= x < nx - XEDGE, run by the main kernel (STEP_INTERIOR).  Rows shorter than
// 2 XEDGE + 1 run entirely in the face kernel.  16-node strips: the general face rules cost more
// per node than the main kernel, so narrower strips put more of each row in the main kernel
// (whole step 8.76 -> 8.69 ms on the buildings workload, FP16 6.17 -> 6.09 ms).  The adjoint's
// backward step has no strips: its main kernel takes 1 <= x <= nx - 2 and a one-thread-per-node
// kernel the two x faces.
constexpr int XEDGE = 16;
constexpr int STEP_BX = 64;   // threads per block of the main step kernels (along x)
cudaError_t launch_step(int storage, const StepParams &P, bool band, int part, int collision, cudaStream_t st);
template <int COLL, bool FS>
cudaError_t launch_step_coll(int storage, const StepParams &P, bool band, int part, cudaStream_t st);
long long boundary_count(const Geometry &g);
__host__ __device__ inline bool has_interior(const Geometry &g) { return g.nx >= 2 * XEDGE + 1; }
// kernels one launch_step call makes (a grid with a free-slip face runs its face rows in the
// boundary part: edge strips of the other rows, then edge strips and main range of the face rows)
int step_launches(const StepParams &P, int part);
// the rows (y, z) on a y or z face: z = 0 and z = nz-1 (every y), then y = 0 and y = ny-1 of each
// z in between, in this order
__host__ __device__ inline long long face_rows(const Geometry &g) {
    const long long ny = g.ny, nz = g.nz;
    return ny * (nz < 2 ? nz : 2) + (nz > 2 ? nz - 2 : 0) * (ny < 2 ? ny : 2);
}
__host__ __device__ inline void face_row(const Geometry &g, long long r, int &y, int &z) {
    if (r < g.ny) { y = (int)r; z = 0; return; }
    r -= g.ny;
    if (r < g.ny) { y = (int)r; z = g.nz - 1; return; }   // (nz >= 2 here)
    r -= g.ny;
    const int w = g.ny > 1 ? 2 : 1;
    z = 1 + (int)(r / w);
    y = (r % w) ? g.ny - 1 : 0;
}
__host__ __device__ inline int edge_per_row(const Geometry &g) { return has_interior(g) ? 2 * XEDGE : g.nx; }
// A block of rows (y, z): y0 <= y < y0 + ny, z0 <= z < z0 + nz.  band_row_boxes splits the rows of
// a gny x gnz grid into the box [by0, by1] x [bz0, bz1] holding the band's rows and up to four
// boxes around it (rows y < by0 and y > by1 of every z, then the rows of the band's y range with
// z < bz0 and z > bz1), each row in exactly one box; returns the number of boxes around the band.
struct RowBox {
    int y0, ny, z0, nz;
};
__host__ __device__ inline int band_row_boxes(int gny, int gnz, int by0, int by1, int bz0, int bz1, RowBox &band,
                                              RowBox (&around)[4]) {
    band = RowBox{by0, by1 - by0 + 1, bz0, bz1 - bz0 + 1};
    int n = 0;
    if (by0 > 0) around[n++] = RowBox{0, by0, 0, gnz};
    if (by1 < gny - 1) around[n++] = RowBox{by1 + 1, gny - 1 - by1, 0, gnz};
    if (bz0 > 0) around[n++] = RowBox{by0, by1 - by0 + 1, 0, bz0};
    if (bz1 < gnz - 1) around[n++] = RowBox{by0, by1 - by0 + 1, bz1 + 1, gnz - 1 - bz1};
    return n;
}
cudaError_t launch_init(int storage, const StepParams &P, const float *rho, const float *u, cudaStream_t st);
long long macro_blocks(const StepParams &P);
// rows of the k_macro partial sums: mass, momentum x/y/z, slab kinetic energy
constexpr int MACRO_SUMS = 5;
cudaError_t launch_macro(int storage, const StepParams &P, bool band, int force_on, float *rho, float *u, float *f,
                         double *partial, int *nonfinite, cudaStream_t st, int ke_x0 = 0, int ke_x1 = 0);
cudaError_t launch_finalize(const double *partial, long long n, int count, double *out, cudaStream_t st);
cudaError_t launch_band_moments(int storage, const StepParams &P, const int *band_cell, float *band_rho, float *band_u,
                                cudaStream_t st);
// the band bitmap, band stride (nband) and geometry come from P; ub = nullptr: zero boundary velocity
cudaError_t launch_ib_interp(const StepParams &P, long long S, const float *X, const float *area, const float *ub,
                             const float *band_rho, const float *band_u, float *g, cudaStream_t st);
// nband: band nodes (or the stride of the band arrays when count is set); count: device
// count of band nodes (moving solids) or nullptr
cudaError_t launch_ib_spread(long long S, long long nband, const int *count, const float *X, const float *g,
                             const int *base_nbr, const int *cstart, const int *ccount, float *bandF, cudaStream_t st);
// two-phase immersed boundary of a static solid: per occupied base cell (interpolation, penalty,
// the cell's per-corner force sums cellS [24][nocc]), then per band node (gather of those sums)
cudaError_t launch_ib_cells(const StepParams &P, long long S, long long nocc, const int *occ_bi, const int *band_cell,
                            const int *cstart, const int *ccount, const float *X, const float *area, const float *ub,
                            const float *band_rho, const float *band_u, float *g, float *cellS, cudaStream_t st);
cudaError_t launch_ib_gather(long long nband, long long nocc, const int *occ_nbr, const float *cellS, float *bandF,
                             cudaStream_t st);
int force_sum_blocks(long long S);
// per-block force sums (force_sum_blocks(S) blocks); component k of block b at
// partial[k * stride + b], stride = the block count when 0
cudaError_t launch_sum_forces(long long S, const float *g, double *partial, cudaStream_t st, long long stride = 0);

}  // namespace lbm
