/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D3Q27 central-moment MRT kinetic solver with
 * direct-forcing immersed boundaries (arXiv 2101.11856, "GPU Optimization for
 * High-Quality Kinetic Fluid Simulation").
 *
 * One context = one simulation on one GPU and one CUDA stream.  The library owns every
 * device buffer it allocates (populations, immersed-boundary data, scratch); callers
 * own the arrays they pass in and out.  Array arguments may be host or device pointers
 * (the library checks with cudaPointerGetAttributes) and are never retained after the
 * call returns.  Calls on one context are not thread-safe.
 *
 * Lattice units throughout: dx = dt = 1, c_s^2 = 1/3.  Fields are stored x-fastest:
 * cell (x, y, z) has flat index x + nx * (y + ny * z).  Vector fields are
 * structure-of-arrays: u[0..N) = u_x, u[N..2N) = u_y, u[2N..3N) = u_z.
 *
 * Every function returns LBM_OK (0) or a negative error code; lbm_last_error() gives
 * a message for the last failure on a context.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------- */
#define LBM_OK         0
#define LBM_EINVAL    -1   /* bad argument: dims < 1, nu <= 0, non-finite or out-of-domain samples, ... */
#define LBM_ENOMEM    -2   /* a device or host allocation failed                                      */
#define LBM_ECUDA     -3   /* a CUDA runtime call failed                                              */
#define LBM_EUNSTABLE -4   /* non-finite density or velocity detected by lbm_check                   */
#define LBM_ETIMEOUT  -5   /* a host-side wait exceeded its wall-clock limit, or a step kernel's bounded wait ran out */
#define LBM_ESTATE    -6   /* called in the wrong state (e.g. step before set_state)                 */

/* ---- population storage ---------------------------------------------------------- */
#define LBM_STORE_F32  0   /* deviations f_i - w_i rho0 stored as float     (216 B per cell update) */
#define LBM_STORE_F16  1   /* deviations stored as IEEE half, math in FP32   (108 B per cell update) */
#define LBM_STORE_BF16 2   /* deviations stored as bfloat16, math in FP32    (108 B per cell update) */

/* ---- domain faces (order -x, +x, -y, +y, -z, +z) --------------------------------- */
#define LBM_FACE_PERIODIC 0  /* both faces of an axis must be periodic together            */
#define LBM_FACE_NOSLIP   1  /* half-way bounce-back (the paper's Algorithm 1)             */
#define LBM_FACE_INLET    2  /* -x only: moving-wall bounce-back at u_in(y, z, t)          */
#define LBM_FACE_OUTLET   3  /* +x only: zero-gradient ghost layer                         */
#define LBM_FACE_FREESLIP 4  /* y and z faces only: half-way specular reflection (the
                                population from the tangential neighbour, its normal
                                component reversed); no-slip and the inlet win at edges,
                                the outlet ghost is read at the mirrored source; not
                                covered by lbm_adjoint (LBM_EINVAL)                        */

typedef struct lbm_ctx lbm_ctx;

typedef struct lbm_config {
    int storage;                 /* LBM_STORE_*                                                */
    int face_type[6];            /* LBM_FACE_* for -x, +x, -y, +y, -z, +z                      */
    double rho0;                 /* reference density of the deviation storage and the inlet  */
    double u_in;                 /* inlet base velocity (x component)                          */
    double inlet_noise;          /* relative amplitude of the seeded uniform inlet noise       */
    unsigned long long seed;     /* SplitMix64 seed of the inlet noise                         */
    double inflow_coef[16];      /* a_mn, m, n = 1..4 (row-major in m) of the inflow profile   */
    double omega_bulk;           /* rate of the trace of the second-order central moments     */
    double omega_hi[4];          /* rates of the third-, fourth-, fifth-, sixth-order moments */
    void *cuda_stream;           /* cudaStream_t the context launches on (NULL = legacy)       */
    int collision;               /* LBM_COLL_*: the collision of Eq. 4                         */
} lbm_config;

/* Collision models (lbm_config.collision).  LBM_COLL_ACM is the method: central-moment MRT
 * with the rates of Eq. 5 (Sec. 2.1).  The other two are the comparison models of the
 * results in Sec. 6.1, under the same streaming, faces, Guo forcing and immersed boundary:
 * LBM_COLL_BGK relaxes every non-conserved moment at the shear rate (single-relaxation BGK
 * with the D3Q27 product equilibrium), LBM_COLL_RAW is Eq. 5 with the velocity-independent
 * raw moments c_x^p c_y^q c_z^r in place of the central ones and the same rate groups
 * (omega_bulk and omega_hi apply to it as to ACM; BGK ignores them).  Only LBM_COLL_ACM has
 * an adjoint: lbm_adjoint on a context of another model returns LBM_EINVAL. */
#define LBM_COLL_ACM 0
#define LBM_COLL_BGK 1
#define LBM_COLL_RAW 2

/* Fill *cfg with defaults: FP32 storage, all faces periodic, rho0 = 1, no inlet, no noise,
 * seed 2101, zero inflow coefficients, omega_bulk = omega_hi[*] = 1, default stream,
 * collision LBM_COLL_ACM. */
void lbm_config_default(lbm_config *cfg);

/* Create a solver on an nx * ny * nz D3Q27 lattice (Eq. 1) with kinematic viscosity nu
 * (shear rate omega_s = 1 / (3 nu + 1/2), the low-order rate set by nu in Eq. 5) and the
 * uniform body force forcing[3] (Guo-style force term G of Eq. 4; NULL = no force).
 * cfg = NULL takes lbm_config_default.  Allocates the population array (27 planes of
 * nx*ny*nz values of the storage type, AA in-place layout) on the current CUDA device.
 * Errors: LBM_EINVAL (a dim < 1, ny or nz > 65535, more than 2e9 cells, nu <= 0, bad faces),
 * LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(lbm_ctx **out, int nx, int ny, int nz, double nu,
               const double forcing[3], const lbm_config *cfg);

/* Release every buffer of the context (NULL is accepted). */
int lbm_destroy(lbm_ctx *h);

/* Initialise the populations to the equilibrium of the given fields, f_i = f_eq_i(rho, u)
 * (product-form discrete Maxwellian), and reset the step counter to 0.
 * rho: N floats; u: 3N floats (SoA).  Host or device pointers; host fields go through a
 * device staging buffer of 16 N bytes that the context keeps for later host transfers
 * (lbm_set_state, lbm_macroscopic), and the call returns after they were read. */
int lbm_set_state(lbm_ctx *h, const float *rho, const float *u);

/* Install the immersed solid (Sec. 3.1): count samples at positions samples[3*s+a]
 * (x, y, z interleaved, lattice units), per-sample area weights area[s] (NULL = 1) and
 * boundary velocities u_b[3*s+a] (NULL = 0).  Every sample must satisfy
 * 0 <= X_a < n_a - 1 on each axis (its 2x2x2 interpolation stencil lies in the domain);
 * otherwise LBM_EINVAL and the previous solid is kept.  The library sorts the samples by
 * base cell and builds the band of nodes the 2x2x2 kernel touches (Eqs. 6-8).
 * count = 0 removes the solid.  Host or device pointers. */
int lbm_set_solids(lbm_ctx *h, const float *samples, long long count,
                   const float *area, const float *u_b);

/* Advance n time steps (Algorithm 2: streaming, moments, immersed boundary, collision
 * with forcing, domain faces), asynchronously on the context's stream.  Each step is one
 * fused stream+collide kernel over the nodes 16 <= x < nx-16, one over the two 16-node
 * edge strips of every row (the inlet/outlet/x-periodic rules), and three small
 * immersed-boundary kernels when a solid is installed: the band moments, then for a static
 * solid the interpolation and penalty per occupied base cell with each cell's spreading sums
 * and the gather of those sums per band node, for a moving one the interpolation per sample and
 * the spreading per band node (plus the re-pose of a moving solid and the tracer advection
 * when those are set).  On a grid with a free-slip face the rows
 * on a y or z face run in two more kernels (strips and main range) that carry the mirror
 * rule, and the first two skip them.
 * Errors: LBM_ESTATE before lbm_set_state, LBM_ECUDA. */
int lbm_step(lbm_ctx *h, int n);

/* Density and Guo-shifted velocity u = (sum c f + F/2)/rho used by the most recent
 * collision (Eq. 2); before any step, the fields given to lbm_set_state.
 * rho: N floats, u: 3N floats (SoA); either may be NULL.  Host or device pointers;
 * with host pointers the call returns after the copy completed (through the context's
 * staging buffer, see lbm_set_state). */
int lbm_macroscopic(lbm_ctx *h, float *rho, float *u);

/* lbm_set_state and lbm_macroscopic with the host copies queued instead of waited for, so
 * that they overlap the steps queued around them (the step's inputs uploaded while the
 * previous batch of steps runs, its outputs read back while the next one runs).
 * lbm_set_state_async queues the copy of host rho (N floats) and u (3N floats) on the
 * context's host-to-device copy stream into one of two device staging buffers (16 N bytes
 * each, taken in turn; a buffer is reused once the initialisation that read it is done),
 * then the initialisation f_i = f_eq_i(rho, u) on the context's stream behind the copy; the
 * step counter is 0 for the steps queued after it.  lbm_macroscopic_async queues the density
 * and Guo-shifted velocity of the current state (as lbm_macroscopic) into a device staging
 * buffer (16 N bytes) on the context's stream and their copy to host rho / u (either may be
 * NULL) on the device-to-host copy stream behind it.  The staging buffers and both copy
 * streams are made on first use and kept by the context.  The host buffers must stay valid
 * and unchanged (inputs) or unread (outputs) until lbm_synchronize returns; only page-locked
 * host memory lets the copies overlap.  Device pointers behave as in the blocking calls.
 * Errors: as lbm_set_state / lbm_macroscopic; LBM_ENOMEM for the staging buffers. */
int lbm_set_state_async(lbm_ctx *h, const float *rho, const float *u);
int lbm_macroscopic_async(lbm_ctx *h, float *rho, float *u);

/* FP64 global diagnostics of the most recent step: total mass sum rho, total momentum
 * sum rho u, and the drag on the solid -sum_s g_s (Algorithm 2, total force).
 * Any pointer may be NULL.  Host pointers; the call waits for the stream. */
int lbm_reductions(lbm_ctx *h, double *mass, double mom[3], double drag[3]);

/* Penalty forces g_s = rho_s (u_b - u_s) dA_s (Eq. 7) of the most recent step, in the
 * caller's sample order: g[3*s+a].  Host or device pointer. */
int lbm_ib_forces(lbm_ctx *h, float *g);

/* Post-collision populations f_i(x) of the current time in canonical (non-AA) layout,
 * converted to float: f[i*N + cell], i in the library's velocity order (lbm_velocity).
 * Host or device pointer. */
int lbm_populations(lbm_ctx *h, float *f);

/* Velocity c_i of the library's direction i (0 <= i < 27); returns LBM_EINVAL otherwise. */
int lbm_velocity(int i, int c[3]);

/* Number of time steps taken since lbm_set_state / lbm_load. */
long long lbm_time(const lbm_ctx *h);

/* Scan the most recent macroscopic state for non-finite values: LBM_OK or LBM_EUNSTABLE. */
int lbm_check(lbm_ctx *h);

/* Wait for the context's stream and the copy streams of the asynchronous host transfers
 * with a wall-clock limit in seconds (<= 0: no limit), polling with cudaEventQuery:
 * LBM_OK, LBM_ETIMEOUT or LBM_ECUDA. */
int lbm_synchronize(lbm_ctx *h, double timeout_s);

/* Loss of the adjoint problem: L = w_drag * (1/n) sum_{t=1..n} D_x(t)
 *                                 + w_ke * 1/2 sum_{ke_x0 <= x < ke_x1} rho |u|^2 (at step n),
 * D(t) = -sum_s g_s(t) the drag on the solid (Algorithm 2, total force) and rho, u the
 * macroscopic fields of the last collision (Eq. 2). */
typedef struct lbm_loss {
    double w_drag;
    double w_ke;
    int ke_x0, ke_x1;            /* slab of the kinetic-energy term, 0 <= ke_x0 <= ke_x1 <= nx */
} lbm_loss;

/* Hand-written adjoint (the paper has no adjoint; the forward operator is Algorithm 2 with
 * Eqs. 3-8).  Runs n steps forward from the current state (the state advances by n, as with
 * lbm_step), evaluates L and back-propagates through every step: transposed streaming with
 * the faces, the vector-Jacobian product of the central-moment collision recomputed in
 * registers, and the transposes of IB interpolation/spreading with the derivatives of the
 * trilinear weights.  States are recomputed out of place from checkpoints taken every K
 * steps (memory: about n/K + K population arrays plus two FP32 adjoint arrays; K = n stores
 * every state and recomputes nothing).
 * Outputs (host pointers, any may be NULL): dL_dinflow[16] = dL/da_mn of the inflow profile
 * (row-major in m; 0 without an inlet), dL_dpos[3*count] = dL/dX_s in the caller's sample
 * order, *L.  Gradients are accumulated in FP64.  The device workspace (checkpoints, states,
 * adjoint arrays) stays with the context for later calls and is freed by lbm_destroy.
 * Errors: LBM_ESTATE, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_adjoint(lbm_ctx *h, int n, int K, const lbm_loss *loss, double *dL_dinflow, double *dL_dpos, double *L);

/* Checkpoint: serialise the state (header + populations in canonical layout in the
 * storage type + outlet ghost plane + step counter) into buf.  The header records the dims,
 * the storage type and a 64-bit hash of the configuration the state evolves under (nu, body
 * force, face types, collision model and rates, rho0, inlet velocity, noise amplitude and
 * seed, inflow coefficients).  With buf = NULL only *bytes is set to the required size.
 * Host pointer. */
int lbm_save(lbm_ctx *h, void *buf, size_t *bytes);

/* Restore a checkpoint written by lbm_save into a context with the same dims, storage and
 * configuration hash; anything else is LBM_EINVAL and leaves the context unchanged.  Only the
 * populations, the outlet ghost plane and the step counter are restored: the solid, its
 * motion and the tracers are the context's own and are not part of a checkpoint. */
int lbm_load(lbm_ctx *h, const void *buf, size_t bytes);

/* Per-kernel device timing (CUDA events on the context's stream around every launch).
 * lbm_profile(h, 1) enables and clears the counters; lbm_profile(h, 0) disables. */
#define LBM_KERNEL_STEP        0   /* fused stream + collide, 16 <= x < nx-16              */
#define LBM_KERNEL_BAND        1   /* immersed-boundary band moments                      */
#define LBM_KERNEL_INTERP      2   /* interpolation + penalty (Eqs. 6-7)                   */
#define LBM_KERNEL_SPREAD      3   /* spreading (Eq. 8)                                    */
#define LBM_KERNEL_BOUNDARY    4   /* fused stream + collide, the 16-node strips at both
                                      row ends (whole rows when nx < 33)                   */
#define LBM_KERNEL_OTHER       5   /* init, macroscopic, reductions, copies, density      */
#define LBM_KERNEL_TRACER      6   /* smoke tracer advection                              */
#define LBM_KERNEL_MOTION      7   /* moving solids: pose, re-sort and band rebuild       */
#define LBM_NUM_KERNEL_KINDS   8
int lbm_profile(lbm_ctx *h, int enable);
/* ms[k], launches[k] for k < LBM_NUM_KERNEL_KINDS; waits for the stream. */
int lbm_kernel_times(lbm_ctx *h, double ms[LBM_NUM_KERNEL_KINDS], long long launches[LBM_NUM_KERNEL_KINDS]);

/* ---- Moving and rotating solids (Algorithm 2 (c): after the penalty forces are spread the
 * total force and torque are reduced and the solid samples are updated; the paper's dynamic
 * solids are a rotating torus and a moving airplane, Sec. 6).  Prescribed rigid motion: the
 * samples of lbm_set_solids are the pose at the current time t0, with rotation centre
 * `center`; at time t0 + tau the centre is center + velocity tau and the samples are rotated
 * by omega tau (radians) about `axis` (Rodrigues).  Step t runs its immersed-boundary stage
 * with the samples at the pose of time t - 1 (the update that follows the previous step's
 * IB stage) and boundary velocity u_b = velocity + omega axis x (X - centre).  At the start
 * of every step the library re-poses the samples in FP64, re-sorts them by base cell (stable
 * radix sort) and rebuilds the band and the spreading lists on the device. */
typedef struct lbm_motion {
    double center[3];            /* rotation centre of the samples' current pose (lattice units) */
    double velocity[3];          /* translation per step                                         */
    double axis[3];              /* rotation axis (any length; zero vector: no rotation)         */
    double omega;                /* angular velocity, radians per step                           */
} lbm_motion;

/* Start (m != NULL) or stop (m = NULL: the samples stay at their last pose) the motion of
 * the solid of lbm_set_solids; lbm_set_solids ends any motion.  Needs a solid.  Replaces
 * the boundary velocities by the rigid-body ones.  A step whose pose would bring a sample
 * within 1e-3 of the domain's faces (the sphere of radius max |X0 - centre| about the
 * centre) returns LBM_EINVAL before running.  After this call lbm_adjoint returns
 * LBM_EINVAL (static solids only).  Errors: LBM_EINVAL, LBM_ESTATE (no solid), LBM_ENOMEM. */
int lbm_set_motion(lbm_ctx *h, const lbm_motion *m);

/* Current sample positions (of the last step's IB stage), count*3 floats in the caller's
 * order of lbm_set_solids (host or device pointer). */
int lbm_solid_samples(lbm_ctx *h, float *X);

/* Torque on the solid from the last step: sum_s (X_s - c) x (-g_s) in FP64 about c = center,
 * or about the motion's current centre when center is NULL (the origin without motion). */
int lbm_solid_torque(lbm_ctx *h, const double center[3], double torque[3]);

/* ---- Smoke tracers (Sec. 6: smoke particles traced on the GPU and their density projected
 * onto a uniform volume grid for rendering; the paper prints no formulas, so the readings
 * are stated here).  Positions are in lattice units, node (i, j, k) at (i, j, k).
 *
 * While tracers exist, every lbm_step also writes the velocity field of the step (FP32,
 * 12 bytes per cell) and then moves each tracer by the explicit midpoint rule with dt = 1:
 * x_mid = x + u(x)/2, x' = x + u(x_mid), u the trilinear interpolation of the step's
 * Guo-shifted velocity (periodic axes wrap; along a non-periodic axis of n nodes the base
 * node is min(floor(x), n-2)).  Periodic coordinates are wrapped into [0, n) after each
 * stage.  A tracer whose midpoint or end point leaves [0, n-1] along a non-periodic axis is
 * re-injected at lo + (hi - lo) U, U_a = (SplitMix64(seed, ((t-1) P + i) 3 + a) >> 40) 2^-24
 * (t the 1-based step, P the tracer count, i the tracer's index): smoke injected
 * continuously at a fixed tracer count. */
typedef struct lbm_emitter {
    double lo[3], hi[3];         /* re-injection box [lo, hi) in lattice units               */
    unsigned long long seed;     /* SplitMix64 seed of the re-injection positions            */
} lbm_emitter;

/* Set (count > 0) or remove (count = 0) the tracers.  X: host or device pointer to count*3
 * floats (x, y, z per tracer), each inside the domain ([0, n) along periodic axes, [0, n-1]
 * along the others); non-periodic axes need n >= 2.  em: the re-injection box, inside the
 * same domain (lo <= hi); required unless every axis is periodic.  Allocates about
 * 50 bytes per tracer and 12 bytes per cell on the device; count < 2^28.  The library keeps
 * the tracers in its own (spatially sorted) order; lbm_tracers returns them in the caller's
 * order.  Tracers are not part of lbm_save checkpoints.
 * Errors: LBM_EINVAL (bad position, box or count; X or em NULL), LBM_ENOMEM. */
int lbm_set_tracers(lbm_ctx *h, const float *X, long long count, const lbm_emitter *em);

/* Number of tracers. */
long long lbm_tracer_count(const lbm_ctx *h);

/* Copy the tracer positions to X (host or device, count*3 floats as in lbm_set_tracers). */
int lbm_tracers(lbm_ctx *h, float *X);

/* Voxels of the density grid of spacing s (integer >= 1, voxel j at coordinate j s): n/s
 * along a periodic axis (n divisible by s, else LBM_EINVAL), ceil((n-1)/s) + 1 along a
 * non-periodic one.  dims = {gx, gy, gz}. */
int lbm_tracer_dims(const lbm_ctx *h, int s, int dims[3]);

/* Density projection: every tracer adds unit mass to the 8 voxels around x/s with the
 * trilinear (cloud-in-cell) weights (periodic axes wrap; along a non-periodic axis the base
 * voxel is min(floor(x/s), g-2)).  out: host or device, gx*gy*gz floats, x fastest.  The
 * tracers are sorted by base voxel (stable radix sort) and every voxel sums the runs of its
 * eight lower neighbours in FP64 in a fixed order, so the result is deterministic.
 * Works with zero tracers (all zeros).  Errors: LBM_EINVAL (s, out NULL, grid >= 2^31
 * voxels), LBM_ENOMEM (workspace: 4 bytes per voxel, 8 with a host out). */
int lbm_tracer_density(lbm_ctx *h, int s, float *out);

/* Replace the 16 inflow-profile coefficients a_mn (layout of lbm_config.inflow_coef) of a
 * context whose -x face is an inlet; takes effect from the next step (lbm_step, lbm_adjoint).
 * Errors: LBM_EINVAL (no inlet, NULL or non-finite coef), LBM_ENOMEM. */
int lbm_set_inflow(lbm_ctx *h, const double coef[16]);

/* Which kernel runs the main range of a step with 16-bit storage (LBM_STORE_F16 / _BF16), the
 * method's collision and nx even.  bulk = 0 (the default): one node pair per thread, each thread
 * loading its 27 pair values itself.  bulk = 1 (used when nx % 8 == 0): a persistent kernel in
 * which one thread of each CTA issues tiled tensor copies (cp.async.bulk.tensor over a 4-D map
 * (x, y, z, direction plane) of the population array, completion counted on an mbarrier) of a
 * 240-node row tile's 27 source segments into a three-stage shared-memory ring, two tiles ahead of
 * the threads that collide the node pairs from there; every wait for a copy is bounded (about a
 * second of SM clocks), and a wait that runs out makes the next lbm_synchronize or lbm_check return
 * LBM_ETIMEOUT.  Both give bit-identical results (the same values in the same FP32 arithmetic); on
 * GB300 the first is faster (the second keeps 4 warps per CTA in step with its tiles).  bulk = 2
 * is a self-test of the bounded wait: the second kernel with every barrier waiting for 16 bytes
 * that no copy delivers, so every wait runs out (about a second), no tile is updated and the next
 * lbm_synchronize or lbm_check returns LBM_ETIMEOUT; the state is invalid afterwards (call
 * lbm_set_state or lbm_load).  Takes effect from the next step.  Errors: LBM_EINVAL for NULL h or
 * bulk outside 0..2. */
int lbm_set_pair_kernel(lbm_ctx *h, int bulk);

/* Number of band nodes (nodes within the 2x2x2 stencil of a sample) of the solid. */
long long lbm_band_size(const lbm_ctx *h);

/* Number of solid samples S of the last lbm_set_solids (0 without a solid; -1 for NULL h):
 * the length of the per-sample outputs of lbm_ib_forces, lbm_solid_samples and the position
 * gradient of lbm_adjoint (3 S values each). */
long long lbm_solid_count(const lbm_ctx *h);

/* Grid size of the context: dims = {nx, ny, nz}.  LBM_EINVAL for NULL arguments. */
int lbm_dims(const lbm_ctx *h, int dims[3]);

/* Allocation-free FP64 sum of per-sample forces: out[a] = sum_s g[3*s + a] (the paper has
 * no counterpart; this is a service for callers that cannot call cudaMalloc at the point
 * where they need the sum, e.g. code running while allocation is forbidden or a memory
 * pool is locked).  g: device pointer to count*3 floats in the layout of lbm_ib_forces;
 * out: device pointer to 3 doubles, written on cuda_stream (NULL = legacy stream).
 * No cudaMalloc, cudaFree or allocating library call is made: the partial sums live in a
 * fixed 48 KiB __device__ array that every GPU loading the library holds until exit.
 * The first call on a device looks up that array's address (cudaGetSymbolAddress) and keeps
 * it; make that first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) after it in the same process.  All calls on a device share the array, so
 * calls that overlap on the GPU race; serialise them.  count may be 0 (out = 0);
 * count > LBM_STATIC_MAX_SAMPLES, a NULL out, or a NULL g with count > 0 give LBM_EINVAL.
 * A CUDA error already pending on the calling thread gives LBM_ECUDA without a launch and is
 * left pending; LBM_ECUDA is otherwise a failure of this call's own launches. */
#define LBM_STATIC_MAX_SAMPLES (2048LL * 256LL * 64LL)
int lbm_sum_forces_static(const float *g, long long count, double *out, void *cuda_stream);

/* Message of the last error on h (or of the last failed lbm_create when h is NULL). */
const char *lbm_last_error(const lbm_ctx *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
