/*
 * lbm.h -- C-ABI of the GB300 (sm_103a) half-range finite-difference lattice
 * Boltzmann library (liblbm.so).
 *
 * Method: Ghiroldi & Gibelli, "A finite-difference lattice Boltzmann approach for
 * gas microflows" (arXiv:1308.0692).  The library marches the discrete,
 * linearised BGKW equation (Eq. 1) on a half-range (or full-range) Gauss-Hermite
 * velocity set (Table 1, tensor product in 2-D) with Maxwell diffuse walls
 * (Eqs. 8-9), using the paper's fully discrete scheme: first-order time
 * splitting, first-order upwind transport, explicit Euler relaxation.
 *
 * Conventions shared by every call:
 *   - Every function returns an lbm_status; nothing is thrown or aborted across
 *     the ABI.  On failure lbm_last_error() (thread-local) describes the cause.
 *   - Opaque objects (lbm_vset, lbm_sim) are owned by the library: free them with
 *     lbm_vset_destroy / lbm_destroy.  Host arrays are owned by the caller.
 *   - Host field arrays are FP64, row-major [ny][nx] (cell index c = y*nx + x).
 *     Distribution arrays are structure-of-arrays [n][ny][nx] (index a*ncells + c)
 *     of the perturbation h_a = (f_a - w_a) / u_ref, u_ref = max(|u_bottom|,|u_top|)
 *     (1 when both are zero).
 *   - Device work is enqueued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  lbm_step is asynchronous;
 *     lbm_residual, lbm_moments, lbm_face_flux and lbm_get_state synchronise that
 *     stream.
 *   - Units are those of Eq. (1): lengths in units of l (plate gap / cavity side),
 *     velocities in units of sqrt(R T0), densities in units of the reference.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,       /* invalid argument (sizes, Kn <= 0, CFL, NULL pointers, ...) */
    LBM_ENOMEM = 2,       /* device or host allocation failed, or caller buffer too small */
    LBM_ECUDA = 3,        /* a CUDA runtime call failed */
    LBM_ENONFINITE = 4,   /* a reduction met a NaN or Inf */
    LBM_ETIMEOUT = 5,     /* a bounded device-side wait gave up */
    LBM_EUNSUPPORTED = 6  /* valid request with no kernel (e.g. a velocity-set size) */
} lbm_status;

typedef enum { LBM_HALF_RANGE_GH = 0, LBM_FULL_RANGE_GH = 1 } lbm_vset_kind;
typedef enum { LBM_COUETTE = 0, LBM_CAVITY = 1 } lbm_geometry;
typedef enum { LBM_FP64 = 0, LBM_FP32_PERTURB = 1 } lbm_precision;

typedef struct lbm_vset lbm_vset;
typedef struct lbm_sim lbm_sim;

/* One boundary-value problem (the two flows of the paper's examples).
 *   geom      LBM_COUETTE: nx columns periodic in x, ny cells between plates at
 *             y = 0 (speed u_bottom along x) and y = 1 (speed u_top); square cells
 *             of side 1/ny.  LBM_CAVITY: unit square, nx x ny cells, diffuse walls
 *             on all faces, bottom moving at u_bottom, top (the lid) at u_top,
 *             side walls at rest.
 *   kn        Knudsen number of Eq. (1), > 0; +inf switches collisions off.
 *   cfl       dt = cfl / (max|xi_x|/dx + max|xi_y|/dy), the x term dropped for a single
 *             periodic Couette column, then dt <= kn.  0 < cfl <= 1.
 *   prec      LBM_FP64: FP64 storage and arithmetic.  LBM_FP32_PERTURB: FP32 storage
 *             and arithmetic of h; FP64 wall sums and reductions.
 *   residual_every  the relative residual ||h^{n+1}-h^n|| / ||h^{n+1}|| is evaluated
 *             on every step whose index (counted from 1 since lbm_init) is a multiple
 *             of it (>= 1); lbm_residual returns the latest one. */
typedef struct {
    int geom;
    int nx, ny;
    double kn;
    double u_bottom, u_top;
    double cfl;
    int prec;
    int residual_every;
} lbm_problem;

/* Build the 2-D tensor-product velocity set (Table 1 and the paragraph after it).
 *   kind LBM_HALF_RANGE_GH: n = N Gauss nodes per half-axis of the weight
 *        exp(-xi^2/2)/sqrt(2 pi) on [0, inf), mirrored; M = 2N nodes per axis, M^2
 *        velocities (N = 2: D2Q^h_16, N = 4: D2Q^h_64, N = 6: D2Q^h_144).  1 <= N <= 8.
 *   kind LBM_FULL_RANGE_GH: n = M Gauss-Hermite nodes per axis on the whole line
 *        (M = 3: the standard D2Q9).  2 <= M <= 16.
 * Computed on the host in double-double arithmetic and rounded to FP64.
 * Velocity a = iy*M + ix has xi = (node[ix], node[iy]), weight wt[ix]*wt[iy];
 * nodes ascending.  *out receives a new object (free with lbm_vset_destroy). */
lbm_status lbm_make_velocity_set(int kind, int n, lbm_vset **out);

/* Query a velocity set.  *n_vel = M^2, *m = M.  Arrays, when non-NULL, receive
 * xi_x[n_vel], xi_y[n_vel], w[n_vel] (caller-sized). */
lbm_status lbm_vset_query(const lbm_vset *vs, int *n_vel, int *m, double *xi_x, double *xi_y,
                          double *w);
void lbm_vset_destroy(lbm_vset *vs);

/* Device bytes a simulation of this problem needs when the caller provides the memory. */
lbm_status lbm_sim_bytes(const lbm_vset *vs, const lbm_problem *prob, size_t *bytes);

/* Create a simulation (Eqs. 1, 5-9 on the grid of `prob`).
 *   init_h      host FP64 [n][ny][nx] initial perturbation, or NULL for the cold start
 *               h = 0 (f_a = w_a: rho = 1, u = 0).
 *   device_buf  caller-owned device memory of at least lbm_sim_bytes() bytes, 256-byte
 *               aligned, which must outlive the simulation; NULL = the library allocates
 *               (and frees in lbm_destroy).
 *   stream      cudaStream_t on which all device work of this simulation is ordered.
 * Returns LBM_EUNSUPPORTED for a velocity-set size without a compiled kernel
 * (supported: M in {3, 4, 6, 8, 12}). */
lbm_status lbm_init(const lbm_vset *vs, const lbm_problem *prob, const double *init_h,
                    void *device_buf, size_t buf_bytes, void *stream, lbm_sim **out);
void lbm_destroy(lbm_sim *sim);

/* Coefficients the simulation uses: time step dt, relaxation factor omega = dt/Kn,
 * reference speed u_ref (any pointer may be NULL). */
lbm_status lbm_coeffs(const lbm_sim *sim, double *dt, double *omega, double *u_ref);

/* Advance nsteps >= 0 time steps (asynchronous, stream-ordered).  Each step is one
 * fused pass: upwind transport with wall ghosts (Eqs. 8-9), moments (Eqs. 6-7),
 * relaxation towards w_a (rho + xi_a . j) (Eqs. 1, 5). */
lbm_status lbm_step(lbm_sim *sim, long nsteps);

/* Result of lbm_solve. */
typedef struct {
    long steps;             /* time steps of the march (FP32: of the FP32 march) */
    long correction_steps;  /* FP32 refinement: steps of all correction marches */
    int sweeps;             /* FP32 refinement: defect-correction sweeps applied */
    double residual;        /* last per-step residual of the march */
    double defect;          /* FP32 with refinement: ||M(h) - h|| / ||M(h)|| of the final
                               state, one step M evaluated in FP64; otherwise = residual */
} lbm_solve_info;

/* March to the steady state: whole residual intervals (residual_every steps) until the
 * residual drops below tol or max_steps steps were taken (synchronises once per interval).
 * Any march also stops when its residual has not improved by 1 % over 20 consecutive
 * checks (the FP32 rounding floor of the per-step change, about 1e-8 of ||h|| on a 128^2
 * cavity, lies above a 1e-8 target).  FP32 simulations may apply refine_sweeps
 * mixed-precision refinement sweeps: the march then stops at max(tol, 5e-8), and each sweep
 * takes the defect D = M(h) - h of the stored FP32 state under one FP64 step, marches the
 * correction delta <- L(delta) + D of the homogeneous problem (walls without driving) in
 * FP32 until its per-step change is below refine_tol * ||h|| (refine_tol <= 0: 0.1 * tol),
 * and adds h += delta; sweeps stop once the FP64 defect ||D|| / ||M(h)|| -- the FP64
 * march's residual evaluated on the refined state -- is below tol, or when it stops halving
 * (FP32 rounding floor).  This removes the bias of the FP32 fixed
 * point (the FP32 operator's rounding amplified by the conditioning of the slow modes),
 * which plain FP32 storage cannot.  refine_sweeps must be 0 for FP64 simulations. */
lbm_status lbm_solve(lbm_sim *sim, double tol, long max_steps, int refine_sweeps, double refine_tol,
                     lbm_solve_info *info);

/* Time splitting of transport and relaxation.  LBM_SPLIT_LIE (default; the paper's
 * first-order splitting): transport then relaxation, the stored state is h^n.
 * LBM_SPLIT_STRANG (symmetric second-order splitting, an extension the paper points to):
 * relaxation over dt/2, transport over dt, relaxation over dt/2 (explicit Euler half steps).
 * The library stores g^n = R(dt/2) h^n, whose step is transport then one relaxation with
 * the factor (1 - omega/2)^2 (two half relaxations share their equilibrium, which
 * relaxation does not change); lbm_get_state/lbm_state_device/the residual and the face
 * fluxes refer to g, lbm_moments and lbm_set_moments to the physical h (rho and u are the
 * same; the non-equilibrium part of P is scaled by 1/(1 - omega/2)).  Call before the
 * first step (else LBM_EINVAL). */
#define LBM_SPLIT_LIE 0
#define LBM_SPLIT_STRANG 1
/* as LBM_SPLIT_STRANG with exact half relaxations g -> E + exp(-omega/2) (g - E): the stored
 * state then advances with the factor exp(-omega), and P converts with exp(omega/2) */
#define LBM_SPLIT_STRANG_EXACT 2
lbm_status lbm_set_splitting(lbm_sim *sim, int scheme);
lbm_status lbm_get_splitting(const lbm_sim *sim, int *scheme);

/* Transport order.  1 (default): the paper's first-order upwind.  2: a second-order
 * finite-volume transport (an extension of the paper's scheme): per direction the face flux
 * nu [h_u + (1 - nu)/2 (h_u - h_uu)] (h_u, h_uu the two upwind cells; first order where h_uu
 * lies beyond a wall; nu times the wall-emitted population across a wall face), wall
 * densities (Eq. 9) balancing that outflow.  With LBM_SPLIT_STRANG_EXACT the steady state
 * converges at second order in the grid spacing.  Order 2 has its own kernels: the segment
 * kernel (load path 0; warps per segment 1 for M <= 4 and FP32 M = 6, 2 for FP64 M = 6 and
 * FP32 M = 8, 4 for FP64 M = 8, 4 or 6 for M = 12 and 12 for FP64 M = 12; 6 by default for
 * M = 12) and, on FP32 cavities with nx a multiple of 64, nx >= 128 and ny >= 12, the
 * second-order column march on the strip-tiled state (load path 8: ring of five row slots,
 * 9: four slots with bulk asynchronous stores; M = 12 with 6 warps, M = 8 with 4), which
 * marches the cells two or more cells from every wall while the segment kernel takes rows
 * 0, 1, ny-2, ny-1 and the 32-cell side segments; any other load path returns
 * LBM_EUNSUPPORTED.  Order 2 has no FP32 refinement (lbm_solve with refine_sweeps > 0
 * returns LBM_EUNSUPPORTED), and lbm_face_flux and the wall shear of lbm_moments use its
 * face values.  Setting the order returns the sim to load path 0 and the planar layout.
 * Call before the first step. */
lbm_status lbm_set_transport(lbm_sim *sim, int order);
lbm_status lbm_get_transport(const lbm_sim *sim, int *order);

/* Kernel variant: the number of warps that share one 32-cell segment (1, 2, 3, 4 or 6
 * dividing M; each warp owns M/warps velocity rows), and the load path of the wall-free
 * segments: 0 registers, 1 registers with all loads issued ahead of the arithmetic,
 * 2 TMA (bulk asynchronous copies into shared memory, FP32 cavities with nx and the cell
 * count multiples of 4 and the planar state layout; M = 8 or 12), 3 as 2 with the wall
 * segments in the same launch,
 * 4 to 7 the interior as a column march (persistent blocks march 64-cell strips row by
 * row, each row's lines copied once by TMA into a ring of 4 (path 4), 5 (path 5) or 2
 * (path 6, two blocks per SM) row slots; path 7 is path 4 with each row's relaxation
 * deferred until after the next row's transport, its moments exchanged through mbarrier
 * phases instead of a block barrier (steps without the residual); FP32 cavities with nx a
 * multiple of 64, nx >= 128, ny >= 10; M = 12 with 6 or 12 warps (6 only for paths 6 and
 * 7), M = 8 with 2 or 4 warps (path 5)),
 * 8 the column march of path 4 on a strip-tiled state, 9 the same with the stores too as
 * bulk asynchronous copies from shared memory (M = 12 with 6 warps, M = 8 with 4, M = 4 with 2): choosing
 * path 8 or 9 moves the current state into that layout (lbm_state_tiling), where one
 * row of a 64-cell strip, all velocities, is one contiguous stretch of memory, so that a
 * warp copies its lines of a row with one bulk copy; any other path moves it back to the
 * planar layout.  Host transfers (lbm_get_state, lbm_set_state and their _f32 forms, lbm_set_moments,
 * lbm_warm_start) and the diagnostics stay planar on the host side; lbm_solve's refinement
 * sweeps run on the planar layout and return the state to the tiled one.
 * It changes speed, not results beyond rounding order.
 * lbm_init picks a default; lbm_set_variant returns LBM_EUNSUPPORTED for a combination
 * without a compiled kernel.  Used by the autotuner.  Call between steps only. */
lbm_status lbm_set_variant(lbm_sim *sim, int warps_per_segment, int load_path);
lbm_status lbm_get_variant(const lbm_sim *sim, int *warps_per_segment, int *load_path);

/* Latest relative residual r and the step count at which it was evaluated
 * (synchronises).  LBM_ENONFINITE if the state contains NaN/Inf. */
lbm_status lbm_residual(lbm_sim *sim, double *r, long *step);

/* Macroscopic fields of the current state, Eq. (1) units, linearised about rho = 1:
 *   rho = 1 + u_ref sum h, u = u_ref sum xi h / rho, P_ij = delta_ij + u_ref sum xi_i xi_j h.
 * Each output is host FP64 [ny][nx] or NULL (with pxx, pxy and pyy all NULL their sums are
 * not formed; a strip-tiled FP32 state is read through its tiles in place, the wall shear
 * from a planar copy in the other state buffer).  wall_shear (NULL or double[4]) receives
 * the mean tangential momentum flux through the bottom, top, left and right walls
 * (the drag the gas exerts; left/right are 0 for Couette).  Synchronises. */
lbm_status lbm_moments(lbm_sim *sim, double *rho, double *ux, double *uy, double *pxx,
                       double *pxy, double *pyy, double *wall_shear);

/* Momentum flux through the cell faces, u_ref sum xi_x xi_y h_upwind, with the wall
 * ghost as upwind value on a wall face.  flux_y (NULL or host [ny+1][nx]): horizontal
 * faces, row j between cells j-1 and j (j = 0 bottom wall, j = ny top wall).  flux_x
 * (NULL or host [ny][nx+1], cavity only): vertical faces.  Synchronises. */
lbm_status lbm_face_flux(lbm_sim *sim, double *flux_y, double *flux_x);

/* Copy the current state to / from host FP64 [n][ny][nx].  get synchronises. */
lbm_status lbm_get_state(lbm_sim *sim, double *h);
lbm_status lbm_set_state(lbm_sim *sim, const double *h);
/* The same with host FP32 [n][ny][nx] (not in the paper).  For an LBM_FP32_PERTURB
 * simulation these move the stored values themselves, half the bytes of the FP64 calls, and
 * lbm_set_state_f32(sim, x) leaves the state lbm_set_state(sim, y) leaves for any y that
 * rounds to x.  For an LBM_FP64 simulation get rounds to nearest and set widens exactly.
 * Both synchronise the simulation's stream.  Buffers are the caller's (pinned memory gives
 * the full host-device copy rate). */
lbm_status lbm_get_state_f32(lbm_sim *sim, float *h);
lbm_status lbm_set_state_f32(lbm_sim *sim, const float *h);

/* Replace the current state by the one with the given moments per cell: moments is host
 * FP64 [6][ny][nx] = rho, u_x, u_y, P_xx, P_xy, P_yy in Eq. (1) units (what lbm_moments
 * returns).  The populations are the second-order Hermite expansion about the rest
 * equilibrium, h_a = w_a [rho' + xi_a . j' + 1/2 sum_ij (P'_ij - rho' delta_ij)(xi_i xi_j -
 * delta_ij)], rho' = (rho - 1)/u_ref, j' = rho u / u_ref, P' = (P - I)/u_ref, whose moments
 * are the given ones on velocity sets exact to degree 4 (half-range N >= 3, full-range
 * M >= 3).  The initial condition in moment form; lbm_init's init_h is the full state.
 * Synchronises. */
lbm_status lbm_set_moments(lbm_sim *sim, const double *moments);

/* Device pointer of the current state (FP64 or FP32 elements per the precision) and
 * the step counter.  The pointer changes after every step (double buffering).  In the
 * planar layout [a][y][x] the value of velocity a at cell (x, y) is at element
 * a * plane_pitch + y * row_pitch + x (lbm_state_layout: plane_pitch = nx ny, row_pitch =
 * nx); lbm_state_layout returns LBM_EUNSUPPORTED while the state is strip-tiled (load path
 * 8 or 9).  Host arrays of the ABI (lbm_init, lbm_get_state, lbm_set_state) are planar. */
lbm_status lbm_state_device(lbm_sim *sim, void **ptr, long *step);
lbm_status lbm_state_layout(const lbm_sim *sim, long *plane_pitch, long *row_pitch);
/* The strip-tiled layout of load paths 8 and 9 (all outputs 0 while the state is planar): tiles of
 * tile_width = 64 cells in x, tile t holding x in [64 t - x_shift, 64 t - x_shift + 64)
 * with x_shift = 32 (so that the column march's 64-cell strips are whole tiles), the value
 * of velocity a at cell (x, y) at element
 *   ((x + x_shift) / 64) * tile_pitch + y * row_pitch + a * 64 + (x + x_shift) % 64,
 * row_pitch = 64 n, tile_pitch = ny row_pitch.  The buffer holds nx / 64 + 1 tiles; the
 * positions outside the grid are padding.  Not in the paper: a memory layout for the
 * march's access pattern. */
lbm_status lbm_state_tiling(const lbm_sim *sim, int *tile_width, int *x_shift, long *tile_pitch,
                            long *row_pitch);

/* Squared norms of device vectors, FP64 accumulation (the residual reduction):
 *   out[0] = sum (a_i - b_i)^2, out[1] = sum a_i^2, i < count; b may be NULL (then
 *   out[0] = out[1]).
 *   prec      element type of a and b (LBM_FP64 or LBM_FP32_PERTURB: float).
 *   scratch   device memory of at least lbm_norms_scratch_bytes(count) bytes for the
 *             per-block partial sums (caller-owned).
 *   out       device pointer to 2 doubles (written stream-ordered).
 * Deterministic (fixed summation order).  Not part of the paper: the residual
 * definition the march uses, exported for callers that keep their own buffers. */
lbm_status lbm_norms_scratch_bytes(long count, size_t *bytes);
lbm_status lbm_norms(const void *a, const void *b, long count, int prec, void *scratch,
                     size_t scratch_bytes, double *out, void *stream);

/* lbm_norms without any allocation, for callers that cannot allocate device memory
 * at all -- e.g. code that runs while someone else's CUDA graph is being captured,
 * hosts without a device allocator, or latency-critical paths where cudaMalloc may
 * block -- and cannot pass a scratch buffer either.  The paper has no counterpart.
 *   a, b, count, prec, out, stream  as for lbm_norms (b may be NULL).
 * The per-block partial sums live in a 512 KiB array inside the library that every GPU
 * loading the library holds until process exit; count is therefore limited to
 * 67,108,864 elements (one partial pair per 2048 elements): larger counts return
 * LBM_EINVAL.  Each call whose stream is not being captured looks up the array's device
 * address with the call's device current (so a cudaDeviceReset in between is harmless);
 * a call made while its stream is being captured reuses the address found by the last
 * uncaptured call on that device, so make one uncaptured call on each device before any
 * stream capture that includes this call, and again after a cudaDeviceReset.  count = 0
 * writes out = {0, 0}.  Calls share the array: each call writes every slot it reads, so nothing has to be
 * cleared, but calls that overlap on the GPU (other streams, concurrent graph launches)
 * race on it and must be serialised by the caller.  Never calls cudaMalloc or cudaFree.
 * Results equal lbm_norms up to summation order. */
lbm_status lbm_norms_noalloc(const void *a, const void *b, long count, int prec, double *out,
                             void *stream);

/* FP64 fused multiply-adds per second this GPU sustains (8 SMs' worth of blocks per SM, eight
 * independent FMA chains of `iters` steps per thread, timed with CUDA events on `stream`;
 * synchronises).  Not in the paper: the measured ceiling of the FP64 march, which is bound by
 * the FP64 pipe rather than by memory on this GPU.  LBM_EINVAL for iters < 1. */
lbm_status lbm_probe_fp64_rate(long iters, double *fma_per_s, void *stream);

/* ---- Batched sweeps: many independent instances in one persistent launch ----
 * A batch holds independent problems (Couette channels and cavities of any size, Kn and
 * wall speeds; one shared velocity set, precision and residual_every) packed in one
 * device allocation.  lbm_batch_advance enqueues one cooperative, persistent kernel
 * launch (captured into a CUDA graph on a non-default stream) that advances every
 * unconverged instance by nsteps time steps: work items are (instance, 32-cell segment)
 * pairs taken round-robin by the resident blocks, a grid-wide barrier with a bounded wait
 * separates steps, and every residual_every steps instances whose residual is below tol
 * are frozen (their items are skipped from then on); with tol > 0 so is an instance whose
 * residual has not improved by 1 % over 20 checks (the FP32 rounding floor: its status
 * then reports it as stalled, not converged, with the residual it reached).  Supported: FP32 perturbation
 * storage with 4 or 8 nodes per axis (D2Q^h_16 / D2Q16, D2Q^h_64); wall densities are
 * summed in FP64, the ghosts evaluated in FP32.  A barrier that gives up makes the next
 * lbm_batch_poll return LBM_ETIMEOUT. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_bytes(const lbm_vset *vs, const lbm_problem *insts, int count, size_t *bytes);
lbm_status lbm_batch_init(const lbm_vset *vs, const lbm_problem *insts, int count, void *device_buf,
                          size_t buf_bytes, void *stream, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);
/* Schedule: warps per segment (1, 2 or 4), resident blocks per SM (<= 0: the occupancy
 * maximum), item order (0 given order, 1 largest instance first, 2 segments interleaved
 * across instances).  Chosen by the autotuner; any choice gives the same results. */
lbm_status lbm_batch_set_schedule(lbm_batch *b, int warps_per_segment, int blocks_per_sm, int order);
lbm_status lbm_batch_get_schedule(const lbm_batch *b, int *warps_per_segment, int *blocks_per_sm,
                                  int *order, int *grid);
/* Column march of cavity instances (on by default where the velocity set has 4 or 8 nodes
 * per axis): cavity instances are advanced by a second persistent kernel in which a group
 * of warps marches a 32-column strip up a chunk of rows, each warp owning one or two
 * velocity rows, streaming the rows through a shared-memory ring (each value read once per
 * step) and forming the wall densities inline; Couette instances always take the segment
 * kernel.  on = 0 puts every instance on the segment kernel (same results up to FP32
 * summation order).  Cavity states are stored strip-tiled (32-cell strips, velocity pairs
 * interleaved; host transfers keep the planar order).  The warp groups take items of all
 * the launch's steps from one counter, and an item waits only for its own instance's
 * previous step (no grid-wide barrier between steps).  rows_per_chunk: rows of one march
 * item (>= 4), or 0 to let the library plan it at every rebuild of the item lists (about
 * 1.3 items per resident warp group and step with eight or more live cavities, 1.7 with
 * fewer, 4 to 128 rows).  warps_per_item: M (one velocity row per warp), M / 2 (two rows
 * per warp, two items per block of eight warps), for M = 8 also 2 (four rows per warp, four
 * items per block); 0 the default: four rows per warp for M = 8, two for M = 4.
 * lbm_batch_get_march reports the switch, the rows per chunk in use, the number of march
 * items per step, the march kernel's grid and its warps per item (outputs may be NULL). */
lbm_status lbm_batch_set_march(lbm_batch *b, int on, int rows_per_chunk, int warps_per_item);
lbm_status lbm_batch_get_march(const lbm_batch *b, int *on, int *rows_per_chunk, int *items, int *grid,
                               int *warps_per_item);
lbm_status lbm_batch_advance(lbm_batch *b, int nsteps, double tol);     /* asynchronous */
/* Limit of every bounded wait (the segment kernel's grid barrier, the column march's wait
 * for an instance's previous step and for its row copies), in SM clock cycles (default 4e9,
 * about 2 s).  Exposed so that tests can make a wait give up and check the error path. */
lbm_status lbm_batch_set_timeout(lbm_batch *b, long long cycles);
lbm_status lbm_batch_poll(lbm_batch *b, int *n_active, long *step);     /* synchronises */
/* Back to the cold start (h = 0 everywhere, step 0, nothing converged). */
lbm_status lbm_batch_reset(lbm_batch *b);
/* Autotuner: times steps_per_trial steps of every schedule (warps per segment x blocks
 * per SM x item order) on this batch, keeps the fastest and resets the batch to the cold
 * start.  Outputs may be NULL. */
lbm_status lbm_batch_tune(lbm_batch *b, int steps_per_trial, int *best_warps_per_segment,
                          int *best_blocks_per_sm, int *best_order, double *best_ms_per_step);
/* Instance i: steps taken (the step at which it was frozen, or all steps so far), last
 * residual, and converged = 1 only if it was frozen because its residual fell below the
 * tolerance (0 while it marches, and 0 if the stagnation rule froze it above the
 * tolerance: see lbm_batch_stalled).  Synchronises the batch's stream. */
lbm_status lbm_batch_status(lbm_batch *b, int i, long *steps, double *residual, int *converged);
/* stalled = 1 if instance i was frozen by the stagnation rule (no 1 % improvement of its
 * residual over 20 checks, the FP32 rounding floor) with its residual still at or above the
 * tolerance; lbm_batch_status gives that residual and the step.  Not in the paper. */
lbm_status lbm_batch_stalled(lbm_batch *b, int i, int *stalled);
lbm_status lbm_batch_get_state(lbm_batch *b, int i, double *h);
/* Initial state of instance i before the first lbm_batch_advance: host FP64 [n][ny][nx],
 * or the warm start of a cavity instance from the network (see lbm_warm_start). */
lbm_status lbm_batch_set_state(lbm_batch *b, int i, const double *h);
typedef struct lbm_mlp lbm_mlp;
lbm_status lbm_batch_warm_start(lbm_batch *b, int i, lbm_mlp *mlp, double kn, double u_w);
/* Moments of instance i (as lbm_moments) into device FP64 [6][ny][nx]: rho, ux, uy, pxx,
 * pxy, pyy.  Stream-ordered. */
lbm_status lbm_batch_moments(lbm_batch *b, int i, double *out_dev);
/* Mixed-precision refinement of every instance, all instances at once (the batched form of
 * lbm_solve's refinement sweeps; not in the paper).  Each sweep evaluates the defect
 * D = M(h) - h of the stored FP32 state under one step in FP64 arithmetic (Eqs. 1, 5-9 of
 * the linearised scheme), marches the corrections delta <- L(delta) + D of the homogeneous
 * problems (walls without driving) in FP32 in one persistent launch per 5 * residual_every
 * steps until each instance's per-step change is below refine_tol * ||M(h)|| (refine_tol
 * <= 0: 0.1 * tol; an instance whose change has not improved by 1 % over 20 residual checks,
 * or that reached max_steps correction steps, stops there), and adds h += delta.  An
 * instance takes sweeps until its FP64 defect ||D|| / ||M(h)|| is below tol, the defect
 * stops halving (the FP32 rounding floor), or max_sweeps.  Refines the state each instance
 * stands at (its convergence step, or the current step) in place; step counts and
 * convergence flags are unchanged.  info (may be NULL) receives one record per instance.
 * The first call allocates a workspace of four state copies (freed with the batch).
 * Synchronises the batch's stream. */
typedef struct {
    long correction_steps;   /* correction steps over all sweeps */
    int sweeps;              /* sweeps taken (0: the defect was already below tol) */
    double defect;           /* final FP64 defect ||M(h) - h|| / ||M(h)|| */
} lbm_batch_refine_info;
lbm_status lbm_batch_refine(lbm_batch *b, double tol, int max_sweeps, double refine_tol, long max_steps,
                            lbm_batch_refine_info *info);

/* ---- Hybrid half-range / full-range coupling (not in the paper's algorithms) ----
 * The coupling the paper's conclusion proposes (half-range sets accurate in the Knudsen
 * layers, the full-range set with 2^d times fewer velocities they reduce to in the bulk),
 * in this project's reading, for the Couette channel (geom LBM_COUETTE, one periodic
 * column, nx = 1, plates u_bottom at y = 0 and u_top at y = 1) and the lid-driven cavity
 * (LBM_CAVITY, nx x ny, bottom u_bottom, lid u_top, sides at rest) of Eqs. 1, 5-9: cells
 * within `layer` cells of a wall carry D2Q^h_{(2N)^2}, the others the full-range
 * Gauss-Hermite set of N nodes per axis (D2Q_{N^2}).  Across an interface the upwind
 * values are the tensor Hermite projection (order N - 1) of the neighbour's distribution;
 * the flux through an interface face is the half-range one (both half-spaces summed in the
 * half-range set), and the full-range cell's transported state is corrected by
 * (lam + mu_x xi_x + mu_y xi_y) w so that its mass and momentum exchange through that face
 * equals it: mass and momentum are conserved exactly, a state at rest stays at rest.
 * layer = 0 is the full-range march, a layer beyond the half width the half-range march.
 * dt = cfl / (max|xi_x|/dx + max|xi_y|/dy) over the sets present (the x term dropped for the
 * column), dt <= Kn.  FP64 by default; lbm_hybrid_set_precision(hb, LBM_FP32_PERTURB) switches
 * the march to FP32 storage and arithmetic (the interface projections and face moments
 * too, with FP32 tables) with the mixed-precision refinement of lbm_hybrid_refine (below).  State layout
 * (host FP64, packed): cell after cell
 * (c = y * nx + x), each cell's values in its own set's order a = iy * M + ix (M = 2N
 * half-range, N full-range); lbm_hybrid_query reports the total.  2 <= N <= 6.
 * lbm_hybrid_step is stream-ordered; lbm_hybrid_residual returns ||h^{n+1} - h^n|| /
 * ||h^{n+1}|| of the last step taken (synchronises); lbm_hybrid_solve marches in blocks of
 * `every` steps until that residual is below tol or max_steps (in FP32 also once it has not
 * improved by 1 % over 20 checks: the FP32 rounding floor); lbm_hybrid_velocity writes
 * (u_x, u_y) per cell (host [ny][nx]); lbm_hybrid_face_flux (column only) the x-momentum
 * flux through the ny + 1 faces (host [ny + 1], interface faces in the half-range
 * evaluation; LBM_EUNSUPPORTED for the cavity). */
typedef struct lbm_hybrid lbm_hybrid;
lbm_status lbm_hybrid_init(int geom, int n_half, int nx, int ny, double kn, double u_bottom, double u_top, int layer,
                           double cfl, void *stream, lbm_hybrid **out);
void lbm_hybrid_destroy(lbm_hybrid *hb);
lbm_status lbm_hybrid_query(const lbm_hybrid *hb, long *unknowns, int *half_range_cells, double *dt);
lbm_status lbm_hybrid_set_state(lbm_hybrid *hb, const double *h);
lbm_status lbm_hybrid_get_state(lbm_hybrid *hb, double *h);
lbm_status lbm_hybrid_step(lbm_hybrid *hb, long nsteps);
lbm_status lbm_hybrid_residual(lbm_hybrid *hb, double *r);
lbm_status lbm_hybrid_solve(lbm_hybrid *hb, double tol, long max_steps, int every, long *steps, double *r);
lbm_status lbm_hybrid_velocity(lbm_hybrid *hb, double *ux, double *uy);
lbm_status lbm_hybrid_face_flux(lbm_hybrid *hb, double *pxy);
/* Precision of the hybrid march: LBM_FP64 (default) or LBM_FP32_PERTURB; the current state is
 * converted.  Allocates the FP32 buffers on first use.  Not in the paper. */
lbm_status lbm_hybrid_set_precision(lbm_hybrid *hb, int prec);
/* Mixed-precision refinement of the FP32 hybrid state (the hybrid form of lbm_solve's
 * sweeps; not in the paper): D = M64(h) - h by one FP64 hybrid step of the stored state,
 * the correction march delta <- L(delta) + D of the homogeneous problem (walls without
 * driving) in FP32 from delta = 0, residual checks every `every` steps, until its per-step
 * change is below refine_tol ||M64(h)|| (refine_tol <= 0: 0.1 tol) or has not improved by
 * 1 % over 20 checks or max_steps, then h += delta; at most max_sweeps sweeps, stopping once
 * the FP64 defect ||D|| / ||M64(h)|| is below tol or stops halving.  Outputs the correction
 * steps taken and that defect (may be NULL).  LBM_EINVAL for an FP64 hybrid. */
lbm_status lbm_hybrid_refine(lbm_hybrid *hb, double tol, int max_sweeps, double refine_tol, long max_steps, int every,
                             long *correction_steps, double *defect);

/* ---- Learned warm start (not in the paper) ----
 * A coordinate MLP 4 -> 256 -> 256 -> 256 -> 6 with exact-erf GELU maps the features
 * (2x-1, 2y-1, (2 log10 Kn + 1)/3, (u_w - 0.0125)/0.0075) of a cavity cell to the
 * normalised moments ((rho-1)/u_w, u_x/u_w, u_y/u_w, (P_xx-1)/u_w, P_xy/u_w, (P_yy-1)/u_w).
 * BF16 weights and activations enter hand-written tensor-core GEMMs that accumulate in
 * FP32; FP32 master weights are updated by Adam (beta 0.9/0.999, eps 1e-8).
 * Parameters are flattened as W1 [256][4], b1 [256], W2 [256][256], b2, W3, b3,
 * W4 [6][256], b4 [6] (row-major).  All x/t/y pointers are device FP32, row-major
 * [M][4] / [M][6]; work is ordered on the MLP's stream. */
lbm_status lbm_mlp_param_count(long *count);
lbm_status lbm_mlp_create(int max_batch, unsigned long long seed, void *stream, lbm_mlp **out);
void lbm_mlp_destroy(lbm_mlp *mlp);
lbm_status lbm_mlp_set_params(lbm_mlp *mlp, const float *flat_host);   /* resets Adam */
lbm_status lbm_mlp_get_params(lbm_mlp *mlp, float *flat_host);
lbm_status lbm_mlp_forward(lbm_mlp *mlp, const float *x_dev, int m, float *y_dev);
/* Mean-squared-error loss and its gradient (flattened like the parameters, host FP32;
 * grad may be NULL) without updating; synchronises. */
lbm_status lbm_mlp_loss_grad(lbm_mlp *mlp, const float *x_dev, const float *t_dev, int m, double *loss,
                             float *grad_flat_host);
/* One Adam step on a batch; loss (may be NULL) is the batch loss before the update. */
lbm_status lbm_mlp_train_step(lbm_mlp *mlp, const float *x_dev, const float *t_dev, int m, float lr,
                              double *loss);
/* Features of every cell of an nx x ny cavity (device [nx*ny][4]). */
lbm_status lbm_mlp_features(lbm_mlp *mlp, int nx, int ny, double kn, double u_w, float *x_dev);
/* Replace the state of a cavity simulation by the second-order Hermite expansion of the
 * moments the network predicts for (kn, u_w):
 *   h_a = w_a [rho' + xi_a . j' + 1/2 sum_ij (P'_ij - rho' delta_ij)(xi_i xi_j - delta_ij)].
 * The network's max_batch must cover nx*ny.  Synchronises. */
lbm_status lbm_warm_start(lbm_sim *sim, lbm_mlp *mlp, double kn, double u_w);

/* Work split of the column-march interior kernel (load paths 4, 5) for an nx x ny cavity
 * run by `blocks` persistent blocks (host logic only, no GPU needed): the number of 64-cell
 * strips and of row chunks; items = strips x chunks.  LBM_EUNSUPPORTED where the march does
 * not apply (nx not a multiple of 64, nx < 128 or ny < 10). */
lbm_status lbm_march_plan(int nx, int ny, int blocks, int *strips, int *chunks);

/* A non-blocking CUDA stream owned by the caller, created and destroyed through the library
 * (no counterpart in the paper: plumbing for callers whose stream sources are pooled, so
 * that concurrent simulations driven from several host threads get streams of their own).
 * lbm_stream_create writes the cudaStream_t to *stream; lbm_stream_destroy synchronises
 * and destroys it (NULL is ignored). */
lbm_status lbm_stream_create(void **stream);
void lbm_stream_destroy(void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
