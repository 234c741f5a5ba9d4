/*
 * gamer_hydro.h -- C ABI of the GB300-native relaxing-TVD patch-group hydro
 * path of GAMER (Schive, Tsai & Chiueh, arXiv 0907.3390).
 *
 * The library advances the ideal-gas Euler equations (Sec. 2.2, Eqs.
 * MassConserve..EOS) on a hierarchy of 8^3-cell patches grouped into 16^3
 * patch groups (Sec. 3.1) with the second-order relaxing TVD scheme
 * (Eqs. 1DEuler..FullstepValue), dimensional splitting xyz / zyx (Sec. 2.2),
 * ghost zones of 3 cells from same-level neighbours or Min-Mod
 * interpolation from the level one coarser (Sec. 2.2, Sec. 3.1),
 * restriction and coarse-fine flux correction (Sec. 2.1, step 3), the CFL
 * time step (Sec. 3.4, Eq. CFL) and conservation / positivity checks.
 *
 * Conventions shared by every call
 * --------------------------------
 * - All field, map and flux pointers inside gamer_level_t are DEVICE
 *   pointers owned by the caller; the structs themselves are host memory.
 * - Conserved state of a level: u[5][8*n_groups][8][8][8], variables
 *   (rho, rho vx, rho vy, rho vz, e), x fastest; patch group g owns patches
 *   8g..8g+7, local patch index (pz*2 + py)*2 + px.  Element type float for
 *   GAMER_FP32 handles, double for GAMER_FP64 handles.  u and u_out must be
 *   16-byte aligned (GAMER_ERR_ARG otherwise).
 * - nbr[n_groups][26]: neighbour d = (dz+1)*9 + (dy+1)*3 + (dx+1) with 13
 *   (the group itself) skipped: a same-level group index >= 0, -1 when that
 *   region exists only on the coarser level (ghosts interpolated), -2 for
 *   an outflow (zero-gradient) domain face.  Periodic wrap is encoded by the
 *   map.  Ghost cells never come from two levels down (proper nesting,
 *   Sec. 2.1); maps violating it are rejected with GAMER_ERR_MAP.
 * - parent[n_groups]: patch index on the level below (NULL on level 0).
 * - child[8*n_groups]: patch-group index on the level above, or -1 (NULL on
 *   the finest level).
 * - Every call returns GAMER_OK (0) or a negative status; the message of the
 *   last failure is available from gamer_hydro_last_error().  No call
 *   throws.  Asynchronous calls are ordered on the handle's stream.
 */
#ifndef GAMER_HYDRO_H
#define GAMER_HYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GAMER_OK = 0,
    GAMER_ERR_ARG = -1,          /* bad argument                              */
    GAMER_ERR_CUDA = -2,         /* a CUDA call failed                        */
    GAMER_ERR_MAP = -3,          /* inconsistent neighbour / parent / child map */
    GAMER_ERR_TIMEOUT = -4,      /* a bounded device-side wait gave up        */
    GAMER_ERR_UNSUPPORTED = -5,  /* valid request the library does not offer */
    GAMER_ERR_STATE = -6         /* call out of order for the handle          */
};

enum { GAMER_LIMITER_VANLEER = 0, GAMER_LIMITER_MINMOD = 1 };
enum { GAMER_FP32 = 0, GAMER_FP64 = 1 };
enum { GAMER_TIME_STEPS_UNIFORM = 0, GAMER_TIME_STEPS_INDIVIDUAL = 1 };
enum { GAMER_FLAG_DENSITY_GRADIENT = 0, GAMER_FLAG_PRESSURE_GRADIENT = 1, GAMER_FLAG_DENSITY = 2 };

typedef struct gamer_hydro_s *gamer_hydro_t;

/* One refinement level.  face_flux is optional: [n_groups][3][3][5][16][16]
 * of the element type (net interface fluxes on the interior-relative planes
 * 0, 8, 16 of each axis, for the 16x16 interior rows), every plane written
 * by each step; when NULL and the hierarchy has more than one level the
 * handle allocates its own, into which FP32 steps may write only what the
 * coarse-fine fix-ups read. */
typedef struct {
    int32_t n_groups;
    int32_t reserved;
    double dh;                 /* cell width of this level                   */
    const void *u;             /* in:  pre-step state                        */
    void *u_out;               /* out: post-step state, must not alias u     */
    const int32_t *nbr;
    const int32_t *parent;
    const int32_t *child;
    void *face_flux;
} gamer_level_t;

/* A hierarchy snapshot.  `version` identifies the maps (nbr, parent,
 * child, n_groups, dh): the library validates them and builds its work
 * lists once per version, so a caller that changes a map must change the
 * version.  The u / u_out pointers may change on every call. */
typedef struct {
    int32_t n_levels;
    int32_t reserved;
    const gamer_level_t *levels;   /* host array of n_levels entries */
    uint64_t version;
} gamer_hierarchy_t;

/* Create a solver handle.
 * gamma: ratio of specific heats, > 1 (Eq. EOS).
 * limiter: GAMER_LIMITER_VANLEER (Eq. vanLeer) or GAMER_LIMITER_MINMOD.
 * ghost_width: must be 3, the ghost depth the seven-point stencil needs
 *   (Sec. 2.2); other values give GAMER_ERR_UNSUPPORTED.
 * precision: GAMER_FP32 (batched persistent kernel, FP64 reductions) or
 *   GAMER_FP64 (plain path, one thread block per patch group).
 * The handle uses the current CUDA device and the legacy default stream
 * until gamer_hydro_set_stream().  Every level's sweep parity starts at 0
 * (xyz).  Errors: GAMER_ERR_ARG (gamma <= 1, unknown limiter/precision,
 * out == NULL), GAMER_ERR_CUDA. */
int gamer_hydro_create(double gamma, int limiter, int ghost_width, int precision,
                       gamer_hydro_t *out);

/* Release the handle and everything it allocated.  NULL is accepted. */
int gamer_hydro_destroy(gamer_hydro_t h);

/* Stream (a cudaStream_t, or NULL for the legacy stream) on which every
 * later call of this handle is ordered. */
int gamer_hydro_set_stream(gamer_hydro_t h, void *cuda_stream);

/* Sweep order of the next advance of `level`: parity 0 = forward xyz,
 * 1 = backward zyx (Sec. 2.2: forward then backward sweep with one dt).
 * Every advance of a level flips its parity; these two calls let a caller
 * read it for a checkpoint and set it on resume.  level in [0, 32). */
int gamer_hydro_set_parity(gamer_hydro_t h, int level, int parity);
int gamer_hydro_get_parity(gamer_hydro_t h, int level, int *parity);

/* Time step from Eq. CFL: dt = cfl * min over levels of
 * dh_l / max over cells of (c_s + max(|vx|,|vy|,|vz|)), read from every
 * level's u.  The per-group maxima and the reduction are exact (max is
 * order-independent); the division is FP64.  Synchronous: waits for the
 * handle's stream and writes *dt_out on the host.  A level whose signal
 * speed is not finite makes *dt_out NaN. */
int gamer_hydro_cfl_dt(gamer_hydro_t h, const gamer_hierarchy_t *H, double cfl,
                       double *dt_out);

/* One sweep set (xyz or zyx by the level's parity) of every patch group of
 * `level` with time step dt (Sec. 3.1): ghost zones gathered on the device
 * (same-level copy, Min-Mod interpolation from levels[level-1].u, outflow
 * clamp), the three sweeps of the relaxing TVD scheme, the 16^3 interior
 * written to levels[level].u_out and, on multi-level hierarchies, the face
 * fluxes.  Asynchronous on the handle's stream.  The coarse data read is
 * levels[level-1].u, so every level of a step must be advanced before any
 * level is corrected (gamer_hydro_fixup) or swapped by the caller. */
int gamer_hydro_advance(gamer_hydro_t h, const gamer_hierarchy_t *H, int level,
                        double dt);

/* Coarse-fine correction of `level` from level+1 (Sec. 2.1, step 3): in
 * levels[level].u_out, covered cells become the mean of their 8 children
 * from levels[level+1].u_out, and leaf cells next to a refined neighbour
 * patch get the coarse face flux replaced by the mean of the 4 fine face
 * fluxes (Berger-Colella).  dt must be the dt of the advance.  Call for
 * level = n_levels-2 down to 0 after all advances.  Asynchronous. */
int gamer_hydro_fixup(gamer_hydro_t h, const gamer_hierarchy_t *H, int level,
                      double dt);

/* Whole step of the level evolution with a uniform dt: every level
 * advanced (the FP32 handle uses ONE persistent launch whose device work
 * queue spans the patch groups of all levels), then the fix-ups from the
 * finest level down.  Flips every level's parity (all levels must share
 * it, else GAMER_ERR_STATE).  Asynchronous.  The caller swaps u and u_out
 * of every level afterwards. */
int gamer_hydro_advance_all(gamer_hydro_t h, const gamer_hierarchy_t *H, double dt);

/* One whole step with the time step kept on the device: the sweep sets and
 * fix-ups of gamer_hydro_advance_all with the handle's device dt, then the
 * diagnostics of the new state (per-group exact speed maxima, FP64 leaf
 * sums, bad-cell count; fused into the sweep launch for single-level FP32
 * hierarchies) and the dt of the next step from Eq. CFL with factor cfl.
 * Following the forward/backward sweep pairing of Sec. 2.2 the new dt is
 * taken only when the next step is an xyz step; a zyx step reuses the dt of
 * the xyz step before it.  The first call on a hierarchy version (or after
 * any call that set dt from the host) computes dt from the current state
 * first.  The sequence is captured once per (hierarchy version, u/u_out
 * pointers, parity, cfl) as a CUDA graph and replayed on the handle's
 * stream: no host round trip per step.  For a single-level FP32 hierarchy
 * the graph is one kernel: the CTA of the sweep launch that finishes last
 * reduces the diagnostics, sets the device dt and writes the step result
 * to mapped pinned host memory.  A handle's launches share its work-queue
 * counters, so they must stay ordered on one stream.  Asynchronous; the caller swaps u
 * and u_out afterwards and may read the result with
 * gamer_hydro_step_result. */
int gamer_hydro_step(gamer_hydro_t h, const gamer_hierarchy_t *H, double cfl);

/* A forward and a backward sweep set with one dt (Sec. 2.2): the xyz set
 * and then the zyx set, each as in gamer_hydro_step, the new state back in
 * u (u_out is scratch; the caller does NOT swap).  Every level must be at
 * parity 0 (an xyz set next, else GAMER_ERR_STATE) and is at parity 0
 * again afterwards.  dt comes from the device as in gamer_hydro_step and
 * is taken new from Eq. CFL after the pair.  For a single-level FP32
 * hierarchy the pair is ONE persistent launch: a group's zyx set starts as
 * soon as the xyz results of the group and of its 26 neighbours are
 * published, so the two sets overlap and share one start-up and one tail;
 * waits are bounded (about a second), and a wait that gave up makes
 * gamer_hydro_step_result return GAMER_ERR_TIMEOUT.  Other hierarchies run
 * the two sets as two steps, the diagnostics only after the second (the
 * xyz set keeps dt either way).  Captured as a CUDA graph like
 * gamer_hydro_step.  Asynchronous; results via gamer_hydro_step_result. */
int gamer_hydro_step_pair(gamer_hydro_t h, const gamer_hierarchy_t *H, double cfl);

/* Test hook for the failure path of the fused pair launch: the next
 * gamer_hydro_step_pair on a single-level FP32 hierarchy does not publish
 * the xyz result of patch group `group` (level 0), a mark that nothing else
 * sets.  The zyx items that read it wait until their bound runs out (about
 * a second), later waits give up at once, the launch finishes, and
 * gamer_hydro_step_result returns GAMER_ERR_TIMEOUT; the state that step
 * leaves is not valid, the handle and the CUDA context stay usable.  The
 * hook applies to one call (that call is launched directly, not through a
 * graph); -1 clears it, a group outside the level publishes everything.
 * GAMER_ERR_ARG for group < -1. */
int gamer_hydro_test_withhold(gamer_hydro_t h, int group);

/* FP64 handles: at most n patch groups per kernel launch of a level's
 * sweep set (default 2048; each launch runs one thread block per group).
 * n = 1 gives the plain one-group-per-launch layout of the paper's solver
 * loop (Sec. 3.1 launches N_g groups at a time), the baseline the batched
 * kernels are compared with.  Results do not depend on n.  Waits for the
 * handle's stream and drops its cached graphs.  GAMER_ERR_ARG for n < 1,
 * GAMER_ERR_UNSUPPORTED for FP32 handles (one persistent launch covers
 * every group). */
int gamer_hydro_set_launch_groups(gamer_hydro_t h, int n);

/* Time stepping of multi-level hierarchies (Sec. 2.1).
 * GAMER_TIME_STEPS_UNIFORM (default): one dt for every level, as the paper
 * does with self-gravity.  GAMER_TIME_STEPS_INDIVIDUAL: every level takes
 * two steps of half its parent's dt, as the paper allows for pure
 * hydrodynamics; gamer_hydro_step_pair then advances level 0 by two steps
 * of dt (xyz then zyx) and level l by 2^(l+1) steps of dt / 2^l.  A level's
 * step is its sweep set, then the two steps of the finer level, whose
 * coarse ghosts are interpolated linearly in time between the level's
 * state before and after its sweep set (weight 0, then 1/2), then the
 * level's fix-up (restriction; flux correction against the finer fluxes
 * averaged over the finer level's two steps).  Every level's new state is
 * back in u (no swap).  dt follows Eq. CFL with the factors 2^l:
 * cfl * min_l 2^l dh_l / s_l (also from gamer_hydro_cfl_dt and
 * gamer_hydro_diagnose).  gamer_hydro_step refuses multi-level hierarchies
 * in this mode (GAMER_ERR_UNSUPPORTED); gamer_hydro_advance and
 * gamer_hydro_advance_all keep one dt for every level.  Changing the mode
 * waits for the handle's stream and drops its cached graphs and buffers;
 * the individual mode holds a second face-flux buffer per level. */
int gamer_hydro_set_time_steps(gamer_hydro_t h, int mode);

/* Flag step of the refinement-map rebuild (Sec. 2.1 step 4) on level
 * `level` of H (its u).  A cell is flagged when
 *   GAMER_FLAG_DENSITY_GRADIENT / GAMER_FLAG_PRESSURE_GRADIENT: the largest
 *     relative change of density / pressure across one cell width,
 *     max over x, y, z of |q(+1) - q(-1)| / (2 |q|), reaches threshold
 *     (Eqs. ShockTube_RefineCriterion, BlastWave_RefineCriterion; a
 *     neighbour that only exists on the coarser level counts as the cell
 *     itself, outflow edges as zero gradient);
 *   GAMER_FLAG_DENSITY: rho > threshold;
 * evaluated in the handle's precision (single precision is the paper's
 * GPU precision) in the order of these definitions; the relative change
 * and rho are compared with threshold in FP64.  Every flagged cell
 * has a flag buffer, the cube of 1 + 2 n_buffer cells around it
 * (0 <= n_buffer <= 8); masks (device, [8 n_groups] uint32) receives per
 * patch the bit (dz+1)*9 + (dy+1)*3 + (dx+1) of every patch offset that
 * the buffers of its cells reach (bit 13: the patch itself).  The caller
 * combines the masks into flags and rebuilds the maps (the library's
 * Python side does, in paper_0907_3390_gb300/regrid.py).  Asynchronous. */
int gamer_hydro_flag(gamer_hydro_t h, const gamer_hierarchy_t *H, int level, int criterion, double threshold,
                     int n_buffer, uint32_t *masks);

/* Refinement step: the data of a rebuilt level l+1 whose n_new patch groups
 * have the parent patches parent_new (device, patch indices on level l =
 * `level` of H).  Group i copies group inherit[i] (device, or -1) of the
 * previous state u_old of that level (n_old groups, device, may be NULL if
 * nothing inherits); the others are filled cell by cell by Min-Mod
 * interpolation (R8) from level l's u.  u_new: device [5][8 n_new][8][8][8],
 * 16-byte aligned.  The parents must be properly nested (their 26
 * neighbours on level l exist), else GAMER_ERR_MAP; this is checked on the
 * host, so the call synchronises the device. */
int gamer_hydro_refine_fill(gamer_hydro_t h, const gamer_hierarchy_t *H, int level, int n_new,
                            const int32_t *parent_new, const int32_t *inherit, const void *u_old, int n_old,
                            void *u_new);

/* Red-black SOR Poisson solver of the refined levels (Sec. 2.3, Eqs.
 * DiscretePoisson, Residual, SOR), one patch group per thread block, with
 * no handle.  phi: device [n_groups][18][18][18] (x fastest), the 16^3
 * interior's initial guess inside the Dirichlet ghost layer, which is kept;
 * rho: device [n_groups][16][16][16]; coef = 4 pi G dh^2.  One iteration
 * updates the even interior cells (i + j + k even, interior indices) by
 *   R = (phi(i+1) + phi(j+1) + phi(k+1) + phi(i-1) + phi(j-1) + phi(k-1)
 *        - 6 phi) - coef rho,   phi <- phi + (omega / 6) R
 * and then the odd ones with the updated even values; a group stops after
 * the iteration in which the one-norm of its residuals falls to tol times
 * the one-norm of coef rho (tol = 0: never; the norms are then not
 * formed at all, and otherwise summed in the data's precision per warp),
 * or after max_iter iterations.  iters: device [n_groups] iteration counts, or NULL.
 * precision: GAMER_FP32 or GAMER_FP64 (the data's type; FP64 follows the
 * oracle's order of operations, so with tol = 0 it matches it bit for bit).
 * 0 < omega < 2.  Work runs on cuda_stream (NULL: legacy stream),
 * asynchronously.  The preparation of rho and of the ghost layer
 * (interpolation from the coarser level) and the potential correction of
 * the paper are not part of this call.  Errors: GAMER_ERR_ARG,
 * GAMER_ERR_CUDA; message from gamer_hydro_last_error(NULL). */
int gamer_poisson_sor(int precision, int n_groups, const void *rho, void *phi, double coef, double omega,
                      int max_iter, double tol, int32_t *iters, void *cuda_stream);

/* Gravity operator G of the split scheme (Sec. 2.3): the gravity source
 * terms of Eqs. MomConserve and EnergyConserve, without the flux terms,
 * applied to one level for a time dt, with no handle.  The hydro sweeps and
 * G alternate as xyzGGzyx, the two G of a double step taken as one call
 * with twice the hydro dt.  u: device [5][8 n_groups][8][8][8] (the level
 * storage), updated in place; phi: device [n_groups][18][18][18] (x
 * fastest), each group's potential with one ghost layer (the layout
 * gamer_poisson_sor works on).  Per cell and axis k,
 *   d_k = (phi(-1) - phi(+1)) * (dt / (2 dh))       (3-point difference: g_k dt)
 *   m_k <- m_k + rho d_k
 *   e   <- e + 0.5 (((m_x + m'_x) d_x + (m_y + m'_y) d_y) + (m_z + m'_z) d_z)
 * with m' the new momentum (the exact solution over dt with rho and g
 * fixed: the thermal energy does not change).  precision: GAMER_FP32 or
 * GAMER_FP64 (the type of u and phi; FP64 follows the oracle's order of
 * operations and matches it bit for bit).  dh > 0, dt >= 0, both finite.
 * Work runs on cuda_stream (NULL: legacy stream), asynchronously.  Errors:
 * GAMER_ERR_ARG (checked before any CUDA call), GAMER_ERR_CUDA; message
 * from gamer_hydro_last_error(NULL). */
int gamer_gravity_update(int precision, int n_groups, void *u, const void *phi, double dh, double dt,
                         void *cuda_stream);

/* Inputs of the SOR problems of refined level `level` >= 1 of H (Sec. 2.3):
 * for every patch group of that level, phi_blocks [n][18][18][18] (x
 * fastest; the layout gamer_poisson_sor and gamer_gravity_update take) gets
 * at every cell -- the one-cell ghost layer, which is the Dirichlet
 * boundary, and the 16^3 interior, the initial guess -- the Min-Mod
 * interpolation (as for the coarse-fine ghosts of the hydro step) of
 * phi_c, the potential of level-1 in the level layout [8 n_c][8][8][8];
 * rho_blocks [n][16][16][16] (x fastest) gets the group's density from the
 * level's state u.  All pointers are device memory of the handle's
 * precision.  The maps are validated as for the step (GAMER_ERR_MAP);
 * GAMER_ERR_ARG for level 0 or missing pointers.  Asynchronous, on the
 * handle's stream.  The root level's potential (an FFT solve in the paper)
 * is the caller's. */
int gamer_poisson_prepare(gamer_hydro_t h, const gamer_hierarchy_t *H, int level, const void *phi_c,
                          void *phi_blocks, void *rho_blocks);

/* Result of the last gamer_hydro_step or gamer_hydro_step_pair: the dt it
 * used, the dt the next step will use, the leaf sums of u * dh^3 and the
 * bad-cell count of the new state.  Waits for that step.  Any output
 * pointer may be NULL.  GAMER_ERR_STATE if no step has completed,
 * GAMER_ERR_TIMEOUT if a dependency wait of a pair launch gave up. */
int gamer_hydro_step_result(gamer_hydro_t h, double *dt_used, double *dt_next, double sums[5],
                            int64_t *n_bad);

/* Conservation and positivity check over leaf cells (patches whose child
 * is -1) of every level's u: sums[v] = sum of u_v * dh^3 (FP64,
 * deterministic fixed-order reduction), *n_bad = number of cells with
 * rho <= 0, P <= 0 or a non-finite variable.  Synchronous. */
int gamer_hydro_check(gamer_hydro_t h, const gamer_hierarchy_t *H, double sums[5],
                      int64_t *n_bad);

/* gamer_hydro_cfl_dt and gamer_hydro_check in one pass over the data
 * (either output pointer may be NULL).  Synchronous. */
int gamer_hydro_diagnose(gamer_hydro_t h, const gamer_hierarchy_t *H, double cfl,
                         double *dt_out, double sums[5], int64_t *n_bad);

/* The CFL time step and the conservation / positivity check of
 * gamer_hydro_diagnose, without a handle and without allocating any device
 * memory.  *dt_out is the shared-time-step dt of Eq. CFL, each level
 * limited by its own dh (what gamer_hydro_diagnose returns for a handle in
 * the default shared-time-step mode; a handle with individual time steps
 * scales level l's limit by 2^l instead, so the two differ there).  The paper has no counterpart; this is for callers that cannot
 * call cudaMalloc -- a thread that must not synchronise the device (as
 * cudaMalloc/cudaFree may), code running inside a memory arena that owns
 * all of the GPU's memory, a periodic health check that must not disturb
 * the caller's allocator.
 * The per-group scratch is one fixed array in the library's device memory
 * (3.4 MB, held by every GPU that loads the library until the process
 * exits) covering at most 65536 patch groups summed over levels; larger
 * hierarchies get GAMER_ERR_ARG.  The caller passes the inputs (H: every
 * level's u, n_groups, dh, and child below the finest level) and the host
 * outputs (dt_out, sums, n_bad: any may be NULL); gamma and precision are
 * those of the data.  Work runs on cuda_stream (NULL: legacy stream) and
 * the call waits for it.  Every call looks the scratch address up in the
 * current device's context (cudaGetSymbolAddress, which allocates
 * nothing), so the address stays right after a context reset; the first
 * call on a device may load the library's device code, so make that first
 * call before any stream capture.  All calls in the process share the
 * scratch and each call rewrites every part it reads, so no state carries
 * over; calls that overlap on the GPU (other threads, other streams) race
 * on it and must be serialised by the caller.  Errors: GAMER_ERR_ARG,
 * GAMER_ERR_CUDA; the message is available from
 * gamer_hydro_last_error(NULL) on this thread. */
int gamer_hydro_diagnose_noalloc(double gamma, int precision, const gamer_hierarchy_t *H,
                                 double cfl, void *cuda_stream, double *dt_out, double sums[5],
                                 int64_t *n_bad);

/* Autotuner: times the launch configurations the library offers on the
 * caller's hierarchy and keeps the fastest for the handle.  FP32 handles
 * choose between the pipelined persistent kernel (512 threads: the next
 * work item's ghost slabs gathered by warps idle in sweeps 2 and 3) and the
 * non-pipelined one (256 or 512 threads per patch group), each with one CTA
 * per SM or with a balanced grid (fewer CTAs, same number of rounds); FP64
 * handles choose 128 or 256 threads per patch group.  The timing runs
 * whole steps with dt = 0, so it overwrites every level's u_out and face
 * fluxes but never u.  With cache_path given, a line
 * "<GPU>|<precision>|lim<L>|levels<N>|groups2^<B>=<config>" is looked up
 * first (no timing when found) and appended after a timing.  Synchronous.
 * Captured step graphs are discarded. */
int gamer_hydro_tune(gamer_hydro_t h, const gamer_hierarchy_t *H, const char *cache_path);

/* Human-readable launch configuration of the handle, written into buf
 * (len bytes, NUL-terminated). */
int gamer_hydro_get_config(gamer_hydro_t h, char *buf, int len);

/* Profiling hook: CUDA events (cudaEvent_t, created with timing enabled)
 * that every later advance_all / step records immediately before and after
 * its sweep launches, so the caller can time the dominant kernel with
 * cudaEventElapsedTime.  While events are set, gamer_hydro_step launches
 * its sequence directly instead of replaying a graph (events recorded
 * inside a graph cannot be timed).  Both NULL turns it off.  The events
 * stay owned by the caller and must outlive their use. */
int gamer_hydro_set_profiling(gamer_hydro_t h, void *ev_before, void *ev_after);

/* Message of the last failed call on this handle ("" if none).  With a NULL
 * handle, the message of the last failed handle-free call on this thread
 * (gamer_hydro_create, gamer_hydro_diagnose_noalloc).
 * The string stays valid until the next call on the handle. */
const char *gamer_hydro_last_error(gamer_hydro_t h);

#ifdef __cplusplus
}
#endif
#endif /* GAMER_HYDRO_H */
