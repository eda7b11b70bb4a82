/*
 * mdbs.h -- C-ABI of the GB300 micro-continuum multiphase Darcy-Brinkman-Stokes
 * volume-of-fluid step (Carrillo, Bourg & Soulaine, "A micro-continuum
 * approach for multiphase flow in hybrid-scale porous media", arXiv 2003.08374).
 *
 * One call of mdbs_step advances one or more pressure-velocity time steps of
 * the model of section 2 (Eq. 21: total mass, saturation and momentum
 * equations with the multiscale closures of section 2.3, Eqs. 41-45) by the
 * solution algorithm of section 3.2: explicit flux-corrected saturation update,
 * property update, momentum predictor (Eq. 50), PISO pressure correction
 * (Eqs. 51-53).  Every step runs in CUDA kernels on the current device; there is
 * no CPU path.
 *
 * Grid and layout.  Uniform Cartesian grid, spacing h, nx*ny*nz cells (nz == 1:
 * two-dimensional run, no z faces).  Scalars (porosity, permeability, alpha, p)
 * are cell-centred; velocities live on cell faces (staggered/MAC), so the face
 * velocity times the face area is the conservative volumetric flux.  All host
 * arrays are float64, x fastest:
 *   cells   : nx*ny*nz         index i + nx*(j + ny*k)
 *   x faces : (nx+1)*ny*nz     index i + (nx+1)*(j + ny*k), i in [0, nx]
 *   y faces : nx*(ny+1)*nz     index i + nx*(j + (ny+1)*k)
 *   z faces : nx*ny*(nz+1)     index i + nx*(j + ny*k)  (ignored when nz == 1)
 * Face velocities are positive along +x, +y, +z.
 *
 * Boundaries.  Each of the six sides (x-, x+, y-, y+, z-, z+) is a no-slip
 * wall, an inlet (normal velocity inlet_u into the domain, saturation
 * inlet_alpha, zero normal pressure gradient) or an outlet (p = 0 on the face,
 * zero normal gradient of velocity and saturation).  At least one side must be
 * an outlet, which makes the pressure equation non-singular.
 *
 * Ownership.  The caller owns every host array; the library copies them in and
 * out and keeps no pointer to them.  A simulation owns its device memory until
 * mdbs_destroy.  Calls on one simulation are not thread safe.
 *
 * Errors.  Every int-returning call returns MDBS_OK (0) or a negative code; a
 * message is kept per simulation (mdbs_last_error).  After MDBS_ERR_DIVERGED or
 * MDBS_ERR_CUDA the fields hold the state reached when the error was found; after
 * MDBS_ERR_NOT_CONVERGED every requested step was taken, with the last CG iterate
 * of each solve that stopped at max_cg.
 */
#ifndef MDBS_H
#define MDBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MDBS_OK 0
#define MDBS_ERR_ARG (-1)           /* bad size, pointer, option or field value */
#define MDBS_ERR_OOM (-2)           /* device allocation failed */
#define MDBS_ERR_CUDA (-3)          /* a CUDA call failed */
#define MDBS_ERR_DIVERGED (-4)      /* a non-finite value appeared in the fields */
#define MDBS_ERR_NOT_CONVERGED (-5) /* a pressure solve stopped at max_cg above p_tol (the step was taken) */

#define MDBS_BC_WALL 0
#define MDBS_BC_INLET 1
#define MDBS_BC_OUTLET 2

#define MDBS_BROOKS_COREY 0
#define MDBS_VAN_GENUCHTEN 1

/* Density of porous cells in the momentum equation.  MDBS_RHO_MOBILITY: the
 * mobility-weighted rho* = (rho_l M_l + rho_g M_g) / M of Eq. 45 (main
 * text).  MDBS_RHO_SATURATION: the saturation-weighted rho of Appendix B, with
 * the porous capillary force extended by M^-1 (M_l a_g - M_g a_l)(rho_l - rho_g) g
 * so that the Darcy momentum balance is unchanged (Appendix B shows the two are
 * equivalent). */
#define MDBS_RHO_MOBILITY 0
#define MDBS_RHO_SATURATION 1

#define MDBS_FP64 0        /* FP64 everywhere */
#define MDBS_MIXED 1       /* FP32 multigrid preconditioner inside FP64 flexible CG */
#define MDBS_MIXED_BF16 2  /* as MDBS_MIXED with coarse-level coefficients stored in BF16 */

typedef struct {
  int32_t nx, ny, nz; /* cells per axis; nz == 1 selects a 2-D run */
  double h;           /* cell size [m] */
} mdbs_grid;

/* Fluid pair (Table 1): l = wetting liquid, g = non-wetting phase. */
typedef struct {
  double rho_l, mu_l, rho_g, mu_g; /* densities [kg/m^3], viscosities [Pa s] */
  double sigma;                    /* interfacial tension [N/m] (Eq. 27) */
  double g[3];                     /* gravity [m/s^2] */
} mdbs_fluids;

/* Relative permeability and capillary pressure closures (Appendix A, Table 2). */
typedef struct {
  int32_t kr_model, pc_model;  /* MDBS_BROOKS_COREY or MDBS_VAN_GENUCHTEN */
  double kr_m;                 /* exponent m of the kr model */
  double a_l_irr, a_g_irr;     /* irreducible saturations of the kr effective saturation */
  double pc0, pc_beta, pc_m;   /* entry pressure [Pa], Brooks-Corey beta, Van Genuchten m */
  double a_pc_irr, a_pc_max;   /* bounds of the p_c effective saturation */
  double pc_eps;               /* the p_c effective saturation is clamped to [eps, 1-eps] */
  int32_t porous_density;      /* MDBS_RHO_MOBILITY (default) or MDBS_RHO_SATURATION */
} mdbs_closures;

typedef struct {
  double dt;        /* time step [s] (the first one when cfl > 0) */
  double cfl;       /* > 0: next dt = min(cfl h / max|u_f/phi_f|, 1.2 dt, dt_max) */
  double dt_max;    /* upper bound of the adaptive time step */
  double c_alpha;   /* interface compression coefficient C_alpha (Eq. 22) */
  double p_tol;     /* pressure solve stops at ||b - A p||_2 <= p_tol ||b||_2 */
  int32_t n_corr;   /* PISO correctors per step (section 3.2: at least 2) */
  int32_t mom_sweeps; /* Jacobi sweeps of the momentum predictor */
  int32_t max_cg;   /* CG iteration cap per pressure solve */
  int32_t mg_nu1, mg_nu2;     /* red-black Gauss-Seidel pre/post sweep pairs per level */
  int32_t mg_coarse_sweeps;   /* sweep pairs (forward, then as many backward) on the coarsest level */
  int32_t precision;          /* MDBS_FP64, MDBS_MIXED or MDBS_MIXED_BF16 */
  int32_t bc[6];              /* side types, order x-, x+, y-, y+, z-, z+ */
  double inlet_u;             /* inlet normal velocity into the domain [m/s] */
  double inlet_alpha;         /* inlet saturation */
} mdbs_options;

typedef struct {
  int64_t steps;          /* steps taken since mdbs_set_fields */
  double time;            /* simulated time [s] */
  double dt;              /* time step of the next step [s] */
  int32_t cg_iters[8];    /* CG iterations per corrector of the last step */
  double cg_resid[8];     /* final relative residual per corrector of the last step */
  int64_t cg_iters_total; /* since mdbs_set_fields */
  int32_t not_converged;  /* pressure solves that stopped at max_cg */
  double mass;            /* sum of porosity * alpha * cell volume [m^3] */
  double boundary_in;     /* time-integrated net liquid volume entering through boundaries [m^3] */
  double alpha_min, alpha_max;
  int64_t kernel_launches; /* CUDA kernels this library launched since mdbs_set_fields */
} mdbs_stats;

typedef struct mdbs_sim mdbs_sim;

/*
 * Creates a simulation on the current CUDA device (problem statement of
 * section 2: porosity field, Eqs. 7-8; absolute permeability k0, Eq. 30; fluid
 * pair; contact angle, Eq. 40).
 *   porosity     : host, nx*ny*nz, each in (0, 1]; exactly 1 marks a solid-free cell
 *   permeability : host, nx*ny*nz, k0 [m^2] > 0 where porosity < 1 (ignored elsewhere)
 *   contact_angle_deg : angle through the wetting phase at the free/porous interface
 * Returns MDBS_ERR_ARG for invalid sizes or values, MDBS_ERR_OOM / MDBS_ERR_CUDA on
 * device failure; *out is NULL then.  Velocities and pressure start at zero; call
 * mdbs_set_fields before stepping.
 */
int mdbs_create(const mdbs_grid* grid, const double* porosity, const double* permeability,
                const mdbs_fluids* fluids, double contact_angle_deg, const mdbs_closures* closures,
                const mdbs_options* options, mdbs_sim** out);

/*
 * Sets the state (saturation alpha_l in [0, 1], Eq. 8; face velocities, Eq. 10;
 * pressure, Eq. 9) from host arrays laid out as above; uz may be NULL in 2-D.
 * Wall and inlet face velocities are overwritten by their boundary values.
 * Resets the statistics (the simulated time and the time step, too).
 * MDBS_ERR_ARG if alpha is not finite or lies outside [0, 1] by more than 1e-9 or
 * than the extremes this simulation's own steps reached (transport through a velocity
 * field divergence-free only to the pressure tolerance moves alpha outside [0, 1] by
 * dt |div(A u)| / (phi V) per step; a get_fields / set_fields round trip of such a
 * state is accepted); the check runs on the device and a rejected call leaves the
 * state unchanged.  A non-finite pressure or velocity is copied in and reported:
 * MDBS_ERR_DIVERGED (the state is set; mdbs_step then reports it too).
 */
int mdbs_set_fields(mdbs_sim* sim, const double* alpha, const double* ux, const double* uy,
                    const double* uz, const double* p);

/*
 * Advances n >= 1 time steps (section 3.2).  Runs on the simulation's stream and
 * returns after the last step has finished on the device.  MDBS_ERR_DIVERGED if
 * a non-finite value appears; MDBS_ERR_NOT_CONVERGED if a pressure solve (Eq. 53) of
 * these steps stopped at max_cg with its relative residual above p_tol (the steps
 * were taken; mdbs_stats.not_converged counts such solves since mdbs_set_fields).
 */
int mdbs_step(mdbs_sim* sim, int32_t n);

/*
 * Copies the state -- the unknowns of the model's summary (section 2.2, Eq. 21):
 * saturation alpha_l (Eq. 8), single-field face velocities (Eq. 10) and pressure
 * (Eq. 9) -- to host arrays laid out as above (any pointer may be NULL to skip it;
 * uz is ignored in 2-D).  Waits for the simulation's stream.  MDBS_ERR_CUDA if a copy
 * fails.
 */
int mdbs_get_fields(const mdbs_sim* sim, double* alpha, double* ux, double* uy, double* uz,
                    double* p);

/* Ends a simulation made by mdbs_create (its device memory goes back to cudaFree or to
 * the allocator hook that provided it).  No counterpart in the paper.  Waits for the
 * simulation's work; NULL is accepted.  A simulation still in a batch must leave it
 * (mdbs_batch_remove / mdbs_batch_destroy) first. */
void mdbs_destroy(mdbs_sim* sim);

/* ---------------- batches ---------------- */

/*
 * Many independent simulations advanced together: every phase of the step
 * (saturation update, properties, momentum, each CG iteration and multigrid
 * level) is ONE kernel launch over all member domains, whatever their sizes, and
 * the whole batched step is one CUDA graph.  Each member keeps its own device
 * memory, fields, time step and statistics (mdbs_get_fields / mdbs_get_stats work
 * on members as usual).  Every member's pressure solve stops at its own tolerance:
 * converged members drop out of the remaining CG iterations, which run while any
 * member iterates.  A member's results are identical alone and in any batch.
 *   sims : n >= 1 distinct simulations, each after mdbs_set_fields, with identical
 *          n_corr, mom_sweeps, p_tol, max_cg, multigrid options and precision class
 *          (FP64 or mixed); time steps, grids and physics may differ.
 * While in a batch a member cannot be stepped alone (MDBS_ERR_ARG); destroying the
 * batch releases the members, not their memory.  Member fields may be read or reset
 * between batch steps.
 */
typedef struct mdbs_batch mdbs_batch;
int mdbs_batch_create(mdbs_sim* const* sims, int32_t n, mdbs_batch** out);
/* Membership changes between batch steps (continuous batching): add a simulation
 * that meets mdbs_batch_create's conditions, or remove a member (which becomes a
 * simulation of its own again, fields and statistics intact).  The batch's launch
 * plan and CUDA graph are rebuilt; members' results are unaffected.  A batch keeps
 * at least one member: removing the last one is MDBS_ERR_ARG, as are NULL
 * arguments, a simulation already in a batch (add) or not in this one (remove).
 * On a CUDA error the batch keeps its previous members. */
int mdbs_batch_add(mdbs_batch* batch, mdbs_sim* sim);
int mdbs_batch_remove(mdbs_batch* batch, mdbs_sim* sim);
/* Advances every member n >= 1 steps; MDBS_ERR_DIVERGED names the first diverged member,
 * MDBS_ERR_NOT_CONVERGED (when no member diverged) the first member whose pressure
 * solve stopped at max_cg above p_tol. */
int mdbs_batch_step(mdbs_batch* batch, int32_t n);
/* Runs the batch's kernels on the given cudaStream_t (NULL: legacy default stream). */
int mdbs_batch_set_stream(mdbs_batch* batch, void* cuda_stream);
const char* mdbs_batch_last_error(const mdbs_batch* batch);
void mdbs_batch_destroy(mdbs_batch* batch);

/* ---------------- execution schedule and autotuning ---------------- */

/*
 * How the pressure solver's multigrid kernels are scheduled (no counterpart in the
 * paper: the schedule decides speed only).  Every schedule computes every value
 * with the same arithmetic in the same order, so results are bitwise identical
 * under any schedule; only the time per step changes.
 *   smooth_rows : 1, 2, 4 or 8 rows of 256 cells per CTA work item in the
 *                 finest-level red-black sweeps (fewer rows: more CTAs in flight)
 *   tail_cells  : 0 .. 262144; levels with at most this many cells run, with all
 *                 coarser ones, inside one kernel with tail_ctas CTAs per domain
 *                 (fewer launches, less parallelism)
 *   tail_ctas   : 1, 2, 4 or 8; CTAs of 1024 threads per domain in that kernel (more
 *                 than one: a thread-block cluster synchronised by cluster barriers)
 *   snake       : 0 or 1; 1 alternates the traversal direction of consecutive
 *                 kernels over one level, so each starts on the cache lines the
 *                 previous one touched last
 *   sweep_kz    : 0, 4, 8, 16 or 32; > 0 runs each red-black sweep pair of an FP32
 *                 level (mixed precisions) as ONE fused launch over tiles of 60 x 6
 *                 columns and chunks of sweep_kz planes (every array read once per
 *                 pair); 0, and every FP64 level, runs two half sweeps (then
 *                 smooth_rows applies)
 *   coarse_coop : 0 or 1; 1 runs every level between the finest one and the tail,
 *                 and the tail itself (one CTA per domain; tail_ctas then does not
 *                 apply), in ONE cooperative launch whose phases are separated by
 *                 grid-wide barriers instead of kernel boundaries (with sweep_kz 0 and
 *                 at least one such level; otherwise it has no effect)
 *   vec_sweeps  : 0 or 1; 1 runs the half sweeps of every level whose n_x is a
 *                 multiple of 4 (FP64) or 8 (FP32), with FP32 or FP64 coefficients,
 *                 with each thread updating 2 (FP64) or 4 (FP32) consecutive cells of a
 *                 colour run through 16-byte loads and stores (smooth_rows then does not
 *                 apply to those levels)
 * Default: {1, 4096, 0, 0, 1, 0, 0}.  Values outside these sets give MDBS_ERR_ARG.
 */
typedef struct {
  int32_t smooth_rows;
  int32_t tail_cells;
  int32_t snake;
  int32_t sweep_kz;
  int32_t tail_ctas;
  int32_t coarse_coop;
  int32_t vec_sweeps;
} mdbs_tuning;

/* Sets or reads the schedule of a simulation that is not in a batch (the step
 * graph is rebuilt at the next step), or of a batch (default: its first member's). */
int mdbs_set_tuning(mdbs_sim* sim, const mdbs_tuning* tuning);
int mdbs_get_tuning(const mdbs_sim* sim, mdbs_tuning* out);
int mdbs_batch_set_tuning(mdbs_batch* batch, const mdbs_tuning* tuning);
int mdbs_batch_get_tuning(const mdbs_batch* batch, mdbs_tuning* out);

/*
 * Picks the fastest schedule for this simulation (or batch) by timing real steps:
 * starting from the current schedule it tries the alternatives of snake, then of
 * sweep_kz (mixed precisions only), then of smooth_rows (when the half sweeps
 * run), then of coarse_coop, then of (tail_cells, tail_ctas) pairs, then of
 * vec_sweeps (coordinate descent), each for one untimed and
 * trial_steps >= 1 timed steps (CUDA events on the simulation's stream), and keeps
 * a change only when it is faster.  The device state (fields, step scalars) is
 * copied aside first and restored after every trial, so the simulation continues
 * exactly as if mdbs_autotune had not run (the statistics, too).  Needs free device
 * memory for one copy of the simulation's (or every member's) arena:
 * MDBS_ERR_OOM otherwise, with nothing changed.  *chosen (may be NULL) receives
 * the schedule kept; trial_ms (may be NULL, capacity entries) receives the
 * per-step time of every trial in order, and *trials (may be NULL) their count.
 */
int mdbs_autotune(mdbs_sim* sim, int32_t trial_steps, mdbs_tuning* chosen, double* trial_ms, int32_t capacity,
                  int32_t* trials);
int mdbs_batch_autotune(mdbs_batch* batch, int32_t trial_steps, mdbs_tuning* chosen, double* trial_ms,
                        int32_t capacity, int32_t* trials);

/* ---------------- helpers ---------------- */

/* Statistics of the last step (see mdbs_stats). */
int mdbs_get_stats(const mdbs_sim* sim, mdbs_stats* out);

/* Last error message of sim, or of the last failed mdbs_create when sim is NULL. */
const char* mdbs_last_error(const mdbs_sim* sim);

/* Runs the simulation's kernels on the given cudaStream_t (NULL: legacy default
 * stream).  The caller keeps ownership of the stream. */
int mdbs_set_stream(mdbs_sim* sim, void* cuda_stream);

/*
 * Device-memory hook (no counterpart in the paper; lets a host framework such as
 * PyTorch's caching allocator own the memory): when set, the two bulk device
 * allocations of every later mdbs_create -- the simulation's field arena and its
 * pressure-solver block, together mdbs_bytes_required bytes -- come from
 * alloc(bytes, ctx) and go back through free(ptr, ctx) at mdbs_destroy, with the
 * hook that allocated them.  alloc must return device memory aligned to 256 bytes
 * (else mdbs_create fails with MDBS_ERR_ARG) or NULL (MDBS_ERR_OOM).  Both NULL
 * restores cudaMalloc / cudaFree; exactly one NULL is MDBS_ERR_ARG.  Small
 * bookkeeping buffers still use the CUDA runtime.  Process-wide; not thread-safe
 * against concurrent mdbs_create.
 */
typedef void* (*mdbs_alloc_fn)(size_t bytes, void* ctx);
typedef void (*mdbs_free_fn)(void* ptr, void* ctx);
int mdbs_set_allocator(mdbs_alloc_fn alloc, mdbs_free_fn free_fn, void* ctx);

/* Device bytes mdbs_create allocates for this grid and precision. */
size_t mdbs_bytes_required(const mdbs_grid* grid, int32_t precision);

/*
 * Per-kernel device timing (a measurement aid with no counterpart in the paper):
 * when enabled, each launch of kernel only_id (every kernel when only_id is -1)
 * is bracketed by CUDA events on the simulation's stream and the elapsed times
 * are summed per kernel.  Enabling or disabling resets the sums.  Each timed
 * launch adds two event records of host overhead.
 */
int mdbs_profile_enable(mdbs_sim* sim, int32_t enable, int32_t only_id);
/* Number of kernel ids understood by mdbs_profile_read. */
int32_t mdbs_profile_count(void);
/* Name, summed device time [ms] and timed launches of kernel id since enabling
 * (sim may be NULL to read the name only); MDBS_ERR_ARG for an id outside
 * [0, mdbs_profile_count()). */
int mdbs_profile_read(const mdbs_sim* sim, int32_t id, const char** name, double* total_ms, int64_t* launches);

/*
 * Copies an internal device array to host memory for inspection (names: "rho",
 * "mu", "drag", "pc", "cf", "Ml", "Mg", "kappa", "mx", "my", "mz", "Tx", "Ty", "Tz",
 * "Dd", "b", "aL", "Rp", "Rm", "aPx", "aPy", "aPz", "rhs0x", "rhs0y", "rhs0z", "Bx", "By",
 * "Bz", "hbyax", "hbyay", "hbyaz", "FLOx", "FLOy", "FLOz", "AFx", "AFy", "AFz").
 * Returns the element count (and copies min(count, capacity) values when out is
 * not NULL), or MDBS_ERR_ARG for an unknown name.
 */
int64_t mdbs_debug_array(const mdbs_sim* sim, const char* name, double* out, int64_t capacity);

/*
 * Self-test of the bounded device waits (no counterpart in the paper).  Kernels that
 * wait on asynchronous copies (the fused sweeps' mbarriers) give up after one second,
 * record the failure (the step then returns MDBS_ERR_CUDA) and return, so a lost
 * copy never hangs the GPU.  This call runs one such wait on an mbarrier that
 * nothing completes: MDBS_OK when the wait gave up as designed and the device still
 * runs work afterwards; *waited_s receives the device-measured wait (about 1 s).
 * Error text via mdbs_last_error(NULL).
 */
int mdbs_check_bounded_wait(double* waited_s);

/* ---------------- allocation-free helper ---------------- */

/* Capacity of the file-scope scratch array used by mdbs_field_stats_static:
 * per-block partial results, 4 doubles per block (16 KiB in all), held by every
 * device that loads the library until the process exits. */
#define MDBS_STATIC_STATS_MAX_BLOCKS 512
/* Largest cell count mdbs_field_stats_static accepts. */
#define MDBS_STATIC_STATS_MAX_CELLS ((int64_t)2147483647)

/*
 * Field statistics without any device allocation.  The paper has no counterpart:
 * this is a library service.  It computes, on the GPU, the same quantities that
 * mdbs_set_fields / mdbs_step leave in mdbs_stats (liquid volume
 * sum porosity*alpha*cell_volume, alpha min, alpha max) plus the count of
 * non-finite alpha or p values, for fields that the caller already holds on the
 * device.  It exists for callers that must not allocate: code that runs while a
 * CUDA graph is being captured (cudaMalloc is not allowed there), serving loops
 * that cannot afford the device-wide synchronisation an allocation may cause,
 * and embedders that do not let a library own device memory at all.
 *   cells        : number of cells, 1 .. MDBS_STATIC_STATS_MAX_CELLS, else MDBS_ERR_ARG
 *   cell_volume  : h^3 [m^3], > 0
 *   porosity, alpha, p : device arrays of `cells` float64 values (x-fastest)
 *   out          : device array of 4 float64: volume, alpha min, alpha max, non-finite count
 *   stream       : cudaStream_t the two kernels are queued on (NULL: legacy default stream)
 * Allocates nothing: its scratch is a file-scope __device__ array of
 * MDBS_STATIC_STATS_MAX_BLOCKS * 4 doubles shared by every call.  The first call on a
 * device looks up that array's device address with the device current; make that first
 * call before any stream capture.  The address is kept for the life of the process: after
 * cudaDeviceReset on a device it is stale, so do not call this function on that device
 * again.  Calls whose kernels overlap on the GPU race on the shared scratch: serialise
 * them (one stream, or events).  Each call overwrites every scratch value it reads, so
 * nothing needs clearing between calls.  Returns MDBS_OK, MDBS_ERR_ARG or MDBS_ERR_CUDA;
 * the result is ready when the stream reaches it.  A CUDA error already pending on the
 * calling thread (from the caller's earlier work) gives MDBS_ERR_CUDA without a launch
 * and stays pending; an error of this call's own launches is cleared.
 */
int mdbs_field_stats_static(int64_t cells, double cell_volume, const double* porosity, const double* alpha,
                            const double* p, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
