/*
 * best.h -- C ABI of the GB300 collision-integral library (libbest.so).
 *
 * The library evaluates the momentum-resolved collision integral C_a[f](p_i)
 * of the Boltzmann equation (Eq. (1)-(3) of the paper) for n_in -> n_out
 * processes by VEGAS adaptive Monte Carlo in 3(n_total - 2) dimensions
 * (Sec. 2D, App. A), at every grid point of a comoving momentum grid, and
 * steps log f in time with Euler or Heun (Sec. 3C).
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_dev are device pointers owned by the caller (for
 *     example torch tensors' data_ptr()); they must stay valid until the
 *     work queued on `stream` has finished.  Host pointers are read during
 *     the call only.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Every call that takes a stream only enqueues work on
 *     it and returns without synchronising (except where stated), so its
 *     results are valid once the stream reaches that point.
 *   - Distributions are laid out species-major: f[s * n_grid + i] is f of
 *     species s at grid point i, FP64.
 *   - No call throws across the ABI.  Each returns a best_status;
 *     best_last_error() gives a one-line description of the last failure
 *     on that context.  A context must not be used from two host threads
 *     at once.
 */
#ifndef BEST_H
#define BEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BEST_OK = 0,
    BEST_ERR_INVALID = 1,   /* bad argument or configuration */
    BEST_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    BEST_ERR_OOM = 3,       /* device allocation failed */
    BEST_ERR_NUMERIC = 4,   /* non-positive or non-finite f, or a NaN result */
    BEST_ERR_TIMEOUT = 5    /* reserved: no device wait in this library spins */
} best_status;

/* Quantum statistics of a species (Sec. 3A): eta = 0 (MB), +1 (BE), -1 (FD). */
typedef enum { BEST_MB = 0, BEST_BE = 1, BEST_FD = 2 } best_stat;

/* Arithmetic of the per-sample integrand.  Accumulators, VEGAS refinement,
 * spline construction and time stepping are FP64 in both. */
typedef enum { BEST_FP64 = 0, BEST_FP32 = 1 } best_precision;

#define BEST_MAX_LEGS 6        /* n_total <= 6: up to 12 VEGAS dimensions */
#define BEST_MAX_SPECIES 8
#define BEST_MAX_PROCESSES 16
#define BEST_MAX_MASS_KNOTS 8

/* Comoving momentum grid shared by all species (Sec. 3A): n points over
 * [q_min, q_max], logarithmic (log_spaced != 0) or linear; 4 <= n <= 4096. */
typedef struct {
    int32_t n;
    int32_t log_spaced;
    double q_min, q_max;
} best_grid;

/* A species: statistics and mass m(t) (Sec. 3A): m(t) = mass0 + mass1 * t,
 * or, with 2 <= n_mass_knots <= BEST_MAX_MASS_KNOTS, the piecewise-linear
 * interpolation of (mass_t[k], mass_m[k]) (mass_t strictly increasing, masses
 * >= 0), constant before the first and after the last knot; a step in the
 * mass (the paper's example of a phase transition) is a steep ramp between two
 * close knots. */
typedef struct {
    int32_t stat;          /* best_stat */
    int32_t n_mass_knots;  /* 0: the linear law */
    double mass0, mass1;
    double mass_t[BEST_MAX_MASS_KNOTS], mass_m[BEST_MAX_MASS_KNOTS];
} best_species;

/* Matrix element.  The paper registers |M|^2 as a callable of the momenta
 * (Sec. 3A), which a kernel cannot call; here |M|^2 = coupling^2 P(s) with
 * P(s) = me_coef[0] + me_coef[1] s + me_coef[2] s^2 + me_coef[3] s^3 and
 * s = (sum of the initial energies)^2 - |sum of the initial momenta|^2 of the
 * sample (physical units).  All-zero me_coef is rejected; {1, 0, 0, 0} is
 * the constant |M|^2 = coupling^2 of all the paper's examples. */
/* Adaptive stratified sampling (strat = 1; the vegas library's default
 * since 2021, Lepage, J. Comput. Phys. 439 (2021) 110386): a task draws
 * 8 floor(N/8) samples in items of 8; the map's unit cube is cut into M^D
 * hypercubes, M the largest integer with 4 M^D <= items and
 * M^D <= strat_max_hcubes; each hypercube gets m_h >= 1 items (uniform at
 * first), samples uniform inside it; the estimate is the volume-weighted sum
 * of the hypercube means; after each iteration
 * m_h = 1 + floor((J - H) d_h / sum d) with d_h = s_h^strat_beta (s_h the
 * sample standard deviation in h), leftovers one each to the first
 * hypercubes.  The allocation persists like the maps and is checkpointed.
 * The fixed-sample integral of best_collision_vjp / _jvp does not stratify. */
/* A process n_in -> n_out (Sec. 3A, App. D) with constant |M|^2 = coupling^2.
 * species[0 .. n_in-1] are the initial legs, species[n_in .. n_in+n_out-1]
 * the final legs.  neval is the number of samples per VEGAS iteration per
 * task (one task = one grid point, one pinned side, gain or loss); a
 * non-NULL neval_per_point (host array of grid.n entries, copied during
 * best_collision_init) overrides it per grid point.  nitn VEGAS iterations
 * per evaluation, damping alpha, nbins increments per dimension (2..256).
 * The Gaussian of Eq. (11) has width sigma_E (width_mode 0), or the
 * fractional width of App. C, sigma = w (E_in + E_out) / 2 per sample, with
 * w = width fixed (width_mode 1) or adapted after every evaluation
 * (width_mode 2): with r = sqrt(sum err_t^2) / sum |I_t| over the process's
 * tasks, w /= width_factor when r < width_rel_lo, w *= width_factor when
 * r > width_rel_hi, then clamped to [width_min, width_max]; the new w is
 * used from the next evaluation on. */
typedef struct {
    int32_t n_in, n_out;
    int32_t species[BEST_MAX_LEGS];
    double coupling;
    double sigma_E;
    int64_t neval;
    const int64_t* neval_per_point;
    int32_t nitn;
    int32_t nbins;
    double alpha;
    int32_t width_mode;    /* 0: sigma_E; 1: fractional w; 2: fractional, adapted */
    int32_t pad_;
    double width;          /* initial w (modes 1, 2) */
    double width_rel_lo, width_rel_hi, width_factor, width_min, width_max;   /* mode 2 */
    int32_t strat;         /* 1: adaptive stratified sampling (see below) */
    int32_t strat_max_hcubes;   /* 1 .. 2^20 */
    double strat_beta;     /* >= 0 */
    double me_coef[4];     /* |M|^2 = coupling^2 (c0 + c1 s + c2 s^2 + c3 s^3), see below */
    int32_t budget;        /* 1: variance-driven budgets (see below) */
    int32_t sides;         /* side integrals of Eq. (7) evaluated: 0 all; 1 observed leg initial only;
                              2 observed leg final only (e.g. C_3 alone, Sec. 5D) */
    int64_t neval_min, neval_max;   /* budget = 1: bounds of a task's samples per iteration */
} best_process;

/* Variance-driven budgets (budget = 1; the paper reuses each grid point's
 * integrator from step to step, Sec. 3D, and its budget per point need not
 * be uniform): the first evaluation uses the configured budgets (neval or
 * neval_per_point); after every evaluation each of the process's tasks t
 * gets N_t' = lambda v_t with v_t = N_t (err_t / I_t)^2 its relative variance
 * per sample (0 where I_t = 0 or a value is not finite), rounded down to a
 * multiple of 256 and held within [neval_min, neval_max]; lambda is found by
 * 200 bisection steps so that sum_t min(max(lambda v_t, neval_min),
 * neval_max) stays at the sum of the configured budgets of the process's
 * tasks in this context.  All on the device (no host round trip, so the
 * steps stay capturable); the budgets persist like the maps and are
 * checkpointed.  Needs 2 <= neval_min <= neval_max <= 2^31 with
 * neval_max * dim <= 2^33; not combined with strat. */

typedef struct {
    best_grid grid;
    int32_t n_species;
    int32_t n_processes;
    const best_species* species;     /* host array [n_species] */
    const best_process* processes;   /* host array [n_processes] */
    int32_t precision;               /* best_precision */
    int32_t tail_points;             /* grid points in each end fit of Eq. (13), >= 2 */
    uint64_t seed;                   /* Philox key */
    double e_cut;                    /* samples with any E_k < e_cut weigh 0 (App. A) */
    int32_t expansion;               /* 0: a = 1; 1: a(t) = a0 (t / t0)^(1/2) (Sec. 3E) */
    int32_t pad_;
    double a0, t0;
    double eps_dt;                   /* bound on max |dt C/f| of Eq. (16) */
    int32_t point_lo, point_hi;      /* shard: grid points [point_lo, point_hi) only; 0, 0 = all
                                        (see best_step_stage) */
} best_config;

typedef struct best_ctx best_ctx;

/*
 * Builds a context: validates the configuration, enumerates the side
 * integrals and tasks of the identical-particle decomposition (Eq. (7),
 * Eq. (8); roles of App. A), allocates and owns all device state (VEGAS
 * maps, one per task, kept across calls as in Sec. 3D; spline tables;
 * accumulators; the work partition), and picks the launch shape for the
 * current device.  Synchronous.  On failure *out is NULL and the status says
 * why (best_last_error(NULL) describes it).
 */
best_status best_collision_init(const best_config* cfg, best_ctx** out);

/*
 * One collision-integral sweep at time t (host value): C_dev[s*n+i] =
 * C_a(p_i) of Eq. (7) for every species and grid point, err_dev the Monte
 * Carlo standard error (sqrt of sum mult^2 (sigma_gain^2 + sigma_loss^2)).
 * f_dev: [n_species * n_grid] FP64, f > 0.  Runs nitn VEGAS iterations per
 * task, refines every map after every iteration and advances the context's
 * evaluation counter (part of the Philox counter).  err_dev may be NULL.
 */
best_status best_collision_eval(best_ctx* ctx, const double* f_dev, double t,
                                double* C_dev, double* err_dev, void* stream);

/*
 * One log-space Euler step (Eq. (14)) with the step bound of Eq. (16):
 * logf_dev [n_species * n_grid] is updated in place; *t_dev (device FP64)
 * is the current time and advances by the step used; *dt_dev (device FP64)
 * holds the requested step on entry and the step used on return,
 * dt = min(dt_requested, eps_dt / max |C/f|).  C_dev, if not NULL, receives
 * C[f(t)].  No host synchronisation: the call can be captured in a CUDA
 * graph.
 */
best_status best_step_euler(best_ctx* ctx, double* logf_dev, double* t_dev,
                            double* dt_dev, double* C_dev, void* stream);

/*
 * One Heun step (Eq. (15)): k1 = C[f] at t, f* = exp(log f + dt k1/f),
 * k2 = C[f*] at t + dt, log f += dt/2 (k1/f + k2/f*), dt bounded by
 * Eq. (16) from k1.  Arguments as for best_step_euler.
 */
best_status best_step_heun(best_ctx* ctx, double* logf_dev, double* t_dev,
                           double* dt_dev, double* C_dev, void* stream);

/*
 * Sharded runs (the paper's MPI design over grid points, Sec. 3D): each
 * process builds its context with config.point_lo/point_hi, so that it holds
 * only the tasks of its grid points; best_collision_eval writes C and err for
 * those points and zero elsewhere, so the processes' C arrays add up to the
 * full C (an all-reduce sum, or an all-gather of the slices).  Task ids and
 * hence the Philox streams are those of the whole grid: the shards draw
 * exactly the samples a whole-grid context would.  The adaptive width
 * (width_mode 2) needs every task in one context and is rejected in a shard.
 *
 * best_collision_eval_log: best_collision_eval from log f (f = exp(log f)).
 * best_step_stage: one stage of a step from the assembled C, every process
 * applying it to its copy of the whole distribution (same arithmetic as
 * best_step_euler / best_step_heun, Eq. (14)-(16)); all pointers device:
 *   method 0 (Euler), stage 0: k1 = C(f) at t: dt = min(*dt_dev, eps/max|k1/f|),
 *       log f += dt k1/f, *t_dev += dt, *dt_dev = dt.
 *   method 1 (Heun), stage 0: k1 = C(f) at t: dt as above, fstar = exp(log f +
 *       dt k1/f), *dt_dev = dt (t unchanged); evaluate k2 = C(fstar) at t + dt;
 *   method 1, stage 1: log f += dt/2 (k1/f + k2/fstar), *t_dev += dt.
 * logf, k1, k2, fstar: [n_species*n_grid]; asynchronous on `stream`.
 */
best_status best_collision_eval_log(best_ctx* ctx, const double* logf_dev, double t, double* C_dev,
                                    double* err_dev, void* stream);
best_status best_step_stage(best_ctx* ctx, int32_t method, int32_t stage, double* logf_dev, const double* k1_dev,
                            const double* k2_dev, double* fstar_dev, double* t_dev, double* dt_dev, void* stream);

/*
 * n_steps Euler (method 0, Eq. (14)) or Heun (method 1, Eq. (15)) steps
 * replayed from a CUDA graph: the first call (and any call whose logf / t /
 * dt pointers or method differ from the previous one) captures one step on
 * `stream` into a graph owned by the context; every call then launches it
 * n_steps times.  Each step starts from the requested step dt_request
 * (written into *dt_dev inside the graph) and bounds it by Eq. (16); on
 * return *dt_dev holds the step used by the last step.  `stream` must be a
 * created stream (not the legacy or per-thread default stream).  Results
 * are bitwise identical to n_steps calls of best_step_euler / best_step_heun
 * with *dt_dev reset to dt_request before each.
 */
best_status best_evolve(best_ctx* ctx, int32_t method, int32_t n_steps, double* logf_dev,
                        double* t_dev, double* dt_dev, double dt_request, void* stream);

/*
 * Project autotuner of the sample kernel's launch shape: runs one sweep of
 * f_dev at time t with each compiled variant of the sample kernel -- its
 * register budget (2..10 CTAs per SM), threads per CTA (128, 256, 512) and
 * samples a lane evaluates per step (1, or 2 in packed FP32x2 arithmetic);
 * the persistent grid and the work partition follow from the variant's
 * occupancy -- times the sample-kernel launches with CUDA events, keeps the
 * fastest, and restores the VEGAS maps, the per-task scales, the budgets and
 * the evaluation counter, so that the context's later results do not depend
 * on whether it was tuned (beyond summation order in the FP32 path).
 * Synchronous; allocates a temporary copy of the maps.  *ctas_per_sm (may be
 * NULL) receives the chosen budget; best_launch_shape reports the rest.
 */
/* The sample kernel's current launch shape: CTAs per SM of its register
 * budget, threads per CTA and samples per lane per step (any may be NULL). */
best_status best_launch_shape(const best_ctx* ctx, int32_t* ctas_per_sm, int32_t* threads,
                              int32_t* samples_per_lane);

best_status best_autotune(best_ctx* ctx, const double* f_dev, double t, int32_t* ctas_per_sm,
                          void* stream);

/*
 * Vector-Jacobian product of the fixed-sample collision integral (the paper
 * has no gradients; Eq. (3), (7), (12) define the function).  C~ is C of
 * Eq. (7) estimated with one VEGAS iteration per task on the context's
 * current maps and a reserved Philox iteration index, the evaluation counter
 * left unchanged: common random numbers, so repeated calls use identical
 * samples and C~ is a deterministic, piecewise smooth function of f, the
 * masses and the couplings.  For L = sum_{a,i} v[a*n+i] C~_a(p_i) the call
 * writes C~ (C_dev [n_species*n_grid]), dL/df (gf_dev [n_species*n_grid],
 * through the spline and the Eq. (13) tail fits), dL/dm_s (gm_dev
 * [n_species], at the masses m_s(t)) and dL/dcoupling (gcoupling_dev
 * [n_processes]).  Samples are recomputed, not stored.  Maps and the
 * counter are not modified.  Gradient sums use FP64 atomics, so their last
 * bits can vary between calls.
 */
best_status best_collision_vjp(best_ctx* ctx, const double* f_dev, double t, const double* v_dev,
                               double* C_dev, double* gf_dev, double* gm_dev, double* gcoupling_dev,
                               void* stream);

/*
 * Jacobian-vector product of the same fixed-sample collision integral C~ as
 * best_collision_vjp (same maps, reserved Philox iteration index and
 * evaluation counter, so the same samples): writes C~ (C_dev) and
 * JU = (dC~/df) u (JU_dev), both [n_species*n_grid], for a direction u_dev
 * in the grid values f (masses and couplings held fixed).  Forward mode: the
 * tangent of every sample's weight through the spline of u (the spline
 * coefficients are linear in f) and the Eq. (13) tail fits, accumulated per
 * task in FP64 in a fixed order, so repeated calls give identical bits.
 * Device pointers; asynchronous on `stream`; maps and counter untouched.
 */
best_status best_collision_jvp(best_ctx* ctx, const double* f_dev, double t, const double* u_dev,
                               double* C_dev, double* JU_dev, void* stream);

/*
 * One implicit (backward) Euler step in log space, the implicit counterpart
 * of Eq. (14): log f(t+dt) = g solves
 *     R(g) = g - log f(t) - dt C~(e^g) / e^g = 0
 * with C~ the fixed-sample collision integral at time t + dt (masses and
 * a(t) there).  Newton's method; each linear system J_R d = -R is solved by
 * GMRES with at most krylov_dim (1..64) Arnoldi steps, stopped when its
 * residual is below krylov_rtol * ||R||_2; J_R x = x - dt[(J (f x))/f -
 * (C~/f) x] costs one best_collision_jvp launch set per product.  Steps are
 * damped by halving until ||R||_2 decreases.  Stops when ||R||_inf <= tol or
 * after max_newton iterations.  train != 0 first runs one full VEGAS sweep
 * (all iterations, Sec. 3B) at f(t), time t + dt, to adapt the maps (and
 * advances the evaluation counter); train == 0 keeps the current maps.
 * logf_dev [n_species*n_grid] (device) holds log f(t) on entry and, when
 * Newton converged, log f(t+dt) on return; otherwise it is unchanged and the
 * call returns BEST_ERR_NUMERIC.  info (host, may be NULL, 5 doubles):
 * Newton iterations, Krylov products, final ||R||_inf, converged (1/0),
 * step halvings.  Synchronous (the Krylov loop reads residual norms).
 */
best_status best_step_implicit_euler(best_ctx* ctx, double* logf_dev, double t, double dt, int32_t train,
                                     double tol, int32_t max_newton, int32_t krylov_dim, double krylov_rtol,
                                     double* info, void* stream);

/*
 * Checkpoint of a context's evolving state (the paper checkpoints its
 * integrator states with the distributions, Sec. 3F): the VEGAS maps of
 * every task, the per-task accumulation scales, the evaluation counter and
 * the time state (and the variance-driven budgets, when a process has them),
 * behind a header with a hash of the configuration.  With
 * the same distribution values, time and step, a context restored from a
 * state continues bit for bit like the one that saved it.  Both calls are
 * synchronous; buffers are host memory of at least best_state_size bytes.
 * Loading a state saved from a different configuration returns
 * BEST_ERR_INVALID.
 */
int64_t best_state_size(const best_ctx* ctx);
best_status best_save_state(best_ctx* ctx, void* host_buf, int64_t size);
best_status best_load_state(best_ctx* ctx, const void* host_buf, int64_t size);

/*
 * Number and energy densities of every species at time t, the conservation
 * diagnostics of a thermalisation run (Sec. 5C): n_s = Int q^2 f dq /
 * (2 pi^2 a^3) and rho_s = Int q^2 E(q/a) f dq / (2 pi^2 a^3) over the grid
 * range on the not-a-knot spline of f (unclamped, no tails), 4-point
 * Gauss-Legendre per interval, FP64.  f_dev [n_species*n_grid], n_dev and
 * rho_dev [n_species]: device pointers; asynchronous on `stream`.  Rebuilds
 * the context's spline tables and time state (the next evaluation or step
 * rebuilds them again).
 */
best_status best_moments(best_ctx* ctx, const double* f_dev, double t, double* n_dev, double* rho_dev,
                         void* stream);

/*
 * Stratification of task t (host outputs, each may be NULL): strata per
 * dimension *M, hypercubes *H (0: the task is not stratified) and, when m is
 * not NULL and *H > 0, the items per hypercube m[0 .. H) that the next
 * iteration uses (synchronous).
 */
best_status best_get_strata(best_ctx* ctx, int32_t task, int32_t* M, int32_t* H, int32_t* m);

/*
 * Fractional Gaussian widths (App. C), one per process, as used by the next
 * evaluation: w[p] (0 for width_mode 0) and rel[p], the relative error r of
 * the last evaluation that updated it (0 before any).  Either pointer may be
 * NULL; host arrays of n_processes.  best_set_widths overrides w for the
 * processes with width_mode != 0 (each value must be > 0; synchronous).
 * The widths are part of the state saved by best_save_state.
 */
best_status best_get_widths(best_ctx* ctx, double* w, double* rel);
best_status best_set_widths(best_ctx* ctx, const double* w);

/* The species' masses m_s(t) at time t (Sec. 3A), by the formula the
 * kernels use (equal to theirs up to rounding): m (caller-owned host array of
 * n_species) receives them.  No device work.  BEST_ERR_INVALID when ctx or m is NULL or t is
 * not finite. */
best_status best_species_masses(const best_ctx* ctx, double t, double* m);

/* Context geometry. */
int32_t best_num_tasks(const best_ctx* ctx);
int32_t best_num_side_integrals(const best_ctx* ctx);

/* Samples per VEGAS iteration of every task (host array [n_tasks], in the
 * order of best_get_task_results) that the next sweep will use: the
 * configured budgets, or the variance-driven ones set after the last sweep.
 * Synchronises `stream`. */
best_status best_get_budgets(best_ctx* ctx, int64_t* neval, void* stream);

/* The work partition of VEGAS iteration `iteration` as the next sweep will
 * use it (built on the host, or rebuilt on the device after variance-driven
 * budgets changed): groups[t] (caller-owned host array [n_tasks]) receives
 * the number of sample groups the iteration's segments of task t cover, 0
 * for a task not active in that iteration, or -1 when its segments do not
 * tile [0, groups) exactly (a gap, an overlap or an out-of-order segment).
 * A sample group is the samples of one Philox block set: 2 (FP64) or 4
 * (FP32) uniforms per block shared over D-dimensional samples, so a task of
 * N samples has ceil(N / G) groups (for stratified tasks, whole items of 8
 * samples).  Synchronises the device.  BEST_ERR_INVALID when ctx or groups
 * is NULL or the iteration is out of range. */
best_status best_partition_groups(best_ctx* ctx, int32_t iteration, int64_t* groups);

/* The chunk bounds of the dynamic work partition of one VEGAS iteration
 * (host arithmetic only, no device access; the sample kernel's CTAs take the
 * chunks in order from an atomic counter).  `cost`: the iteration's
 * estimated cost in the partition's units (per sample group, its samples x
 * (dimensions + 6)); `grid`: the persistent grid's CTAs.  *chunks receives
 * the chunk count, 16 x grid; bounds (caller-owned host array of n int64,
 * n >= *chunks + 1) receives the chunk starts: bounds[0] = 0, bounds[*chunks]
 * = cost, non-decreasing.  With cost >= 16 x grid x 98304 (98304: 8192
 * samples of a 2 -> 2 task) the chunks come in 8 stages of 2 x grid equal
 * chunks, the stages covering 1/2, 1/4, ... of the cost and the last one the
 * remainder; with less, max(grid, cost / 98304) equal chunks and empty ones
 * after them.  BEST_ERR_INVALID when cost < 0, grid < 1, chunks is NULL, or
 * bounds is NULL or too short (*chunks is set first, so a call with n = 0
 * asks for the count). */
best_status best_chunk_bounds(int64_t cost, int32_t grid, int64_t* bounds, int32_t n, int32_t* chunks);

/* Integrand evaluations of one sweep: in VEGAS iteration `iteration` (one
 * launch of the sample kernel), or in all iterations when iteration < 0.
 * With variance-driven budgets these are the next sweep's budgets as the
 * device holds them (the call then synchronises the device; -1 on a CUDA
 * error). */
int64_t best_sweep_samples(const best_ctx* ctx, int32_t iteration);

/*
 * Copies per-task results of the last completed sweep to host memory
 * (synchronises the stream): mean[t] and err[t] are the combined VEGAS
 * estimate of task t and its standard error.  Task numbering:
 * t = (side_integral * n_grid + grid_point) * 2 + term, term 0 = gain,
 * 1 = loss; side integrals ordered by process, side (initial first), then
 * observed species.  In a shard (config.point_lo/point_hi) the numbering is
 * t = (side_integral * (point_hi - point_lo) + grid_point - point_lo) * 2 +
 * term; the same numbering indexes maps, strata and the state blob.  Either
 * pointer may be NULL.
 */
best_status best_get_task_results(best_ctx* ctx, double* mean, double* err, void* stream);

/*
 * Copies (to) / from host memory the VEGAS map edges of every task:
 * task t, dimension d, edge b at edges[t * 3*(BEST_MAX_LEGS-2) * (nbins_max+1)
 * + d * (nbins_max+1) + b], nbins_max the largest nbins of any process.
 * Synchronous.  best_map_stride() returns 3*(BEST_MAX_LEGS-2)*(nbins_max+1).
 */
int64_t best_map_stride(const best_ctx* ctx);
best_status best_get_maps(best_ctx* ctx, double* edges_host);
best_status best_set_maps(best_ctx* ctx, const double* edges_host);

/* Reads / sets the evaluation counter that enters every Philox counter.
 * Synchronous. */
best_status best_get_call_counter(best_ctx* ctx, uint32_t* call);
best_status best_set_call_counter(best_ctx* ctx, uint32_t call);

/*
 * Synchronises `stream` and reports errors that the device recorded since
 * the last check: BEST_ERR_NUMERIC when an input f was not positive and
 * finite, a(t) was not positive, or a result was not finite; BEST_ERR_CUDA
 * for a failed launch.  Clears the recorded error.
 */
best_status best_check(best_ctx* ctx, void* stream);

/*
 * Timing of the sample kernel, for measurement.  While enabled, every launch
 * of the sample kernel is bracketed by a pair of CUDA events recorded on the
 * launching stream (events are created on first use and reused).
 * best_profile_read waits for the recorded events, returns the summed kernel
 * time in milliseconds and the number of launches since the last read or
 * enable, and starts a new count.  When best_evolve captures its step graph
 * with timing enabled, the events become part of the graph and the read
 * returns the launches of the last replayed step.
 */
best_status best_profile_enable(best_ctx* ctx, int32_t enable);
best_status best_profile_read(best_ctx* ctx, double* sample_kernel_ms, int64_t* launches);

/* Number of kernels the last eval / Euler / Heun call enqueued. */
int32_t best_last_launch_count(const best_ctx* ctx);

/*
 * One VEGAS iteration of one task without allocating device memory.  The
 * paper has no counterpart: this serves callers that cannot call cudaMalloc
 * where they run -- a host application whose device memory is handed out
 * only by its own pool allocator (a framework that reserved the GPU's memory
 * up front, a service held to a fixed memory budget), or a latency-bound
 * loop that must not take the device-wide synchronisation a cudaMalloc or
 * cudaFree may cause.  It calls no cudaMalloc, cudaFree or other allocating
 * routine, and needs no context.
 *
 * Inputs: cfg (host, as for best_collision_init; precision selects the
 * FP32 or FP64 sample kernel), task (task id in the enumeration of
 * best_get_task_results), f_dev [n_species * n_grid] FP64, time t (host),
 * edges_dev (device FP64, the task's VEGAS map, [D][nbins + 1] with
 * D = 3 (n_legs - 2); read only), the iteration index and evaluation
 * counter that enter the Philox counter.  Output out_dev (device FP64,
 * 2 + D * nbins values): out[0] = sum of the task's sample weights w,
 * out[1] = sum of w^2, out[2 + d*nbins + b] = sum of w^2 over the samples
 * falling in increment b of dimension d (the training data of the map).
 * The estimate of the iteration is out[0] / neval with variance
 * (out[1]/neval - mean^2) / (neval - 1).  Grid values that the spline build
 * rejects (a value <= 0 or not finite) make every out[] value NaN (the
 * context path's BEST_ERR_NUMERIC); the call itself still returns BEST_OK,
 * since it does not wait for the GPU.
 *
 * Device scratch comes from one static array of about 3.5 MiB that every
 * GPU loading the library holds until the process exits.  Limits: grid.n
 * <= 512, nbins <= 64; larger sizes return BEST_ERR_INVALID with a message
 * in best_last_error(NULL).  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and give wrong results; order
 * them on one stream.
 */
best_status best_vegas_iteration_noalloc(const best_config* cfg, int32_t task, const double* f_dev,
                                         double t, const double* edges_dev, uint32_t iteration,
                                         uint32_t call, double* out_dev, void* stream);

/* Description of the last failure on ctx (or of the last failed init when
 * ctx is NULL); never NULL. */
const char* best_last_error(const best_ctx* ctx);

/* Frees the context and its device memory.  Synchronises the device. */
void best_collision_destroy(best_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BEST_H */
