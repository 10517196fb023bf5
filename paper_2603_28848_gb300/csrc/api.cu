// Host side of the C ABI declared in include/best.h: configuration checks,
// the identical-particle decomposition into tasks (Sec. 2C, App. A), the
// static work partition of the persistent sample kernel, device memory and
// the launch sequences of a sweep, an Euler step and a Heun step.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"
#include "philox.cuh"

namespace best {
// kernels.cu
__global__ void set_time_kernel(Geometry, TimeState*, const double*, double, int, const MassLaw*);
__global__ void spline_build_kernel(Geometry, const double*, int, const double*, TimeState*, SpeciesConst*,
                                    double*, double*, float*);
__global__ void prepare_kernel(Geometry, const SideDesc*, const TaskDesc*, const double*, const double*,
                               const TimeState*, const double*, TaskConst*, TaskAcc*, int, const double*,
                               const SpeciesConst*, SegConst32*);
__global__ void moments_kernel(Geometry, const double*, const double*, const TimeState*, double*, double*);
__global__ void width_control_kernel(Geometry, const SideDesc*, const TaskDesc*, const TaskAcc*, const WidthCtl*,
                                     double*, double*);
__global__ void refine_kernel(Geometry, const SideDesc*, const TaskDesc*, const TaskConst*, const int32_t*,
                              const int32_t*, const Segment*, const double*, double*, TaskAcc*, TaskConst*,
                              const double*, SegConst32*, float2*);
__global__ void map32_kernel(Geometry, const TaskDesc*, int, const double*, float2*);
__global__ void strat_init_kernel(const TaskDesc*, int32_t*, uint32_t*, int);
__global__ void strat_refine_kernel(const TaskDesc*, const int32_t*, const double*, int32_t*, double*, double*,
                                    uint32_t*, double*);
__global__ void assemble_kernel(Geometry, const SideDesc*, TaskAcc*, TimeState*, double*, double*, double*);
__global__ void step_first_kernel(Geometry, double*, const double*, const double*, double*, double*, TimeState*,
                                  double*, int);
__global__ void heun_correct_kernel(Geometry, double*, const double*, const double*, const double*, double*,
                                    double*, TimeState*);
__global__ void stage_kernel(Geometry, int, int, double*, const double*, const double*, double*, double*, double*,
                             TimeState*);
// variants.cu
int eval_variants(bool f32, int nmax, SampleVariant* v, bool strat);
// vjp.cu
void* vjp_kernel_ptr(bool f32, int nmax, bool me);
void* jvp_kernel_ptr(bool f32, int nmax, bool me);
__global__ void jvp_seed_kernel(Geometry, const SideDesc*, const TaskDesc*, const TaskConst*, const SpeciesConst*,
                                const double*, double*);
__global__ void jvp_finish_kernel(Geometry, const SideDesc*, const TaskDesc*, const TaskConst*, const double*, double*,
                                  double*);
__global__ void spline_tangent_kernel(Geometry, const double*, const double*, const double*, const SpeciesConst*,
                                      const TimeState*, double*, float*, double*);
__global__ void nk_exp_kernel(int, const double*, double*);
__global__ void nk_axpy_kernel(int, const double*, const double*, double, double*);
__global__ void nk_direction_kernel(int, const double*, const double*, double*);
__global__ void nk_residual_kernel(int, const double*, const double*, const double*, const double*, double, double*,
                                   double*, double*);
__global__ void gmres_start_kernel(int, int, const double*, double*, double*);
__global__ void gmres_arnoldi_kernel(int, int, int, double, const double*, const double*, const double*, double*,
                                     double*, double*, double*, double*, double*);
__global__ void gmres_update_kernel(int, int, int, const double*, const double*, const double*, double*);
__global__ void vjp_seed_kernel(Geometry, const SideDesc*, const TaskDesc*, const TaskConst*, const double*, double*);
__global__ void vjp_task_kernel(Geometry, const int32_t*, const int32_t*, const Segment*, const double*, int, double*);
__global__ void vjp_finish_kernel(Geometry, const SideDesc*, const TaskDesc*, const TaskConst*, const SpeciesConst*,
                                  const TimeState*, const double*, const double*, const double*, const double*,
                                  double*, double*, double*, double*, double*, int);
__global__ void spline_adjoint_kernel(Geometry, const double*, const double*, const SpeciesConst*, const TimeState*,
                                      const double*, const double*, double*, double*);
__global__ void budget_kernel(const BudgetCtl*, const TaskAcc*, TaskDesc*, double*);
__global__ void plan_kernel(const TaskDesc*, int, const PlanDev*, int, int, int64_t*);
}  // namespace best

using namespace best;

namespace {

thread_local char g_init_error[512] = "no error";

// Work of one VEGAS iteration index: the active tasks and their segments.
struct IterPlan {
    int n_active = 0;
    int n_segs = 0;
    int64_t partial_doubles = 0;
    int32_t* d_active = nullptr;     // [n_active] task ids
    int32_t* d_task_seg = nullptr;   // [n_active + 1]
    Segment* d_segs = nullptr;       // [n_segs]
    int32_t* d_cta_seg = nullptr;    // [chunks + 1]
};

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

}  // namespace

struct best_ctx {
    std::string err = "no error";
    Geometry geo{};
    int precision = 0;
    int nmax_legs = 0;
    int grid = 0;                   // CTAs of the persistent sample kernel
    int n_chunks = 0;               // chunks of the work partition (chunk_count(grid))
    int32_t* d_chunk_ctr = nullptr; // [max_nitn + 1] chunk counters: sample kernel per iteration, adjoint / tangent
    size_t eval_smem = 0;
    size_t spline_smem = 0;
    size_t refine_smem = 0;
    int refine_threads = 128;       // one thread per entry of a task's reduced record, 128 to 512
    void* eval_fn = nullptr;
    int n_variants = 0;             // sample-kernel variants (register budget, CTA size, samples per step)
    SampleVariant variants[kMaxVariants] = {};
    int variant = 0;
    int eval_threads = kThreads;    // threads per CTA of the selected variant
    int64_t partial_capacity = 0;   // doubles allocated at d_partials
    int launches = 0;
    int max_nitn = 0;
    std::vector<SideDesc> sides;
    std::vector<TaskDesc> tasks;
    std::vector<IterPlan> plans;
    // device state
    SideDesc* d_sides = nullptr;
    TaskDesc* d_tasks = nullptr;
    TaskConst* d_tconst = nullptr;
    SegConst32* d_tconst32 = nullptr;  // FP32 segment constants per task (FP32 sample kernel)
    float2* d_map32 = nullptr;      // FP32 kernels' map tables [task][map32_stride] (FP32 contexts)
    TaskAcc* d_acc = nullptr;
    SpeciesConst* d_sconst = nullptr;
    TimeState* d_ts = nullptr;
    double* d_edges = nullptr;
    double* d_knots = nullptr;
    float* d_knots32 = nullptr;
    double* d_coef64 = nullptr;
    float* d_coef32 = nullptr;
    double* d_fgrid = nullptr;
    MassLaw* d_mass_law = nullptr;  // [species]
    std::vector<MassLaw> mass_law;
    double* d_partials = nullptr;
    double* d_k1 = nullptr;
    double* d_k2 = nullptr;
    double* d_fstar = nullptr;
    double* d_prev = nullptr;       // |estimate| of every task from the last sweep (0: none)
    // CUDA graph of one step (best_evolve), keyed by its arguments
    cudaGraphExec_t graph = nullptr;
    double* g_logf = nullptr;
    double* g_t = nullptr;
    double* g_dt = nullptr;
    int g_method = -1;
    int g_launches = 0;
    size_t g_events = 0;            // timing events recorded by one replay
    double* d_dtreq = nullptr;      // requested step, read by the graph
    // adjoint (best_collision_vjp)
    double* d_gcoef = nullptr;      // [species][n-1][4]
    double* d_vjp_tot = nullptr;    // [task][16]
    double* d_u = nullptr;          // [task]
    double* d_gtail = nullptr;      // [species][4]
    double* d_coupling = nullptr;   // [process]
    double* d_dcoef64 = nullptr;    // tangent spline of the JVP direction [species][n-1][4]
    float* d_dcoef32 = nullptr;
    double* d_dtail = nullptr;      // [species][4]
    size_t jvp_smem = 0;
    bool jvp_ready = false;         // shared-memory attribute of the tangent kernel set
    // fractional Gaussian widths (App. C), one per process
    double* d_width = nullptr;
    double* d_width_rel = nullptr;
    WidthCtl* d_wctl = nullptr;
    std::vector<int> width_mode;
    bool any_adaptive = false;
    bool any_me = false;            // some process has an s-dependent |M|^2
    // adaptive stratified sampling (VEGAS+)
    bool any_strat = false;
    int64_t strat_total_h = 0, strat_total_items = 0;
    int32_t* d_strat_m = nullptr;   // items per hypercube, all stratified tasks
    double* d_strat_d = nullptr;    // per-hypercube sum w, then allocation weights (scratch)
    double* d_strat_s2 = nullptr;   // per-hypercube sum w^2 (scratch)
    uint32_t* d_item_h = nullptr;   // hypercube of every item
    double* d_item_rec = nullptr;   // (sum w, sum w^2) per item
    double* d_strat_est = nullptr;  // [task][4] iteration estimate, variance, underflow flag
    // implicit Euler (best_step_implicit_euler): Krylov basis and work vectors
    double* d_nk = nullptr;
    int nk_m = 0;
    int n_processes = 0;
    size_t vjp_smem = 0;
    // variance-driven budgets: per-process controls, the device budgets as last
    // read back (for host-built partitions), and the device partition builder
    bool any_budget = false;
    std::vector<BudgetCtl> bctl;
    BudgetCtl* d_bctl = nullptr;
    double* d_bv = nullptr;         // [task] relative variance per sample (scratch)
    int64_t* d_plan_scratch = nullptr;
    PlanDev* d_plandev = nullptr;   // [max_nitn]
    std::vector<int64_t> neval_now;
    // timing of the sample kernel (best_profile_*)
    bool profiling = false;
    std::vector<cudaEvent_t> ev;    // start/stop pairs
    size_t ev_used = 0;
};

namespace {

best_status fail(best_ctx* c, best_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else snprintf(g_init_error, sizeof(g_init_error), "%s", buf);
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? BEST_ERR_OOM : BEST_ERR_CUDA,   \
                        "%s: %s", #call, cudaGetErrorString(e_));                             \
        }                                                                                     \
    } while (0)

// Roles of App. A for an observed leg: conserved leg and integrated legs.
void roles(int n_in, int n_out, int obs, int* cons, int* integ) {
    const int n = n_in + n_out;
    const bool obs_in = obs < n_in;
    bool first_in;
    if (n_in != n_out) first_in = n_in < n_out;
    else first_in = obs_in;
    int c = -1;
    for (int k = first_in ? 0 : n_in; k < (first_in ? n_in : n); ++k)
        if (k != obs) { c = k; break; }
    if (c < 0)
        for (int k = first_in ? n_in : 0; k < (first_in ? n : n_in); ++k)
            if (k != obs) { c = k; break; }
    *cons = c;
    int j = 0;
    for (int k = 0; k < n; ++k)
        if (k != obs && k != c) integ[j++] = k;
}

void free_all(best_ctx* c) {
    for (auto& p : c->plans) {
        cudaFree(p.d_active); cudaFree(p.d_task_seg); cudaFree(p.d_segs); cudaFree(p.d_cta_seg);
    }
    c->plans.clear();
    void* bufs[] = {c->d_sides, c->d_tasks, c->d_tconst, c->d_tconst32, c->d_map32, c->d_acc, c->d_sconst, c->d_ts, c->d_edges,
                    c->d_knots, c->d_knots32, c->d_coef64, c->d_coef32, c->d_fgrid, c->d_mass_law,
                    c->d_partials, c->d_k1, c->d_k2, c->d_fstar, c->d_prev, c->d_dtreq,
                    c->d_gcoef, c->d_vjp_tot, c->d_u, c->d_gtail, c->d_coupling, c->d_dcoef64,
                    c->d_dcoef32, c->d_dtail, c->d_nk, c->d_width, c->d_width_rel, c->d_wctl,
                    c->d_strat_m, c->d_strat_d, c->d_strat_s2, c->d_item_h, c->d_item_rec, c->d_strat_est};
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    for (void* b : bufs) cudaFree(b);
    cudaFree(c->d_bctl); cudaFree(c->d_bv); cudaFree(c->d_plan_scratch); cudaFree(c->d_plandev);
    cudaFree(c->d_chunk_ctr);
}

best_status validate(const best_config* cfg) {
    best_ctx* ctx = nullptr;
    if (!cfg) return fail(ctx, BEST_ERR_INVALID, "cfg is NULL");
    const best_grid& g = cfg->grid;
    if (g.n < 4 || g.n > 4096) return fail(ctx, BEST_ERR_INVALID, "grid.n must be in [4, 4096]");
    if (!(g.q_min > 0.0) || !(g.q_max > g.q_min) || !std::isfinite(g.q_max))
        return fail(ctx, BEST_ERR_INVALID, "need 0 < q_min < q_max");
    if (cfg->n_species < 1 || cfg->n_species > BEST_MAX_SPECIES || !cfg->species)
        return fail(ctx, BEST_ERR_INVALID, "n_species must be in [1, %d]", BEST_MAX_SPECIES);
    if (cfg->n_processes < 1 || cfg->n_processes > BEST_MAX_PROCESSES || !cfg->processes)
        return fail(ctx, BEST_ERR_INVALID, "n_processes must be in [1, %d]", BEST_MAX_PROCESSES);
    if (cfg->precision != BEST_FP64 && cfg->precision != BEST_FP32)
        return fail(ctx, BEST_ERR_INVALID, "precision must be BEST_FP64 or BEST_FP32");
    if (cfg->tail_points < 2 || cfg->tail_points > g.n)
        return fail(ctx, BEST_ERR_INVALID, "tail_points must be in [2, grid.n]");
    if (cfg->expansion && (!(cfg->a0 > 0.0) || !(cfg->t0 > 0.0)))
        return fail(ctx, BEST_ERR_INVALID, "expansion needs a0 > 0 and t0 > 0");
    if (!(cfg->eps_dt > 0.0)) return fail(ctx, BEST_ERR_INVALID, "eps_dt must be > 0");
    for (int s = 0; s < cfg->n_species; ++s) {
        const best_species& sp = cfg->species[s];
        if (sp.stat < 0 || sp.stat > 2) return fail(ctx, BEST_ERR_INVALID, "species %d: bad stat", s);
        if (!std::isfinite(sp.mass0) || !std::isfinite(sp.mass1))
            return fail(ctx, BEST_ERR_INVALID, "species %d: bad mass", s);
        if (sp.n_mass_knots != 0) {
            if (sp.n_mass_knots < 2 || sp.n_mass_knots > BEST_MAX_MASS_KNOTS)
                return fail(ctx, BEST_ERR_INVALID, "species %d: n_mass_knots must be 0 or in [2, %d]", s,
                            BEST_MAX_MASS_KNOTS);
            for (int k = 0; k < sp.n_mass_knots; ++k) {
                if (!std::isfinite(sp.mass_t[k]) || !std::isfinite(sp.mass_m[k]) || sp.mass_m[k] < 0.0 ||
                    (k > 0 && !(sp.mass_t[k] > sp.mass_t[k - 1])))
                    return fail(ctx, BEST_ERR_INVALID, "species %d: mass knots need increasing finite times and "
                                "finite masses >= 0", s);
            }
        }
    }
    if (cfg->point_hi != 0 && !(cfg->point_lo >= 0 && cfg->point_lo < cfg->point_hi && cfg->point_hi <= g.n))
        return fail(ctx, BEST_ERR_INVALID, "shard: need 0 <= point_lo < point_hi <= grid.n (or both 0)");
    const bool shard = cfg->point_hi != 0 && !(cfg->point_lo == 0 && cfg->point_hi == g.n);
    for (int p = 0; p < cfg->n_processes; ++p) {
        const best_process& pr = cfg->processes[p];
        const int n = pr.n_in + pr.n_out;
        if (pr.n_in < 1 || pr.n_out < 1 || n < 3 || n > BEST_MAX_LEGS)
            return fail(ctx, BEST_ERR_INVALID, "process %d: need 3 <= n_in + n_out <= %d", p, BEST_MAX_LEGS);
        for (int k = 0; k < n; ++k)
            if (pr.species[k] < 0 || pr.species[k] >= cfg->n_species)
                return fail(ctx, BEST_ERR_INVALID, "process %d: leg %d has a bad species", p, k);
        if (!(pr.sigma_E > 0.0)) return fail(ctx, BEST_ERR_INVALID, "process %d: sigma_E must be > 0", p);
        if (pr.width_mode < 0 || pr.width_mode > 2)
            return fail(ctx, BEST_ERR_INVALID, "process %d: width_mode must be 0, 1 or 2", p);
        if (shard && pr.width_mode == 2)
            return fail(ctx, BEST_ERR_INVALID, "process %d: the adaptive width needs every task in one context "
                        "(a shard would adapt on its own points only)", p);
        if (pr.width_mode != 0 && !(pr.width > 0.0 && std::isfinite(pr.width)))
            return fail(ctx, BEST_ERR_INVALID, "process %d: width must be > 0", p);
        if (pr.width_mode == 2 &&
            !(pr.width_min > 0.0 && pr.width_min <= pr.width && pr.width <= pr.width_max &&
              std::isfinite(pr.width_max) && pr.width_factor > 1.0 && std::isfinite(pr.width_factor) &&
              pr.width_rel_lo >= 0.0 && pr.width_rel_lo < pr.width_rel_hi))
            return fail(ctx, BEST_ERR_INVALID,
                        "process %d: adaptive width needs 0 < width_min <= width <= width_max, width_factor > 1, "
                        "0 <= width_rel_lo < width_rel_hi", p);
        {
            bool finite = true, zero = true;
            for (int k = 0; k < 4; ++k) {
                finite = finite && std::isfinite(pr.me_coef[k]);
                zero = zero && pr.me_coef[k] == 0.0;
            }
            if (!finite || zero)
                return fail(ctx, BEST_ERR_INVALID, "process %d: me_coef must be finite and not all zero", p);
        }
        if (pr.strat != 0 && pr.strat != 1) return fail(ctx, BEST_ERR_INVALID, "process %d: strat must be 0 or 1", p);
        if (pr.strat && (!(pr.strat_beta >= 0.0) || !std::isfinite(pr.strat_beta) || pr.strat_max_hcubes < 1 ||
                         pr.strat_max_hcubes > (1 << 20)))
            return fail(ctx, BEST_ERR_INVALID, "process %d: stratification needs strat_beta >= 0 and "
                        "1 <= strat_max_hcubes <= 2^20", p);
        if (pr.budget != 0 && pr.budget != 1) return fail(ctx, BEST_ERR_INVALID, "process %d: budget must be 0 or 1", p);
        if (pr.sides < 0 || pr.sides > 2) return fail(ctx, BEST_ERR_INVALID, "process %d: sides must be 0, 1 or 2", p);
        if (pr.budget && (pr.strat || pr.neval_min < 2 || pr.neval_min > pr.neval_max ||
                          pr.neval_max > (int64_t(1) << 31) || pr.neval_max * 3 * (n - 2) > (int64_t(1) << 33)))
            return fail(ctx, BEST_ERR_INVALID, "process %d: variance-driven budgets need 2 <= neval_min <= neval_max, "
                        "neval_max <= 2^31, neval_max * dim <= 2^33, and no stratification", p);
        if (pr.nitn < 1 || pr.nitn > 1000) return fail(ctx, BEST_ERR_INVALID, "process %d: nitn in [1,1000]", p);
        if (pr.nbins < 2 || pr.nbins > 256) return fail(ctx, BEST_ERR_INVALID, "process %d: nbins in [2,256]", p);
        if (!(pr.alpha >= 0.0)) return fail(ctx, BEST_ERR_INVALID, "process %d: alpha must be >= 0", p);
        for (int i = 0; i < g.n; ++i) {
            const int64_t N = pr.neval_per_point ? pr.neval_per_point[i] : pr.neval;
            // the Philox block index of a task's last sample must fit the 32-bit counter word
            if (N < 2 || N > (int64_t(1) << 31) || N * 3 * (n - 2) > (int64_t(1) << 33))
                return fail(ctx, BEST_ERR_INVALID, "process %d: need 2 <= neval, neval * dim <= 2^33", p);
            if (pr.strat && N < 2 * kItem)
                return fail(ctx, BEST_ERR_INVALID, "process %d: stratified sampling needs neval >= %d", p, 2 * kItem);
        }
    }
    return BEST_OK;
}

// |M|^2 / coupling^2 = P(s) of a process into its side descriptor.
void set_matrix_element(SideDesc& sd, const best_process& pr) {
    for (int k = 0; k < 4; ++k) sd.me_coef[k] = pr.me_coef[k];
    sd.me_on = !(pr.me_coef[0] == 1.0 && pr.me_coef[1] == 0.0 && pr.me_coef[2] == 0.0 && pr.me_coef[3] == 0.0);
}

int group_size(int D, bool f32) {
    const int per = f32 ? 4 : 2;
    int a = D, b = per;
    while (b) { int t = a % b; a = b; b = t; }
    return per / a;
}

// CTAs of 256 threads for map32_kernel: one thread per table entry, at most
// 4096 CTAs (the kernel strides over the rest).
int map32_blocks(const Geometry& g) {
    const int64_t entries = static_cast<int64_t>(g.n_tasks) * map32_stride(g);
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((entries + 255) / 256, 4096)));
}

// Dynamic shared memory of the sample kernel with `threads` per CTA: spline
// tables of all species, the map table, per-warp histograms, the reduction
// scratch and (FP32) the per-warp sample queues, in the kernel's layout.
size_t sample_smem(const best_ctx* ctx, int threads) {
    const Geometry& g = ctx->geo;
    const bool f32 = ctx->precision == BEST_FP32;
    const size_t rs = f32 ? 4 : 8;
    const size_t spl = static_cast<size_t>(g.n_species) * 4 * (g.n_grid - 1) + g.n_grid;
    // the kernel's table stride: 12 dimensions, or in the extended instantiations
    // (stratified tasks or an s-dependent |M|^2) those of their NMAX (4 or 6 legs)
    const bool ext = ctx->any_strat || ctx->any_me;
    const int dims = ext ? (ctx->nmax_legs <= 4 ? 6 : 12) : kMaxDim;
    const size_t map_elems = static_cast<size_t>(dims) * g.nbins_max;
    const size_t hist_elems = static_cast<size_t>(threads / 32) * map_elems;
    const size_t queue = ctx->any_strat ? strat_queue_floats(ctx->nmax_legs) : kQueueSlots * queue_words(ctx->nmax_legs);
    return rs * ((spl + 3) & ~size_t(3)) + 2 * rs * map_elems + rs * ((hist_elems + 3) & ~size_t(3)) +
           2 * 32 * sizeof(double) + (f32 ? sizeof(float) * (threads / 32) * queue : 0);
}

// Partition of the active tasks of one iteration into n_chunks chunks cut at
// chunk_bound() (shape from chunk_shape()) of an estimate of the cost of a
// sample group (its samples times the number of dimensions plus a constant).
// Segments come out ordered by task, so each task's segment records are
// contiguous.
best_status build_plan(best_ctx* ctx, int it, IterPlan& plan) {
    const bool f32 = ctx->precision == BEST_FP32;
    std::vector<int32_t> active;
    for (size_t t = 0; t < ctx->tasks.size(); ++t)
        if (ctx->tasks[t].nitn > it) active.push_back(static_cast<int32_t>(t));
    const int A = static_cast<int>(active.size());
    // work units: sample groups, or for stratified tasks items of kItem
    // samples (kItem / G groups), so that a segment holds whole items
    std::vector<int64_t> groups(A), unit(A), cost(A), cum(A + 1, 0);
    for (int a = 0; a < A; ++a) {
        const TaskDesc& td = ctx->tasks[active[a]];
        const int G = group_size(td.dim, f32);
        const int64_t N = ctx->any_budget ? ctx->neval_now[active[a]] : td.neval;
        unit[a] = td.strat_H > 0 ? kItem / G : 1;
        groups[a] = (N + G - 1) / G / unit[a];
        cost[a] = static_cast<int64_t>(G) * unit[a] * (td.dim + 6);
        cum[a + 1] = cum[a] + groups[a] * cost[a];
    }
    const int64_t W = cum[A];
    const int B = ctx->grid, K = ctx->n_chunks;
    const ChunkShape sh = chunk_shape(W, B);
    std::vector<Segment> segs;
    std::vector<int32_t> cta_seg(K + 1, 0);
    std::vector<int32_t> seg_active;
    int a0 = 0;
    for (int b = 0; b < K; ++b) {
        cta_seg[b] = static_cast<int32_t>(segs.size());
        const int64_t lo = chunk_bound(W, b, sh), hi = chunk_bound(W, b + 1, sh);
        while (a0 < A && cum[a0 + 1] <= lo) ++a0;
        for (int a = a0; a < A && cum[a] < hi; ++a) {
            const int64_t c = cost[a];
            const int64_t g0 = std::max<int64_t>(0, (lo - cum[a] + c - 1) / c);
            const int64_t g1 = std::min<int64_t>(groups[a], (hi - cum[a] + c - 1) / c);
            if (g1 <= g0) continue;
            Segment s{};
            s.task = active[a];
            s.g0 = g0 * unit[a];
            s.g1 = g1 * unit[a];
            segs.push_back(s);
            seg_active.push_back(a);
        }
    }
    cta_seg[K] = static_cast<int32_t>(segs.size());
    // partial records and per-task segment ranges
    std::vector<int32_t> task_seg(A + 1, 0);
    int64_t off = 0;
    for (size_t k = 0; k < segs.size(); ++k) {
        segs[k].part = off;
        const TaskDesc& td = ctx->tasks[segs[k].task];
        off += record_doubles(td.dim, td.nbins);
    }
    {
        size_t k = 0;
        for (int a = 0; a < A; ++a) {
            task_seg[a] = static_cast<int32_t>(k);
            while (k < segs.size() && seg_active[k] == a) ++k;
        }
        task_seg[A] = static_cast<int32_t>(k);
        if (k != segs.size()) return fail(ctx, BEST_ERR_INVALID, "internal: segments not ordered by task");
    }
    plan.n_active = A;
    plan.n_segs = static_cast<int>(segs.size());
    plan.partial_doubles = off;
    if (ctx->any_budget) {
        // the device rebuilds this partition when the budgets change: room for
        // the largest one (each chunk boundary splits at most one task)
        int64_t cap = 0, rmax = 0;
        for (int a = 0; a < A; ++a) {
            const TaskDesc& td = ctx->tasks[active[a]];
            cap += record_doubles(td.dim, td.nbins);
            rmax = std::max(rmax, record_doubles(td.dim, td.nbins));
        }
        plan.partial_doubles = std::max(off, cap + static_cast<int64_t>(K) * rmax);
    }
    CK(dalloc(&plan.d_active, A));
    CK(dalloc(&plan.d_task_seg, A + 1));
    CK(dalloc(&plan.d_segs, ctx->any_budget ? static_cast<size_t>(A) + K : segs.size()));
    CK(dalloc(&plan.d_cta_seg, K + 1));
    CK(cudaMemcpy(plan.d_active, active.data(), A * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(plan.d_task_seg, task_seg.data(), (A + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(plan.d_segs, segs.data(), segs.size() * sizeof(Segment), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(plan.d_cta_seg, cta_seg.data(), (K + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    return BEST_OK;
}

// Selects sample-kernel variant v: raises its shared-memory limit, sizes the
// persistent grid from its occupancy and rebuilds the work partition.
best_status set_variant(best_ctx* ctx, int v) {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    void* fn = ctx->variants[v].fn;
    const int threads = ctx->variants[v].threads;
    ctx->eval_smem = sample_smem(ctx, threads);
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, fn));
    if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) < ctx->eval_smem)
        CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ctx->eval_smem)));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, ctx->eval_smem));
    if (occ < 1) return fail(ctx, BEST_ERR_INVALID, "sample kernel does not fit on an SM");
    // a captured step graph refers to the old partition: drop it
    if (ctx->graph) {
        CK(cudaGraphExecDestroy(ctx->graph));
        ctx->graph = nullptr;
    }
    ctx->eval_fn = fn;
    ctx->variant = v;
    ctx->eval_threads = threads;
    ctx->grid = nsm * occ;
    ctx->n_chunks = chunk_count(ctx->grid);
    for (auto& pl : ctx->plans) {
        cudaFree(pl.d_active); cudaFree(pl.d_task_seg); cudaFree(pl.d_segs); cudaFree(pl.d_cta_seg);
    }
    ctx->plans.assign(ctx->max_nitn, IterPlan{});
    if (ctx->any_budget) {
        std::vector<TaskDesc> cur(ctx->tasks.size());
        CK(cudaMemcpy(cur.data(), ctx->d_tasks, cur.size() * sizeof(TaskDesc), cudaMemcpyDeviceToHost));
        ctx->neval_now.resize(cur.size());
        for (size_t t = 0; t < cur.size(); ++t) ctx->neval_now[t] = cur[t].neval;
    }
    int64_t part_max = 0;
    for (int it = 0; it < ctx->max_nitn; ++it) {
        best_status s = build_plan(ctx, it, ctx->plans[it]);
        if (s != BEST_OK) return s;
        part_max = std::max(part_max, ctx->plans[it].partial_doubles);
    }
    if (part_max > ctx->partial_capacity) {
        cudaFree(ctx->d_partials);
        ctx->d_partials = nullptr;
        ctx->partial_capacity = 0;
        CK(dalloc(&ctx->d_partials, static_cast<size_t>(part_max)));
        ctx->partial_capacity = part_max;
    }
    if (ctx->any_budget) {
        std::vector<PlanDev> pd(ctx->max_nitn);
        int amax = 0;
        for (int it = 0; it < ctx->max_nitn; ++it) {
            const IterPlan& pl = ctx->plans[it];
            pd[it] = PlanDev{pl.n_active, 0, pl.d_active, pl.d_task_seg, pl.d_segs, pl.d_cta_seg};
            amax = std::max(amax, pl.n_active);
        }
        cudaFree(ctx->d_plandev);
        cudaFree(ctx->d_plan_scratch);
        ctx->d_plandev = nullptr;
        ctx->d_plan_scratch = nullptr;
        CK(dalloc(&ctx->d_plandev, pd.size()));
        CK(cudaMemcpy(ctx->d_plandev, pd.data(), pd.size() * sizeof(PlanDev), cudaMemcpyHostToDevice));
        CK(dalloc(&ctx->d_plan_scratch, static_cast<size_t>(amax) + 1 + 2 * static_cast<size_t>(ctx->n_chunks)));
    }
    return BEST_OK;
}

// Kernels of one collision sweep after set_time: spline, task constants,
// nitn x (sample kernel + refinement), assembly into C / err.
best_status enqueue_sweep(best_ctx* ctx, const double* src, int src_mode, double* C, double* err,
                          cudaStream_t st) {
    const Geometry& g = ctx->geo;
    spline_build_kernel<<<g.n_species, 256, ctx->spline_smem, st>>>(
        g, src, src_mode, ctx->d_knots, ctx->d_ts, ctx->d_sconst, ctx->d_fgrid, ctx->d_coef64, ctx->d_coef32);
    prepare_kernel<<<(g.n_tasks + 127) / 128, 128, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_knots,
                                                            ctx->d_fgrid, ctx->d_ts, ctx->d_prev, ctx->d_tconst,
                                                            ctx->d_acc, 1, ctx->d_width, ctx->d_sconst,
                                                            ctx->d_tconst32);
    ctx->launches += 2;
    if (ctx->d_map32) {
        map32_kernel<<<map32_blocks(g), 256, 0, st>>>(g, ctx->d_tasks, g.n_tasks, ctx->d_edges, ctx->d_map32);
        ctx->launches += 1;
    }
    const bool f32 = ctx->precision == BEST_FP32;
    CK(cudaMemsetAsync(ctx->d_chunk_ctr, 0, sizeof(int32_t) * ctx->max_nitn, st));
    for (int it = 0; it < ctx->max_nitn; ++it) {
        const IterPlan& pl = ctx->plans[it];
        if (pl.n_active == 0) continue;
        EvalParams P;
        P.geo = g;
        P.sides = ctx->d_sides;
        P.tasks = ctx->d_tasks;
        P.tconst = ctx->d_tconst;
        P.tconst32 = ctx->d_tconst32;
        P.sconst = ctx->d_sconst;
        P.ts = ctx->d_ts;
        P.edges = ctx->d_edges;
        P.map32 = ctx->d_map32;
        P.segs = pl.d_segs;
        P.cta_seg = pl.d_cta_seg;
        P.n_chunks = ctx->n_chunks;
        P.chunk_counter = ctx->d_chunk_ctr + it;
        P.coef = f32 ? static_cast<const void*>(ctx->d_coef32) : static_cast<const void*>(ctx->d_coef64);
        P.knots = f32 ? static_cast<const void*>(ctx->d_knots32) : static_cast<const void*>(ctx->d_knots);
        P.partials = ctx->d_partials;
        P.item_h = ctx->d_item_h;
        P.strat_m = ctx->d_strat_m;
        P.item_rec = ctx->d_item_rec;
        P.itn = static_cast<uint32_t>(it);
        P.smem_spline_elems = g.n_species * 4 * (g.n_grid - 1) + g.n_grid;
        const PhiloxKey key = philox_key(g.seed);
        for (int r = 0; r < 20; ++r) P.rk[r] = key.k[r];
        void* args[] = {&P};
        // inside a stream capture the events must become event-record nodes
        unsigned rec_flags = cudaEventRecordDefault;
        if (ctx->profiling) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            CK(cudaStreamIsCapturing(st, &cs));
            if (cs == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
            while (ctx->ev.size() < ctx->ev_used + 2) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->ev.push_back(e);
            }
            CK(cudaEventRecordWithFlags(ctx->ev[ctx->ev_used], st, rec_flags));
        }
        CK(cudaLaunchKernel(ctx->eval_fn, dim3(ctx->grid), dim3(ctx->eval_threads), args, ctx->eval_smem, st));
        if (ctx->profiling) {
            CK(cudaEventRecordWithFlags(ctx->ev[ctx->ev_used + 1], st, rec_flags));
            ctx->ev_used += 2;
        }
        if (ctx->any_strat) {
            strat_refine_kernel<<<pl.n_active, 256, 0, st>>>(ctx->d_tasks, pl.d_active, ctx->d_item_rec,
                                                             ctx->d_strat_m, ctx->d_strat_d, ctx->d_strat_s2,
                                                             ctx->d_item_h, ctx->d_strat_est);
            ctx->launches += 1;
        }
        refine_kernel<<<pl.n_active, ctx->refine_threads, ctx->refine_smem, st>>>(
            g, ctx->d_sides, ctx->d_tasks, ctx->d_tconst, pl.d_active, pl.d_task_seg, pl.d_segs,
            ctx->d_partials, ctx->d_edges, ctx->d_acc, ctx->d_tconst, ctx->d_strat_est, ctx->d_tconst32,
            ctx->d_map32);
        ctx->launches += 2;
    }
    const int total = g.n_species * g.n_grid;
    assemble_kernel<<<(total + 255) / 256, 256, 0, st>>>(g, ctx->d_sides, ctx->d_acc, ctx->d_ts, C, err,
                                                         ctx->d_prev);
    ctx->launches += 1;
    if (ctx->any_adaptive) {
        width_control_kernel<<<ctx->n_processes, 256, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_acc,
                                                               ctx->d_wctl, ctx->d_width, ctx->d_width_rel);
        ctx->launches += 1;
    }
    if (ctx->any_budget) {
        // next sweep's budgets from this sweep's estimates, then its partition
        budget_kernel<<<static_cast<int>(ctx->bctl.size()), 1024, 0, st>>>(ctx->d_bctl, ctx->d_acc, ctx->d_tasks,
                                                                          ctx->d_bv);
        plan_kernel<<<1, 1024, 0, st>>>(ctx->d_tasks, ctx->max_nitn, ctx->d_plandev, ctx->grid, f32 ? 1 : 0,
                                        ctx->d_plan_scratch);
        ctx->launches += 2;
    }
    CK(cudaGetLastError());
    return BEST_OK;
}

}  // namespace

namespace best {

__global__ void store_scalar_kernel(double* dst, double v) { *dst = v; }
__global__ void copy_scalar_kernel(double* dst, const double* src) { *dst = *src; }

// Checks a configuration like best_collision_init does (messages go to the
// fixed-size buffer read by best_last_error(NULL); nothing is allocated).
best_status check_config(const best_config* cfg) { return validate(cfg); }

best_status report(best_status st, const char* msg) { return fail(nullptr, st, "%s", msg); }

// Side integral and task descriptors of task `task` in the enumeration of
// best_collision_init, built without heap memory.  Returns false when the
// task id is out of range.
bool describe_task(const best_config* cfg, int32_t task, SideDesc* out_sd, TaskDesc* out_td) {
    const int n_grid = cfg->grid.n;
    int si = 0;
    for (int p = 0; p < cfg->n_processes; ++p) {
        const best_process& pr = cfg->processes[p];
        const int n_in = pr.n_in, n_out = pr.n_out, n = n_in + n_out;
        int s_in[BEST_MAX_LEGS], s_out[BEST_MAX_LEGS];
        for (int k = 0; k < n_in; ++k) s_in[k] = pr.species[k];
        for (int k = 0; k < n_out; ++k) s_out[k] = pr.species[n_in + k];
        std::sort(s_in, s_in + n_in);
        std::sort(s_out, s_out + n_out);
        const bool symmetric = n_in == n_out && std::equal(s_in, s_in + n_in, s_out);
        for (int side = 0; side < (symmetric ? 1 : 2); ++side) {
            if (pr.sides && side != pr.sides - 1) continue;
            const int offset = side == 0 ? 0 : n_in;
            const int cnt = side == 0 ? n_in : n_out;
            const int* sorted = side == 0 ? s_in : s_out;
            for (int u = 0; u < cnt; ++u) {
                if (u > 0 && sorted[u] == sorted[u - 1]) continue;     // distinct species, ascending
                const int a = sorted[u];
                if (task / (2 * n_grid) == si) {
                    SideDesc sd{};
                    sd.n = n;
                    sd.n_in = n_in;
                    sd.obs = -1;
                    sd.mult = 0;
                    for (int k = 0; k < cnt; ++k) {
                        if (pr.species[offset + k] != a) continue;
                        if (sd.obs < 0) sd.obs = offset + k;
                        ++sd.mult;
                    }
                    sd.species_obs = a;
                    sd.process = p;
                    sd.side = side;
                    roles(n_in, n_out, sd.obs, &sd.cons, sd.integ);
                    for (int k = 0; k < n; ++k) {
                        sd.leg_species[k] = pr.species[k];
                        const bool kin = k < n_in;
                        if (kin) sd.in_mask |= 1 << k;
                        if (kin == (side == 0)) sd.own_mask |= 1 << k;
                    }
                    sd.coupling2 = pr.coupling * pr.coupling;
                    const int st_obs = cfg->species[a].stat;
                    sd.eta_obs = st_obs == BEST_BE ? 1.0 : (st_obs == BEST_FD ? -1.0 : 0.0);
                    sd.sigma = pr.sigma_E;
                    sd.width_mode = pr.width_mode;
                    sd.width0 = pr.width;
                    set_matrix_element(sd, pr);
                    TaskDesc td{};
                    td.si = 0;
                    td.point = (task / 2) % n_grid;
                    td.term = task % 2;
                    td.gid = static_cast<uint32_t>(task);
                    td.nitn = 1;
                    td.neval = pr.neval_per_point ? pr.neval_per_point[td.point] : pr.neval;
                    td.dim = 3 * (n - 2);
                    td.nbins = pr.nbins;
                    td.alpha = pr.alpha;
                    *out_sd = sd;
                    *out_td = td;
                    return true;
                }
                ++si;
            }
        }
    }
    return false;
}

}  // namespace best

extern "C" {

best_status best_collision_init(const best_config* cfg, best_ctx** out) {
    if (!out) return fail(nullptr, BEST_ERR_INVALID, "out is NULL");
    *out = nullptr;
    best_status vs = validate(cfg);
    if (vs != BEST_OK) return vs;
    best_ctx* ctx = new best_ctx();
    auto bail = [&](best_status s) {
        snprintf(g_init_error, sizeof(g_init_error), "%s", ctx->err.c_str());
        free_all(ctx);
        delete ctx;
        return s;
    };
    Geometry& g = ctx->geo;
    g.n_grid = cfg->grid.n;
    g.log_spaced = cfg->grid.log_spaced ? 1 : 0;
    g.q_min = cfg->grid.q_min;
    g.q_max = cfg->grid.q_max;
    g.log_step = g.log_spaced ? std::log(g.q_max / g.q_min) / (g.n_grid - 1) : (g.q_max - g.q_min) / (g.n_grid - 1);
    g.inv_step = 1.0 / (g.log_spaced ? g.log_step / 0.6931471805599453 : g.log_step);
    g.lq0_step = g.log_spaced ? std::log2(g.q_min) * g.inv_step : 0.0;
    g.n_species = cfg->n_species;
    g.expansion = cfg->expansion ? 1 : 0;
    g.a0 = cfg->a0;
    g.t0 = cfg->t0;
    g.e_cut = cfg->e_cut;
    g.eps_dt = cfg->eps_dt;
    g.seed = cfg->seed;
    g.tail_points = cfg->tail_points;
    g.precision = cfg->precision;
    g.pt_lo = cfg->point_hi > 0 ? cfg->point_lo : 0;
    g.pt_hi = cfg->point_hi > 0 ? cfg->point_hi : cfg->grid.n;
    ctx->precision = cfg->precision;
    const bool f32 = cfg->precision == BEST_FP32;

    // ---- side integrals (Eq. (7), Eq. (8)) and tasks -----------------------------
    int nb_max = 2;
    for (int p = 0; p < cfg->n_processes; ++p) {
        const best_process& pr = cfg->processes[p];
        const int n_in = pr.n_in, n_out = pr.n_out, n = n_in + n_out;
        std::vector<int> a_in(pr.species, pr.species + n_in), a_out(pr.species + n_in, pr.species + n);
        std::vector<int> s_in = a_in, s_out = a_out;
        std::sort(s_in.begin(), s_in.end());
        std::sort(s_out.begin(), s_out.end());
        const bool symmetric = s_in == s_out;
        nb_max = std::max(nb_max, pr.nbins);
        ctx->nmax_legs = std::max(ctx->nmax_legs, n);
        ctx->max_nitn = std::max(ctx->max_nitn, pr.nitn);
        for (int side = 0; side < (symmetric ? 1 : 2); ++side) {
            if (pr.sides && side != pr.sides - 1) continue;   // a restricted set of side integrals
            const std::vector<int>& sp = side == 0 ? a_in : a_out;
            const int offset = side == 0 ? 0 : n_in;
            std::vector<int> distinct = sp;
            std::sort(distinct.begin(), distinct.end());
            distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
            for (int a : distinct) {
                SideDesc sd{};
                sd.n = n;
                sd.n_in = n_in;
                sd.obs = offset + static_cast<int>(std::find(sp.begin(), sp.end(), a) - sp.begin());
                sd.mult = static_cast<int>(std::count(sp.begin(), sp.end(), a));
                sd.species_obs = a;
                sd.process = p;
                sd.side = side;
                roles(n_in, n_out, sd.obs, &sd.cons, sd.integ);
                for (int k = 0; k < n; ++k) {
                    sd.leg_species[k] = pr.species[k];
                    const bool kin = k < n_in;
                    if (kin) sd.in_mask |= 1 << k;
                    if (kin == (side == 0)) sd.own_mask |= 1 << k;
                }
                sd.coupling2 = pr.coupling * pr.coupling;
                const int st_obs = cfg->species[a].stat;
                sd.eta_obs = st_obs == BEST_BE ? 1.0 : (st_obs == BEST_FD ? -1.0 : 0.0);
                sd.sigma = pr.sigma_E;
                sd.width_mode = pr.width_mode;
                sd.width0 = pr.width;
                set_matrix_element(sd, pr);
                ctx->sides.push_back(sd);
            }
        }
    }
    g.n_side = static_cast<int>(ctx->sides.size());
    for (int p = 0; p < cfg->n_processes; ++p) {
        bool any = false;
        for (const SideDesc& sd : ctx->sides) any = any || sd.process == p;
        if (!any)
            return bail(fail(ctx, BEST_ERR_INVALID, "process %d: its sides setting leaves no side integral (a "
                             "process with equal initial and final species has only the initial side)", p));
    }
    g.nbins_max = nb_max;
    g.map_stride = kMaxDim * (nb_max + 1);
    for (int si = 0; si < g.n_side; ++si) {
        const SideDesc& sd = ctx->sides[si];
        const best_process& pr = cfg->processes[sd.process];
        for (int i = g.pt_lo; i < g.pt_hi; ++i)
            for (int term = 0; term < 2; ++term) {
                TaskDesc td{};
                td.si = si;
                td.point = i;
                td.term = term;
                td.gid = static_cast<uint32_t>((si * g.n_grid + i) * 2 + term);
                td.nitn = pr.nitn;
                td.neval = pr.neval_per_point ? pr.neval_per_point[i] : pr.neval;
                td.dim = 3 * (sd.n - 2);
                td.nbins = pr.nbins;
                td.alpha = pr.alpha;
                if (pr.strat) {
                    // items of kItem samples; M the largest with 4 M^D <= J and M^D <= max hypercubes
                    const int64_t J = td.neval / kItem;
                    int64_t M = 1;
                    auto pw = [](int64_t b, int e) { int64_t r = 1; for (int k = 0; k < e; ++k) r *= b; return r; };
                    while (4 * pw(M + 1, td.dim) <= J && pw(M + 1, td.dim) <= pr.strat_max_hcubes) ++M;
                    td.neval = kItem * J;
                    td.strat_M = static_cast<int32_t>(M);
                    td.strat_H = static_cast<int32_t>(pw(M, td.dim));
                    td.strat_J = J;
                    td.strat_off_h = ctx->strat_total_h;
                    td.strat_off_item = ctx->strat_total_items;
                    td.strat_beta = pr.strat_beta;
                    ctx->strat_total_h += td.strat_H;
                    ctx->strat_total_items += J;
                    ctx->any_strat = true;
                }
                ctx->tasks.push_back(td);
            }
    }
    g.n_tasks = static_cast<int>(ctx->tasks.size());
    if (static_cast<int64_t>(g.n_tasks) >= (int64_t(1) << 31)) return bail(fail(ctx, BEST_ERR_INVALID, "too many tasks"));
    // variance-driven budgets: a process's tasks are contiguous (side integrals by process)
    for (int p = 0; p < cfg->n_processes; ++p) {
        const best_process& pr = cfg->processes[p];
        if (!pr.budget) continue;
        BudgetCtl c{};
        c.first = -1;
        for (int t = 0; t < g.n_tasks; ++t) {
            if (ctx->sides[ctx->tasks[t].si].process != p) continue;
            if (c.first < 0) c.first = t;
            c.count = t - c.first + 1;
            c.total += static_cast<double>(ctx->tasks[t].neval);
        }
        if (c.first < 0) continue;
        c.n_min = pr.neval_min;
        c.n_max = pr.neval_max;
        ctx->bctl.push_back(c);
    }
    ctx->any_budget = !ctx->bctl.empty();

    // ---- launch shape of the sample kernel -------------------------------------------------
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(ctx, BEST_ERR_CUDA, "no CUDA device"));
    for (const SideDesc& sd : ctx->sides) ctx->any_me = ctx->any_me || sd.me_on;
    // stratified tasks and s-dependent |M|^2 run in the extended instantiations
    ctx->geo.nbins_max = nb_max;                   // (sample_smem reads it)
    {
        SampleVariant all[kMaxVariants];
        const int nv = eval_variants(f32, ctx->nmax_legs, all, ctx->any_strat || ctx->any_me);
        // variants whose tables do not fit one CTA's shared memory are left out
        int max_optin = 0;
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        ctx->n_variants = 0;
        for (int v = 0; v < nv; ++v)
            if (sample_smem(ctx, all[v].threads) <= static_cast<size_t>(max_optin))
                ctx->variants[ctx->n_variants++] = all[v];
        if (ctx->n_variants == 0)
            return bail(fail(ctx, BEST_ERR_INVALID, "spline and map tables need %zu B of shared memory (max %d)",
                             sample_smem(ctx, kThreads), max_optin));
        cudaFuncAttributes fa{};
        ctx->spline_smem = 5 * sizeof(double) * g.n_grid;
        for (const void* fn : {reinterpret_cast<const void*>(&spline_build_kernel),
                               reinterpret_cast<const void*>(&spline_tangent_kernel),
                               reinterpret_cast<const void*>(&spline_adjoint_kernel)}) {
            if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
                return bail(fail(ctx, BEST_ERR_CUDA, "cannot query the spline kernels"));
            if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) < ctx->spline_smem &&
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(ctx->spline_smem)) != cudaSuccess)
                return bail(fail(ctx, BEST_ERR_CUDA, "cannot set shared memory of the spline kernels"));
        }
        ctx->refine_smem = sizeof(double) * (5 * static_cast<size_t>(kMaxDim) * nb_max + 4 * kMaxDim + 2);
        // the refinement's first phase sums each entry of the records (2 + D nb) over the task's
        // segments, one entry per thread where they fit: a chain of dependent loads per entry
        ctx->refine_threads = std::min(512, std::max(128, (2 + 3 * (ctx->nmax_legs - 2) * nb_max + 31) / 32 * 32));
        if (cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(&refine_kernel)) != cudaSuccess)
            return bail(fail(ctx, BEST_ERR_CUDA, "cannot query the refinement kernel"));
        if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) < ctx->refine_smem &&
            cudaFuncSetAttribute(reinterpret_cast<const void*>(&refine_kernel),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ctx->refine_smem)) != cudaSuccess)
            return bail(fail(ctx, BEST_ERR_CUDA, "cannot set shared memory of the refinement kernel"));
    }

    // ---- device state ----------------------------------------------------------------------------
    const int S = g.n_species, n = g.n_grid, T = g.n_tasks;
    std::vector<double> knots(n);
    for (int j = 0; j < n; ++j) {
        if (g.log_spaced) knots[j] = g.q_min * std::pow(g.q_max / g.q_min, static_cast<double>(j) / (n - 1));
        else knots[j] = g.q_min + (g.q_max - g.q_min) * j / (n - 1);
    }
    knots[0] = g.q_min;
    knots[n - 1] = g.q_max;
    std::vector<float> knots32(knots.begin(), knots.end());
    std::vector<SpeciesConst> sconst(S);
    ctx->mass_law.assign(S, MassLaw{});
    for (int s = 0; s < S; ++s) {
        sconst[s] = SpeciesConst{};
        sconst[s].stat = cfg->species[s].stat;
        sconst[s].eta = cfg->species[s].stat == BEST_BE ? 1.0 : (cfg->species[s].stat == BEST_FD ? -1.0 : 0.0);
        MassLaw& L = ctx->mass_law[s];
        L.m0 = cfg->species[s].mass0;
        L.m1 = cfg->species[s].mass1;
        L.n = cfg->species[s].n_mass_knots;
        for (int k = 0; k < L.n; ++k) {
            L.t[k] = cfg->species[s].mass_t[k];
            L.m[k] = cfg->species[s].mass_m[k];
        }
    }
    std::vector<double> edges(static_cast<size_t>(T) * g.map_stride, 0.0);
    for (int t = 0; t < T; ++t) {
        const TaskDesc& td = ctx->tasks[t];
        for (int d = 0; d < td.dim; ++d)
            for (int b = 0; b <= td.nbins; ++b)
                edges[static_cast<size_t>(t) * g.map_stride + d * (td.nbins + 1) + b] =
                    b == td.nbins ? 1.0 : static_cast<double>(b) / td.nbins;
    }
    TimeState ts{};
    ts.a = 1.0;
    ts.inv_a = 1.0;
#define CKI(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return bail(fail(ctx, e_ == cudaErrorMemoryAllocation ? BEST_ERR_OOM : BEST_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_))); } while (0)
    CKI(dalloc(&ctx->d_sides, g.n_side));
    CKI(dalloc(&ctx->d_tasks, T));
    CKI(dalloc(&ctx->d_tconst, T));
    CKI(dalloc(&ctx->d_tconst32, T));
    if (ctx->precision == BEST_FP32) CKI(dalloc(&ctx->d_map32, static_cast<size_t>(T) * map32_stride(g)));
    CKI(dalloc(&ctx->d_acc, T));
    CKI(dalloc(&ctx->d_chunk_ctr, static_cast<size_t>(ctx->max_nitn) + 1));
    CKI(dalloc(&ctx->d_sconst, S));
    CKI(dalloc(&ctx->d_ts, 1));
    CKI(dalloc(&ctx->d_edges, static_cast<size_t>(T) * g.map_stride));
    CKI(dalloc(&ctx->d_knots, n));
    CKI(dalloc(&ctx->d_knots32, n));
    CKI(dalloc(&ctx->d_coef64, static_cast<size_t>(S) * (n - 1) * 4));
    CKI(dalloc(&ctx->d_coef32, static_cast<size_t>(S) * (n - 1) * 4));
    CKI(dalloc(&ctx->d_fgrid, static_cast<size_t>(S) * n));
    CKI(dalloc(&ctx->d_mass_law, S));
    CKI(dalloc(&ctx->d_k1, static_cast<size_t>(S) * n));
    CKI(dalloc(&ctx->d_k2, static_cast<size_t>(S) * n));
    CKI(dalloc(&ctx->d_fstar, static_cast<size_t>(S) * n));
    CKI(dalloc(&ctx->d_prev, static_cast<size_t>(T)));
    CKI(dalloc(&ctx->d_dtreq, 1));
    CKI(dalloc(&ctx->d_gcoef, static_cast<size_t>(S) * (n - 1) * 4));
    CKI(dalloc(&ctx->d_vjp_tot, static_cast<size_t>(T) * 16));
    CKI(dalloc(&ctx->d_u, static_cast<size_t>(T)));
    CKI(dalloc(&ctx->d_gtail, static_cast<size_t>(S) * 4));
    CKI(dalloc(&ctx->d_coupling, static_cast<size_t>(cfg->n_processes)));
    CKI(dalloc(&ctx->d_dcoef64, static_cast<size_t>(S) * (n - 1) * 4));
    CKI(dalloc(&ctx->d_dcoef32, static_cast<size_t>(S) * (n - 1) * 4));
    CKI(dalloc(&ctx->d_dtail, static_cast<size_t>(S) * 4));
    {
        const int P = cfg->n_processes;
        CKI(dalloc(&ctx->d_width, static_cast<size_t>(P)));
        CKI(dalloc(&ctx->d_width_rel, static_cast<size_t>(P)));
        CKI(dalloc(&ctx->d_wctl, static_cast<size_t>(P)));
        std::vector<double> w0(P), zero(P, 0.0);
        std::vector<WidthCtl> wc(P);
        ctx->width_mode.assign(P, 0);
        for (int p = 0; p < P; ++p) {
            const best_process& pr = cfg->processes[p];
            w0[p] = pr.width_mode == 0 ? 0.0 : pr.width;
            wc[p] = WidthCtl{pr.width_mode, 0, pr.width_rel_lo, pr.width_rel_hi, pr.width_factor, pr.width_min,
                             pr.width_max};
            ctx->width_mode[p] = pr.width_mode;
            if (pr.width_mode == 2) ctx->any_adaptive = true;
        }
        CKI(cudaMemcpy(ctx->d_width, w0.data(), P * sizeof(double), cudaMemcpyHostToDevice));
        CKI(cudaMemcpy(ctx->d_width_rel, zero.data(), P * sizeof(double), cudaMemcpyHostToDevice));
        CKI(cudaMemcpy(ctx->d_wctl, wc.data(), P * sizeof(WidthCtl), cudaMemcpyHostToDevice));
    }
    {
        std::vector<double> lam(cfg->n_processes);
        for (int p = 0; p < cfg->n_processes; ++p) lam[p] = cfg->processes[p].coupling;
        CKI(cudaMemcpy(ctx->d_coupling, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice));
        ctx->n_processes = cfg->n_processes;
        const size_t rs = f32 ? 4 : 8;
        const size_t spl = static_cast<size_t>(S) * 4 * (n - 1) + n;
        const size_t ngc = static_cast<size_t>(S) * 4 * (n - 1);
        const size_t map_elems = static_cast<size_t>(kMaxDim) * nb_max;
        const size_t queue = sizeof(float) * (kThreads / 32) * kQueueSlots;   // FP32 per-warp sample queues
        ctx->vjp_smem = rs * ((spl + 3) & ~size_t(3)) + 2 * rs * map_elems + sizeof(double) * ngc +
                        12 * 8 * sizeof(double) +
                        (f32 ? sizeof(float) * ngc + queue * vjp_queue_words(ctx->nmax_legs, false) : 0);
        ctx->jvp_smem = rs * ((spl + 3) & ~size_t(3)) + 2 * rs * map_elems + 12 * 8 * sizeof(double) + rs * ngc +
                        (f32 ? queue * vjp_queue_words(ctx->nmax_legs, true) : 0);
    }
    CKI(cudaMemset(ctx->d_prev, 0, sizeof(double) * T));
    CKI(cudaMemcpy(ctx->d_sides, ctx->sides.data(), g.n_side * sizeof(SideDesc), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_tasks, ctx->tasks.data(), T * sizeof(TaskDesc), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_sconst, sconst.data(), S * sizeof(SpeciesConst), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_ts, &ts, sizeof(TimeState), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_edges, edges.data(), edges.size() * sizeof(double), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_knots, knots.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_knots32, knots32.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(ctx->d_mass_law, ctx->mass_law.data(), S * sizeof(MassLaw), cudaMemcpyHostToDevice));
    CKI(dalloc(&ctx->d_strat_est, static_cast<size_t>(T) * 4));
    CKI(cudaMemset(ctx->d_strat_est, 0, sizeof(double) * 4 * T));
    if (ctx->any_strat) {
        CKI(dalloc(&ctx->d_strat_m, static_cast<size_t>(ctx->strat_total_h)));
        CKI(dalloc(&ctx->d_strat_d, static_cast<size_t>(ctx->strat_total_h)));
        CKI(dalloc(&ctx->d_strat_s2, static_cast<size_t>(ctx->strat_total_h)));
        CKI(dalloc(&ctx->d_item_h, static_cast<size_t>(ctx->strat_total_items)));
        CKI(dalloc(&ctx->d_item_rec, static_cast<size_t>(ctx->strat_total_items) * 2));
        strat_init_kernel<<<T, 256>>>(ctx->d_tasks, ctx->d_strat_m, ctx->d_item_h, 1);
        CKI(cudaGetLastError());
    }
    if (ctx->any_budget) {
        CKI(dalloc(&ctx->d_bctl, ctx->bctl.size()));
        CKI(cudaMemcpy(ctx->d_bctl, ctx->bctl.data(), ctx->bctl.size() * sizeof(BudgetCtl), cudaMemcpyHostToDevice));
        CKI(dalloc(&ctx->d_bv, static_cast<size_t>(T)));
    }
    {
        best_status sv = set_variant(ctx, 0);
        if (sv != BEST_OK) return bail(sv);
    }
    CKI(cudaDeviceSynchronize());
#undef CKI
    *out = ctx;
    return BEST_OK;
}

best_status best_collision_eval(best_ctx* ctx, const double* f_dev, double t, double* C_dev, double* err_dev,
                                void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!f_dev || !C_dev) return fail(ctx, BEST_ERR_INVALID, "f_dev and C_dev must not be NULL");
    if (!std::isfinite(t)) return fail(ctx, BEST_ERR_INVALID, "t must be finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->launches = 0;
    set_time_kernel<<<1, 32, 0, st>>>(ctx->geo, ctx->d_ts, nullptr, t, 0, ctx->d_mass_law);
    ctx->launches += 1;
    return enqueue_sweep(ctx, f_dev, 0, C_dev, err_dev, st);
}

best_status best_collision_eval_log(best_ctx* ctx, const double* logf_dev, double t, double* C_dev,
                                    double* err_dev, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!logf_dev || !C_dev) return fail(ctx, BEST_ERR_INVALID, "logf_dev and C_dev must not be NULL");
    if (!std::isfinite(t)) return fail(ctx, BEST_ERR_INVALID, "t must be finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->launches = 0;
    set_time_kernel<<<1, 32, 0, st>>>(ctx->geo, ctx->d_ts, nullptr, t, 0, ctx->d_mass_law);
    ctx->launches += 1;
    return enqueue_sweep(ctx, logf_dev, 1, C_dev, err_dev, st);
}

best_status best_step_stage(best_ctx* ctx, int32_t method, int32_t stage, double* logf_dev, const double* k1_dev,
                            const double* k2_dev, double* fstar_dev, double* t_dev, double* dt_dev, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (method != 0 && method != 1) return fail(ctx, BEST_ERR_INVALID, "method must be 0 (Euler) or 1 (Heun)");
    if (stage != 0 && !(method == 1 && stage == 1)) return fail(ctx, BEST_ERR_INVALID, "stage must be 0, or 1 for Heun");
    if (!logf_dev || !k1_dev || !t_dev || !dt_dev) return fail(ctx, BEST_ERR_INVALID, "logf, k1, t and dt must not be NULL");
    if (method == 1 && !fstar_dev) return fail(ctx, BEST_ERR_INVALID, "Heun needs fstar");
    if (stage == 1 && !k2_dev) return fail(ctx, BEST_ERR_INVALID, "the Heun corrector needs k2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    stage_kernel<<<1, 1024, 0, st>>>(ctx->geo, method, stage, logf_dev, k1_dev, k2_dev, fstar_dev, t_dev, dt_dev,
                                     ctx->d_ts);
    ctx->launches = 1;
    CK(cudaGetLastError());
    return BEST_OK;
}

static best_status step_common(best_ctx* ctx, double* logf, double* t_dev, double* dt_dev, double* C_dev,
                               void* stream, bool heun) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!logf || !t_dev || !dt_dev) return fail(ctx, BEST_ERR_INVALID, "logf, t and dt must not be NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Geometry& g = ctx->geo;
    ctx->launches = 0;
    double* k1 = C_dev ? C_dev : ctx->d_k1;
    set_time_kernel<<<1, 32, 0, st>>>(g, ctx->d_ts, t_dev, 0.0, 1, ctx->d_mass_law);
    ctx->launches += 1;
    best_status s = enqueue_sweep(ctx, logf, 1, k1, nullptr, st);
    if (s != BEST_OK) return s;
    step_first_kernel<<<1, 1024, 0, st>>>(g, logf, ctx->d_fgrid, k1, t_dev, dt_dev, ctx->d_ts, ctx->d_fstar,
                                          heun ? 1 : 0);
    ctx->launches += 1;
    if (heun) {
        set_time_kernel<<<1, 32, 0, st>>>(g, ctx->d_ts, t_dev, 0.0, 2, ctx->d_mass_law);
        ctx->launches += 1;
        s = enqueue_sweep(ctx, ctx->d_fstar, 0, ctx->d_k2, nullptr, st);
        if (s != BEST_OK) return s;
        heun_correct_kernel<<<1, 1024, 0, st>>>(g, logf, ctx->d_fstar, k1, ctx->d_k2, t_dev, dt_dev, ctx->d_ts);
        ctx->launches += 1;
    }
    CK(cudaGetLastError());
    return BEST_OK;
}

best_status best_step_euler(best_ctx* ctx, double* logf_dev, double* t_dev, double* dt_dev, double* C_dev,
                            void* stream) {
    return step_common(ctx, logf_dev, t_dev, dt_dev, C_dev, stream, false);
}

best_status best_step_heun(best_ctx* ctx, double* logf_dev, double* t_dev, double* dt_dev, double* C_dev,
                           void* stream) {
    return step_common(ctx, logf_dev, t_dev, dt_dev, C_dev, stream, true);
}

best_status best_evolve(best_ctx* ctx, int32_t method, int32_t n_steps, double* logf_dev, double* t_dev,
                        double* dt_dev, double dt_request, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (method != 0 && method != 1) return fail(ctx, BEST_ERR_INVALID, "method must be 0 (Euler) or 1 (Heun)");
    if (n_steps < 0) return fail(ctx, BEST_ERR_INVALID, "n_steps must be >= 0");
    if (!logf_dev || !t_dev || !dt_dev) return fail(ctx, BEST_ERR_INVALID, "logf, t and dt must not be NULL");
    if (!(dt_request > 0.0)) return fail(ctx, BEST_ERR_INVALID, "dt_request must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread)
        return fail(ctx, BEST_ERR_INVALID, "best_evolve needs a created (non-default) stream to capture on");
    const bool same = ctx->graph && ctx->g_logf == logf_dev && ctx->g_t == t_dev && ctx->g_dt == dt_dev &&
                      ctx->g_method == method;
    if (!same) {
        if (ctx->graph) {
            CK(cudaGraphExecDestroy(ctx->graph));
            ctx->graph = nullptr;
        }
        // With profiling enabled the timing events are captured too: after the
        // replays they hold the sample-kernel times of the last replayed step.
        ctx->ev_used = 0;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        copy_scalar_kernel<<<1, 1, 0, st>>>(dt_dev, ctx->d_dtreq);
        best_status s = step_common(ctx, logf_dev, t_dev, dt_dev, nullptr, stream, method == 1);
        cudaGraph_t gr = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(st, &gr);
        ctx->g_events = ctx->ev_used;
        if (s != BEST_OK) {
            if (gr) cudaGraphDestroy(gr);
            return s;
        }
        if (ec != cudaSuccess) return fail(ctx, BEST_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&ctx->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (ei != cudaSuccess) {
            ctx->graph = nullptr;
            return fail(ctx, BEST_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
        }
        ctx->g_logf = logf_dev;
        ctx->g_t = t_dev;
        ctx->g_dt = dt_dev;
        ctx->g_method = method;
        ctx->g_launches = ctx->launches + 1;
    }
    store_scalar_kernel<<<1, 1, 0, st>>>(ctx->d_dtreq, dt_request);
    CK(cudaGetLastError());
    for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(ctx->graph, st));
    if (n_steps > 0) ctx->ev_used = ctx->g_events;     // events of the last replay
    ctx->launches = 1 + n_steps * ctx->g_launches;
    return BEST_OK;
}

best_status best_launch_shape(const best_ctx* ctx, int32_t* ctas_per_sm, int32_t* threads,
                              int32_t* samples_per_lane) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    const SampleVariant& v = ctx->variants[ctx->variant];
    if (ctas_per_sm) *ctas_per_sm = v.mb;
    if (threads) *threads = v.threads;
    if (samples_per_lane) *samples_per_lane = v.spl;
    return BEST_OK;
}

best_status best_autotune(best_ctx* ctx, const double* f_dev, double t, int32_t* ctas_per_sm, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!f_dev) return fail(ctx, BEST_ERR_INVALID, "f_dev must not be NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(st));
    const Geometry& g = ctx->geo;
    const size_t ne = static_cast<size_t>(g.n_tasks) * g.map_stride;
    double *edges0 = nullptr, *prev0 = nullptr, *Ctmp = nullptr;
    TaskDesc* tasks0 = nullptr;                   // the budgets live in the task descriptors
    TimeState ts0;
    auto release = [&]() { cudaFree(edges0); cudaFree(prev0); cudaFree(Ctmp); cudaFree(tasks0); };
    if (dalloc(&edges0, ne) != cudaSuccess || dalloc(&prev0, g.n_tasks) != cudaSuccess ||
        dalloc(&Ctmp, static_cast<size_t>(g.n_species) * g.n_grid) != cudaSuccess ||
        dalloc(&tasks0, g.n_tasks) != cudaSuccess) {
        release();
        return fail(ctx, BEST_ERR_OOM, "autotune: no memory for the state backup");
    }
    auto restore = [&]() -> best_status {
        CK(cudaMemcpyAsync(ctx->d_edges, edges0, ne * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_prev, prev0, g.n_tasks * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_tasks, tasks0, g.n_tasks * sizeof(TaskDesc), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_ts, &ts0, sizeof(TimeState), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return BEST_OK;
    };
    best_status s = BEST_OK;
    do {
        if (cudaMemcpy(edges0, ctx->d_edges, ne * sizeof(double), cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemcpy(prev0, ctx->d_prev, g.n_tasks * sizeof(double), cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemcpy(tasks0, ctx->d_tasks, g.n_tasks * sizeof(TaskDesc), cudaMemcpyDeviceToDevice) != cudaSuccess ||
            cudaMemcpy(&ts0, ctx->d_ts, sizeof(TimeState), cudaMemcpyDeviceToHost) != cudaSuccess) {
            s = fail(ctx, BEST_ERR_CUDA, "autotune: state backup failed");
            break;
        }
        const bool prof = ctx->profiling;
        int best_v = ctx->variant;
        double best_ms = 1e300;
        for (int v = 0; v < ctx->n_variants && s == BEST_OK; ++v) {
            // restored first: the partition is built from the restored budgets
            if ((s = restore()) != BEST_OK) break;
            if ((s = set_variant(ctx, v)) != BEST_OK) break;
            ctx->profiling = true;
            ctx->ev_used = 0;
            s = best_collision_eval(ctx, f_dev, t, Ctmp, nullptr, stream);
            double ms = 0.0;
            int64_t n = 0;
            if (s == BEST_OK) s = best_profile_read(ctx, &ms, &n);
            ctx->profiling = prof;
            ctx->ev_used = 0;
            if (s == BEST_OK && ms < best_ms) {
                best_ms = ms;
                best_v = v;
            }
        }
        if (s != BEST_OK) break;
        if ((s = restore()) != BEST_OK) break;
        s = set_variant(ctx, best_v);
        if (ctas_per_sm) *ctas_per_sm = ctx->variants[best_v].mb;
    } while (false);
    release();
    return s;
}

// CTAs of the persistent adjoint / tangent sample kernel fn: as many as fit
// on the device at once (the kernel takes the partition's chunks from a
// counter, so its grid need not match the sample kernel's).
static cudaError_t adjoint_grid(const best_ctx* ctx, const void* fn, size_t smem, int* grid) {
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
    *grid = std::max(1, std::min(nsm * std::max(occ, 1), ctx->n_chunks));
    return e;
}

best_status best_collision_vjp(best_ctx* ctx, const double* f_dev, double t, const double* v_dev, double* C_dev,
                               double* gf_dev, double* gm_dev, double* gcoupling_dev, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!f_dev || !v_dev || !C_dev || !gf_dev || !gm_dev || !gcoupling_dev)
        return fail(ctx, BEST_ERR_INVALID, "f, v, C, gf, gm and gcoupling must not be NULL");
    if (!std::isfinite(t)) return fail(ctx, BEST_ERR_INVALID, "t must be finite");
    const Geometry& g = ctx->geo;
    const bool f32 = ctx->precision == BEST_FP32;
    void* fn = vjp_kernel_ptr(f32, ctx->nmax_legs, ctx->any_me);
    int max_optin = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (ctx->vjp_smem > static_cast<size_t>(max_optin))
        return fail(ctx, BEST_ERR_INVALID, "adjoint tables need %zu B of shared memory (max %d)", ctx->vjp_smem, max_optin);
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, fn));
    if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) < ctx->vjp_smem)
        CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ctx->vjp_smem)));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->launches = 0;
    set_time_kernel<<<1, 32, 0, st>>>(g, ctx->d_ts, nullptr, t, 0, ctx->d_mass_law);
    spline_build_kernel<<<g.n_species, 256, ctx->spline_smem, st>>>(
        g, f_dev, 0, ctx->d_knots, ctx->d_ts, ctx->d_sconst, ctx->d_fgrid, ctx->d_coef64, ctx->d_coef32);
    prepare_kernel<<<(g.n_tasks + 127) / 128, 128, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_knots, ctx->d_fgrid,
                                                            ctx->d_ts, ctx->d_prev, ctx->d_tconst, ctx->d_acc, 0,
                                                            ctx->d_width, ctx->d_sconst, ctx->d_tconst32);
    if (ctx->d_map32)
        map32_kernel<<<map32_blocks(g), 256, 0, st>>>(g, ctx->d_tasks, g.n_tasks, ctx->d_edges, ctx->d_map32);
    vjp_seed_kernel<<<(g.n_tasks + 127) / 128, 128, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_tconst, v_dev,
                                                             ctx->d_u);
    CK(cudaMemsetAsync(ctx->d_gcoef, 0, sizeof(double) * g.n_species * (g.n_grid - 1) * 4, st));
    const IterPlan& pl = ctx->plans[0];
    VjpParams V{};
    EvalParams& P = V.E;
    P.geo = g;
    P.sides = ctx->d_sides;
    P.tasks = ctx->d_tasks;
    P.tconst = ctx->d_tconst;
    P.tconst32 = ctx->d_tconst32;
    P.sconst = ctx->d_sconst;
    P.ts = ctx->d_ts;
    P.edges = ctx->d_edges;
    P.map32 = ctx->d_map32;
    P.segs = pl.d_segs;
    P.cta_seg = pl.d_cta_seg;
    P.n_chunks = ctx->n_chunks;
    P.chunk_counter = ctx->d_chunk_ctr + ctx->max_nitn;
    P.coef = f32 ? static_cast<const void*>(ctx->d_coef32) : static_cast<const void*>(ctx->d_coef64);
    P.knots = f32 ? static_cast<const void*>(ctx->d_knots32) : static_cast<const void*>(ctx->d_knots);
    P.partials = ctx->d_partials;
    P.itn = 0xFFFFu;                                   // the adjoint's reserved iteration index
    P.smem_spline_elems = g.n_species * 4 * (g.n_grid - 1) + g.n_grid;
    const PhiloxKey key = philox_key(g.seed);
    for (int r = 0; r < 20; ++r) P.rk[r] = key.k[r];
    V.task_u = ctx->d_u;
    V.gcoef = ctx->d_gcoef;
    V.dcoef = nullptr;
    V.dtail = nullptr;
    void* args[] = {&V};
    int vgrid = 0;
    CK(adjoint_grid(ctx, fn, ctx->vjp_smem, &vgrid));
    CK(cudaMemsetAsync(P.chunk_counter, 0, sizeof(int32_t), st));
    CK(cudaLaunchKernel(fn, dim3(vgrid), dim3(kThreads), args, ctx->vjp_smem, st));
    vjp_task_kernel<<<(pl.n_active + 127) / 128, 128, 0, st>>>(g, pl.d_active, pl.d_task_seg, pl.d_segs,
                                                               ctx->d_partials, pl.n_active, ctx->d_vjp_tot);
    vjp_finish_kernel<<<1, 32, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_tconst, ctx->d_sconst, ctx->d_ts, v_dev,
                                        ctx->d_u, ctx->d_vjp_tot, ctx->d_coupling, C_dev, gf_dev, gm_dev,
                                        gcoupling_dev, ctx->d_gtail, ctx->n_processes);
    spline_adjoint_kernel<<<g.n_species, 32, ctx->spline_smem, st>>>(g, ctx->d_knots, ctx->d_fgrid, ctx->d_sconst,
                                                                     ctx->d_ts, ctx->d_gcoef, ctx->d_gtail, gf_dev,
                                                                     gm_dev);
    ctx->launches = ctx->d_map32 ? 10 : 9;
    CK(cudaGetLastError());
    return BEST_OK;
}

namespace {
struct StateHeader {
    uint64_t magic;         // "BESTSTT1"
    uint64_t config_hash;   // FNV-1a of the task and side descriptors and the grid
    int64_t n_tasks;
    int64_t map_stride;
};
constexpr uint64_t kStateMagic = 0x3154545354534542ull;

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t k = 0; k < n; ++k) {
        h ^= c[k];
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t config_hash(const best_ctx* ctx) {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, ctx->sides.data(), ctx->sides.size() * sizeof(SideDesc));
    h = fnv1a(h, ctx->tasks.data(), ctx->tasks.size() * sizeof(TaskDesc));
    const double grid[3] = {ctx->geo.q_min, ctx->geo.q_max, static_cast<double>(ctx->geo.n_grid)};
    h = fnv1a(h, grid, sizeof(grid));
    h = fnv1a(h, &ctx->geo.seed, sizeof(ctx->geo.seed));
    return h;
}
}  // namespace

// Fixed-sample C~ and its tangent J u (the launches of best_collision_jvp).
// setup: time state, spline of f and per-task constants, needed whenever f or
// t changed since the previous call.
static best_status enqueue_jvp(best_ctx* ctx, const double* f_dev, double t, const double* u_dev, double* C_dev,
                               double* JU_dev, cudaStream_t st, bool setup) {
    const Geometry& g = ctx->geo;
    const bool f32 = ctx->precision == BEST_FP32;
    void* fn = jvp_kernel_ptr(f32, ctx->nmax_legs, ctx->any_me);
    if (!ctx->jvp_ready) {
        int max_optin = 0, dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (ctx->jvp_smem > static_cast<size_t>(max_optin))
            return fail(ctx, BEST_ERR_INVALID, "tangent tables need %zu B of shared memory (max %d)", ctx->jvp_smem,
                        max_optin);
        cudaFuncAttributes fa{};
        CK(cudaFuncGetAttributes(&fa, fn));
        if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) < ctx->jvp_smem)
            CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(ctx->jvp_smem)));
        ctx->jvp_ready = true;
    }
    if (setup) {
        set_time_kernel<<<1, 32, 0, st>>>(g, ctx->d_ts, nullptr, t, 0, ctx->d_mass_law);
        spline_build_kernel<<<g.n_species, 256, ctx->spline_smem, st>>>(
            g, f_dev, 0, ctx->d_knots, ctx->d_ts, ctx->d_sconst, ctx->d_fgrid, ctx->d_coef64, ctx->d_coef32);
        prepare_kernel<<<(g.n_tasks + 127) / 128, 128, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_knots,
                                                                ctx->d_fgrid, ctx->d_ts, ctx->d_prev, ctx->d_tconst,
                                                                ctx->d_acc, 0, ctx->d_width, ctx->d_sconst,
                                                                ctx->d_tconst32);
        if (ctx->d_map32) {
            map32_kernel<<<map32_blocks(g), 256, 0, st>>>(g, ctx->d_tasks, g.n_tasks, ctx->d_edges, ctx->d_map32);
            ctx->launches += 1;
        }
        ctx->launches += 3;
    }
    jvp_seed_kernel<<<(g.n_tasks + 127) / 128, 128, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_tconst,
                                                             ctx->d_sconst, u_dev, ctx->d_u);
    spline_tangent_kernel<<<g.n_species, 256, ctx->spline_smem, st>>>(g, u_dev, ctx->d_knots, ctx->d_fgrid,
                                                                      ctx->d_sconst, ctx->d_ts, ctx->d_dcoef64,
                                                                      ctx->d_dcoef32, ctx->d_dtail);
    const IterPlan& pl = ctx->plans[0];
    VjpParams V{};
    EvalParams& P = V.E;
    P.geo = g;
    P.sides = ctx->d_sides;
    P.tasks = ctx->d_tasks;
    P.tconst = ctx->d_tconst;
    P.tconst32 = ctx->d_tconst32;
    P.sconst = ctx->d_sconst;
    P.ts = ctx->d_ts;
    P.edges = ctx->d_edges;
    P.map32 = ctx->d_map32;
    P.segs = pl.d_segs;
    P.cta_seg = pl.d_cta_seg;
    P.n_chunks = ctx->n_chunks;
    P.chunk_counter = ctx->d_chunk_ctr + ctx->max_nitn;
    P.coef = f32 ? static_cast<const void*>(ctx->d_coef32) : static_cast<const void*>(ctx->d_coef64);
    P.knots = f32 ? static_cast<const void*>(ctx->d_knots32) : static_cast<const void*>(ctx->d_knots);
    P.partials = ctx->d_partials;
    P.itn = 0xFFFFu;                                   // same samples as best_collision_vjp
    P.smem_spline_elems = g.n_species * 4 * (g.n_grid - 1) + g.n_grid;
    const PhiloxKey key = philox_key(g.seed);
    for (int r = 0; r < 20; ++r) P.rk[r] = key.k[r];
    V.task_u = ctx->d_u;
    V.gcoef = nullptr;
    V.dcoef = f32 ? static_cast<const void*>(ctx->d_dcoef32) : static_cast<const void*>(ctx->d_dcoef64);
    V.dtail = ctx->d_dtail;
    void* args[] = {&V};
    int vgrid = 0;
    CK(adjoint_grid(ctx, fn, ctx->jvp_smem, &vgrid));
    CK(cudaMemsetAsync(P.chunk_counter, 0, sizeof(int32_t), st));
    CK(cudaLaunchKernel(fn, dim3(vgrid), dim3(kThreads), args, ctx->jvp_smem, st));
    vjp_task_kernel<<<(pl.n_active + 127) / 128, 128, 0, st>>>(g, pl.d_active, pl.d_task_seg, pl.d_segs,
                                                               ctx->d_partials, pl.n_active, ctx->d_vjp_tot);
    jvp_finish_kernel<<<1, 32, 0, st>>>(g, ctx->d_sides, ctx->d_tasks, ctx->d_tconst, ctx->d_vjp_tot, C_dev, JU_dev);
    ctx->launches += 5;
    CK(cudaGetLastError());
    return BEST_OK;
}

best_status best_collision_jvp(best_ctx* ctx, const double* f_dev, double t, const double* u_dev, double* C_dev,
                               double* JU_dev, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!f_dev || !u_dev || !C_dev || !JU_dev) return fail(ctx, BEST_ERR_INVALID, "f, u, C and JU must not be NULL");
    if (!std::isfinite(t)) return fail(ctx, BEST_ERR_INVALID, "t must be finite");
    ctx->launches = 0;
    return enqueue_jvp(ctx, f_dev, t, u_dev, C_dev, JU_dev, static_cast<cudaStream_t>(stream), true);
}

// Newton-Krylov implicit Euler (kernels in newton.cu).
static best_status nk_buffers(best_ctx* ctx, int m) {
    const int64_t N = static_cast<int64_t>(ctx->geo.n_species) * ctx->geo.n_grid;
    if (ctx->nk_m >= m && ctx->d_nk) return BEST_OK;
    if (ctx->d_nk) cudaFree(ctx->d_nk);
    ctx->d_nk = nullptr;
    ctx->nk_m = 0;
    const size_t total = static_cast<size_t>(N) * (m + 1 + 10) + static_cast<size_t>(m + 1) * m + 3 * m + 2 + 8;
    CK(cudaMalloc(&ctx->d_nk, total * sizeof(double)));
    ctx->nk_m = m;
    return BEST_OK;
}

static best_status read_stat(best_ctx* ctx, const double* d_stat, double* h_stat, cudaStream_t st) {
    CK(cudaMemcpyAsync(h_stat, d_stat, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return BEST_OK;
}

best_status best_step_implicit_euler(best_ctx* ctx, double* logf_dev, double t, double dt, int32_t train,
                                     double tol, int32_t max_newton, int32_t krylov_dim, double krylov_rtol,
                                     double* info, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!logf_dev) return fail(ctx, BEST_ERR_INVALID, "logf must not be NULL");
    if (!std::isfinite(t) || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, BEST_ERR_INVALID, "need finite t, dt > 0");
    if (!(tol > 0.0)) return fail(ctx, BEST_ERR_INVALID, "tol must be > 0");
    if (max_newton < 1) return fail(ctx, BEST_ERR_INVALID, "max_newton must be >= 1");
    if (krylov_dim < 1 || krylov_dim > 64) return fail(ctx, BEST_ERR_INVALID, "krylov_dim must be in [1, 64]");
    if (!(krylov_rtol > 0.0 && krylov_rtol < 1.0)) return fail(ctx, BEST_ERR_INVALID, "krylov_rtol must be in (0, 1)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Geometry& g = ctx->geo;
    const int N = g.n_species * g.n_grid;
    const int m = krylov_dim;
    best_status s = nk_buffers(ctx, m);
    if (s != BEST_OK) return s;
    ctx->launches = 0;
    const int mm = ctx->nk_m;               // layout follows the allocated Krylov dimension
    double* V = ctx->d_nk;
    double* gn = V + static_cast<size_t>(N) * (mm + 1);
    double* ga = gn + N;                    // accepted iterate
    double* gt = ga + N;                    // trial iterate
    double* f = gt + N;
    double* r = f + N;
    double* Qd = r + N;
    double* d = Qd + N;
    double* C = d + N;
    double* JU = C + N;
    double* u = JU + N;
    double* H = u + N;
    double* cs = H + static_cast<size_t>(mm + 1) * mm;
    double* sn = cs + mm;
    double* gvec = sn + mm;
    double* stat = gvec + mm + 2;
    double hs[8] = {};
    const int eb = (N + 255) / 256;
    const double t1 = t + dt;

    if (train) {
        set_time_kernel<<<1, 32, 0, st>>>(g, ctx->d_ts, nullptr, t1, 0, ctx->d_mass_law);
        ctx->launches += 1;
        s = enqueue_sweep(ctx, logf_dev, 1, ctx->d_k1, nullptr, st);
        if (s != BEST_OK) return s;
    }
    CK(cudaMemcpyAsync(gn, logf_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ga, logf_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(u, 0, N * sizeof(double), st));
    nk_exp_kernel<<<eb, 256, 0, st>>>(N, ga, f);
    ctx->launches += 1;
    s = enqueue_jvp(ctx, f, t1, u, C, JU, st, true);
    if (s != BEST_OK) return s;
    nk_residual_kernel<<<1, 1024, 0, st>>>(N, ga, gn, C, f, dt, r, Qd, stat);
    ctx->launches += 1;
    s = read_stat(ctx, stat, hs, st);
    if (s != BEST_OK) return s;
    if (hs[4] != 0.0) return fail(ctx, BEST_ERR_NUMERIC, "implicit Euler: non-finite residual at the initial iterate");
    double rn2 = hs[0], rinf = hs[1];
    int newton = 0, krylov = 0, halvings = 0;
    while (rinf > tol && newton < max_newton) {
        gmres_start_kernel<<<1, 1024, 0, st>>>(N, mm, r, V, gvec);
        ctx->launches += 1;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            nk_direction_kernel<<<eb, 256, 0, st>>>(N, f, V + static_cast<size_t>(j) * N, u);
            ctx->launches += 1;
            s = enqueue_jvp(ctx, f, t1, u, C, JU, st, false);
            if (s != BEST_OK) return s;
            gmres_arnoldi_kernel<<<1, 1024, 0, st>>>(N, mm, j, dt, f, Qd, JU, V, H, cs, sn, gvec, stat);
            ctx->launches += 1;
            ++krylov;
            s = read_stat(ctx, stat, hs, st);
            if (s != BEST_OK) return s;
            k = j + 1;
            if (hs[2] <= krylov_rtol * rn2 || !(hs[3] > 1e-300 * rn2)) break;
        }
        gmres_update_kernel<<<1, 1024, 0, st>>>(N, mm, k, V, H, gvec, d);
        ctx->launches += 1;
        // backtracking on ||R||_2 (Armijo with slope -||R||^2 of the exact Newton direction)
        double lambda = 1.0;
        for (int ls = 0;; ++ls) {
            nk_axpy_kernel<<<eb, 256, 0, st>>>(N, ga, d, lambda, gt);
            nk_exp_kernel<<<eb, 256, 0, st>>>(N, gt, f);
            CK(cudaMemsetAsync(u, 0, N * sizeof(double), st));
            ctx->launches += 2;
            s = enqueue_jvp(ctx, f, t1, u, C, JU, st, true);
            if (s != BEST_OK) return s;
            nk_residual_kernel<<<1, 1024, 0, st>>>(N, gt, gn, C, f, dt, r, Qd, stat);
            ctx->launches += 1;
            s = read_stat(ctx, stat, hs, st);
            if (s != BEST_OK) return s;
            const bool ok = hs[4] == 0.0 && hs[0] <= (1.0 - 1e-4 * lambda) * rn2;
            if (ok || ls == 10) {
                if (hs[4] != 0.0) return fail(ctx, BEST_ERR_NUMERIC, "implicit Euler: non-finite residual");
                std::swap(ga, gt);
                rn2 = hs[0];
                rinf = hs[1];
                break;
            }
            lambda *= 0.5;
            ++halvings;
        }
        ++newton;
    }
    const bool converged = rinf <= tol;
    if (info) {
        info[0] = newton;
        info[1] = krylov;
        info[2] = rinf;
        info[3] = converged ? 1.0 : 0.0;
        info[4] = halvings;
    }
    if (!converged)
        return fail(ctx, BEST_ERR_NUMERIC, "implicit Euler: Newton stopped at ||R||_inf = %.3e > tol %.3e after %d iterations",
                    rinf, tol, newton);
    CK(cudaMemcpyAsync(logf_dev, ga, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return BEST_OK;
}

int64_t best_state_size(const best_ctx* ctx) {
    if (!ctx) return 0;
    const int64_t T = ctx->geo.n_tasks;
    return static_cast<int64_t>(sizeof(StateHeader)) + 8 * T * ctx->geo.map_stride + 8 * T +
           static_cast<int64_t>(sizeof(TimeState)) + 16 * static_cast<int64_t>(ctx->n_processes) +
           4 * ctx->strat_total_h + (ctx->any_budget ? 8 * T : 0);
}

best_status best_save_state(best_ctx* ctx, void* host_buf, int64_t size) {
    if (!ctx || !host_buf) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    if (size < best_state_size(ctx)) return fail(ctx, BEST_ERR_INVALID, "state buffer too small");
    CK(cudaDeviceSynchronize());
    char* p = static_cast<char*>(host_buf);
    StateHeader hd{kStateMagic, config_hash(ctx), ctx->geo.n_tasks, ctx->geo.map_stride};
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const size_t ne = static_cast<size_t>(ctx->geo.n_tasks) * ctx->geo.map_stride;
    CK(cudaMemcpy(p, ctx->d_edges, ne * sizeof(double), cudaMemcpyDeviceToHost));
    p += ne * sizeof(double);
    CK(cudaMemcpy(p, ctx->d_prev, ctx->geo.n_tasks * sizeof(double), cudaMemcpyDeviceToHost));
    p += ctx->geo.n_tasks * sizeof(double);
    CK(cudaMemcpy(p, ctx->d_ts, sizeof(TimeState), cudaMemcpyDeviceToHost));
    p += sizeof(TimeState);
    CK(cudaMemcpy(p, ctx->d_width, ctx->n_processes * sizeof(double), cudaMemcpyDeviceToHost));
    p += ctx->n_processes * sizeof(double);
    CK(cudaMemcpy(p, ctx->d_width_rel, ctx->n_processes * sizeof(double), cudaMemcpyDeviceToHost));
    p += ctx->n_processes * sizeof(double);
    if (ctx->strat_total_h > 0)
        CK(cudaMemcpy(p, ctx->d_strat_m, ctx->strat_total_h * sizeof(int32_t), cudaMemcpyDeviceToHost));
    p += ctx->strat_total_h * sizeof(int32_t);
    if (ctx->any_budget) {
        std::vector<TaskDesc> cur(ctx->geo.n_tasks);
        CK(cudaMemcpy(cur.data(), ctx->d_tasks, cur.size() * sizeof(TaskDesc), cudaMemcpyDeviceToHost));
        for (size_t t = 0; t < cur.size(); ++t) std::memcpy(p + 8 * t, &cur[t].neval, 8);
    }
    return BEST_OK;
}

best_status best_load_state(best_ctx* ctx, const void* host_buf, int64_t size) {
    if (!ctx || !host_buf) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    if (size < best_state_size(ctx)) return fail(ctx, BEST_ERR_INVALID, "state buffer too small");
    const char* p = static_cast<const char*>(host_buf);
    StateHeader hd;
    std::memcpy(&hd, p, sizeof(hd));
    if (hd.magic != kStateMagic) return fail(ctx, BEST_ERR_INVALID, "not a libbest state");
    if (hd.n_tasks != ctx->geo.n_tasks || hd.map_stride != ctx->geo.map_stride || hd.config_hash != config_hash(ctx))
        return fail(ctx, BEST_ERR_INVALID, "state was saved from a different configuration");
    p += sizeof(hd);
    CK(cudaDeviceSynchronize());
    const size_t ne = static_cast<size_t>(ctx->geo.n_tasks) * ctx->geo.map_stride;
    CK(cudaMemcpy(ctx->d_edges, p, ne * sizeof(double), cudaMemcpyHostToDevice));
    p += ne * sizeof(double);
    CK(cudaMemcpy(ctx->d_prev, p, ctx->geo.n_tasks * sizeof(double), cudaMemcpyHostToDevice));
    p += ctx->geo.n_tasks * sizeof(double);
    CK(cudaMemcpy(ctx->d_ts, p, sizeof(TimeState), cudaMemcpyHostToDevice));
    p += sizeof(TimeState);
    CK(cudaMemcpy(ctx->d_width, p, ctx->n_processes * sizeof(double), cudaMemcpyHostToDevice));
    p += ctx->n_processes * sizeof(double);
    CK(cudaMemcpy(ctx->d_width_rel, p, ctx->n_processes * sizeof(double), cudaMemcpyHostToDevice));
    p += ctx->n_processes * sizeof(double);
    if (ctx->strat_total_h > 0) {
        // the allocation, then the items rebuilt from it
        CK(cudaMemcpy(ctx->d_strat_m, p, ctx->strat_total_h * sizeof(int32_t), cudaMemcpyHostToDevice));
        strat_init_kernel<<<ctx->geo.n_tasks, 256>>>(ctx->d_tasks, ctx->d_strat_m, ctx->d_item_h, 0);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
    }
    p += ctx->strat_total_h * sizeof(int32_t);
    if (ctx->any_budget) {
        // the budgets, then the partition built from them
        std::vector<TaskDesc> cur(ctx->geo.n_tasks);
        CK(cudaMemcpy(cur.data(), ctx->d_tasks, cur.size() * sizeof(TaskDesc), cudaMemcpyDeviceToHost));
        for (size_t t = 0; t < cur.size(); ++t) std::memcpy(&cur[t].neval, p + 8 * t, 8);
        CK(cudaMemcpy(ctx->d_tasks, cur.data(), cur.size() * sizeof(TaskDesc), cudaMemcpyHostToDevice));
        plan_kernel<<<1, 1024>>>(ctx->d_tasks, ctx->max_nitn, ctx->d_plandev, ctx->grid,
                                 ctx->precision == BEST_FP32 ? 1 : 0, ctx->d_plan_scratch);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
    }
    return BEST_OK;
}

best_status best_moments(best_ctx* ctx, const double* f_dev, double t, double* n_dev, double* rho_dev,
                         void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!f_dev || !n_dev || !rho_dev) return fail(ctx, BEST_ERR_INVALID, "f, n and rho must not be NULL");
    if (!std::isfinite(t)) return fail(ctx, BEST_ERR_INVALID, "t must be finite");
    const Geometry& g = ctx->geo;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    set_time_kernel<<<1, 32, 0, st>>>(g, ctx->d_ts, nullptr, t, 0, ctx->d_mass_law);
    spline_build_kernel<<<g.n_species, 256, ctx->spline_smem, st>>>(
        g, f_dev, 0, ctx->d_knots, ctx->d_ts, ctx->d_sconst, ctx->d_fgrid, ctx->d_coef64, ctx->d_coef32);
    moments_kernel<<<g.n_species, 256, 0, st>>>(g, ctx->d_knots, ctx->d_coef64, ctx->d_ts, n_dev, rho_dev);
    ctx->launches = 3;
    CK(cudaGetLastError());
    return BEST_OK;
}

best_status best_get_strata(best_ctx* ctx, int32_t task, int32_t* M, int32_t* H, int32_t* m) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (task < 0 || task >= ctx->geo.n_tasks) return fail(ctx, BEST_ERR_INVALID, "task out of range");
    const TaskDesc& td = ctx->tasks[task];
    if (M) *M = td.strat_M;
    if (H) *H = td.strat_H;
    if (m && td.strat_H > 0) {
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(m, ctx->d_strat_m + td.strat_off_h, td.strat_H * sizeof(int32_t), cudaMemcpyDeviceToHost));
    }
    return BEST_OK;
}

best_status best_species_masses(const best_ctx* ctx, double t, double* m) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!m || !std::isfinite(t)) return fail(const_cast<best_ctx*>(ctx), BEST_ERR_INVALID, "need m and a finite t");
    for (size_t s = 0; s < ctx->mass_law.size(); ++s) m[s] = mass_at(ctx->mass_law[s], t);
    return BEST_OK;
}

best_status best_get_widths(best_ctx* ctx, double* w, double* rel) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    CK(cudaDeviceSynchronize());
    if (w) CK(cudaMemcpy(w, ctx->d_width, ctx->n_processes * sizeof(double), cudaMemcpyDeviceToHost));
    if (rel) CK(cudaMemcpy(rel, ctx->d_width_rel, ctx->n_processes * sizeof(double), cudaMemcpyDeviceToHost));
    return BEST_OK;
}

best_status best_set_widths(best_ctx* ctx, const double* w) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    if (!w) return fail(ctx, BEST_ERR_INVALID, "w is NULL");
    std::vector<double> cur(ctx->n_processes);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(cur.data(), ctx->d_width, cur.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int p = 0; p < ctx->n_processes; ++p) {
        if (ctx->width_mode[p] == 0) continue;
        if (!(w[p] > 0.0) || !std::isfinite(w[p]))
            return fail(ctx, BEST_ERR_INVALID, "process %d: width must be > 0", p);
        cur[p] = w[p];
    }
    CK(cudaMemcpy(ctx->d_width, cur.data(), cur.size() * sizeof(double), cudaMemcpyHostToDevice));
    return BEST_OK;
}

int32_t best_num_tasks(const best_ctx* ctx) { return ctx ? ctx->geo.n_tasks : 0; }
int32_t best_num_side_integrals(const best_ctx* ctx) { return ctx ? ctx->geo.n_side : 0; }
int64_t best_map_stride(const best_ctx* ctx) { return ctx ? ctx->geo.map_stride : 0; }
int32_t best_last_launch_count(const best_ctx* ctx) { return ctx ? ctx->launches : 0; }

int64_t best_sweep_samples(const best_ctx* ctx, int32_t iteration) {
    if (!ctx) return 0;
    std::vector<TaskDesc> cur;
    if (ctx->any_budget) {
        // the budgets of the next sweep, as the device holds them (synchronises)
        cur.resize(ctx->tasks.size());
        if (cudaMemcpy(cur.data(), ctx->d_tasks, cur.size() * sizeof(TaskDesc), cudaMemcpyDeviceToHost) != cudaSuccess)
            return -1;
    }
    const std::vector<TaskDesc>& ts = ctx->any_budget ? cur : ctx->tasks;
    int64_t tot = 0;
    for (const TaskDesc& td : ts) {
        if (iteration < 0) tot += td.neval * td.nitn;
        else if (td.nitn > iteration) tot += td.neval;
    }
    return tot;
}

best_status best_get_budgets(best_ctx* ctx, int64_t* neval, void* stream) {
    if (!ctx || !neval) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    std::vector<TaskDesc> cur(ctx->tasks.size());
    CK(cudaMemcpy(cur.data(), ctx->d_tasks, cur.size() * sizeof(TaskDesc), cudaMemcpyDeviceToHost));
    for (size_t t = 0; t < cur.size(); ++t) neval[t] = cur[t].neval;
    return BEST_OK;
}

best_status best_chunk_bounds(int64_t cost, int32_t grid, int64_t* bounds, int32_t n, int32_t* chunks) {
    if (!chunks || grid < 1 || cost < 0) return fail(nullptr, BEST_ERR_INVALID, "chunk bounds: invalid argument");
    const int K = chunk_count(grid);
    *chunks = K;
    if (!bounds || n < K + 1) return fail(nullptr, BEST_ERR_INVALID, "chunk bounds: bounds needs %d entries", K + 1);
    const ChunkShape sh = chunk_shape(cost, grid);
    for (int c = 0; c <= K; ++c) bounds[c] = chunk_bound(cost, c, sh);
    return BEST_OK;
}

best_status best_partition_groups(best_ctx* ctx, int32_t iteration, int64_t* groups) {
    if (!ctx || !groups) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    if (iteration < 0 || iteration >= ctx->max_nitn) return fail(ctx, BEST_ERR_INVALID, "iteration out of range");
    CK(cudaDeviceSynchronize());
    const IterPlan& pl = ctx->plans[iteration];
    const int T = ctx->geo.n_tasks;
    for (int t = 0; t < T; ++t) groups[t] = 0;
    if (pl.n_active == 0) return BEST_OK;
    // the device may have rebuilt the partition: read its current shape
    std::vector<int32_t> active(pl.n_active), task_seg(pl.n_active + 1), cta_seg(ctx->n_chunks + 1);
    CK(cudaMemcpy(active.data(), pl.d_active, active.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(task_seg.data(), pl.d_task_seg, task_seg.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cta_seg.data(), pl.d_cta_seg, cta_seg.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    const int n_segs = cta_seg[ctx->n_chunks];
    if (n_segs < 0 || cta_seg[0] != 0) return fail(ctx, BEST_ERR_INVALID, "internal: malformed partition");
    std::vector<Segment> segs(n_segs);
    if (n_segs > 0) CK(cudaMemcpy(segs.data(), pl.d_segs, n_segs * sizeof(Segment), cudaMemcpyDeviceToHost));
    for (int c = 0; c < ctx->n_chunks; ++c)
        if (cta_seg[c + 1] < cta_seg[c]) return fail(ctx, BEST_ERR_INVALID, "internal: malformed partition");
    for (int a = 0; a < pl.n_active; ++a) {
        const int t = active[a];
        int64_t next = 0;
        bool ok = task_seg[a] <= task_seg[a + 1] && task_seg[a + 1] <= n_segs;
        for (int k = task_seg[a]; ok && k < task_seg[a + 1]; ++k) {
            ok = segs[k].task == t && segs[k].g0 == next && segs[k].g1 > segs[k].g0;
            next = segs[k].g1;
        }
        groups[t] = ok ? next : -1;
    }
    return BEST_OK;
}

best_status best_get_task_results(best_ctx* ctx, double* mean, double* err, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    std::vector<TaskAcc> acc(ctx->geo.n_tasks);
    CK(cudaMemcpy(acc.data(), ctx->d_acc, acc.size() * sizeof(TaskAcc), cudaMemcpyDeviceToHost));
    for (size_t t = 0; t < acc.size(); ++t) {
        if (mean) mean[t] = acc[t].mean;
        if (err) err[t] = acc[t].err;
    }
    return BEST_OK;
}

best_status best_get_maps(best_ctx* ctx, double* edges_host) {
    if (!ctx || !edges_host) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(edges_host, ctx->d_edges, sizeof(double) * ctx->geo.n_tasks * ctx->geo.map_stride,
                  cudaMemcpyDeviceToHost));
    return BEST_OK;
}

best_status best_set_maps(best_ctx* ctx, const double* edges_host) {
    if (!ctx || !edges_host) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(ctx->d_edges, edges_host, sizeof(double) * ctx->geo.n_tasks * ctx->geo.map_stride,
                  cudaMemcpyHostToDevice));
    return BEST_OK;
}

best_status best_get_call_counter(best_ctx* ctx, uint32_t* call) {
    if (!ctx || !call) return fail(ctx, BEST_ERR_INVALID, "NULL argument");
    CK(cudaDeviceSynchronize());
    TimeState ts;
    CK(cudaMemcpy(&ts, ctx->d_ts, sizeof(TimeState), cudaMemcpyDeviceToHost));
    *call = ts.call;
    return BEST_OK;
}

best_status best_set_call_counter(best_ctx* ctx, uint32_t call) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(reinterpret_cast<char*>(ctx->d_ts) + offsetof(TimeState, call), &call, sizeof(uint32_t),
                  cudaMemcpyHostToDevice));
    return BEST_OK;
}

best_status best_check(best_ctx* ctx, void* stream) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    CK(cudaGetLastError());
    int32_t e = 0;
    CK(cudaMemcpy(&e, reinterpret_cast<char*>(ctx->d_ts) + offsetof(TimeState, error), sizeof(int32_t),
                  cudaMemcpyDeviceToHost));
    if (e != 0) {
        const int32_t z = 0;
        CK(cudaMemcpy(reinterpret_cast<char*>(ctx->d_ts) + offsetof(TimeState, error), &z, sizeof(int32_t),
                      cudaMemcpyHostToDevice));
        return fail(ctx, BEST_ERR_NUMERIC, "non-positive or non-finite f, or a non-finite result");
    }
    return BEST_OK;
}

best_status best_profile_enable(best_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    ctx->profiling = enable != 0;
    ctx->ev_used = 0;
    // events for two sweeps of launches, created now rather than during a capture
    const size_t want = 4 * static_cast<size_t>(ctx->max_nitn) + 8;
    while (ctx->profiling && ctx->ev.size() < want) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->ev.push_back(e);
    }
    return BEST_OK;
}

best_status best_profile_read(best_ctx* ctx, double* sample_kernel_ms, int64_t* launches) {
    if (!ctx) return fail(nullptr, BEST_ERR_INVALID, "ctx is NULL");
    double total = 0.0;
    for (size_t k = 0; k + 1 < ctx->ev_used; k += 2) {
        CK(cudaEventSynchronize(ctx->ev[k + 1]));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[k], ctx->ev[k + 1]));
        total += ms;
    }
    if (sample_kernel_ms) *sample_kernel_ms = total;
    if (launches) *launches = static_cast<int64_t>(ctx->ev_used / 2);
    ctx->ev_used = 0;
    return BEST_OK;
}

const char* best_last_error(const best_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error; }

void best_collision_destroy(best_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
