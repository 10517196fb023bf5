// Device-side data layout of libbest shared by its translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/best.h"

namespace best {

constexpr int kMaxLegs = BEST_MAX_LEGS;
constexpr int kMaxDim = 3 * (BEST_MAX_LEGS - 2);
constexpr int kThreads = 256;          // threads per CTA of the sample kernel
constexpr int kQueueSlots = 64;        // FP32 sample kernel: queued samples per warp

// 32-bit words per queued sample of an n-leg task: the kinematic weight, the
// comoving radii of the n-2 integrated legs, the conserved leg's comoving
// momentum and energy, and the 3(n-2) map increments packed 4 per word.
__host__ __device__ constexpr int queue_words(int nleg) {
    return 1 + (nleg - 2) + 2 + (3 * (nleg - 2) + 3) / 4;
}

// The same for the adjoint (tangent = false) and tangent sample kernels: the
// kinematic weight, the comoving radii, then for the adjoint 1/E of each
// integrated leg; the conserved leg's comoving momentum and energy; for the
// adjoint also 1/E_cons, dE / sigma^2, the fractional-width term and
// d log P / d E.
__host__ __device__ constexpr int vjp_queue_words(int nleg, bool tangent) {
    return tangent ? 3 + (nleg - 2) : 7 + 2 * (nleg - 2);
}
constexpr int kItem = 8;               // samples per item of stratified sampling (a multiple of every group size)

// Stratified sampling in the FP32 sample kernel: the items a lane takes
// between two flushes of its warp's sample queue, and the floats of one
// warp's queue: the plain queue words of each sample plus its item's slot in
// the warp's round of 32 kStratItemsPerLane items and 1 / m_h, then the
// round's per-item sums of w and w^2.
constexpr int kStratItemsPerLane = 2;
__host__ __device__ constexpr int strat_queue_floats(int nleg) {
    return kQueueSlots * (queue_words(nleg) + 2) + 2 * 32 * kStratItemsPerLane;
}
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

// One side integral of Eq. (7): a process, the side of the observed leg and
// the observed species, with the roles of App. A already assigned.
struct SideDesc {
    int32_t n;              // legs
    int32_t n_in;
    int32_t obs;            // observed leg
    int32_t cons;           // conserved leg
    int32_t mult;           // n_S^a of Eq. (7)
    int32_t species_obs;
    int32_t process;
    int32_t side;           // 0: observed leg initial, 1: final
    int32_t leg_species[kMaxLegs];
    int32_t integ[kMaxLegs];   // integrated legs in dimension order
    int32_t own_mask;       // bit k: leg k on the observed side
    int32_t in_mask;        // bit k: leg k initial
    double coupling2;       // |M|^2
    double sigma;           // sigma_E
    double eta_obs;         // eta of the observed species
    int32_t width_mode;     // 0: sigma_E; 1: fractional w; 2: fractional, adapted (App. C)
    int32_t me_on;          // |M|^2 depends on s (me_coef other than {1, 0, 0, 0})
    double width0;          // initial fractional width
    double me_coef[4];      // |M|^2 / coupling^2 = c0 + c1 s + c2 s^2 + c3 s^3
};

// One task: side integral x grid point x {gain, loss}.
struct TaskDesc {
    int32_t si;
    int32_t point;
    int32_t term;           // 0 gain, 1 loss
    int32_t nitn;
    int64_t neval;
    int32_t dim;
    int32_t nbins;
    double alpha;
    // adaptive stratified sampling (VEGAS+); strat_H == 0: off
    int32_t strat_M;        // strata per dimension
    int32_t strat_H;        // hypercubes M^D
    int64_t strat_J;        // items of kItem samples (neval = kItem * strat_J)
    int64_t strat_off_h;    // offset of the task's hypercube arrays
    int64_t strat_off_item; // offset of the task's item arrays
    double strat_beta;      // damping exponent of the allocation
    uint32_t gid;           // task id in the whole grid's numbering (the Philox stream's task word)
    int32_t pad2_;
};

// Per-task values recomputed at the start of every sweep (FP64).
struct TaskConst {
    double K;               // constant factor of the weight (see eval kernel)
    double scale;           // the kernel accumulates w / (K * scale)
    double obs_factor;      // f_obs (loss) or 1 + eta f_obs (gain)
    double f_obs;           // f_a(q_i), the grid value of the observed leg
    double E_obs;           // energy of the observed leg
    double p_obs;           // physical momentum of the observed leg
    double wfrac;           // fractional width w of App. C this sweep (0: absolute sigma_E)
    double c0;              // obs_factor / scale, 0 when the observed leg is cut (App. A)
    double gauss_k;         // exponent factor of the Gaussian: -log2(e) / (2 sigma^2), or -2 log2(e) / w^2
    double inv_sig2_abs;    // 1 / sigma_E^2
    double four_over_w2;    // 4 / w^2 with a fractional width, else 0
    double inv_E_obs;       // 1 / E_obs
};

// FP32 constants of one task's segment set-up in the FP32 sample kernel,
// rounded once per sweep from the FP64 values (seg_const32, in the prepare
// kernel; c0 again when the refinement rescales the task), so that the
// sample kernel's threads only load them: FP64 arithmetic and conversions
// run at a small fraction of the FP32 rate.  Leg arrays hold the
// integrated legs in dimension order (entries past n - 2 unused).
struct SegConst32 {
    float pobs_sig, sgn_obs_E, sgn_cons, m2c, cac, cbc;
    float inv_a, a, c0, gauss_k, e_obs;
    float cons_inw, obs_in_p, obs_in_E, e_cut, eta_c;
    float tlo_a, tlo_b, thi_a, thi_b;
    float q0, lq0_step, qN, inv_step;
    float mass_c, inv_sig2_abs, four_over_w2, inv_E_obs, obs_inw;   // (adjoint and tangent kernels)
    float me[4];
    float sig[kMaxLegs - 2], sgnE[kMaxLegs - 2], m2[kMaxLegs - 2], ca[kMaxLegs - 2], cb[kMaxLegs - 2],
        inw[kMaxLegs - 2], mass[kMaxLegs - 2];
    int32_t spc[kMaxLegs - 2], fd[kMaxLegs - 2];
    int32_t sp_cons, fd_c, frac, me_on, obs_cut;
};

// Mass law of one species: m(t) = m0 + m1 t, or with n >= 2 knots the
// piecewise-linear interpolation of (t[k], m[k]) (t increasing), constant
// beyond the first and last knot.
struct MassLaw {
    double m0, m1;
    int32_t n;
    int32_t pad_;
    double t[BEST_MAX_MASS_KNOTS], m[BEST_MAX_MASS_KNOTS];
};

__host__ __device__ inline double mass_at(const MassLaw& L, double t) {
    if (L.n < 2) return L.m0 + L.m1 * t;
    if (t <= L.t[0]) return L.m[0];
    for (int k = 1; k < L.n; ++k)
        if (t <= L.t[k]) return L.m[k - 1] + (L.m[k] - L.m[k - 1]) * ((t - L.t[k - 1]) / (L.t[k] - L.t[k - 1]));
    return L.m[L.n - 1];
}

// Width controller of one process (App. C).
struct WidthCtl {
    int32_t mode;           // width_mode of the process
    int32_t pad_;
    double rel_lo, rel_hi, factor, w_min, w_max;
};

// Per-task VEGAS iteration combination accumulators (FP64).
struct TaskAcc {
    double sum_inv_var;     // sum 1/var_k
    double sum_mean_inv_var;// sum mean_k/var_k
    double sum_exact;       // sum of means of zero-variance iterations
    double n_exact;         // number of zero-variance iterations
    double mean;            // combined result (written by the assemble kernel)
    double err;
};

// A contiguous piece of one task's samples handled by one CTA.
struct Segment {
    int32_t task;
    int32_t pad_;
    int64_t g0, g1;         // sample groups [g0, g1) of the task
    int64_t part;           // offset (in doubles) of this segment's partial record
};

// Time-dependent scalars of the current sweep, resident on the device so
// that whole steps can be captured in a CUDA graph.
struct TimeState {
    double t;               // time of the current sweep
    double a;               // scale factor a(t)
    double dt;              // step used by the current Euler / Heun step
    double t_step;          // time at the start of the current step
    double mass[BEST_MAX_SPECIES];
    double inv_a;           // 1 / a(t)
    uint32_t call;          // evaluation counter (Philox counter word 2)
    int32_t error;          // sticky numeric-error flag (BEST_ERR_NUMERIC)
};

// Spline table of one species (FP64 master copy; the FP32 copy mirrors it).
struct SpeciesConst {
    double eta;             // +1 BE, -1 FD, 0 MB
    double tail_lo_a, tail_lo_b, tail_hi_a, tail_hi_b;
    int32_t stat;
    int32_t pad_;
};

// Everything the kernels of one context need, by value.
struct Geometry {
    int32_t n_grid;
    int32_t log_spaced;
    double q_min, q_max;
    double log_step;        // ln(q_{j+1}/q_j) (log grid) or step (linear grid)
    int32_t n_species;
    int32_t n_tasks;
    int32_t n_side;
    int32_t map_stride;     // doubles per task in the edges array
    int32_t nbins_max;
    int32_t expansion;
    double a0, t0;
    double e_cut;
    double eps_dt;
    uint64_t seed;
    int32_t tail_points;
    int32_t precision;
    int32_t pt_lo, pt_hi;   // grid points of this context's tasks (a shard), [pt_lo, pt_hi)
    double inv_step;        // spline interval index: 1 / (log2 step) (log grid) or 1 / step (linear grid)
    double lq0_step;        // log grid: log2(q_min) * inv_step
};

// The FP32 segment constants of task td (side sd, constants tc) at the
// sweep's time state: the roles and signs of the legs (App. A), masses,
// statistical-factor coefficients of Eq. (5), the Gaussian's exponent
// factor of Eq. (11), the conserved leg's Eq. (13) end fits and the spline
// index constants, each rounded to FP32 from FP64 exactly as the sample
// kernel needs them.
__device__ inline SegConst32 seg_const32(const SideDesc& sd, const TaskDesc& td, const TaskConst& tc,
                                         const TimeState& ts, const SpeciesConst* sconst, const Geometry& g) {
    SegConst32 C{};
    const int NI = sd.n - 2;
    const int cons = sd.cons;
    const bool cons_in = (sd.in_mask >> cons) & 1;
    const float flip = cons_in ? -1.0f : 1.0f;     // p_cons = flip * sum_{k != c} s_k p_k
    const bool is_loss = td.term == 1;
    {
        const float s_obs = ((sd.in_mask >> sd.obs) & 1) ? 1.0f : -1.0f;
        C.pobs_sig = flip * s_obs * static_cast<float>(tc.p_obs);
        C.sgn_obs_E = s_obs * static_cast<float>(tc.E_obs);
    }
    for (int j = 0; j < NI; ++j) {
        const int k = sd.integ[j];
        const bool kin = (sd.in_mask >> k) & 1;
        const bool own = (sd.own_mask >> k) & 1;
        const int sp = sd.leg_species[k];
        const double eta = sconst[sp].eta;
        C.sig[j] = flip * (kin ? 1.0f : -1.0f);
        C.sgnE[j] = kin ? 1.0f : -1.0f;
        const double m = ts.mass[sp];
        C.m2[j] = static_cast<float>(m * m);
        C.mass[j] = static_cast<float>(m);
        const bool enh = own != is_loss;
        C.ca[j] = enh ? 1.0f : 0.0f;
        C.cb[j] = enh ? static_cast<float>(eta) : 1.0f;
        C.spc[j] = sp;
        C.fd[j] = sconst[sp].stat == BEST_FD;
        C.inw[j] = ((sd.in_mask >> sd.integ[j]) & 1) ? 1.0f : 0.0f;
    }
    {
        const int sp = sd.leg_species[cons];
        const bool own = (sd.own_mask >> cons) & 1;
        const double eta = sconst[sp].eta;
        const double m = ts.mass[sp];
        C.sgn_cons = cons_in ? 1.0f : -1.0f;
        C.m2c = static_cast<float>(m * m);
        C.mass_c = static_cast<float>(m);
        const bool enh = own != is_loss;
        C.cac = enh ? 1.0f : 0.0f;
        C.cbc = enh ? static_cast<float>(eta) : 1.0f;
        C.sp_cons = sp;
        C.eta_c = static_cast<float>(eta);
        C.fd_c = sconst[sp].stat == BEST_FD;
        C.tlo_a = static_cast<float>(sconst[sp].tail_lo_a);
        C.tlo_b = static_cast<float>(sconst[sp].tail_lo_b);
        C.thi_a = static_cast<float>(sconst[sp].tail_hi_a);
        C.thi_b = static_cast<float>(sconst[sp].tail_hi_b);
    }
    C.a = static_cast<float>(ts.a);
    C.inv_a = static_cast<float>(ts.inv_a);
    C.c0 = static_cast<float>(tc.c0);
    C.frac = tc.wfrac > 0.0;
    C.gauss_k = static_cast<float>(tc.gauss_k);
    C.e_obs = static_cast<float>(tc.E_obs);
    C.me_on = sd.me_on != 0;
    for (int k = 0; k < 4; ++k) C.me[k] = static_cast<float>(sd.me_coef[k]);
    {
        const bool obs_in = (sd.in_mask >> sd.obs) & 1;
        C.obs_in_p = obs_in ? static_cast<float>(tc.p_obs) : 0.0f;
        C.obs_in_E = obs_in ? static_cast<float>(tc.E_obs) : 0.0f;
        C.cons_inw = cons_in ? 1.0f : 0.0f;
        C.obs_inw = obs_in ? 1.0f : 0.0f;
    }
    C.obs_cut = tc.E_obs < g.e_cut;
    C.inv_sig2_abs = static_cast<float>(tc.inv_sig2_abs);
    C.four_over_w2 = static_cast<float>(tc.four_over_w2);
    C.inv_E_obs = static_cast<float>(tc.inv_E_obs);
    C.e_cut = static_cast<float>(g.e_cut);
    C.q0 = static_cast<float>(g.q_min);
    C.lq0_step = static_cast<float>(g.lq0_step);
    C.qN = static_cast<float>(g.q_max);
    C.inv_step = static_cast<float>(g.inv_step);
    return C;
}

// The FP32 kernels' map table of one task: for dimension d and increment b,
// the left end and the width of increment b in the physical variable (r
// comoving, theta, phi - pi), from the FP64 edges in [0, 1] rounded to FP32;
// entry d * nb + b of the task's kMaxDim * nbins_max entries.  Written by
// map32_kernel (every sweep) and by the refinement for the tasks it refines.
__host__ __device__ inline int map32_stride(const Geometry& g) { return kMaxDim * g.nbins_max; }
__device__ inline float2 map32_entry(const double* e_task, int d, int b, int nb, const Geometry& g) {
    const double e0 = e_task[d * (nb + 1) + b];
    const double e1 = e_task[d * (nb + 1) + b + 1];
    double lo, sc;
    switch (d % 3) {
        case 0: lo = g.q_min; sc = g.q_max - g.q_min; break;   // r (comoving)
        case 1: lo = 0.0; sc = kPi; break;                     // theta
        default: lo = -kPi; sc = kTwoPi; break;                // phi - pi
    }
    return make_float2(static_cast<float>(lo + sc * e0), static_cast<float>(sc * (e1 - e0)));
}

// Arguments of the sample kernel.
struct EvalParams {
    Geometry geo;
    const SideDesc* sides;
    const TaskDesc* tasks;
    const TaskConst* tconst;
    const SegConst32* tconst32; // FP32 segment constants per task (FP32 sample kernel)
    const SpeciesConst* sconst;
    const TimeState* ts;
    const double* edges;        // [task][map_stride]
    const float2* map32;        // FP32 kernels: [task][map32_stride] map tables (map32_entry)
    const Segment* segs;
    const int32_t* cta_seg;     // segments of chunk c: [cta_seg[c], cta_seg[c+1])
    int32_t n_chunks;           // chunks of the partition
    int32_t pad_chunks_;
    int32_t* chunk_counter;     // next chunk to take (reset to 0 before the launch); NULL: CTA b takes chunk b
    const void* coef;           // [species][n-1][4] in R
    const void* knots;          // [n] in R
    double* partials;
    const uint32_t* item_h;     // stratified: hypercube of every item
    const int32_t* strat_m;     // stratified: items per hypercube
    double* item_rec;           // stratified: (sum w, sum w^2) per item
    uint32_t itn;
    int32_t smem_spline_elems;  // R elements of spline coefficients + knots
    uint32_t rk[20];            // Philox round keys (kernel parameters: read from the constant bank)
};

// Arguments of the adjoint / tangent sample kernel.
struct VjpParams {
    EvalParams E;
    const double* task_u;       // VJP: v_{a,i} mult sign K scale / N;  JVP: dobs u_{a,i} / scale
    double* gcoef;              // VJP: [species][n-1][4] FP64 coefficient gradients (atomics)
    const void* dcoef;          // JVP: tangent spline coefficients of u, [species][n-1][4] in R
    const double* dtail;        // JVP: tail tangents [species][4] = (da, db) low end, (da, db) high end
};

// Variance-driven budgets of one process: its tasks [first, first + count)
// share the fixed total of their configured budgets.
struct BudgetCtl {
    int32_t first, count;
    int64_t n_min, n_max;
    double total;
};
constexpr int kBudgetQuantum = 256;     // budgets are multiples of this many samples (or a bound)
constexpr int kBudgetBisections = 200;

// The device's view of the work partition of one VEGAS iteration index
// (rebuilt on the device when budgets change).  The partition cuts the
// iteration's sample groups into chunks of equal estimated cost; CTAs of the
// persistent grid take chunks from an atomic counter until none is left, so
// that CTAs whose chunks ran faster take more of them.
struct PlanDev {
    int32_t n_active;
    int32_t pad_;
    const int32_t* active;      // [n_active] task ids
    int32_t* task_seg;          // [n_active + 1]
    Segment* segs;              // capacity n_active + grid
    int32_t* cta_seg;           // [chunks + 1]
};

// Chunks of the dynamic partition.  With enough work (W, the iteration's
// estimated cost, at least chunk_count(B) x kMinChunkCost) the partition has
// kChunkStages stages of kChunkSplit x B chunks (B: the persistent grid), the
// stages covering 1/2, 1/4, ... of W and the last stage the remainder, so
// that the chunks taken last (when CTAs run out of work at different times)
// are small.  With less work it has max(B, W / kMinChunkCost) equal chunks,
// so that no chunk is so small that the per-segment set-up (map table,
// histograms, record) outweighs its samples.  Chunks past the last one are
// empty: the kernels always see chunk_count(B) chunks.  Integer arithmetic:
// the host and the device cut identically.
#ifndef BEST_CHUNK_STAGES
#define BEST_CHUNK_STAGES 8
#endif
#ifndef BEST_CHUNK_SPLIT
#define BEST_CHUNK_SPLIT 2
#endif
constexpr int kChunkStages = BEST_CHUNK_STAGES;
constexpr int kChunkSplit = BEST_CHUNK_SPLIT;
constexpr int64_t kMinChunkCost = 8192LL * 12;   // cost of 8192 samples of a 2 -> 2 task
__host__ __device__ inline int chunk_count(int B) { return kChunkStages * kChunkSplit * B; }
struct ChunkShape {
    int stages;             // stages of the partition
    int per;                // chunks per stage
};
__host__ __device__ inline ChunkShape chunk_shape(int64_t W, int B) {
    const int kmax = chunk_count(B);
    const int64_t want = W / kMinChunkCost;
    if (want >= kmax) return ChunkShape{kChunkStages, kChunkSplit * B};
    return ChunkShape{1, want < B ? B : static_cast<int>(want)};
}
__host__ __device__ inline int64_t stage_start(int64_t W, int s, int stages) {
    return s >= stages ? W : W - (W >> s);
}
__host__ __device__ inline int64_t chunk_bound(int64_t W, int c, const ChunkShape& sh) {
    const int s = c / sh.per, j = c - s * sh.per;
    if (s >= sh.stages) return W;
    const int64_t lo = stage_start(W, s, sh.stages);
    return lo + (stage_start(W, s + 1, sh.stages) - lo) * j / sh.per;
}

// One instantiation of the sample kernel the autotuner may pick.
struct SampleVariant {
    void* fn;
    int32_t mb;             // CTAs per SM of its register budget (__launch_bounds__)
    int32_t threads;        // threads per CTA
    int32_t spl;            // samples a lane evaluates per step of the FP32 loop
};
constexpr int kMaxVariants = 12;

// Samples per Philox group of a D-dimensional task stream (FP32: 4 uniforms
// per block, FP64: 2).
__host__ __device__ inline int stream_group(int D, bool f32) {
    const int per = f32 ? 4 : 2;
    int a = D, b = per;
    while (b) { const int t = a % b; a = b; b = t; }
    return per / a;
}

// Doubles per partial record: the sample kernel writes 2 + D nb, the adjoint
// kernel up to 12 values.
__host__ __device__ inline int64_t record_doubles(int D, int nb) {
    const int64_t r = 2 + static_cast<int64_t>(D) * nb;
    return r < 16 ? 16 : r;
}

}  // namespace best
