// FP64 kernels around the sample kernel: time state, spline construction
// (Sec. 3B), per-task constants, iteration reduction and VEGAS refinement,
// assembly of C_a (Eq. (7)) and the Euler / Heun updates (Sec. 3C).
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace best {

// ---------------------------------------------------------------------------
// Time state: a(t) (Sec. 3E) and m_s(t) (Sec. 3A) of the current sweep.
// mode 0: t = t_host; mode 1: t = *t_dev; mode 2: t = *t_dev + state dt.
// ---------------------------------------------------------------------------
__global__ void set_time_kernel(Geometry g, TimeState* ts, const double* t_dev, double t_host,
                                int mode, const MassLaw* law) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = t_host;
    if (mode == 1) t = *t_dev;
    if (mode == 2) t = *t_dev + ts->dt;
    ts->t = t;
    ts->a = g.expansion ? g.a0 * sqrt(t / g.t0) : 1.0;
    ts->inv_a = 1.0 / ts->a;
    if (!(ts->a > 0.0) || !isfinite(ts->a)) ts->error = BEST_ERR_NUMERIC;
    for (int s = 0; s < g.n_species; ++s) ts->mass[s] = mass_at(law[s], t);
}

// Second derivatives M_j of the not-a-knot cubic spline through (q_j, f_j):
// the tridiagonal system for M_1 .. M_{n-2} with the not-a-knot conditions
// (third derivative continuous at q_1 and q_{n-2}) eliminated into its first
// and last rows, solved by the Thomas algorithm; then M_0 and M_{n-1}.
// Called by every thread of the CTA: the rows (sub-, main and
// super-diagonal, right-hand side) are formed in parallel in shared memory,
// then one thread runs the recurrence (one division per row, no global
// loads in the dependent chain).  cp, A, Bd: scratch of n doubles each.
__device__ void notaknot_moments(int n, const double* __restrict__ knots, const double* f, double* cp,
                                 double* M, double* A, double* Bd) {
    const int m = n - 2;    // unknowns M_1 .. M_{n-2}
    auto h = [&](int i) { return knots[i + 1] - knots[i]; };
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = k + 1;
        double a = h(i - 1), b = 2.0 * (h(i - 1) + h(i)), c = h(i);
        const double d = 6.0 * ((f[i + 1] - f[i]) / h(i) - (f[i] - f[i - 1]) / h(i - 1));
        if (k == 0) {
            const double h0 = h(0), h1 = h(1);
            b += h0 * (h0 + h1) / h1;
            c -= h0 * h0 / h1;
            a = 0.0;
        }
        if (k == m - 1) {
            const double hl = h(n - 2), hp = h(n - 3);
            a -= hl * hl / hp;
            b += hl * (hl + hp) / hp;
            c = 0.0;
        }
        A[k] = a;
        Bd[k] = b;
        cp[k] = c;
        M[k + 1] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < m; ++k) {
            const double den = k > 0 ? Bd[k] - A[k] * cp[k - 1] : Bd[k];
            const double r = 1.0 / den;
            cp[k] *= r;
            M[k + 1] = (k > 0 ? M[k + 1] - A[k] * M[k] : M[k + 1]) * r;
        }
        for (int k = m - 2; k >= 0; --k) M[k + 1] -= cp[k] * M[k + 2];
        const double h0 = h(0), h1 = h(1);
        M[0] = ((h0 + h1) * M[1] - h0 * M[2]) / h1;
        const double hl = h(n - 2), hp = h(n - 3);
        M[n - 1] = ((hl + hp) * M[n - 2] - hl * M[n - 3]) / hp;
    }
    __syncthreads();
}

// Least-squares line y = a + b x through the K end points of one end of
// the grid (end 0: j < K; end 1: j >= n - K), x and y given per grid point.
__device__ inline void end_fit(int n, int K, int end, const double* x, const double* y, double* a0, double* b) {
    double xm = 0.0, ym = 0.0;
    for (int k = 0; k < K; ++k) {
        const int j = end == 0 ? k : n - K + k;
        xm += x[j];
        ym += y[j];
    }
    xm /= K;
    ym /= K;
    double sxy = 0.0, sxx = 0.0;
    for (int k = 0; k < K; ++k) {
        const int j = end == 0 ? k : n - K + k;
        const double xc = x[j] - xm;
        sxy += xc * (y[j] - ym);
        sxx += xc * xc;
    }
    *b = sxy / sxx;
    *a0 = ym - *b * xm;
}

// ---------------------------------------------------------------------------
// Spline of one species per CTA: not-a-knot cubic spline of (q_j, f_j)
// through the tridiagonal system for the second derivatives M_j, with the
// not-a-knot conditions (third derivative continuous at q_1 and q_{n-2})
// eliminated into the first and last rows; then the interval coefficients
// and the least-squares end fits of log(1/f + eta) against E(q/a) (Eq. (13)).
// src_mode 0: f given; 1: f = exp(src) (log f).
// Dynamic shared memory: 5 n doubles.
// ---------------------------------------------------------------------------
__global__ void spline_build_kernel(Geometry g, const double* __restrict__ src, int src_mode,
                                    const double* __restrict__ knots, TimeState* ts,
                                    SpeciesConst* sc, double* fgrid, double* coef64,
                                    float* coef32) {
    extern __shared__ double sh[];
    const int n = g.n_grid;
    const int s = blockIdx.x;
    double* f = sh;
    double* cp = sh + n;
    double* M = sh + 2 * n;
    double* X = sh + 3 * n;            // row scratch, then the end fits' abscissae
    double* Y = sh + 4 * n;            // row scratch, then the end fits' ordinates
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double v = src[static_cast<int64_t>(s) * n + j];
        if (src_mode == 1) v = exp(v);
        if (!(v > 0.0) || !isfinite(v)) ts->error = BEST_ERR_NUMERIC;
        f[j] = v;
        fgrid[static_cast<int64_t>(s) * n + j] = v;
    }
    __syncthreads();
    notaknot_moments(n, knots, f, cp, M, X, Y);
    for (int j = threadIdx.x; j < n - 1; j += blockDim.x) {
        const double hj = knots[j + 1] - knots[j];
        const double c0 = f[j];
        const double c1 = (f[j + 1] - f[j]) / hj - hj * (2.0 * M[j] + M[j + 1]) / 6.0;
        const double c2 = 0.5 * M[j];
        const double c3 = (M[j + 1] - M[j]) / (6.0 * hj);
        const int64_t o = (static_cast<int64_t>(s) * (n - 1) + j) * 4;
        coef64[o + 0] = c0; coef64[o + 1] = c1; coef64[o + 2] = c2; coef64[o + 3] = c3;
        coef32[o + 0] = static_cast<float>(c0); coef32[o + 1] = static_cast<float>(c1);
        coef32[o + 2] = static_cast<float>(c2); coef32[o + 3] = static_cast<float>(c3);
    }
    // end fits: E(q_j / a) and log(1/f_j + eta) of the 2K end points in
    // parallel, then one line per end
    const double eta = sc[s].eta;
    const double mass = ts->mass[s];
    const double a = ts->a;
    const int K = g.tail_points;
    for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) {
        const int j = t < K ? t : n - 2 * K + t;
        const double p = knots[j] / a;
        X[j] = sqrt(p * p + mass * mass);
        Y[j] = log(1.0 / f[j] + eta);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double a0, b;
        end_fit(n, K, threadIdx.x, X, Y, &a0, &b);
        if (threadIdx.x == 0) { sc[s].tail_lo_a = a0; sc[s].tail_lo_b = b; }
        else { sc[s].tail_hi_a = a0; sc[s].tail_hi_b = b; }
    }
}

// ---------------------------------------------------------------------------
// Tangent of the spline construction in the direction u (one species per
// CTA): the interval coefficients are linear in f, so the tangent spline is
// the spline of u (no clamping); the end fits y = log(1/f + eta) = a + b E
// move by da, db from dy_j = -u_j / (f_j (1 + eta f_j)).  Dynamic shared
// memory: 5 n doubles.
// ---------------------------------------------------------------------------
__global__ void spline_tangent_kernel(Geometry g, const double* __restrict__ u, const double* __restrict__ knots,
                                      const double* __restrict__ fgrid, const SpeciesConst* __restrict__ sc,
                                      const TimeState* ts, double* dcoef64, float* dcoef32, double* dtail) {
    extern __shared__ double sh[];
    const int n = g.n_grid;
    const int s = blockIdx.x;
    double* du = sh;
    double* cp = sh + n;
    double* M = sh + 2 * n;
    double* X = sh + 3 * n;
    double* Y = sh + 4 * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) du[j] = u[static_cast<int64_t>(s) * n + j];
    __syncthreads();
    notaknot_moments(n, knots, du, cp, M, X, Y);
    for (int j = threadIdx.x; j < n - 1; j += blockDim.x) {
        const double hj = knots[j + 1] - knots[j];
        const double c0 = du[j];
        const double c1 = (du[j + 1] - du[j]) / hj - hj * (2.0 * M[j] + M[j + 1]) / 6.0;
        const double c2 = 0.5 * M[j];
        const double c3 = (M[j + 1] - M[j]) / (6.0 * hj);
        const int64_t o = (static_cast<int64_t>(s) * (n - 1) + j) * 4;
        dcoef64[o + 0] = c0; dcoef64[o + 1] = c1; dcoef64[o + 2] = c2; dcoef64[o + 3] = c3;
        dcoef32[o + 0] = static_cast<float>(c0); dcoef32[o + 1] = static_cast<float>(c1);
        dcoef32[o + 2] = static_cast<float>(c2); dcoef32[o + 3] = static_cast<float>(c3);
    }
    const double eta = sc[s].eta;
    const double mass = ts->mass[s];
    const double a = ts->a;
    const int K = g.tail_points;
    const double* f = fgrid + static_cast<int64_t>(s) * n;
    for (int t = threadIdx.x; t < 2 * K; t += blockDim.x) {
        const int j = t < K ? t : n - 2 * K + t;
        const double p = knots[j] / a;
        X[j] = sqrt(p * p + mass * mass);
        Y[j] = -du[j] / (f[j] * (1.0 + eta * f[j]));
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double da, db;
        end_fit(n, K, threadIdx.x, X, Y, &da, &db);
        dtail[s * 4 + 2 * threadIdx.x] = da;
        dtail[s * 4 + 2 * threadIdx.x + 1] = db;
    }
}

// ---------------------------------------------------------------------------
// Per-task constants of the sweep and reset of the iteration accumulators.
// ---------------------------------------------------------------------------
// Accumulation scale: the kernel sums w_n = w / (K scale).  With a previous
// estimate I of the task (last sweep) scale = |I| / K, so that w_n averages
// to about 1; otherwise scale = f_obs.  The scale is kept within 2^+-100 of
// the observed-leg factor so that obs_factor / scale fits in FP32.
__device__ inline double clamp_scale(double scale, double obs_factor) {
    if (!(obs_factor > 0.0)) return scale > 0.0 && isfinite(scale) ? scale : 1.0;
    const double lo = obs_factor * 7.888609052210118e-31, hi = obs_factor * 1.2676506002282294e30;
    if (!(scale > 0.0) || !isfinite(scale)) return obs_factor;
    return scale < lo ? lo : (scale > hi ? hi : scale);
}

// x^k for a non-negative integer k by repeated squaring (the task constants'
// integer powers: a few multiplications instead of an FP64 pow sequence)
__device__ inline double ipow(double x, int k) {
    double r = 1.0;
    for (; k > 0; k >>= 1) {
        if (k & 1) r *= x;
        x *= x;
    }
    return r;
}

__global__ void prepare_kernel(Geometry g, const SideDesc* __restrict__ sides,
                               const TaskDesc* __restrict__ tasks, const double* __restrict__ knots,
                               const double* __restrict__ fgrid, const TimeState* ts,
                               const double* __restrict__ prev, TaskConst* tconst, TaskAcc* acc, int reset_acc,
                               const double* __restrict__ width, const SpeciesConst* __restrict__ sconst,
                               SegConst32* tconst32) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n_tasks) return;
    const TaskDesc td = tasks[t];
    const SideDesc& sd = sides[td.si];
    const double a = ts->a;
    const double m = ts->mass[sd.species_obs];
    const double p = knots[td.point] / a;
    const double E = sqrt(p * p + m * m);
    const int n = sd.n;
    const int D = 3 * (n - 2);
    const double nbD = ipow(static_cast<double>(td.nbins), D);
    const double two_pi_pow = ipow(kTwoPi, 3 * (n - 1) - 4);
    const double a3 = ipow(ts->inv_a, 3 * (n - 2));             // a^{-3(n-2)}
    TaskConst c;
    c.p_obs = p;
    c.E_obs = E;
    c.f_obs = fgrid[static_cast<int64_t>(sd.species_obs) * g.n_grid + td.point];
    // fractional width (App. C): the per-sample factor sigma_ref / sigma with
    // sigma_ref = w E_obs is applied in the sample kernel
    c.wfrac = sd.width_mode == 0 ? 0.0 : (width ? width[sd.process] : sd.width0);
    const double sigma_ref = sd.width_mode == 0 ? sd.sigma : c.wfrac * E;
    c.K = sd.coupling2 * nbD * a3 /
          (two_pi_pow * ldexp(1.0, n) * E * sigma_ref * sqrt(kTwoPi));
    c.obs_factor = td.term == 1 ? c.f_obs : 1.0 + sd.eta_obs * c.f_obs;
    const double est = prev[t];
    c.scale = clamp_scale(est > 0.0 && c.K > 0.0 ? est / c.K : (c.f_obs > 0.0 ? c.f_obs : 1.0), c.obs_factor);
    // the observed leg's own cut (App. A) removes the whole task
    c.c0 = E < g.e_cut ? 0.0 : c.obs_factor / c.scale;
    c.gauss_k = c.wfrac > 0.0 ? -2.0 * 1.4426950408889634 / (c.wfrac * c.wfrac)
                              : -1.4426950408889634 / (2.0 * sd.sigma * sd.sigma);
    c.inv_sig2_abs = 1.0 / (sd.sigma * sd.sigma);
    c.four_over_w2 = c.wfrac > 0.0 ? 4.0 / (c.wfrac * c.wfrac) : 0.0;
    c.inv_E_obs = 1.0 / E;
    tconst[t] = c;
    if (tconst32) tconst32[t] = seg_const32(sd, td, c, *ts, sconst, g);
    if (!reset_acc) return;
    TaskAcc z;
    z.sum_inv_var = 0.0; z.sum_mean_inv_var = 0.0; z.sum_exact = 0.0; z.n_exact = 0.0;
    z.mean = 0.0; z.err = 0.0;
    acc[t] = z;
}

// ---------------------------------------------------------------------------
// Adaptive stratified sampling (VEGAS+): per-task hypercube allocation m_h
// (items of kItem samples, at least one per hypercube) and the hypercube of
// every item, items in hypercube order.  One CTA of 256 threads per task.
// ---------------------------------------------------------------------------
namespace {

// Exclusive prefix of v over the CTA (v of thread k at position k), with the
// CTA total in *total; s: 256 int64 of shared memory.
__device__ int64_t cta_exclusive_scan(int64_t v, int64_t* s, int64_t* total) {
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {
        const int64_t a = static_cast<int>(threadIdx.x) >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += a;
        __syncthreads();
    }
    const int64_t incl = s[threadIdx.x];
    *total = s[blockDim.x - 1];
    __syncthreads();
    return incl - v;
}

__device__ void strat_write_items(const int32_t* m, int H, int64_t J, uint32_t* item_h, int64_t* s) {
    if (H < static_cast<int>(blockDim.x)) {
        // few (large) hypercubes: every thread fills each hypercube's range
        int64_t base = 0;
        for (int h = 0; h < H; ++h) {
            const int64_t v = m[h];
            for (int64_t k = threadIdx.x; k < v && base + k < J; k += blockDim.x)
                item_h[base + k] = static_cast<uint32_t>(h);
            base += v;
        }
        return;
    }
    int64_t base = 0;
    for (int c0 = 0; c0 < H; c0 += blockDim.x) {
        const int h = c0 + static_cast<int>(threadIdx.x);
        const int64_t v = h < H ? m[h] : 0;
        int64_t tot;
        const int64_t ex = base + cta_exclusive_scan(v, s, &tot);
        for (int64_t k = 0; k < v && ex + k < J; ++k) item_h[ex + k] = static_cast<uint32_t>(h);
        base += tot;
    }
}

__device__ void uniform_allocation(int32_t* m, int H, int64_t J) {
    for (int h = threadIdx.x; h < H; h += blockDim.x)
        m[h] = static_cast<int32_t>(J / H + (h < J % H ? 1 : 0));
}

}  // namespace

// uniform != 0: first (uniform) allocation; otherwise only the items are
// rebuilt from the stored allocation (after a state load).
__global__ void strat_init_kernel(const TaskDesc* __restrict__ tasks, int32_t* strat_m, uint32_t* item_h,
                                  int uniform) {
    __shared__ int64_t s[256];
    const TaskDesc td = tasks[blockIdx.x];
    if (td.strat_H == 0) return;
    int32_t* m = strat_m + td.strat_off_h;
    if (uniform) {
        uniform_allocation(m, td.strat_H, td.strat_J);
        __syncthreads();
    }
    strat_write_items(m, td.strat_H, td.strat_J, item_h + td.strat_off_item, s);
}

// After the sample kernel of an iteration, one CTA per active task: per
// hypercube S1 = sum w, S2 = sum w^2 from its items (fixed order), the
// iteration estimate I = (1/H) sum_h S1_h / n_h and variance
// (1/H^2) sum_h s_h^2 / n_h (n_h = kItem m_h), written to est[4 t ..] with an
// underflow flag (S2 < S1^2 / n violated, i.e. FP32 squares underflowed, in
// hypercubes holding more than 1e-6 of sum_h |S1_h| / n_h); then the
// next allocation m_h = 1 + floor((J - H) d_h / sum d), d_h = (s_h^2)^(beta/2),
// the remaining items one each to h = 0, 1, ... (uniform if every d_h = 0),
// and the items rebuilt.  An underflowed iteration keeps its allocation.
__global__ void strat_refine_kernel(const TaskDesc* __restrict__ tasks, const int32_t* __restrict__ active,
                                    const double* __restrict__ item_rec, int32_t* strat_m, double* strat_d,
                                    double* strat_s2, uint32_t* item_h, double* est) {
    __shared__ int64_t s[256];
    __shared__ double r0[256], r1[256], r2[256], r3[256], r4[256];
    __shared__ int64_t si[256];
    __shared__ int32_t b_h[2][256];          // boundary runs of each thread's item chunk: first, last
    __shared__ double b_1[2][256], b_2[2][256];
    const int t = active[blockIdx.x];
    const TaskDesc td = tasks[t];
    if (td.strat_H == 0) return;
    const int H = td.strat_H;
    const int64_t J = td.strat_J;
    int32_t* m = strat_m + td.strat_off_h;
    double* S1h = strat_d + td.strat_off_h;      // sum w per hypercube, then d_h
    double* S2h = strat_s2 + td.strat_off_h;
    const uint32_t* ih = item_h + td.strat_off_item;
    const double2* rec = reinterpret_cast<const double2*>(item_rec) + td.strat_off_item;
    // per-hypercube sums: each thread scans a contiguous chunk of items
    // (items of a hypercube are contiguous); runs inside a chunk are whole
    // hypercubes and are stored directly, the chunk's first and last runs
    // are added afterwards by one thread in chunk order (deterministic)
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        S1h[h] = 0.0;
        S2h[h] = 0.0;
    }
    __syncthreads();
    {
        const int64_t ch = (J + blockDim.x - 1) / blockDim.x;
        const int64_t i0 = static_cast<int64_t>(threadIdx.x) * ch;
        const int64_t i1 = i0 + ch < J ? i0 + ch : J;
        int32_t cur = -1;
        double s1 = 0.0, s2 = 0.0;
        b_h[0][threadIdx.x] = -1;
        b_h[1][threadIdx.x] = -1;
        // eight items per step, their loads issued together (the run logic
        // below is serial per thread and would otherwise wait on each load)
        constexpr int U = 8;
        for (int64_t i = i0; i < i1; i += U) {
            int32_t hh[U];
            double2 rr[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = i + u < i1;
                hh[u] = in ? static_cast<int32_t>(ih[i + u]) : -1;
                rr[u] = in ? rec[i + u] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t h = hh[u];
                if (h < 0) continue;
                if (h != cur) {
                    if (cur >= 0) {
                        if (b_h[0][threadIdx.x] < 0) {
                            b_h[0][threadIdx.x] = cur; b_1[0][threadIdx.x] = s1; b_2[0][threadIdx.x] = s2;
                        } else {
                            S1h[cur] = s1;
                            S2h[cur] = s2;
                        }
                    }
                    cur = h;
                    s1 = 0.0;
                    s2 = 0.0;
                }
                s1 += rr[u].x;
                s2 += rr[u].y;
            }
        }
        if (cur >= 0) {
            const int k = b_h[0][threadIdx.x] < 0 ? 0 : 1;
            b_h[k][threadIdx.x] = cur; b_1[k][threadIdx.x] = s1; b_2[k][threadIdx.x] = s2;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < static_cast<int>(blockDim.x); ++c)
            for (int k = 0; k < 2; ++k) {
                const int32_t h = b_h[k][c];
                if (h >= 0) {
                    S1h[h] += b_1[k][c];
                    S2h[h] += b_2[k][c];
                }
            }
    }
    __syncthreads();
    double a_mean = 0.0, a_var = 0.0, a_d = 0.0, a_abs = 0.0, a_bad = 0.0;
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        const double S1 = S1h[h], S2 = S2h[h];
        const double n = static_cast<double>(kItem) * static_cast<double>(m[h]);
        const double q = S1 * S1 / n;
        double s2v = (S2 - q) / (n - 1.0);
        s2v = s2v > 0.0 ? s2v : 0.0;
        if (S2 < (1.0 - 1e-6) * q) a_bad += fabs(S1) / n;
        a_abs += fabs(S1) / n;
        a_mean += S1 / n;
        a_var += s2v / n;
        const double d = pow(s2v, 0.5 * td.strat_beta);
        S1h[h] = d;
        a_d += d;
    }
    r0[threadIdx.x] = a_mean;
    r1[threadIdx.x] = a_var;
    r2[threadIdx.x] = a_d;
    r3[threadIdx.x] = a_abs;
    r4[threadIdx.x] = a_bad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (static_cast<int>(threadIdx.x) < o) {
            r0[threadIdx.x] += r0[threadIdx.x + o];
            r1[threadIdx.x] += r1[threadIdx.x + o];
            r2[threadIdx.x] += r2[threadIdx.x + o];
            r3[threadIdx.x] += r3[threadIdx.x + o];
            r4[threadIdx.x] += r4[threadIdx.x + o];
        }
        __syncthreads();
    }
    const double sum_d = r2[0];
    // underflowed hypercubes (FP32 squares of weights near the end of the
    // range) matter only when they carry a noticeable part of the estimate
    const bool underflow = r4[0] > 1e-6 * r3[0];
    if (threadIdx.x == 0) {
        est[4 * t] = r0[0] / H;
        est[4 * t + 1] = r1[0] / (static_cast<double>(H) * H);
        est[4 * t + 2] = underflow ? 1.0 : 0.0;
    }
    if (underflow) return;
    __syncthreads();
    if (sum_d > 0.0) {
        int64_t cnt = 0;
        for (int h = threadIdx.x; h < H; h += blockDim.x) {
            const int32_t v = 1 + static_cast<int32_t>(floor(static_cast<double>(J - H) * S1h[h] / sum_d));
            m[h] = v;
            cnt += v;
        }
        si[threadIdx.x] = cnt;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (static_cast<int>(threadIdx.x) < o) si[threadIdx.x] += si[threadIdx.x + o];
            __syncthreads();
        }
        const int64_t rest = J - si[0];
        __syncthreads();
        if (rest >= 0) {
            for (int h = threadIdx.x; h < H; h += blockDim.x)
                if (h < rest) m[h] += 1;
        } else {
            uniform_allocation(m, H, J);      // rounding overshoot (never seen): start afresh
        }
    } else {
        uniform_allocation(m, H, J);
    }
    __syncthreads();
    strat_write_items(m, H, J, item_h + td.strat_off_item, s);
}

// ---------------------------------------------------------------------------
// End of one VEGAS iteration, one CTA per active task: sum the task's
// segment records in a fixed order (deterministic), form the iteration
// estimate and its variance, add them to the combination accumulators, and
// refine the map (Lepage): smooth the per-increment sums of w^2 with the
// (7,1)/8, (1,6,1)/8, (1,7)/8 stencil, normalise, compress with
// ((1-d)/ln(1/d))^alpha, and re-partition into equal shares of the
// compressed weight.  A normalised share below 1e-30 counts as an empty
// increment (weight 0, like an exact zero) so that the map does not depend on
// where underflow of w^2 falls.  Dynamic shared memory: (3 kMaxDim nbins_max
// + 2 kMaxDim + 2) doubles.
// ---------------------------------------------------------------------------
__global__ void refine_kernel(Geometry g, const SideDesc* __restrict__ sides,
                              const TaskDesc* __restrict__ tasks, const TaskConst* tconst,
                              const int32_t* __restrict__ active, const int32_t* __restrict__ task_seg,
                              const Segment* __restrict__ segs, const double* __restrict__ partials,
                              double* edges, TaskAcc* acc, TaskConst* tconst_next,
                              const double* __restrict__ strat_est, SegConst32* tconst32, float2* map32) {
    extern __shared__ double hist[];
    const int t = active[blockIdx.x];
    const TaskDesc td = tasks[t];
    const int nb = td.nbins;
    const int D = td.dim;
    const int s0 = task_seg[blockIdx.x], s1 = task_seg[blockIdx.x + 1];
    const int L = 2 + D * nb;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        // the records in segment order; eight loads in flight at a time
        double v = 0.0;
        int s = s0;
        for (; s + 8 <= s1; s += 8) {
            double a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = partials[segs[s + u].part + k];
#pragma unroll
            for (int u = 0; u < 8; ++u) v += a[u];
        }
        for (; s < s1; ++s) v += partials[segs[s].part + k];
        hist[k] = v;
    }
    __syncthreads();
    // Sum w^2 >= (sum w)^2 / N holds exactly; if the computed sums violate it,
    // squares of tiny weights underflowed (FP32 path with a poor scale): the
    // iteration is discarded (no estimate, no refinement) and only the scale
    // is corrected for the next iteration.
    const double N = static_cast<double>(td.neval);
    double mean_n, var_n;
    bool underflow;
    if (td.strat_H > 0) {
        // stratified: estimate, variance and underflow flag from strat_refine_kernel
        mean_n = strat_est[4 * t];
        var_n = strat_est[4 * t + 1];
        underflow = strat_est[4 * t + 2] != 0.0;
    } else {
        mean_n = hist[0] / N;
        underflow = hist[1] / N < (1.0 - 1e-6) * mean_n * mean_n;
        var_n = N > 1.0 ? (hist[1] / N - mean_n * mean_n) / (N - 1.0) : 0.0;
        var_n = var_n > 0.0 ? var_n : 0.0;
    }
    if (threadIdx.x == 0) {
        const TaskConst c = tconst[t];
        const double sc = c.K * c.scale;
        const double mean = mean_n * sc;
        const double var = var_n * sc * sc;
        if (!underflow) {
            TaskAcc& A = acc[t];
            if (var > 0.0) {
                A.sum_inv_var += 1.0 / var;
                A.sum_mean_inv_var += mean / var;
            } else {
                A.sum_exact += mean;
                A.n_exact += 1.0;
            }
        }
        if (mean_n != 0.0) {
            const double scale = clamp_scale(fabs(mean_n) * c.scale, c.obs_factor);
            tconst_next[t].scale = scale;
            tconst_next[t].c0 = c.c0 == 0.0 ? 0.0 : c.obs_factor / scale;   // a cut observed leg stays cut
            if (tconst32) tconst32[t].c0 = static_cast<float>(tconst_next[t].c0);
        }
    }
    if (underflow) return;
    // refinement: smoothing and compression in parallel over (dimension,
    // increment); the running sums of the compressed weights per dimension
    // (one thread each, in increment order); then every new edge in
    // parallel: the increment where the running sum reaches k / nb of the
    // total, and the linear interpolation inside it
    double* sm = hist + 2 + D * nb;            // smoothed, then compressed weights [D][nb]
    double* tot = sm + D * nb;                 // per-dimension sums [D], then (FP32 path) their reciprocals [D]
    double* olde = tot + 2 * D;                // old edges [D][nb + 1]
    double* rom = olde + D * (nb + 1);         // reciprocals of the compressed weights [D][nb]
    double* cum = rom + D * nb;                // running sums of the compressed weights [D][nb + 1]
    const double* e_task = edges + static_cast<int64_t>(t) * g.map_stride;
    for (int k = threadIdx.x; k < D * (nb + 1); k += blockDim.x) olde[k] = e_task[k];
    for (int k = threadIdx.x; k < D * nb; k += blockDim.x) {
        const int d = k / nb, b = k - d * nb;
        const double* dd = hist + 2 + d * nb;
        double v;
        if (nb == 1) v = dd[0];
        else if (b == 0) v = (7.0 * dd[0] + dd[1]) / 8.0;
        else if (b == nb - 1) v = (dd[nb - 2] + 7.0 * dd[nb - 1]) / 8.0;
        else v = (dd[b - 1] + 6.0 * dd[b] + dd[b + 1]) / 8.0;
        sm[k] = v;
    }
    __syncthreads();
    const bool f32 = g.precision == BEST_FP32;
    if (threadIdx.x < D) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += sm[threadIdx.x * nb + b];
        tot[threadIdx.x] = t;
        // FP32 path: the totals are sums of FP32 training data, so their
        // reciprocals are finite (an FP64 total can be subnormal)
        tot[D + threadIdx.x] = f32 && t > 0.0 ? 1.0 / t : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < D * nb; k += blockDim.x) {
        const int d = k / nb;
        const double t = tot[d];
        double o = 0.0, r = 0.0;
        if (t > 0.0) {
            if (f32) {
                // the FP32 path's training data carry FP32 rounding: its
                // normalisation, compression and reciprocal are evaluated in
                // FP32 (FP64 division, log and pow run at a small fraction of
                // the FP32 rate on this GPU)
                const float vf = static_cast<float>(sm[k] * tot[D + d]);
                float of = 1.0f;               // v >= 1, or not a number (FP32 training data overflowed)
                if (vf < 1e-30f) of = 0.0f;    // numerically empty increment
                else if (vf < 1.0f) of = powf((1.0f - vf) / -logf(vf), static_cast<float>(td.alpha));
                o = of;
                r = of > 0.0f ? __frcp_rn(of) : 0.0f;
            } else {
                const double v = sm[k] / t;
                if (v < 1e-30) o = 0.0;        // numerically empty increment
                else if (v >= 1.0) o = 1.0;
                else o = pow((1.0 - v) / -log(v), td.alpha);
                // the interpolation below multiplies by these reciprocals (o is
                // 0 or at least (1 / ln 1e30)^alpha)
                r = o > 0.0 ? 1.0 / o : 0.0;
            }
        }
        sm[k] = o;
        rom[k] = r;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        const int d = threadIdx.x;
        const double* om = sm + d * nb;
        double* c = cum + d * (nb + 1);
        double acc = 0.0;
        c[0] = 0.0;
        for (int b = 0; b < nb; ++b) {
            acc += om[b];
            c[b + 1] = acc;
        }
    }
    __syncthreads();
    // new edge k of dimension d: starting from increment 0, step to the next
    // increment while the running sum after it stays below the goal k T / nb
    // (and an increment is left); the running sums are non-decreasing, so the
    // increment reached is the number of j in [1, nb - 1] with cum[j] < goal
    double* e = edges + static_cast<int64_t>(t) * g.map_stride;
    for (int q = threadIdx.x; q < D * (nb + 1); q += blockDim.x) {
        const int d = q / (nb + 1), k = q - d * (nb + 1);
        if (!(tot[d] > 0.0)) continue;                   // no training data: the map is kept
        if (k == 0 || k == nb) {
            e[q] = k == 0 ? 0.0 : 1.0;
            continue;
        }
        const double* c = cum + d * (nb + 1);
        const double target = c[nb] / nb;
        const double goal = k * target;
        int lo = 0, hi = nb - 1;                         // first i in [0, nb - 1] with !(c[i + 1] < goal), else nb - 1
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (c[mid + 1] < goal) lo = mid + 1;
            else hi = mid;
        }
        const int i = lo;
        double fr = (goal - c[i]) * rom[d * nb + i];
        fr = fr < 0.0 ? 0.0 : (fr > 1.0 ? 1.0 : fr);
        const double* oe = olde + d * (nb + 1);
        e[q] = oe[i] + fr * (oe[i + 1] - oe[i]);
    }
    if (map32) {
        // the FP32 kernels' table of the refined map
        __syncthreads();
        float2* m = map32 + static_cast<int64_t>(t) * map32_stride(g);
        for (int k = threadIdx.x; k < D * nb; k += blockDim.x) m[k] = map32_entry(e, k / nb, k % nb, nb, g);
    }
}

// The FP32 kernels' map tables of tasks [0, n_tasks) from their FP64 edges
// (edges [task][map_stride], tables [task][map32_stride]); one thread per
// entry.
__global__ void map32_kernel(Geometry g, const TaskDesc* __restrict__ tasks, int n_tasks,
                             const double* __restrict__ edges, float2* map32) {
    const int stride = map32_stride(g);
    const int64_t total = static_cast<int64_t>(n_tasks) * stride;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int t = static_cast<int>(q / stride), k = static_cast<int>(q - static_cast<int64_t>(t) * stride);
        const int nb = tasks[t].nbins, D = tasks[t].dim;
        if (k < D * nb)
            map32[q] = map32_entry(edges + static_cast<int64_t>(t) * g.map_stride, k / nb, k % nb, nb, g);
    }
}

// ---------------------------------------------------------------------------
// Combination of the iterations per task (inverse-variance weights; zero-
// variance iterations are exact) and assembly of Eq. (7):
// C_a(p_i) = sum_sides mult (I_gain - I_loss), err^2 = sum mult^2
// (sigma_gain^2 + sigma_loss^2).  One thread per (species, grid point), each
// owning the tasks observed there; thread 0 advances the evaluation counter.
// ---------------------------------------------------------------------------
__device__ inline void combine_task(TaskAcc& A) {
    if (A.n_exact > 0.0) {
        A.mean = A.sum_exact / A.n_exact;
        A.err = 0.0;
    } else if (A.sum_inv_var > 0.0) {
        A.mean = A.sum_mean_inv_var / A.sum_inv_var;
        A.err = sqrt(1.0 / A.sum_inv_var);
    } else {
        A.mean = 0.0;
        A.err = 0.0;
    }
}

__global__ void assemble_kernel(Geometry g, const SideDesc* __restrict__ sides, TaskAcc* acc,
                                TimeState* ts, double* C, double* err, double* prev) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n_grid;
    if (k < g.n_species * n) {
        const int s = k / n;
        const int i = k - s * n;
        double c = 0.0, v = 0.0;
        const int nl = g.pt_hi - g.pt_lo;         // points of this context (a shard) in task order
        const bool mine = i >= g.pt_lo && i < g.pt_hi;
        for (int si = 0; si < (mine ? g.n_side : 0); ++si) {
            const SideDesc& sd = sides[si];
            if (sd.species_obs != s) continue;
            const int tg = (si * nl + i - g.pt_lo) * 2;
            TaskAcc& G = acc[tg];
            TaskAcc& L = acc[tg + 1];
            combine_task(G);
            combine_task(L);
            if (G.mean != 0.0) prev[tg] = fabs(G.mean);
            if (L.mean != 0.0) prev[tg + 1] = fabs(L.mean);
            c += sd.mult * (G.mean - L.mean);
            v += static_cast<double>(sd.mult) * sd.mult * (G.err * G.err + L.err * L.err);
        }
        if (!isfinite(c) || !isfinite(v)) ts->error = BEST_ERR_NUMERIC;
        C[k] = c;
        if (err) err[k] = sqrt(v);
    }
    if (k == 0) ts->call += 1u;
}

// ---------------------------------------------------------------------------
// Number and energy densities, one CTA (256 threads) per species:
//   n = Int q^2 f dq / (2 pi^2 a^3),  rho = Int q^2 E(q/a) f dq / (2 pi^2 a^3)
// over [q_min, q_max] on the FP64 not-a-knot spline (unclamped), 4-point
// Gauss-Legendre per grid interval, fixed-order tree reduction.
// ---------------------------------------------------------------------------
__global__ void moments_kernel(Geometry g, const double* __restrict__ knots, const double* __restrict__ coef64,
                               const TimeState* ts, double* n_out, double* rho_out) {
    __shared__ double sn[256], sr[256];
    const int s = blockIdx.x;
    const double a = ts->a, m = ts->mass[s];
    const double xg[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
    const double wg[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};
    double an = 0.0, ar = 0.0;
    for (int j = threadIdx.x; j < g.n_grid - 1; j += blockDim.x) {
        const double* c = coef64 + (static_cast<int64_t>(s) * (g.n_grid - 1) + j) * 4;
        const double lo = knots[j], hi = knots[j + 1];
        const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
        for (int k = 0; k < 4; ++k) {
            const double q = fma(half, xg[k], mid);
            const double tt = q - lo;
            const double f = fma(fma(fma(c[3], tt, c[2]), tt, c[1]), tt, c[0]);
            const double p = q / a;
            const double wq = half * wg[k] * q * q * f;
            an += wq;
            ar += wq * sqrt(fma(p, p, m * m));
        }
    }
    sn[threadIdx.x] = an;
    sr[threadIdx.x] = ar;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sn[threadIdx.x] += sn[threadIdx.x + h];
            sr[threadIdx.x] += sr[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double pref = 1.0 / (2.0 * kPi * kPi * a * a * a);
        n_out[s] = pref * sn[0];
        rho_out[s] = pref * sr[0];
    }
}

// ---------------------------------------------------------------------------
// Adaptive fractional width (App. C), one CTA per process after a sweep:
// r = sqrt(sum err_t^2) / sum |I_t| over the process's tasks (FP64, fixed
// summation order), then w /= factor below rel_lo, w *= factor above rel_hi,
// clamped to [w_min, w_max]; processes with a fixed width are left alone.
// ---------------------------------------------------------------------------
__global__ void width_control_kernel(Geometry g, const SideDesc* __restrict__ sides,
                                     const TaskDesc* __restrict__ tasks, const TaskAcc* __restrict__ acc,
                                     const WidthCtl* __restrict__ ctl, double* width, double* width_rel) {
    __shared__ double r2[256], ra[256];
    const int p = blockIdx.x;
    const WidthCtl c = ctl[p];
    if (c.mode != 2) return;
    double e2 = 0.0, am = 0.0;
    for (int t = threadIdx.x; t < g.n_tasks; t += blockDim.x) {
        if (sides[tasks[t].si].process != p) continue;
        const TaskAcc& A = acc[t];
        e2 = fma(A.err, A.err, e2);
        am += fabs(A.mean);
    }
    r2[threadIdx.x] = e2;
    ra[threadIdx.x] = am;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            r2[threadIdx.x] += r2[threadIdx.x + h];
            ra[threadIdx.x] += ra[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0 || !(ra[0] > 0.0)) return;
    const double rel = sqrt(r2[0]) / ra[0];
    double w = width[p];
    if (rel < c.rel_lo) w /= c.factor;
    else if (rel > c.rel_hi) w *= c.factor;
    width[p] = fmin(fmax(w, c.w_min), c.w_max);
    width_rel[p] = rel;
}

// ---------------------------------------------------------------------------
// Time stepping (Sec. 3C), one CTA of 1024 threads over all species and grid
// points.  max |C/f| is reduced in FP64 and the step used is
// dt = min(dt_requested, eps / max |C/f|) (Eq. (16)).
// ---------------------------------------------------------------------------
__device__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const double r = red[0];
    __syncthreads();
    return r;
}

// Euler (Eq. (14)) or the Heun predictor: dt from k1, logf_out = logf + dt k1/f.
// heun != 0: writes f* = exp(logf + dt k1/f) to fstar and leaves logf alone.
__global__ void step_first_kernel(Geometry g, double* logf, const double* __restrict__ fgrid,
                                  const double* __restrict__ k1, double* t_dev, double* dt_dev,
                                  TimeState* ts, double* fstar, int heun) {
    __shared__ double red[32];
    const int total = g.n_species * g.n_grid;
    double mx = 0.0;
    for (int k = threadIdx.x; k < total; k += blockDim.x) mx = fmax(mx, fabs(k1[k] / fgrid[k]));
    mx = block_max(mx, red);
    double dt = *dt_dev;
    if (mx > 0.0) dt = fmin(dt, g.eps_dt / mx);
    for (int k = threadIdx.x; k < total; k += blockDim.x) {
        const double step = dt * k1[k] / fgrid[k];
        if (heun) fstar[k] = exp(logf[k] + step);
        else logf[k] += step;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ts->dt = dt;
        ts->t_step = *t_dev;
        if (!heun) {
            *t_dev += dt;
            *dt_dev = dt;
        }
        if (!isfinite(dt)) ts->error = BEST_ERR_NUMERIC;
    }
}

// One stage of a step from collision integrals the caller assembled (sharded
// runs), one CTA of 1024 threads; the same arithmetic as step_first_kernel
// and heun_correct_kernel with f = exp(log f).
//   stage 0: dt = min(*dt_dev, eps / max |k1/f|); Euler: log f += dt k1/f,
//            t += dt; Heun: fstar = exp(log f + dt k1/f); *dt_dev = dt.
//   stage 1 (Heun): log f += dt/2 (k1/f + k2/fstar), t += dt.
__global__ void stage_kernel(Geometry g, int heun, int stage, double* logf, const double* __restrict__ k1,
                             const double* __restrict__ k2, double* fstar, double* t_dev, double* dt_dev,
                             TimeState* ts) {
    __shared__ double red[32];
    const int total = g.n_species * g.n_grid;
    if (stage == 0) {
        double mx = 0.0;
        for (int k = threadIdx.x; k < total; k += blockDim.x) mx = fmax(mx, fabs(k1[k] / exp(logf[k])));
        mx = block_max(mx, red);
        double dt = *dt_dev;
        if (mx > 0.0) dt = fmin(dt, g.eps_dt / mx);
        for (int k = threadIdx.x; k < total; k += blockDim.x) {
            const double step = dt * k1[k] / exp(logf[k]);
            if (heun) fstar[k] = exp(logf[k] + step);
            else logf[k] += step;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ts->dt = dt;
            ts->t_step = *t_dev;
            if (!heun) *t_dev += dt;
            *dt_dev = dt;
            if (!isfinite(dt)) ts->error = BEST_ERR_NUMERIC;
        }
    } else {
        const double dt = *dt_dev;
        for (int k = threadIdx.x; k < total; k += blockDim.x)
            logf[k] += 0.5 * dt * (k1[k] / exp(logf[k]) + k2[k] / fstar[k]);
        __syncthreads();
        if (threadIdx.x == 0) *t_dev += dt;
    }
}

// Heun corrector (Eq. (15)): logf += dt/2 (k1/f + k2/f*), f = exp(logf)
// (log f is left untouched by the predictor).
__global__ void heun_correct_kernel(Geometry g, double* logf, const double* __restrict__ fstar, const double* __restrict__ k1,
                                    const double* __restrict__ k2, double* t_dev, double* dt_dev,
                                    TimeState* ts) {
    const int total = g.n_species * g.n_grid;
    const double dt = ts->dt;
    for (int k = threadIdx.x; k < total; k += blockDim.x)
        logf[k] += 0.5 * dt * (k1[k] / exp(logf[k]) + k2[k] / fstar[k]);
    __syncthreads();
    if (threadIdx.x == 0) {
        *t_dev = ts->t_step + dt;
        *dt_dev = dt;
    }
}

}  // namespace best
