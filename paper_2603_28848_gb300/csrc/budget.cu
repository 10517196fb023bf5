// Variance-driven sample budgets and the device-side work partition.
//
// After every sweep, budget_kernel re-sets the samples per iteration of the
// tasks of each process with budget = 1 from the sweep's estimates (the
// integrators are reused from sweep to sweep, Sec. 3D): N_t = lambda v_t with
// v_t = N_t (err_t / I_t)^2, lambda by bisection so that the clipped budgets
// keep the process's total, rounded down to a multiple of kBudgetQuantum and
// held within [n_min, n_max].  plan_kernel then rebuilds the static
// partition of every iteration's sample groups over the persistent grid from
// the new budgets, with the same cost model and arithmetic as the host-built
// partition, so that graph-replayed steps pick the budgets up with no host
// round trip.
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace best {

namespace {

// Sum over the CTA in a fixed order (deterministic); s: blockDim doubles.
__device__ double cta_sum(double v, double* s) {
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (static_cast<int>(threadIdx.x) < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

__device__ double cta_min(double v, double* s) {
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (static_cast<int>(threadIdx.x) < o) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

// Exclusive prefix over the CTA of one int64 per thread, with the total;
// s: blockDim int64.
__device__ int64_t cta_scan(int64_t v, int64_t* s, int64_t* total) {
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

__device__ inline double clip(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

}  // namespace

// One CTA (blockDim a power of two) per process with variance-driven budgets.
// v: scratch of n_tasks doubles.
__global__ void budget_kernel(const BudgetCtl* __restrict__ ctl, const TaskAcc* __restrict__ acc, TaskDesc* tasks,
                              double* v) {
    __shared__ double s[1024];
    const BudgetCtl c = ctl[blockIdx.x];
    const double nmin = static_cast<double>(c.n_min), nmax = static_cast<double>(c.n_max);
    double vmin = INFINITY;
    for (int k = threadIdx.x; k < c.count; k += blockDim.x) {
        const int t = c.first + k;
        const double m = acc[t].mean, e = acc[t].err;
        double x = 0.0;
        if (m != 0.0 && isfinite(m) && isfinite(e)) {
            const double r = e / m;
            x = static_cast<double>(tasks[t].neval) * (r * r);
            if (!isfinite(x)) x = 0.0;
        }
        v[t] = x;
        if (x > 0.0) vmin = fmin(vmin, x);
    }
    vmin = cta_min(vmin, s);
    double lam = 0.0;
    if (vmin < INFINITY) {
        double lo = 0.0, hi = 2.0 * nmax / vmin;
        for (int it = 0; it < kBudgetBisections; ++it) {
            const double mid = 0.5 * (lo + hi);
            double part = 0.0;
            for (int k = threadIdx.x; k < c.count; k += blockDim.x) part += clip(mid * v[c.first + k], nmin, nmax);
            if (cta_sum(part, s) < c.total) lo = mid;
            else hi = mid;
        }
        lam = lo;
    }
    for (int k = threadIdx.x; k < c.count; k += blockDim.x) {
        const int t = c.first + k;
        const double q = static_cast<double>(kBudgetQuantum);
        const double N = q * floor(fmin(lam * v[t], 2.0 * nmax) / q);
        tasks[t].neval = static_cast<int64_t>(clip(N, nmin, nmax));
    }
}

// Rebuilds the partition of every iteration index (one CTA, blockDim a
// power of two): plan p's active tasks are split into segments of sample
// groups, chunk c of the K = chunk_count(B) chunks (B: the persistent grid)
// taking the cost range [chunk_bound(W, c, sh), chunk_bound(W, c + 1, sh)),
// sh = chunk_shape(W, B), with
// cost (groups x group size x unit) x (D + 6) per task, as the host-built
// partition does; segments are ordered by task, the partial records laid out
// in segment order.  scratch: int64 of max(n_active) + 1 + 2 K.
__global__ void plan_kernel(const TaskDesc* __restrict__ tasks, int n_plans, const PlanDev* __restrict__ plans,
                            int B, int f32, int64_t* scratch) {
    __shared__ int64_t s[1024];
    const int K = chunk_count(B);
    for (int p = 0; p < n_plans; ++p) {
        const PlanDev pl = plans[p];
        const int A = pl.n_active;
        int64_t* cum = scratch;                 // [A + 1]
        int64_t* cnt = scratch + A + 1;         // [K] segments of chunk b, then their first index
        int64_t* rec = cnt + K;                 // [K] record doubles of chunk b, then their offset
        // cost prefix of the active tasks
        int64_t carry = 0;
        for (int a0 = 0; a0 < A; a0 += blockDim.x) {
            const int a = a0 + threadIdx.x;
            int64_t w = 0;
            if (a < A) {
                const TaskDesc td = tasks[pl.active[a]];
                const int G = stream_group(td.dim, f32 != 0);
                const int64_t unit = td.strat_H > 0 ? kItem / G : 1;
                const int64_t groups = (td.neval + G - 1) / G / unit;
                w = groups * (static_cast<int64_t>(G) * unit * (td.dim + 6));
            }
            int64_t tot;
            const int64_t ex = cta_scan(w, s, &tot);
            if (a < A) cum[a] = carry + ex;
            carry += tot;
        }
        if (threadIdx.x == 0) cum[A] = carry;
        __syncthreads();
        const int64_t W = carry;
        const ChunkShape sh = chunk_shape(W, B);
        // pass 1: segments and record doubles per chunk; pass 2: write them
        for (int pass = 0; pass < 2; ++pass) {
            for (int b = threadIdx.x; b < K; b += blockDim.x) {
                const int64_t lo = chunk_bound(W, b, sh), hi = chunk_bound(W, b + 1, sh);
                int a = 0, top = A;             // first a with cum[a + 1] > lo
                while (a < top) {
                    const int mid = (a + top) >> 1;
                    if (cum[mid + 1] <= lo) a = mid + 1;
                    else top = mid;
                }
                int64_t k = pass ? cnt[b] : 0, off = pass ? rec[b] : 0;
                for (; a < A && cum[a] < hi; ++a) {
                    const TaskDesc td = tasks[pl.active[a]];
                    const int G = stream_group(td.dim, f32 != 0);
                    const int64_t unit = td.strat_H > 0 ? kItem / G : 1;
                    const int64_t groups = (td.neval + G - 1) / G / unit;
                    const int64_t cg = static_cast<int64_t>(G) * unit * (td.dim + 6);
                    const int64_t g0 = max(int64_t(0), (lo - cum[a] + cg - 1) / cg);
                    const int64_t g1 = min(groups, (hi - cum[a] + cg - 1) / cg);
                    if (g1 <= g0) continue;
                    if (pass) {
                        Segment sg{};
                        sg.task = pl.active[a];
                        sg.g0 = g0 * unit;
                        sg.g1 = g1 * unit;
                        sg.part = off;
                        pl.segs[k] = sg;
                        if (g0 == 0) pl.task_seg[a] = static_cast<int32_t>(k);
                    }
                    ++k;
                    off += record_doubles(td.dim, td.nbins);
                }
                if (!pass) {
                    cnt[b] = k;
                    rec[b] = off;
                }
            }
            __syncthreads();
            if (!pass) {
                // exclusive prefixes over the chunks
                int64_t c1 = 0, c2 = 0;
                for (int b0 = 0; b0 < K; b0 += blockDim.x) {
                    const int b = b0 + threadIdx.x;
                    int64_t t1, t2;
                    const int64_t e1 = cta_scan(b < K ? cnt[b] : 0, s, &t1);
                    const int64_t e2 = cta_scan(b < K ? rec[b] : 0, s, &t2);
                    if (b < K) {
                        cnt[b] = c1 + e1;
                        rec[b] = c2 + e2;
                        pl.cta_seg[b] = static_cast<int32_t>(c1 + e1);
                    }
                    c1 += t1;
                    c2 += t2;
                }
                if (threadIdx.x == 0) {
                    pl.cta_seg[K] = static_cast<int32_t>(c1);
                    pl.task_seg[A] = static_cast<int32_t>(c1);
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

}  // namespace best
