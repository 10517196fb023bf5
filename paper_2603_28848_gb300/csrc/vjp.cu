// Adjoint of the fixed-sample collision integral: instantiations of the
// adjoint sample kernel and the FP64 kernels that turn its per-segment
// records and coefficient gradients into dL/df, dL/dm and dL/dcoupling.
#include <cmath>

#include "vjp_impl.cuh"

namespace best {

template <bool JVP>
void* kernel_ptr(bool f32, int nmax) {
    if (f32) {
        if (nmax <= 4) return reinterpret_cast<void*>(&vjp_kernel<float, 4, JVP>);
        if (nmax == 5) return reinterpret_cast<void*>(&vjp_kernel<float, 5, JVP>);
        return reinterpret_cast<void*>(&vjp_kernel<float, 6, JVP>);
    }
    if (nmax <= 4) return reinterpret_cast<void*>(&vjp_kernel<double, 4, JVP>);
    if (nmax == 5) return reinterpret_cast<void*>(&vjp_kernel<double, 5, JVP>);
    return reinterpret_cast<void*>(&vjp_kernel<double, 6, JVP>);
}

void* vjp_me_kernel_ptr(bool f32, int nmax, bool jvp);     // vjp_me.cu

// me: some process has an s-dependent |M|^2 (the extended instantiations)
void* vjp_kernel_ptr(bool f32, int nmax, bool me) {
    return me ? vjp_me_kernel_ptr(f32, nmax, false) : kernel_ptr<false>(f32, nmax);
}
void* jvp_kernel_ptr(bool f32, int nmax, bool me) {
    return me ? vjp_me_kernel_ptr(f32, nmax, true) : kernel_ptr<true>(f32, nmax);
}

// Adjoint seed of every task: L = sum_{a,i} v_{a,i} C~_a(p_i) and C~ = sum
// mult (I_gain - I_loss), I = K scale (sum w_n) / N, so dL/dw_n = v mult sign
// K scale / N for each of the task's samples.
__global__ void vjp_seed_kernel(Geometry g, const SideDesc* __restrict__ sides, const TaskDesc* __restrict__ tasks,
                                const TaskConst* __restrict__ tconst, const double* __restrict__ v, double* u) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n_tasks) return;
    const TaskDesc td = tasks[t];
    const SideDesc& sd = sides[td.si];
    const double sign = td.term == 0 ? 1.0 : -1.0;
    u[t] = v[static_cast<int64_t>(sd.species_obs) * g.n_grid + td.point] * sd.mult * sign * tconst[t].K *
           tconst[t].scale / static_cast<double>(td.neval);
}

// Tangent seed: d w_n / d f_obs u_obs = (w_n / c0) dobs u_{a,i} / scale.
__global__ void jvp_seed_kernel(Geometry g, const SideDesc* __restrict__ sides, const TaskDesc* __restrict__ tasks,
                                const TaskConst* __restrict__ tconst, const SpeciesConst* __restrict__ sconst,
                                const double* __restrict__ uvec, double* u) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n_tasks) return;
    const TaskDesc td = tasks[t];
    const SideDesc& sd = sides[td.si];
    const double dobs = td.term == 1 ? 1.0 : sconst[sd.species_obs].eta;
    u[t] = dobs * uvec[static_cast<int64_t>(sd.species_obs) * g.n_grid + td.point] / tconst[t].scale;
}

// C~ and dC~ = J u from the tasks' tangent records; one thread, tasks in order.
__global__ void jvp_finish_kernel(Geometry g, const SideDesc* __restrict__ sides, const TaskDesc* __restrict__ tasks,
                                  const TaskConst* __restrict__ tconst, const double* __restrict__ tot, double* C,
                                  double* JU) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = g.n_grid;
    for (int k = 0; k < g.n_species * n; ++k) { C[k] = 0.0; JU[k] = 0.0; }
    for (int t = 0; t < g.n_tasks; ++t) {
        const TaskDesc td = tasks[t];
        const SideDesc& sd = sides[td.si];
        const double* T = tot + static_cast<int64_t>(t) * 16;
        const int64_t ai = static_cast<int64_t>(sd.species_obs) * n + td.point;
        const double f = sd.mult * (td.term == 0 ? 1.0 : -1.0) * tconst[t].K * tconst[t].scale /
                         static_cast<double>(td.neval);
        C[ai] += f * T[0];
        JU[ai] += f * T[1];
    }
}

// Sum of each task's segment records (fixed order), 16 doubles per task.
__global__ void vjp_task_kernel(Geometry g, const int32_t* __restrict__ active, const int32_t* __restrict__ task_seg,
                                const Segment* __restrict__ segs, const double* __restrict__ partials, int n_active,
                                double* tot) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_active) return;
    const int t = active[a];
    double s[16] = {};
    for (int k = task_seg[a]; k < task_seg[a + 1]; ++k)
        for (int v = 0; v < 12; ++v) s[v] += partials[segs[k].part + v];
    for (int v = 0; v < 16; ++v) tot[static_cast<int64_t>(t) * 16 + v] = s[v];
}

// C~, the observed-leg and mass / coupling parts of the gradient, and the
// tail-parameter gradients per species; one thread, tasks in order.
__global__ void vjp_finish_kernel(Geometry g, const SideDesc* __restrict__ sides, const TaskDesc* __restrict__ tasks,
                                  const TaskConst* __restrict__ tconst, const SpeciesConst* __restrict__ sconst,
                                  const TimeState* ts, const double* __restrict__ v, const double* __restrict__ u,
                                  const double* __restrict__ tot, const double* __restrict__ coupling, double* C,
                                  double* gf, double* gm, double* gcoupling, double* gtail, int n_processes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = g.n_grid;
    for (int k = 0; k < g.n_species * n; ++k) { C[k] = 0.0; gf[k] = 0.0; }
    for (int s = 0; s < g.n_species; ++s) {
        gm[s] = 0.0;
        for (int q = 0; q < 4; ++q) gtail[s * 4 + q] = 0.0;
    }
    for (int p = 0; p < n_processes; ++p) gcoupling[p] = 0.0;
    for (int t = 0; t < g.n_tasks; ++t) {
        const TaskDesc td = tasks[t];
        const SideDesc& sd = sides[td.si];
        const TaskConst& c = tconst[t];
        const double* T = tot + static_cast<int64_t>(t) * 16;
        const int a = sd.species_obs;
        const int64_t ai = static_cast<int64_t>(a) * n + td.point;
        const double sign = td.term == 0 ? 1.0 : -1.0;
        const double I = T[0] / static_cast<double>(td.neval) * c.K * c.scale;
        C[ai] += sd.mult * sign * I;
        const double U = u[t];
        const double dobs = td.term == 1 ? 1.0 : sconst[a].eta;
        gf[ai] += U * T[1] * dobs / c.scale;
        gm[a] += U * T[2] * ts->mass[a] / c.E_obs;
        const int sc = sd.leg_species[sd.cons];
        gm[sc] += U * T[3];
        for (int q = 0; q < 4; ++q) gtail[sc * 4 + q] += U * T[4 + q];
        for (int j = 0; j < sd.n - 2; ++j) gm[sd.leg_species[sd.integ[j]]] += U * T[8 + j];
        gcoupling[sd.process] += 2.0 / coupling[sd.process] * sd.mult * sign * I * v[ai];
    }
}

// Transpose of the spline construction for one species per CTA (thread 0):
// the interval coefficients are linear in f through the second derivatives
// M (not-a-knot tridiagonal system), so df = L^T dcoef; plus the tail fits'
// dependence on the end values f_j and, through E(q_j/a), on the mass.
// Dynamic shared memory: 3 n doubles.
__global__ void spline_adjoint_kernel(Geometry g, const double* __restrict__ knots, const double* __restrict__ fgrid,
                                      const SpeciesConst* __restrict__ sconst, const TimeState* ts,
                                      const double* __restrict__ gcoef, const double* __restrict__ gtail,
                                      double* gf, double* gm) {
    extern __shared__ double sh[];
    if (threadIdx.x != 0) return;
    const int n = g.n_grid;
    const int s = blockIdx.x;
    double* gM = sh;
    double* cp = sh + n;
    double* yv = sh + 2 * n;
    const double* gc = gcoef + static_cast<int64_t>(s) * (n - 1) * 4;
    const double* f = fgrid + static_cast<int64_t>(s) * n;
    double* out = gf + static_cast<int64_t>(s) * n;
    auto h = [&](int i) { return knots[i + 1] - knots[i]; };
    for (int j = 0; j < n; ++j) gM[j] = 0.0;
    for (int j = 0; j < n - 1; ++j) {
        const double hj = h(j);
        const double g0 = gc[4 * j], g1 = gc[4 * j + 1], g2 = gc[4 * j + 2], g3 = gc[4 * j + 3];
        out[j] += g0 - g1 / hj;
        out[j + 1] += g1 / hj;
        gM[j] += -g1 * hj / 3.0 + 0.5 * g2 - g3 / (6.0 * hj);
        gM[j + 1] += -g1 * hj / 6.0 + g3 / (6.0 * hj);
    }
    {
        const double h0 = h(0), h1 = h(1);
        gM[1] += gM[0] * (h0 + h1) / h1;
        gM[2] += -gM[0] * h0 / h1;
        const double hl = h(n - 2), hp = h(n - 3);
        gM[n - 2] += gM[n - 1] * (hl + hp) / hp;
        gM[n - 3] += -gM[n - 1] * hl / hp;
    }
    // rows of the interior system (as in the forward solve)
    const int m = n - 2;
    auto row = [&](int k, double* ra, double* rb, double* rc) {
        const int i = k + 1;
        double a = h(i - 1), b = 2.0 * (h(i - 1) + h(i)), c = h(i);
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
        *ra = a; *rb = b; *rc = c;
    };
    // solve A^T y = gM[1 .. n-2]: A^T has sub-diagonal c_{k-1}, diagonal b_k, super-diagonal a_{k+1}
    for (int k = 0; k < m; ++k) {
        double a_k, b_k, c_k;
        row(k, &a_k, &b_k, &c_k);
        double lo = 0.0;
        if (k > 0) {
            double a_p, b_p, c_p;
            row(k - 1, &a_p, &b_p, &c_p);
            lo = c_p;
        }
        double up = 0.0;
        if (k + 1 < m) {
            double a_n, b_n, c_n;
            row(k + 1, &a_n, &b_n, &c_n);
            up = a_n;
        }
        const double rhs = gM[k + 1];
        if (k == 0) {
            cp[0] = up / b_k;
            yv[0] = rhs / b_k;
        } else {
            const double den = b_k - lo * cp[k - 1];
            cp[k] = up / den;
            yv[k] = (rhs - lo * yv[k - 1]) / den;
        }
    }
    for (int k = m - 2; k >= 0; --k) yv[k] -= cp[k] * yv[k + 1];
    // r_i = 6 ((f_{i+1} - f_i)/h_i - (f_i - f_{i-1})/h_{i-1}),  i = k + 1
    for (int k = 0; k < m; ++k) {
        const int i = k + 1;
        const double y = 6.0 * yv[k];
        out[i + 1] += y / h(i);
        out[i] -= y * (1.0 / h(i) + 1.0 / h(i - 1));
        out[i - 1] += y / h(i - 1);
    }
    // tail fits (least squares of y = log(1/f + eta) against x = E(q/a))
    const double eta = sconst[s].eta;
    const double mass = ts->mass[s];
    const double aa = ts->a;
    const int K = g.tail_points;
    for (int end = 0; end < 2; ++end) {
        const double ga = gtail[s * 4 + 2 * end], gb = gtail[s * 4 + 2 * end + 1];
        if (ga == 0.0 && gb == 0.0) continue;
        double xm = 0.0, ym = 0.0;
        for (int k = 0; k < K; ++k) {
            const int j = end == 0 ? k : n - K + k;
            const double p = knots[j] / aa;
            xm += sqrt(p * p + mass * mass);
            ym += log(1.0 / f[j] + eta);
        }
        xm /= K;
        ym /= K;
        double sxx = 0.0, sxy = 0.0;
        for (int k = 0; k < K; ++k) {
            const int j = end == 0 ? k : n - K + k;
            const double p = knots[j] / aa;
            const double x = sqrt(p * p + mass * mass);
            sxx += (x - xm) * (x - xm);
            sxy += (x - xm) * (log(1.0 / f[j] + eta) - ym);
        }
        const double b = sxy / sxx;
        for (int k = 0; k < K; ++k) {
            const int j = end == 0 ? k : n - K + k;
            const double p = knots[j] / aa;
            const double x = sqrt(p * p + mass * mass);
            const double y = log(1.0 / f[j] + eta);
            const double dady = 1.0 / K - xm * (x - xm) / sxx;
            const double dbdy = (x - xm) / sxx;
            const double dydf = -1.0 / (f[j] * (1.0 + eta * f[j]));
            out[j] += (ga * dady + gb * dbdy) * dydf;
            const double dbdx = ((y - ym) - 2.0 * b * (x - xm)) / sxx;
            const double dadx = -b / K - xm * dbdx;
            if (x > 0.0) gm[s] += (ga * dadx + gb * dbdx) * mass / x;
        }
    }
}

}  // namespace best
