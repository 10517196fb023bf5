// Implicit log-space Euler step: g = log f at t + dt solves
//   R(g) = g - g_n - dt C~(e^g) / e^g = 0,
// the backward-Euler counterpart of Eq. (14) on the fixed-sample collision
// integral C~.  Newton's method with the linear systems J_R d = -R solved
// by GMRES (Arnoldi with modified Gram-Schmidt, repeated once, and Givens
// rotations); the Jacobian is never formed: its product with a direction x is
//   J_R x = x - dt [ (J (f x)) / f - (C~ / f) x ],   J = dC~/df,
// one forward-mode tangent launch per product.  The vectors have
// n_species * n_grid entries (at most a few thousand), so the Krylov
// arithmetic runs in one CTA per kernel; the cost is the tangent launches.
#include "internal.cuh"

namespace best {

namespace {

__device__ double nk_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) s += red[k];      // same order in every thread
    return s;
}

__device__ double nk_block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) s = fmax(s, red[k]);
    return s;
}

}  // namespace

// f = exp(g)
__global__ void nk_exp_kernel(int N, const double* __restrict__ g, double* __restrict__ f) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) f[k] = exp(g[k]);
}

// out = g + lambda d
__global__ void nk_axpy_kernel(int N, const double* __restrict__ g, const double* __restrict__ d, double lambda,
                               double* __restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
        out[k] = fma(lambda, d[k], g[k]);
}

// Tangent of f along the log-space direction x: u = f x.
__global__ void nk_direction_kernel(int N, const double* __restrict__ f, const double* __restrict__ x,
                                    double* __restrict__ u) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) u[k] = f[k] * x[k];
}

// r = g - g_n - dt C / f and Qd = C / f; stat[0] = ||r||_2, stat[1] = ||r||_inf,
// stat[4] = 1 if any entry is not finite.  One CTA.
__global__ void nk_residual_kernel(int N, const double* __restrict__ g, const double* __restrict__ gn,
                                   const double* __restrict__ C, const double* __restrict__ f, double dt,
                                   double* __restrict__ r, double* __restrict__ Qd, double* stat) {
    __shared__ double red[32];
    double s2 = 0.0, mx = 0.0, bad = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double q = C[k] / f[k];
        const double rk = g[k] - gn[k] - dt * q;
        Qd[k] = q;
        r[k] = rk;
        if (!isfinite(rk)) bad = 1.0;
        s2 = fma(rk, rk, s2);
        mx = fmax(mx, fabs(rk));
    }
    s2 = nk_block_sum(s2, red);
    mx = nk_block_max(mx, red);
    bad = nk_block_max(bad, red);
    if (threadIdx.x == 0) {
        stat[0] = sqrt(s2);
        stat[1] = mx;
        stat[4] = bad;
    }
}

// V_0 = -r / ||r||, gvec = (||r||, 0, ..., 0).  One CTA.
__global__ void gmres_start_kernel(int N, int m, const double* __restrict__ r, double* __restrict__ V,
                                   double* __restrict__ gvec) {
    __shared__ double red[32];
    double s2 = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) s2 = fma(r[k], r[k], s2);
    const double beta = sqrt(nk_block_sum(s2, red));
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) V[k] = -r[k] * inv;
    for (int k = threadIdx.x; k <= m; k += blockDim.x) gvec[k] = k == 0 ? beta : 0.0;
}

// Arnoldi step j: w = J_R V_j from the tangent JU = J (f V_j); orthogonalise
// against V_0 .. V_j (modified Gram-Schmidt, two passes), store column j of
// the Hessenberg matrix H ((m+1) x m, column major), V_{j+1} = w / ||w||,
// rotate the column with the previous Givens rotations, make rotation j, and
// update the least-squares right-hand side gvec.  stat[2] = |gvec[j+1]| (the
// residual norm of the GMRES iterate), stat[3] = ||w|| (0: breakdown, the
// Krylov space is invariant).  One CTA.
__global__ void gmres_arnoldi_kernel(int N, int m, int j, double dt, const double* __restrict__ f,
                                     const double* __restrict__ Qd, const double* __restrict__ JU,
                                     double* __restrict__ V, double* __restrict__ H, double* __restrict__ cs,
                                     double* __restrict__ sn, double* __restrict__ gvec, double* stat) {
    __shared__ double red[32];
    const double* vj = V + static_cast<int64_t>(j) * N;
    double* w = V + static_cast<int64_t>(j + 1) * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x)
        w[k] = vj[k] - dt * (JU[k] / f[k] - Qd[k] * vj[k]);
    __syncthreads();
    double* h = H + static_cast<int64_t>(j) * (m + 1);
    for (int i = threadIdx.x; i <= m; i += blockDim.x) h[i] = 0.0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i <= j; ++i) {
            const double* vi = V + static_cast<int64_t>(i) * N;
            double d = 0.0;
            for (int k = threadIdx.x; k < N; k += blockDim.x) d = fma(w[k], vi[k], d);
            d = nk_block_sum(d, red);
            for (int k = threadIdx.x; k < N; k += blockDim.x) w[k] = fma(-d, vi[k], w[k]);
            if (threadIdx.x == 0) h[i] += d;
            __syncthreads();
        }
    }
    double s2 = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) s2 = fma(w[k], w[k], s2);
    const double hn = sqrt(nk_block_sum(s2, red));
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) w[k] *= inv;
    if (threadIdx.x == 0) {
        h[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double a = h[i], b = h[i + 1];
            h[i] = cs[i] * a + sn[i] * b;
            h[i + 1] = -sn[i] * a + cs[i] * b;
        }
        const double a = h[j], b = h[j + 1];
        const double rr = hypot(a, b);
        const double c = rr > 0.0 ? a / rr : 1.0, s = rr > 0.0 ? b / rr : 0.0;
        cs[j] = c;
        sn[j] = s;
        h[j] = rr;
        h[j + 1] = 0.0;
        gvec[j + 1] = -s * gvec[j];
        gvec[j] = c * gvec[j];
        stat[2] = fabs(gvec[j + 1]);
        stat[3] = hn;
    }
}

// GMRES update after k Arnoldi steps: y = R_k^{-1} gvec[0:k] (R_k the rotated
// upper-triangular H) and d = V[:, 0:k] y.  One CTA; y in shared memory.
__global__ void gmres_update_kernel(int N, int m, int k, const double* __restrict__ V, const double* __restrict__ H,
                                    const double* __restrict__ gvec, double* __restrict__ d) {
    __shared__ double y[64];
    if (threadIdx.x == 0) {
        for (int i = k - 1; i >= 0; --i) {
            double s = gvec[i];
            for (int c = i + 1; c < k; ++c) s -= H[static_cast<int64_t>(c) * (m + 1) + i] * y[c];
            const double dii = H[static_cast<int64_t>(i) * (m + 1) + i];
            y[i] = dii != 0.0 ? s / dii : 0.0;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(y[i], V[static_cast<int64_t>(i) * N + e], s);
        d[e] = s;
    }
}

}  // namespace best
