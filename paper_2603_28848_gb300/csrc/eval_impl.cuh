// Sample kernel of one VEGAS iteration over every active task (one
// persistent launch for all grid points, species, processes and pinned
// sides).  Included by eval_f32.cu and eval_f64.cu, which instantiate it for
// FP32 and FP64 integrand arithmetic.
//
// Per sample (Sec. 2D, App. A):
//   uniforms (Philox stream) -> VEGAS map -> (r, theta, phi) per integrated
//   leg -> physical momenta p = r/a -> conserved leg from momentum
//   conservation (Eq. (10)) -> energies -> Gaussian delta of Eq. (11) ->
//   statistical factor of Eq. (5) with spline / Eq. (13) lookups -> weight of
//   Eq. (12) -> compensated sums of w and w^2 and per-increment sums of w^2.
//
// Normalisation: the kernel accumulates w_n = w / (K * scale) with the FP64
// per-task constants K = |M|^2 nb^D a^{-3(n-2)} / ((2pi)^{3(n-1)-4} 2^n
// E_obs sigma sqrt(2pi)) and scale = f_obs, so that w_n is O(1) near
// equilibrium and w_n^2 stays inside the FP32 range.  The map table in
// shared memory holds, per dimension and increment, the scaled left edge Y0
// and width dY of the physical variable, so y = Y0 + dY * (x nb - b) and the
// Jacobian times the volume of the linear scaling is nb^D prod dY.
#pragma once

#include <cstdint>

#include "internal.cuh"
#include "philox.cuh"

namespace best {

template <typename R>
struct Real2 { R y0, dy; };

template <typename R> struct RMath;

// 2^x with denormal results flushed to zero (the bare special-function op)
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(x) of a normal positive float, the bare special-function op (the
// FP32 kernels guard its arguments to at least 1e-30: momenta and energies
// squared, never subnormal there).
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <> struct RMath<float> {
    static constexpr bool kF32 = true;
    __device__ static __forceinline__ void sincos_(float x, float* s, float* c) { __sincosf(x, s, c); }
    __device__ static __forceinline__ float rsqrt_(float x) { return rsqrt_ftz(x); }
    static constexpr float kTiny = 1e-30f;         // smallest argument rsqrt_ is given
    __device__ static __forceinline__ float exp2_(float x) { return ex2_ftz(x); }   // (Gaussian: x <= 0)
    __device__ static __forceinline__ float expm1_(float x) { return expm1f(x); }
    __device__ static __forceinline__ float exp_(float x) { return __expf(x); }
    __device__ static __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
};

template <> struct RMath<double> {
    static constexpr bool kF32 = false;
    __device__ static __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
    __device__ static __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static constexpr double kTiny = 0.0;
    __device__ static __forceinline__ double exp2_(double x) { return exp2(x); }
    __device__ static __forceinline__ double expm1_(double x) { return expm1(x); }
    __device__ static __forceinline__ double exp_(double x) { return exp(x); }
    __device__ static __forceinline__ double rcp_(double x) { return 1.0 / x; }
};

// Compensated (Kahan) sum for the FP32 path; a plain sum for FP64.
template <typename R>
struct Acc {
    R s = 0, c = 0;
    __device__ __forceinline__ void add(R x) {
        if constexpr (sizeof(R) == 4) {
            const R y = x - c;
            const R t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ double value() const {
        return static_cast<double>(s) - static_cast<double>(c);
    }
};

// Energy balance E_in - E_out of Eq. (11) accumulated without losing the
// rounding of each addition: in FP32 an error-free transformation (Knuth's
// TwoSum) keeps the running sum s and, in c, the sum of the exact rounding
// errors of the additions, so that s + c is the sum of the terms to about
// FP32 precision of the (small) result rather than of the (large) energies;
// in FP64 a plain sum.
template <typename R>
struct EBal {
    R s, c;
    __device__ __forceinline__ explicit EBal(R x0) : s(x0), c(R(0)) {}
    __device__ __forceinline__ void add(R x) {
        if constexpr (sizeof(R) == 4) {
            const R t = s + x;
            const R xp = t - s;
            const R sp = t - xp;
            c += (s - sp) + (x - xp);
            s = t;
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ R value() const { return s + c; }
};

// Spline lookup tables of one species in shared memory.
template <typename R>
struct SplineView {
    const R* coef;          // [n-1][4]: c0 + c1 t + c2 t^2 + c3 t^3, t = q - q_j
    const R* knot;          // [n]
};


// Per-segment constants held in registers (uniform across the CTA).
template <typename R, int NLEG>
struct SegConst {
    static constexpr int NI = NLEG - 2;
    R pobs_sig;             // sigma_obs * p_obs (z component of the obs leg in p_cons)
    R sgn_obs_E;            // s_obs * E_obs (its share of E_in - E_out)
    R sig[NI];              // +-1: share of integrated leg j in p_cons
    R sgnE[NI];             // +-1: initial / final leg j in E_in - E_out
    R sgn_cons;             // same for the conserved leg
    R m2[NI];               // masses^2
    R m2c;
    R ca[NI], cb[NI];       // statistical factor of leg j: ca + cb f
    R cac, cbc;             // ... of the conserved leg
    int spc[NI];            // species of leg j
    int sp_cons;
    R inv_a, a;
    R c0;                   // obs factor / scale
    R gauss_k;              // -log2(e) / (2 sigma^2); fractional width: -2 log2(e) / w^2
    R e_obs;                // E_obs (fractional width: sigma_ref / sigma = 2 E_obs / (E_in + E_out))
    bool frac;              // fractional width of App. C
    bool me_on;             // |M|^2 / coupling^2 = P(s) not constant
    R me[4];                // P(s) coefficients
    R inw[NI];              // 1: integrated leg j is initial (enters s), else 0
    R cons_inw;             // 1: conserved leg initial
    R obs_in_p, obs_in_E;   // observed leg's p_z and E if it is initial, else 0
    R e_cut;
    R eta_c;                // eta of the conserved leg (tail formula)
    R tlo_a, tlo_b, thi_a, thi_b;   // Eq. (13) end fits of the conserved leg's species
    int fd_c;               // conserved leg is FD (clamp f <= 1)
    int fd[NI];
};

// log2 of a normal positive float, the bare special-function op (no
// subnormal handling: the spline lookups take momenta >= q_0 > 0).
__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Cubic spline value at comoving q inside [q_0, q_{n-1}] (Sec. 3B).
template <typename R>
__device__ __forceinline__ R spline_eval(const SplineView<R>& sv, R q, const Geometry& g,
                                         R inv_step, R q0, R lq0_step) {
    // interval index from the grid formula (a guess within one interval of
    // the exact one; the cubic pieces agree to C^2 at the knots)
    int j;
    if (g.log_spaced) {
        // log2(q / q0) / step = log2(q) / step - log2(q0) / step
        j = static_cast<int>(fmaf(lg2_ftz(static_cast<float>(q)), static_cast<float>(inv_step),
                                  -static_cast<float>(lq0_step)));
    } else {
        j = static_cast<int>(static_cast<float>((q - q0) * inv_step));
    }
    j = min(max(j, 0), g.n_grid - 2);
    const R t = q - sv.knot[j];
    R f;
    if constexpr (sizeof(R) == 4) {
        const float4 c = reinterpret_cast<const float4*>(sv.coef)[j];
        f = fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
    } else {
        const double2* cp = reinterpret_cast<const double2*>(sv.coef) + 2 * j;
        const double2 lo = cp[0], hi = cp[1];
        f = fma(fma(fma(hi.y, t, hi.x), t, lo.y), t, lo.x);
    }
    return f > R(0) ? f : R(0);
}

// 1 / (exp(x) - eta) of the Eq. (13) tails, FP32, without branches: for BE
// small x uses exp(x) - 1 = x (1 + x/2 + x^2/6) to avoid cancellation.
__device__ __forceinline__ float tail_f32(float x, float eta) {
    const float e = __expf(x);
    const float small = x * fmaf(x, fmaf(x, 0.16666667f, 0.5f), 1.0f);
    const float den = (eta == 1.0f && fabsf(x) < 0.03f) ? small : e - eta;
    return den > 0.0f ? __fdividef(1.0f, den) : 0.0f;      // MUFU reciprocal (2 ulp)
}

// Kinematic part of the weight of one sample at the mapped point y (r,
// theta, phi - pi per integrated leg) with map Jacobian jac: momenta, the
// conserved leg from momentum conservation, energies, the Gaussian of
// Eq. (11), the phase-space measure of Eq. (12) and, in the EXT
// instantiation, an s-dependent |M|^2.  Returns 0 for a cut sample and leaves
// what the statistical factor needs in r (comoving radii of the integrated
// legs), qc (comoving momentum of the conserved leg) and Ec (its energy).
template <typename R, int NLEG, bool EXT>
__device__ __forceinline__ R kin_at(const SegConst<R, NLEG>& C, const R* y, R jac, R* r, R& qc, R& Ec) {
    constexpr int NI = NLEG - 2;
    R px = R(0), py = R(0), pz = C.pobs_sig;
    EBal<R> bal(C.sgn_obs_E);
    R Esum = C.e_obs;                   // E_in + E_out (used when C.frac)
    R Qx = R(0), Qy = R(0), Qz = C.obs_in_p, Ein = C.obs_in_E;   // initial state (used when C.me_on)
    R meas = jac;
    R rinvE_prod = R(1);
    bool cut = false;
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        r[j] = y[3 * j];
        R st, ct, sp, cp;
        RMath<R>::sincos_(y[3 * j + 1], &st, &ct);
        RMath<R>::sincos_(y[3 * j + 2], &sp, &cp);   // angle phi - pi
        const R p = r[j] * C.inv_a;
        const R ps = p * st;
        const R sg = C.sig[j];
        px = fma(-sg * ps, cp, px);                    // cos(phi) = -cos(phi - pi)
        py = fma(-sg * ps, sp, py);
        pz = fma(sg * p, ct, pz);
        const R E2 = fma(p, p, C.m2[j]);
        const R rE = RMath<R>::rsqrt_(E2);
        const R E = E2 * rE;
        cut |= E < C.e_cut;
        bal.add(C.sgnE[j] * E);
        Esum += E;
        if (EXT && C.me_on) {
            const R iw = C.inw[j];
            Qx = fma(-iw * ps, cp, Qx);
            Qy = fma(-iw * ps, sp, Qy);
            Qz = fma(iw * p, ct, Qz);
            Ein = fma(iw, E, Ein);
        }
        meas *= r[j] * r[j] * st;
        rinvE_prod *= rE;
    }
    // conserved leg (Eq. (10), App. A)
    const R pc2 = fma(px, px, fma(py, py, pz * pz));
    const R Ec2 = pc2 + C.m2c;
    const R rEc = RMath<R>::rsqrt_(Ec2 > RMath<R>::kTiny ? Ec2 : R(1e-30));
    Ec = Ec2 * rEc;
    cut |= Ec < C.e_cut;
    bal.add(C.sgn_cons * Ec);
    const R dE = bal.value();
    qc = pc2 * (pc2 > RMath<R>::kTiny ? RMath<R>::rsqrt_(pc2) : R(0)) * C.a;
    R gauss;
    if (C.frac) {
        // sigma = w S / 2 with S = E_in + E_out: exponent
        // -2 dE^2 / (w S)^2, normalisation sigma_ref / sigma = 2 E_obs / S
        Esum += Ec;
        const R iS = RMath<R>::rcp_(Esum);
        const R x = dE * iS;
        gauss = RMath<R>::exp2_(C.gauss_k * x * x) * (R(2) * C.e_obs * iS);
    } else {
        gauss = RMath<R>::exp2_(C.gauss_k * dE * dE);
    }
    R w = meas * rinvE_prod * rEc * gauss;
    if (EXT && C.me_on) {
        // |M|^2 / coupling^2 = P(s), s of the initial state (the conserved
        // leg's momentum is (px, py, pz))
        const R cw = C.cons_inw;
        const R qx = fma(cw, px, Qx), qy = fma(cw, py, Qy), qz = fma(cw, pz, Qz);
        const R e = fma(cw, Ec, Ein);
        const R sv = fma(e, e, -fma(qx, qx, fma(qy, qy, qz * qz)));
        w *= fma(fma(fma(C.me[3], sv, C.me[2]), sv, C.me[1]), sv, C.me[0]);
    }
    return cut ? R(0) : w;
}

// Packed FP32x2 helpers (one instruction for both halves on sm_100+).
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// EBal for two samples, the TwoSum steps packed.
struct EBal2 {
    float2 s, c;
    __device__ __forceinline__ explicit EBal2(float x0) : s(make_float2(x0, x0)), c(make_float2(0.0f, 0.0f)) {}
    __device__ __forceinline__ void add(float2 x) {
        const float2 t = add2(s, x);
        const float2 xp = sub2(t, s);
        const float2 sp = sub2(t, xp);
        c = add2(c, add2(sub2(s, sp), sub2(x, xp)));
        s = t;
    }
    __device__ __forceinline__ float2 value() const { return add2(s, c); }
};

// kin_at for two samples at once (constant |M|^2), each FP32 operation
// packed over the pair; the special-function operations stay per sample.
template <int NLEG>
__device__ __forceinline__ float2 kin_pair(const SegConst<float, NLEG>& C, const float2* y, float2 jac, float2* r,
                                           float2& qc, float2& Ec) {
    constexpr int NI = NLEG - 2;
    float2 px = bc2(0.0f), py = bc2(0.0f), pz = bc2(C.pobs_sig);
    EBal2 bal(C.sgn_obs_E);
    float2 Esum = bc2(C.e_obs);
    float2 meas = jac, rinv = bc2(1.0f);
    float emin0 = 3.0e38f, emin1 = 3.0e38f;
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        r[j] = y[3 * j];
        float2 st, ct, sp, cp;
        __sincosf(y[3 * j + 1].x, &st.x, &ct.x);
        __sincosf(y[3 * j + 1].y, &st.y, &ct.y);
        __sincosf(y[3 * j + 2].x, &sp.x, &cp.x);      // angle phi - pi
        __sincosf(y[3 * j + 2].y, &sp.y, &cp.y);
        const float2 p = mul2(r[j], bc2(C.inv_a));
        const float2 ps = mul2(p, st);
        const float2 nps = mul2(ps, bc2(-C.sig[j]));   // cos(phi) = -cos(phi - pi)
        px = fma2(nps, cp, px);
        py = fma2(nps, sp, py);
        pz = fma2(mul2(p, bc2(C.sig[j])), ct, pz);
        const float2 E2 = fma2(p, p, bc2(C.m2[j]));
        const float2 rE = make_float2(rsqrt_ftz(E2.x), rsqrt_ftz(E2.y));
        const float2 E = mul2(E2, rE);
        emin0 = fminf(emin0, E.x);
        emin1 = fminf(emin1, E.y);
        bal.add(mul2(bc2(C.sgnE[j]), E));
        Esum = add2(Esum, E);
        meas = mul2(meas, mul2(mul2(r[j], r[j]), st));
        rinv = mul2(rinv, rE);
    }
    // conserved leg (Eq. (10), App. A)
    const float2 pc2 = fma2(px, px, fma2(py, py, mul2(pz, pz)));
    const float2 Ec2q = add2(pc2, bc2(C.m2c));
    const float2 rEc = make_float2(rsqrt_ftz(Ec2q.x > 1e-30f ? Ec2q.x : 1e-30f), rsqrt_ftz(Ec2q.y > 1e-30f ? Ec2q.y : 1e-30f));
    Ec = mul2(Ec2q, rEc);
    emin0 = fminf(emin0, Ec.x);
    emin1 = fminf(emin1, Ec.y);
    bal.add(mul2(bc2(C.sgn_cons), Ec));
    const float2 dE = bal.value();
    const float2 rpc = make_float2(pc2.x > 1e-30f ? rsqrt_ftz(pc2.x) : 0.0f, pc2.y > 1e-30f ? rsqrt_ftz(pc2.y) : 0.0f);
    qc = mul2(mul2(pc2, rpc), bc2(C.a));
    float2 gauss;
    if (C.frac) {
        // sigma = w S / 2 with S = E_in + E_out: exponent -2 dE^2 / (w S)^2,
        // normalisation sigma_ref / sigma = 2 E_obs / S
        Esum = add2(Esum, Ec);
        const float2 iS = make_float2(__fdividef(1.0f, Esum.x), __fdividef(1.0f, Esum.y));
        const float2 x = mul2(dE, iS);
        const float2 e = mul2(mul2(x, x), bc2(C.gauss_k));
        gauss = mul2(make_float2(ex2_ftz(e.x), ex2_ftz(e.y)), mul2(bc2(2.0f * C.e_obs), iS));
    } else {
        const float2 e = mul2(mul2(dE, dE), bc2(C.gauss_k));
        gauss = make_float2(ex2_ftz(e.x), ex2_ftz(e.y));
    }
    float2 w = mul2(mul2(meas, rinv), mul2(rEc, gauss));
    w.x = emin0 < C.e_cut ? 0.0f : w.x;
    w.y = emin1 < C.e_cut ? 0.0f : w.y;
    return w;
}

// Statistical factor of Eq. (5) of one sample: the observed leg's factor
// over the scale, times c_a + c_b f of every other leg, f from the spline
// (Sec. 3B) or, for the conserved leg outside the grid, the tails of
// Eq. (13).
template <typename R, int NLEG>
__device__ __forceinline__ R stat_at(const SegConst<R, NLEG>& C, const R* r, R qc, R Ec, const R* s_spline,
                                     const R* knots, const Geometry& g, R inv_step, R q0, R lq0_step, R qN,
                                     int ncoef) {
    constexpr int NI = NLEG - 2;
    constexpr bool F32 = RMath<R>::kF32;
    R stat = C.c0;
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        const SplineView<R> sv{s_spline + C.spc[j] * ncoef, knots};
        R f = spline_eval<R>(sv, r[j], g, inv_step, q0, lq0_step);
        f = C.fd[j] ? (f < R(1) ? f : R(1)) : f;
        stat *= fma(C.cb[j], f, C.ca[j]);
    }
    R fc;
    {
        const bool below = qc < q0, above = qc > qN;
        if constexpr (F32) {
            // spline for every lane, the tail only in warps where some lane
            // left the grid, then a select: the warp never diverges on the
            // conserved leg (the mask is the lanes present)
            const SplineView<R> sv{s_spline + C.sp_cons * ncoef, knots};
            fc = spline_eval<R>(sv, fminf(fmaxf(qc, q0), qN), g, inv_step, q0, lq0_step);
            if (__any_sync(__activemask(), below || above)) {
                const float x = below ? fmaf(C.tlo_b, Ec, C.tlo_a) : fmaf(C.thi_b, Ec, C.thi_a);
                const float ft = tail_f32(x, C.eta_c);
                fc = (below || above) ? ft : fc;
            }
        } else {
            if (!below && !above) {
                const SplineView<R> sv{s_spline + C.sp_cons * ncoef, knots};
                fc = spline_eval<R>(sv, qc, g, inv_step, q0, lq0_step);
            } else {
                const R x = below ? C.tlo_a + C.tlo_b * Ec : C.thi_a + C.thi_b * Ec;
                const R den = C.eta_c == R(1) ? RMath<R>::expm1_(x) : RMath<R>::exp_(x) - C.eta_c;
                fc = den > R(0) ? R(1) / den : R(0);
            }
        }
        fc = C.fd_c ? (fc < R(1) ? fc : R(1)) : fc;
    }
    return stat * fma(C.cbc, fc, C.cac);
}

// Weight of one sample (Eq. (12)): statistical factor times kinematic part.
// EXT: the instantiation also supports an s-dependent |M|^2 (see run_segment).
template <typename R, int NLEG, bool EXT>
__device__ __forceinline__ R weight_at(const SegConst<R, NLEG>& C, const R* y, R jac, const R* s_spline,
                                       const R* knots, const Geometry& g, R inv_step, R q0, R lq0_step, R qN,
                                       int ncoef) {
    R r[NLEG - 2], qc, Ec;
    const R kin = kin_at<R, NLEG, EXT>(C, y, jac, r, qc, Ec);
    return stat_at<R, NLEG>(C, r, qc, Ec, s_spline, knots, g, inv_step, q0, lq0_step, qN, ncoef) * kin;
}

// Per-segment constants of run_segment: the roles, signs, masses and
// statistical-factor coefficients of the legs, the Gaussian's exponent and
// the spline-index constants, rounded to R from values that the time-state,
// spline and prepare kernels computed in FP64 once per sweep (so that the
// threads here only select and convert: FP64 arithmetic runs at a small
// fraction of the FP32 rate).
template <typename R, int NLEG>
struct SegSetup {
    SegConst<R, NLEG> C;
    R inv_step, q0, lq0_step, qN;
};

template <typename R, int NLEG>
__device__ __forceinline__ void seg_setup(const EvalParams& P, const SideDesc& sd, const TaskDesc& td,
                                          const TaskConst& tc, SegSetup<R, NLEG>* out) {
    constexpr int NI = NLEG - 2;
    const Geometry& g = P.geo;
    SegConst<R, NLEG> C;
    const TimeState& ts = *P.ts;
    const int cons = sd.cons;
    const bool cons_in = (sd.in_mask >> cons) & 1;
    const R flip = cons_in ? R(-1) : R(1);     // p_cons = flip * sum_{k != c} s_k p_k
    const bool is_loss = td.term == 1;
    {
        const R s_obs = ((sd.in_mask >> sd.obs) & 1) ? R(1) : R(-1);
        C.pobs_sig = flip * s_obs * static_cast<R>(tc.p_obs);
        C.sgn_obs_E = s_obs * static_cast<R>(tc.E_obs);
    }
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        const int k = sd.integ[j];
        const bool kin = (sd.in_mask >> k) & 1;
        const bool own = (sd.own_mask >> k) & 1;
        const int sp = sd.leg_species[k];
        const double eta = P.sconst[sp].eta;
        C.sig[j] = flip * (kin ? R(1) : R(-1));
        C.sgnE[j] = kin ? R(1) : R(-1);
        const double m = ts.mass[sp];
        C.m2[j] = static_cast<R>(m * m);
        const bool enh = own != is_loss;
        C.ca[j] = enh ? R(1) : R(0);
        C.cb[j] = enh ? static_cast<R>(eta) : R(1);
        C.spc[j] = sp;
        C.fd[j] = P.sconst[sp].stat == BEST_FD;
    }
    {
        const int sp = sd.leg_species[cons];
        const bool own = (sd.own_mask >> cons) & 1;
        const double eta = P.sconst[sp].eta;
        const double m = ts.mass[sp];
        C.sgn_cons = cons_in ? R(1) : R(-1);
        C.m2c = static_cast<R>(m * m);
        const bool enh = own != is_loss;
        C.cac = enh ? R(1) : R(0);
        C.cbc = enh ? static_cast<R>(eta) : R(1);
        C.sp_cons = sp;
        C.eta_c = static_cast<R>(eta);
        C.fd_c = P.sconst[sp].stat == BEST_FD;
        C.tlo_a = static_cast<R>(P.sconst[sp].tail_lo_a);
        C.tlo_b = static_cast<R>(P.sconst[sp].tail_lo_b);
        C.thi_a = static_cast<R>(P.sconst[sp].tail_hi_a);
        C.thi_b = static_cast<R>(P.sconst[sp].tail_hi_b);
    }
    C.a = static_cast<R>(ts.a);
    C.inv_a = static_cast<R>(ts.inv_a);
    C.c0 = static_cast<R>(tc.c0);
    C.frac = tc.wfrac > 0.0;
    C.gauss_k = static_cast<R>(tc.gauss_k);
    C.e_obs = static_cast<R>(tc.E_obs);
    C.me_on = sd.me_on != 0;
    for (int k = 0; k < 4; ++k) C.me[k] = static_cast<R>(sd.me_coef[k]);
    {
        const bool obs_in = (sd.in_mask >> sd.obs) & 1;
        C.obs_in_p = obs_in ? static_cast<R>(tc.p_obs) : R(0);
        C.obs_in_E = obs_in ? static_cast<R>(tc.E_obs) : R(0);
        C.cons_inw = cons_in ? R(1) : R(0);
#pragma unroll
        for (int j = 0; j < NI; ++j) C.inw[j] = ((sd.in_mask >> sd.integ[j]) & 1) ? R(1) : R(0);
    }
    C.e_cut = static_cast<R>(g.e_cut);
    out->C = C;
    out->q0 = static_cast<R>(g.q_min);
    out->lq0_step = static_cast<R>(g.lq0_step);
    out->qN = static_cast<R>(g.q_max);
    out->inv_step = static_cast<R>(g.inv_step);
}

// The same for the FP32 kernel from the task's SegConst32 (rounded once per
// sweep by the prepare kernel): loads only.
template <int NLEG>
__device__ __forceinline__ void seg_setup32(const SegConst32& S, SegSetup<float, NLEG>* out) {
    constexpr int NI = NLEG - 2;
    SegConst<float, NLEG> C;
    C.pobs_sig = S.pobs_sig;
    C.sgn_obs_E = S.sgn_obs_E;
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        C.sig[j] = S.sig[j];
        C.sgnE[j] = S.sgnE[j];
        C.m2[j] = S.m2[j];
        C.ca[j] = S.ca[j];
        C.cb[j] = S.cb[j];
        C.spc[j] = S.spc[j];
        C.fd[j] = S.fd[j];
        C.inw[j] = S.inw[j];
    }
    C.sgn_cons = S.sgn_cons;
    C.m2c = S.m2c;
    C.cac = S.cac;
    C.cbc = S.cbc;
    C.sp_cons = S.sp_cons;
    C.eta_c = S.eta_c;
    C.fd_c = S.fd_c;
    C.tlo_a = S.tlo_a;
    C.tlo_b = S.tlo_b;
    C.thi_a = S.thi_a;
    C.thi_b = S.thi_b;
    C.a = S.a;
    C.inv_a = S.inv_a;
    C.c0 = S.c0;
    C.frac = S.frac != 0;
    C.gauss_k = S.gauss_k;
    C.e_obs = S.e_obs;
    C.me_on = S.me_on != 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) C.me[k] = S.me[k];
    C.obs_in_p = S.obs_in_p;
    C.obs_in_E = S.obs_in_E;
    C.cons_inw = S.cons_inw;
    C.e_cut = S.e_cut;
    out->C = C;
    out->q0 = S.q0;
    out->lq0_step = S.lq0_step;
    out->qN = S.qN;
    out->inv_step = S.inv_step;
}

// STRAT: the instantiation also handles stratified tasks and s-dependent
// matrix elements (kept apart so that the plain kernel's register allocation
// is not affected).
template <typename R, int NLEG, bool STRAT, int SPL>
__device__ __forceinline__ void run_segment(const EvalParams& P, const Segment& seg,
                                            const SideDesc& sd, const TaskDesc& td,
                                            const TaskConst& tc, R* s_spline,
                                            Real2<R>* s_map, R* s_hist, double* s_red, float* s_queue,
                                            int map_elems) {
    constexpr int NI = NLEG - 2;
    constexpr int D = 3 * NI;
    constexpr bool F32 = RMath<R>::kF32;
    using SS = StreamShape<D, F32>;
    constexpr int G = SS::kGroup;
    const Geometry& g = P.geo;
    const int nb = td.nbins;
    const int tid = threadIdx.x;

    // ---- map table of this task in shared memory ---------------------------
    if constexpr (F32) {
        // rounded to FP32 once per refinement (map32_kernel, refine_kernel)
        const float2* m32 = P.map32 + static_cast<int64_t>(seg.task) * map32_stride(g);
        for (int k = tid; k < D * nb; k += blockDim.x) {
            const float2 m = m32[k];
            Real2<R> v;
            v.y0 = m.x;
            v.dy = m.y;
            s_map[k] = v;
        }
    } else {
        const double* edges = P.edges + static_cast<int64_t>(seg.task) * g.map_stride;
        for (int k = tid; k < D * nb; k += blockDim.x) {
            const int d = k / nb;
            const int b = k - d * nb;
            const double e0 = edges[d * (nb + 1) + b];
            const double e1 = edges[d * (nb + 1) + b + 1];
            double lo, sc;
            switch (d % 3) {
                case 0: lo = g.q_min; sc = g.q_max - g.q_min; break;   // r (comoving)
                case 1: lo = 0.0; sc = kPi; break;                     // theta
                default: lo = -kPi; sc = kTwoPi; break;                // phi - pi
            }
            Real2<R> v;
            v.y0 = static_cast<R>(lo + sc * e0);
            v.dy = static_cast<R>(sc * (e1 - e0));
            s_map[k] = v;
        }
    }
    // per-warp histograms: atomics from different warps never share an
    // address, and the warps are summed in a fixed order at the end, so the
    // training data do not depend on warp scheduling
    const int nwarps = blockDim.x >> 5;
    for (int k = tid; k < nwarps * map_elems; k += blockDim.x) s_hist[k] = R(0);
    R* w_hist = s_hist + (tid >> 5) * map_elems;

    // ---- per-segment constants ----------------------------------------------
    SegSetup<R, NLEG> setup;
    if constexpr (F32) seg_setup32<NLEG>(P.tconst32[seg.task], &setup);
    else seg_setup<R, NLEG>(P, sd, td, tc, &setup);
    const R nbR = static_cast<R>(nb);
    const int ncoef = 4 * (g.n_grid - 1);
    const R* knots = s_spline + g.n_species * ncoef;
    __syncthreads();
    const SegConst<R, NLEG>& C = setup.C;
    const R q0 = setup.q0, lq0_step = setup.lq0_step, qN = setup.qN, inv_step = setup.inv_step;
    const uint32_t call = P.ts->call;

    // ---- samples ------------------------------------------------------------
    Acc<R> acc_w, acc_w2;
    const int64_t N = td.neval;
    const uint32_t task = td.gid;                 // the stream is keyed by the global task id
    const int32_t g1 = static_cast<int32_t>(seg.g1);
    if (!STRAT || td.strat_H == 0) {
        if constexpr (F32) {
            // Samples with a non-zero kinematic part (close enough to the
            // energy shell for the Gaussian not to underflow) are queued per
            // warp in shared memory; the statistical factor, the sums and the
            // training data are evaluated 32 queued samples at a time, so
            // that those instructions run on full warps of live samples.  The
            // warp runs the loop in step (a lane past the segment's end
            // computes an invalid sample), so its votes see all 32 lanes.
            constexpr int QW = queue_words(NLEG);
            constexpr int NB = (D + 3) / 4;               // words of packed increments
            float* q = s_queue + (tid >> 5) * (kQueueSlots * QW);
            const int lane = tid & 31;
            const uint32_t lanes_below = (1u << lane) - 1u;
            int qn = 0;                                   // queued samples (warp-uniform)
            auto drain = [&](int slot) {
                R r[NI];
#pragma unroll
                for (int j = 0; j < NI; ++j) r[j] = q[(1 + j) * kQueueSlots + slot];
                const R qc = q[(1 + NI) * kQueueSlots + slot];
                const R Ec = q[(2 + NI) * kQueueSlots + slot];
                const R w = stat_at<R, NLEG>(C, r, qc, Ec, s_spline, knots, g, inv_step, q0, lq0_step, qN, ncoef) *
                            q[slot];
                const R w2 = w * w;
                acc_w.add(w);
                acc_w2.add(w2);
                if (w2 != R(0)) {
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        const uint32_t pb = __float_as_uint(q[(3 + NI + k) * kQueueSlots + slot]);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * k + e < D)
                                atomicAdd(&w_hist[(4 * k + e) * nb + ((pb >> (8 * e)) & 0xFFu)], w2);
                    }
                }
            };
            // 32-bit indices: neval * dim <= 2^33 keeps every group index and sample count below 2^32
            const uint32_t g1u = static_cast<uint32_t>(seg.g1), Nu = static_cast<uint32_t>(N);
            // appends one sample per lane (those with keep) to the warp's queue
            // and, once 32 are queued, evaluates them
            auto push = [&](bool keep, float kin, const float* r, float qc, float Ec, const uint32_t* pb) {
                const uint32_t vote = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int slot = qn + __popc(vote & lanes_below);     // < 2 * 32
                    q[slot] = kin;
#pragma unroll
                    for (int j = 0; j < NI; ++j) q[(1 + j) * kQueueSlots + slot] = r[j];
                    q[(1 + NI) * kQueueSlots + slot] = qc;
                    q[(2 + NI) * kQueueSlots + slot] = Ec;
#pragma unroll
                    for (int k = 0; k < NB; ++k) q[(3 + NI + k) * kQueueSlots + slot] = __uint_as_float(pb[k]);
                }
                qn += __popc(vote);
                if (qn >= 32) {
                    __syncwarp();
                    drain(lane);
                    __syncwarp();
                    if (lane < qn - 32) {
#pragma unroll
                        for (int f = 0; f < QW; ++f) q[f * kQueueSlots + lane] = q[f * kQueueSlots + 32 + lane];
                    }
                    __syncwarp();
                    qn -= 32;
                }
            };
            if constexpr (!STRAT && SPL == 2) {
                // Two samples per step in packed FP32x2 arithmetic: the two
                // samples of a group (G even) or of two consecutive groups
                // (G = 1, a lane then takes groups 2k and 2k + 1).  The
                // packed path holds more registers live, so whether it pays
                // depends on the register budget: the autotuner decides.
                constexpr int U = G % 2 == 0 ? 1 : 2;       // groups per lane per trip
                constexpr int S = G * U;                    // samples per lane per trip (even)
                for (uint32_t gb = static_cast<uint32_t>(seg.g0) + (tid & ~31) * U; gb < g1u;
                     gb += blockDim.x * U) {
                    const uint32_t grp0 = gb + lane * U;
                    uint32_t uw[SS::kUniforms * U];
#pragma unroll
                    for (int u = 0; u < U; ++u) group_words<D>(uw + u * SS::kUniforms, grp0 + u, P.itn, call, task, P.rk);
#pragma unroll
                    for (int sp = 0; sp < S; sp += 2) {
                        bool valid[2];
                        float2 y[D];
                        float2 jac = make_float2(1.0f, 1.0f);
                        uint32_t pb[2][NB];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t grp = grp0 + (sp + h) / G;
                            valid[h] = grp < g1u && grp * G + (sp + h) % G < Nu;
#pragma unroll
                            for (int k = 0; k < NB; ++k) pb[h][k] = 0u;
                        }
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            // x nb = word nb / 2^32: the increment is the high and the
                            // fraction the low half of one 32 x 32 -> 64-bit product
                            Real2<float> e[2];
                            float fr[2];
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const uint64_t m = static_cast<uint64_t>(uw[(sp + h) * D + d]) * static_cast<uint32_t>(nb);
                                const uint32_t b = static_cast<uint32_t>(m >> 32);
                                fr[h] = static_cast<float>(static_cast<uint32_t>(m));
                                e[h] = s_map[d * nb + b];
                                pb[h][d >> 2] |= b << (8 * (d & 3));
                            }
                            const float2 dy = make_float2(e[0].dy, e[1].dy);
                            const float2 frac = __fmul2_rn(make_float2(fr[0], fr[1]),
                                                           make_float2(2.3283064365386963e-10f, 2.3283064365386963e-10f));
                            y[d] = __ffma2_rn(dy, frac, make_float2(e[0].y0, e[1].y0));
                            jac = __fmul2_rn(jac, dy);
                        }
                        float2 r2[NI], qc2, Ec2;
                        const float2 kin = kin_pair<NLEG>(C, y, jac, r2, qc2, Ec2);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float r[NI];
#pragma unroll
                            for (int j = 0; j < NI; ++j) r[j] = h ? r2[j].y : r2[j].x;
                            const float kh = h ? kin.y : kin.x;
                            push(valid[h] && kh != 0.0f, kh, r, h ? qc2.y : qc2.x, h ? Ec2.y : Ec2.x, pb[h]);
                        }
                    }
                }
            } else {
                for (uint32_t gb = static_cast<uint32_t>(seg.g0) + (tid & ~31); gb < g1u; gb += blockDim.x) {
                    const uint32_t grp = gb + lane;
                    uint32_t uw[SS::kUniforms];
                    group_words<D>(uw, grp, P.itn, call, task, P.rk);
#pragma unroll
                    for (int sgi = 0; sgi < G; ++sgi) {
                        // samples past the budget (only in a task's last group) and
                        // past the segment are computed and not queued
                        const bool valid = grp < g1u && grp * G + sgi < Nu;
                        R y[D];
                        uint32_t pb[NB];
#pragma unroll
                        for (int k = 0; k < NB; ++k) pb[k] = 0u;
                        R jac = R(1);
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const uint64_t m = static_cast<uint64_t>(uw[sgi * D + d]) * static_cast<uint32_t>(nb);
                            const uint32_t b = static_cast<uint32_t>(m >> 32);
                            const float fr = static_cast<float>(static_cast<uint32_t>(m)) * 2.3283064365386963e-10f;   // 2^-32
                            const Real2<R> e = s_map[d * nb + b];
                            y[d] = fma(e.dy, fr, e.y0);
                            jac *= e.dy;
                            pb[d >> 2] |= b << (8 * (d & 3));
                        }
                        R r[NI], qc, Ec;
                        const R kin = kin_at<R, NLEG, STRAT>(C, y, jac, r, qc, Ec);
                        push(valid && kin != R(0), kin, r, qc, Ec, pb);
                    }
                }
            }
            __syncwarp();
            if (lane < qn) drain(lane);
        } else {
            for (int32_t grp = static_cast<int32_t>(seg.g0) + tid; grp < g1; grp += blockDim.x) {
                R u[SS::kUniforms];                       // 52-bit uniforms
                group_uniforms<D, F32, R>(u, grp, P.itn, call, task, P.rk);
#pragma unroll
                for (int sgi = 0; sgi < G; ++sgi) {
                    // samples past the budget (only in a task's last group) are
                    // computed and given weight 0: no branch inside the group
                    const bool valid = static_cast<uint32_t>(grp) * G + sgi < static_cast<uint32_t>(N);   // N <= 2^31
                    // VEGAS map and scaling to (r, theta, phi - pi)
                    R y[D];
                    int bin[D];
                    R jac = R(1);
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const R t = u[sgi * D + d] * nbR;
                        int b = static_cast<int>(t);
                        b = b < nb - 1 ? b : nb - 1;
                        const R fr = t - static_cast<R>(b);
                        const Real2<R> e = s_map[d * nb + b];
                        y[d] = fma(e.dy, fr, e.y0);
                        jac *= e.dy;
                        bin[d] = b;
                    }
                    R w = weight_at<R, NLEG, STRAT>(C, y, jac, s_spline, knots, g, inv_step, q0, lq0_step, qN, ncoef);
                    w = valid ? w : R(0);
                    const R w2 = w * w;
                    acc_w.add(w);
                    acc_w2.add(w2);
                    // training data: a zero w^2 (far from the energy shell, or
                    // underflow) adds nothing, so such lanes skip the atomics
                    if (w2 != R(0)) {
#pragma unroll
                        for (int d = 0; d < D; ++d) atomicAdd(&w_hist[d * nb + bin[d]], w2);
                    }
                }
            }
        }
    }
    else if constexpr (STRAT) {
        // Adaptive stratified sampling: items of kItem samples, all in
        // hypercube h = item_h[item] with strata (i_0 .. i_{D-1});
        // x_d = (i_d + u_d) / M.  The item's (sum w, sum w^2) go to its own
        // record (summed per hypercube in a fixed order afterwards); the
        // training data weigh w^2 by 1 / m_h.
        constexpr int GPI = kItem / G;                  // groups per item
        const int M = td.strat_M;
        const R invM = R(1) / static_cast<R>(M);
        const uint32_t* ih = P.item_h + td.strat_off_item;
        const int32_t* sm = P.strat_m + td.strat_off_h;
        double2* rec = reinterpret_cast<double2*>(P.item_rec) + td.strat_off_item;
        const int32_t it0 = static_cast<int32_t>(seg.g0) / GPI, it1 = g1 / GPI;
        if constexpr (F32) {
            // The per-warp queue of the plain loop: a warp takes KI items per
            // lane (a round), queues the samples with a non-zero kinematic
            // part together with their item's slot in the round and 1 / m_h,
            // and evaluates them 32 at a time; w and w^2 go to the slot's
            // shared-memory sums.  At the round's end the queue is drained and
            // the round's item records are written.
            constexpr int QW = queue_words(NLEG);
            constexpr int KI = kStratItemsPerLane;
            constexpr int NB = (D + 3) / 4;
            float* q = s_queue + (tid >> 5) * strat_queue_floats(NLEG);
            float* isum = q + kQueueSlots * (QW + 2);          // [2][32 KI]: sum w, sum w^2 per item slot
            const int lane = tid & 31;
            const uint32_t lanes_below = (1u << lane) - 1u;
            int qn = 0;                                       // queued samples (warp-uniform)
            auto drain = [&](int slot) {
                R r[NI];
#pragma unroll
                for (int j = 0; j < NI; ++j) r[j] = q[(1 + j) * kQueueSlots + slot];
                const R qc = q[(1 + NI) * kQueueSlots + slot];
                const R Ec = q[(2 + NI) * kQueueSlots + slot];
                const R w = stat_at<R, NLEG>(C, r, qc, Ec, s_spline, knots, g, inv_step, q0, lq0_step, qN, ncoef) *
                            q[slot];
                const R w2 = w * w;
                acc_w.add(w);
                acc_w2.add(w2);
                const uint32_t is = __float_as_uint(q[QW * kQueueSlots + slot]);
                atomicAdd(&isum[is], w);
                atomicAdd(&isum[32 * KI + is], w2);
                if (w2 != R(0)) {
                    const R w2m = w2 * q[(QW + 1) * kQueueSlots + slot];
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        const uint32_t pb = __float_as_uint(q[(3 + NI + k) * kQueueSlots + slot]);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * k + e < D)
                                atomicAdd(&w_hist[(4 * k + e) * nb + ((pb >> (8 * e)) & 0xFFu)], w2m);
                    }
                }
            };
            auto push = [&](bool keep, float kin, const float* r, float qc, float Ec, const uint32_t* pb, uint32_t is,
                            float inv_m) {
                const uint32_t vote = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int slot = qn + __popc(vote & lanes_below);     // < 2 * 32
                    q[slot] = kin;
#pragma unroll
                    for (int j = 0; j < NI; ++j) q[(1 + j) * kQueueSlots + slot] = r[j];
                    q[(1 + NI) * kQueueSlots + slot] = qc;
                    q[(2 + NI) * kQueueSlots + slot] = Ec;
#pragma unroll
                    for (int k = 0; k < NB; ++k) q[(3 + NI + k) * kQueueSlots + slot] = __uint_as_float(pb[k]);
                    q[QW * kQueueSlots + slot] = __uint_as_float(is);
                    q[(QW + 1) * kQueueSlots + slot] = inv_m;
                }
                qn += __popc(vote);
                if (qn >= 32) {
                    __syncwarp();
                    drain(lane);
                    __syncwarp();
                    if (lane < qn - 32) {
#pragma unroll
                        for (int f = 0; f < QW + 2; ++f) q[f * kQueueSlots + lane] = q[f * kQueueSlots + 32 + lane];
                    }
                    __syncwarp();
                    qn -= 32;
                }
            };
            // the warp runs the rounds in step (a lane past the segment's last
            // item computes samples that are not queued), so its votes see all
            // 32 lanes
            const int32_t stride = static_cast<int32_t>(blockDim.x) * KI;
            for (int32_t ib = it0 + (tid & ~31) * KI; ib < it1; ib += stride) {
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    isum[k * 32 + lane] = 0.0f;
                    isum[32 * KI + k * 32 + lane] = 0.0f;
                }
                __syncwarp();
#pragma unroll 1
                for (int k = 0; k < KI; ++k) {
                    const int32_t item = ib + k * 32 + lane;
                    const bool ivalid = item < it1;
                    const uint32_t h = ivalid ? ih[item] : 0u;
                    const R inv_m = R(1) / static_cast<R>(sm[h]);
                    R xi[D];                                 // i_d as R
                    {
                        uint32_t r = h;
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const uint32_t qq = r / static_cast<uint32_t>(M);
                            xi[d] = static_cast<R>(r - qq * static_cast<uint32_t>(M));
                            r = qq;
                        }
                    }
#pragma unroll 1
                    for (int gi = 0; gi < GPI; ++gi) {
                        const int32_t grp = item * GPI + gi;
                        uint32_t uw[SS::kUniforms];
                        group_words<D>(uw, grp, P.itn, call, task, P.rk);
#pragma unroll
                        for (int sgi = 0; sgi < G; ++sgi) {
                            R y[D];
                            uint32_t pb[NB];
#pragma unroll
                            for (int k2 = 0; k2 < NB; ++k2) pb[k2] = 0u;
                            R jac = R(1);
#pragma unroll
                            for (int d = 0; d < D; ++d) {
                                const float uf = static_cast<float>(uw[sgi * D + d]) * 2.3283064365386963e-10f;   // word 2^-32
                                const R x = fmaf(uf, invM, xi[d] * invM);
                                const R t = x * nbR;
                                int b = static_cast<int>(t);
                                b = b < nb - 1 ? b : nb - 1;
                                const R fr = t - static_cast<R>(b);
                                const Real2<R> e = s_map[d * nb + b];
                                y[d] = fma(e.dy, fr, e.y0);
                                jac *= e.dy;
                                pb[d >> 2] |= static_cast<uint32_t>(b) << (8 * (d & 3));
                            }
                            R r[NI], qc, Ec;
                            const R kin = kin_at<R, NLEG, STRAT>(C, y, jac, r, qc, Ec);
                            push(ivalid && kin != R(0), kin, r, qc, Ec, pb, static_cast<uint32_t>(k * 32 + lane), inv_m);
                        }
                    }
                }
                // the round's samples are all evaluated: its item sums are complete
                __syncwarp();
                if (lane < qn) drain(lane);
                qn = 0;
                __syncwarp();
#pragma unroll
                for (int k = 0; k < KI; ++k) {
                    const int32_t item = ib + k * 32 + lane;
                    if (item < it1)
                        rec[item] = make_double2(static_cast<double>(isum[k * 32 + lane]),
                                                 static_cast<double>(isum[32 * KI + k * 32 + lane]));
                }
                __syncwarp();
            }
        } else {
            // FP64: one thread per item, the item's sums in its registers
            for (int32_t item = it0 + tid; item < it1; item += blockDim.x) {
                const uint32_t h = ih[item];
                const R inv_m = R(1) / static_cast<R>(sm[h]);
                R xi[D];                                     // i_d as R
                {
                    uint32_t r = h;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const uint32_t qq = r / static_cast<uint32_t>(M);
                        xi[d] = static_cast<R>(r - qq * static_cast<uint32_t>(M));
                        r = qq;
                    }
                }
                R s1 = R(0), s2 = R(0);
#pragma unroll 1
                for (int gi = 0; gi < GPI; ++gi) {
                    const int32_t grp = item * GPI + gi;
                    R u[SS::kUniforms];
                    group_uniforms<D, F32, R>(u, grp, P.itn, call, task, P.rk);
#pragma unroll
                    for (int sgi = 0; sgi < G; ++sgi) {
                        R y[D];
                        int bin[D];
                        R jac = R(1);
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const R x = (xi[d] + u[sgi * D + d]) / static_cast<R>(M);
                            const R t = x * nbR;
                            int b = static_cast<int>(t);
                            b = b < nb - 1 ? b : nb - 1;
                            const R fr = t - static_cast<R>(b);
                            const Real2<R> e = s_map[d * nb + b];
                            y[d] = fma(e.dy, fr, e.y0);
                            jac *= e.dy;
                            bin[d] = b;
                        }
                        const R w = weight_at<R, NLEG, STRAT>(C, y, jac, s_spline, knots, g, inv_step, q0, lq0_step,
                                                              qN, ncoef);
                        const R w2 = w * w;
                        s1 += w;
                        s2 += w2;
                        acc_w.add(w);
                        acc_w2.add(w2);
                        if (w2 != R(0)) {
                            const R w2m = w2 * inv_m;
#pragma unroll
                            for (int d = 0; d < D; ++d) atomicAdd(&w_hist[d * nb + bin[d]], w2m);
                        }
                    }
                }
                rec[item] = make_double2(static_cast<double>(s1), static_cast<double>(s2));
            }
        }
    }

    // ---- segment reduction into its partial record (FP64) -------------------
    double vw = acc_w.value(), vw2 = acc_w2.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vw += __shfl_xor_sync(0xffffffffu, vw, o);
        vw2 += __shfl_xor_sync(0xffffffffu, vw2, o);
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        s_red[2 * warp] = vw;
        s_red[2 * warp + 1] = vw2;
    }
    __syncthreads();
    double* part = P.partials + seg.part;
    if (tid == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
            a0 += s_red[2 * k];
            a1 += s_red[2 * k + 1];
        }
        part[0] = a0;
        part[1] = a1;
    }
    for (int k = tid; k < D * nb; k += blockDim.x) {
        // the per-warp histograms summed in their own precision (FP32 for
        // the FP32 kernel: one conversion per entry instead of one per warp)
        R v = R(0);
        for (int w = 0; w < nwarps; ++w) v += s_hist[w * map_elems + k];
        part[2 + k] = static_cast<double>(v);
    }
    __syncthreads();
}

// MB: CTAs per SM the kernel is register-limited to (__launch_bounds__);
// THREADS: threads per CTA; SPL: samples a lane evaluates per step of the
// FP32 loop (1, or 2 in packed FP32x2 arithmetic).  Several combinations are
// instantiated and the autotuner picks one at run time.
template <typename R, int NMAX, int MB, bool STRAT = false, int THREADS = kThreads, int SPL = 1>
__global__ void __launch_bounds__(THREADS, MB)
eval_kernel(EvalParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* s_spline = reinterpret_cast<R*>(smem_raw);
    const int nsp = P.smem_spline_elems;
    Real2<R>* s_map = reinterpret_cast<Real2<R>*>(s_spline + ((nsp + 3) & ~3));
    // map table and per-warp histograms of kDims x nbins_max entries: the
    // largest process the library supports, or, in the extended
    // instantiations, the largest process of their NMAX (the stratified
    // queue's item sums need the room).  A compile-time constant: read as a
    // kernel parameter, the plain 2 -> 2 kernel measured 1.8% slower.
    constexpr int kDims = STRAT ? 3 * (NMAX - 2) : kMaxDim;
    const int map_elems = kDims * P.geo.nbins_max;
    R* s_hist = reinterpret_cast<R*>(s_map + map_elems);      // [warps][map_elems]
    double* s_red = reinterpret_cast<double*>(s_hist + (((THREADS / 32) * map_elems + 3) & ~3));
    float* s_queue = reinterpret_cast<float*>(s_red + 2 * 32);   // FP32: [warps][queue_words][kQueueSlots]

    // spline tables of all species, once per CTA
    {
        const R* gc = static_cast<const R*>(P.coef);
        const int ncoef = 4 * (P.geo.n_grid - 1) * P.geo.n_species;
        for (int k = threadIdx.x; k < ncoef; k += blockDim.x) s_spline[k] = gc[k];
        const R* gk = static_cast<const R*>(P.knots);
        for (int k = threadIdx.x; k < P.geo.n_grid; k += blockDim.x) s_spline[ncoef + k] = gk[k];
    }
    // chunks of the partition: taken from the counter (dynamic), or chunk b
    // by CTA b; every segment writes its own partial record, so the results
    // do not depend on which CTA ran it
    __shared__ int s_chunk;
    for (int c = P.chunk_counter ? -1 : static_cast<int>(blockIdx.x);;) {
        if (P.chunk_counter) {
            __syncthreads();
            if (threadIdx.x == 0) s_chunk = atomicAdd(P.chunk_counter, 1);
            __syncthreads();
            c = s_chunk;
        }
        if (c >= P.n_chunks) break;
        const int s0 = P.cta_seg[c], s1 = P.cta_seg[c + 1];
        for (int si = s0; si < s1; ++si) {
            const Segment seg = P.segs[si];
            const TaskDesc td = P.tasks[seg.task];
            const SideDesc& sd = P.sides[td.si];
            const TaskConst tc = P.tconst[seg.task];
            __syncthreads();
            switch (sd.n) {
                case 3: if constexpr (NMAX >= 3) run_segment<R, 3, STRAT, SPL>(P, seg, sd, td, tc, s_spline, s_map, s_hist, s_red, s_queue, map_elems); break;
                case 4: if constexpr (NMAX >= 4) run_segment<R, 4, STRAT, SPL>(P, seg, sd, td, tc, s_spline, s_map, s_hist, s_red, s_queue, map_elems); break;
                case 5: if constexpr (NMAX >= 5) run_segment<R, 5, STRAT, SPL>(P, seg, sd, td, tc, s_spline, s_map, s_hist, s_red, s_queue, map_elems); break;
                case 6: if constexpr (NMAX >= 6) run_segment<R, 6, STRAT, SPL>(P, seg, sd, td, tc, s_spline, s_map, s_hist, s_red, s_queue, map_elems); break;
                default: break;
            }
        }
        if (!P.chunk_counter) break;
    }
}

}  // namespace best
