// Adjoint sample kernel: vector-Jacobian products of the fixed-sample
// collision integral C~ (one VEGAS iteration per task on the current maps,
// Philox iteration index kVjpIteration) with respect to the grid values f_j,
// the masses and the couplings, by recomputing every sample (nothing is
// stored).  Included by vjp.cu.
//
// Per sample, with w_n the normalised weight of the sample kernel,
//   w_n = c0 * prod_k fac_k * base,  fac_k = ca_k + cb_k f_k,
//   base = prod r^2 sin(theta) / prod E_k (non-observed legs) * G(dE) * J:
//   d w_n / d f_k      = cb_k * c0 * base * prod_{l != k} fac_l  (0 where f is clamped)
//   d w_n / d f_obs    = w_n / c0 * (d obs_factor / d f_obs) / scale
//   d w_n / d E_k      = w_n * (-1/E_k - dE s_k / sigma^2)      (1/E_k and the Gaussian)
//   d E_k / d m        = m / E_k
// f_k from the spline scatters d w_n / d f_k * (1, t, t^2, t^3) into the
// coefficient gradients of its interval; f_k from an Eq. (13) tail,
// f = 1/(exp(z) - eta), z = a + b E, contributes through dz: d f / d z =
// -f (1 + eta f) to (a, b) and, via E_cons, to the mass.
#pragma once

#include "eval_impl.cuh"

namespace best {

constexpr uint32_t kVjpIteration = 0xFFFF;


template <typename R>
struct Hit {
    R f;        // value (clamped)
    R d;        // 1 where f follows the polynomial, 0 where it was clamped
    int j;      // interval
    R t;        // q - q_j
};

template <typename R>
__device__ __forceinline__ Hit<R> spline_hit(const SplineView<R>& sv, R q, const Geometry& g, R inv_step, R q0,
                                             R lq0_step, bool fd) {
    int j;
    if (g.log_spaced) {
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
    Hit<R> h;
    h.j = j;
    h.t = t;
    h.d = R(1);
    if (!(f > R(0))) { f = R(0); h.d = R(0); }
    if (fd && f > R(1)) { f = R(1); h.d = R(0); }
    h.f = f;
    return h;
}

// JVP = false: adjoint (VJP) accumulation; true: forward tangent dC~ = J u,
// with the tangent spline table of u in s_dsp (same layout as s_spline's
// coefficients) and the tail tangents (da, db per end) in V.dtail.
// ME: the instantiation supports an s-dependent |M|^2 (kept apart so that the
// plain instantiations' register allocation is not affected).
template <typename R, int NLEG, bool JVP, bool ME>
__device__ __forceinline__ void vjp_segment(const VjpParams& V, const Segment& seg, const SideDesc& sd,
                                            const TaskDesc& td, const TaskConst& tc, R* s_spline,
                                            Real2<R>* s_map, double* s_gc, double* s_red, R* s_dsp,
                                            float* s_queue) {
    const EvalParams& P = V.E;
    constexpr int NI = NLEG - 2;
    constexpr int D = 3 * NI;
    constexpr bool F32 = RMath<R>::kF32;
    using SS = StreamShape<D, F32>;
    constexpr int G = SS::kGroup;
    const Geometry& g = P.geo;
    const int nb = td.nbins;
    const int tid = threadIdx.x;

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

    // per-segment constants (as in the sample kernel; the FP32 kernel loads
    // them from the task's SegConst32, rounded once per sweep)
    const TimeState& ts = *P.ts;
    const SegConst32* S = F32 ? P.tconst32 + seg.task : nullptr;
    const int cons = sd.cons;
    const bool cons_in = (sd.in_mask >> cons) & 1;
    const R flip = cons_in ? R(-1) : R(1);
    const bool is_loss = td.term == 1;
    const R s_obs = ((sd.in_mask >> sd.obs) & 1) ? R(1) : R(-1);
    const R pobs_sig = F32 ? R(S->pobs_sig) : flip * s_obs * static_cast<R>(tc.p_obs);
    const R sgn_obs_E = F32 ? R(S->sgn_obs_E) : s_obs * static_cast<R>(tc.E_obs);
    R sig[NI], sgnE[NI], m2[NI], ca[NI], cb[NI], mass[NI];
    int spc[NI], fdj[NI];
#pragma unroll
    for (int j = 0; j < NI; ++j) {
        if constexpr (F32) {
            sig[j] = S->sig[j];
            sgnE[j] = S->sgnE[j];
            mass[j] = S->mass[j];
            m2[j] = S->m2[j];
            ca[j] = S->ca[j];
            cb[j] = S->cb[j];
            spc[j] = S->spc[j];
            fdj[j] = S->fd[j];
        } else {
            const int k = sd.integ[j];
            const bool kin = (sd.in_mask >> k) & 1;
            const bool own = (sd.own_mask >> k) & 1;
            const int sp = sd.leg_species[k];
            const double eta = P.sconst[sp].eta;
            sig[j] = flip * (kin ? R(1) : R(-1));
            sgnE[j] = kin ? R(1) : R(-1);
            const double m = ts.mass[sp];
            mass[j] = static_cast<R>(m);
            m2[j] = static_cast<R>(m * m);
            const bool enh = own != is_loss;
            ca[j] = enh ? R(1) : R(0);
            cb[j] = enh ? static_cast<R>(eta) : R(1);
            spc[j] = sp;
            fdj[j] = P.sconst[sp].stat == BEST_FD;
        }
    }
    const int spcn = sd.leg_species[cons];
    const R eta_c = F32 ? R(S->eta_c) : static_cast<R>(P.sconst[spcn].eta);
    const bool fd_c = F32 ? S->fd_c != 0 : P.sconst[spcn].stat == BEST_FD;
    const R sgn_cons = cons_in ? R(1) : R(-1);
    const R mass_c = F32 ? R(S->mass_c) : static_cast<R>(ts.mass[spcn]);
    const R m2c = mass_c * mass_c;
    const bool own_c = (sd.own_mask >> cons) & 1;
    const bool enh_c = own_c != is_loss;
    const R cac = enh_c ? R(1) : R(0);
    const R cbc = enh_c ? eta_c : R(1);
    const R tlo_a = F32 ? R(S->tlo_a) : static_cast<R>(P.sconst[spcn].tail_lo_a);
    const R tlo_b = F32 ? R(S->tlo_b) : static_cast<R>(P.sconst[spcn].tail_lo_b);
    const R thi_a = F32 ? R(S->thi_a) : static_cast<R>(P.sconst[spcn].tail_hi_a);
    const R thi_b = F32 ? R(S->thi_b) : static_cast<R>(P.sconst[spcn].tail_hi_b);
    // (the FP64 quotients below come from the time-state and prepare kernels,
    // once per sweep: FP64 division runs at a small fraction of the FP32 rate)
    const R a = F32 ? R(S->a) : static_cast<R>(ts.a);
    const R inv_a = F32 ? R(S->inv_a) : static_cast<R>(ts.inv_a);
    const bool obs_cut = F32 ? S->obs_cut != 0 : tc.E_obs < g.e_cut;   // every sample of the task is cut
    const R c0 = F32 ? R(S->c0) : static_cast<R>(tc.c0);
    // Gaussian of Eq. (11); fractional width (App. C): sigma = w S / 2 per
    // sample, S = E_in + E_out, with sigma_ref = w E_obs inside K
    const bool frac = tc.wfrac > 0.0;
    const R gauss_k = F32 ? R(S->gauss_k) : static_cast<R>(tc.gauss_k);
    const R inv_sig2_abs = F32 ? R(S->inv_sig2_abs) : static_cast<R>(tc.inv_sig2_abs);
    const R four_over_w2 = F32 ? R(S->four_over_w2) : static_cast<R>(tc.four_over_w2);
    const R e_obs = F32 ? R(S->e_obs) : static_cast<R>(tc.E_obs);
    // |M|^2 / coupling^2 = P(s), s of the initial state
    const bool me_on = ME && sd.me_on != 0;
    R mec[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) mec[k] = F32 ? R(S->me[k]) : static_cast<R>(sd.me_coef[k]);
    const bool obs_in = (sd.in_mask >> sd.obs) & 1;
    const R obs_in_p = F32 ? R(S->obs_in_p) : (obs_in ? static_cast<R>(tc.p_obs) : R(0));
    const R obs_in_E = F32 ? R(S->obs_in_E) : (obs_in ? static_cast<R>(tc.E_obs) : R(0));
    const R obs_inw = obs_in ? R(1) : R(0);
    const R cons_inw = cons_in ? R(1) : R(0);
    R inw[NI];
#pragma unroll
    for (int j = 0; j < NI; ++j) inw[j] = ((sd.in_mask >> sd.integ[j]) & 1) ? R(1) : R(0);
    const R e_cut = F32 ? R(S->e_cut) : static_cast<R>(g.e_cut);
    const R inv_Eobs = F32 ? R(S->inv_E_obs) : static_cast<R>(tc.inv_E_obs);
    const R U = static_cast<R>(V.task_u[seg.task]);     // VJP: adjoint seed; JVP: obs tangent factor
    R dta_lo = R(0), dtb_lo = R(0), dta_hi = R(0), dtb_hi = R(0);
    if constexpr (JVP) {
        dta_lo = static_cast<R>(V.dtail[spcn * 4 + 0]);
        dtb_lo = static_cast<R>(V.dtail[spcn * 4 + 1]);
        dta_hi = static_cast<R>(V.dtail[spcn * 4 + 2]);
        dtb_hi = static_cast<R>(V.dtail[spcn * 4 + 3]);
    }
    const R nbR = static_cast<R>(nb);
    const R q0 = F32 ? R(S->q0) : static_cast<R>(g.q_min), qN = F32 ? R(S->qN) : static_cast<R>(g.q_max);
    const R lq0_step = F32 ? R(S->lq0_step) : static_cast<R>(g.lq0_step);
    const R inv_step = F32 ? R(S->inv_step) : static_cast<R>(g.inv_step);
    const int ncoef = 4 * (g.n_grid - 1);
    const R* knots = s_spline + g.n_species * ncoef;
    __syncthreads();

    // accumulators: sum w_n, d/d f_obs (w_n / c0), mass via E_obs, E_cons,
    // each integrated leg, tail (a, b) at the low and high ends
    Acc<R> acc_w, acc_fobs, acc_mobs, acc_mc, acc_tla, acc_tlb, acc_tha, acc_thb;
    Acc<R> acc_m[NI];
    Acc<R> acc_dw;                              // JVP: tangent of w_n
    const int64_t N = td.neval;
    const uint32_t task = td.gid;                 // the stream is keyed by the global task id
    const int32_t g1 = static_cast<int32_t>(seg.g1);

    // Statistical factors of one sample from its kinematic part base (0 for
    // a cut or invalid sample), the comoving radii r of the integrated legs,
    // 1/E of each (rE), the conserved leg's comoving momentum qc, energy Ec
    // and 1/Ec, dE / sigma^2 (dEs), the fractional-width term and
    // d log P / d E of the initial legs; then the sums and the derivatives.
    auto accumulate = [&](R base, const R* r, const R* rE, R qc, R Ec, R rEc, R dEs, R sig_term, R me_d) {
        R fac[NI + 1], dfac[NI + 1], tl[NI + 1];
        int jl[NI + 1];
#pragma unroll
        for (int j = 0; j < NI; ++j) {
            const SplineView<R> sv{s_spline + spc[j] * ncoef, knots};
            const Hit<R> h = spline_hit<R>(sv, r[j], g, inv_step, q0, lq0_step, fdj[j]);
            fac[j] = fma(cb[j], h.f, ca[j]);
            dfac[j] = cb[j] * h.d;
            jl[j] = h.j;
            tl[j] = h.t;
        }
        const bool below = qc < q0, above = qc > qN;
        const bool inside = !below && !above;
        R fc, dfdz = R(0);
        {
            const SplineView<R> sv{s_spline + spcn * ncoef, knots};
            const Hit<R> h = spline_hit<R>(sv, inside ? qc : (below ? q0 : qN), g, inv_step, q0, lq0_step, fd_c);
            jl[NI] = h.j;
            tl[NI] = h.t;
            if (inside) {
                fc = h.f;
                dfac[NI] = cbc * h.d;
            } else {
                const R x = below ? fma(tlo_b, Ec, tlo_a) : fma(thi_b, Ec, thi_a);
                R ft;
                if constexpr (F32) {
                    ft = tail_f32(x, eta_c);
                } else {
                    const R den = eta_c == R(1) ? expm1(x) : exp(x) - eta_c;
                    ft = den > R(0) ? R(1) / den : R(0);
                }
                dfdz = -ft * fma(eta_c, ft, R(1));
                if (fd_c && ft > R(1)) { ft = R(1); dfdz = R(0); }
                fc = ft;
                dfac[NI] = cbc;
            }
        }
        fac[NI] = fma(cbc, fc, cac);
        // products excluding each factor
        R pre[NI + 2];
        pre[0] = R(1);
#pragma unroll
        for (int k = 0; k <= NI; ++k) pre[k + 1] = pre[k] * fac[k];
        const R F = pre[NI + 1];
        const R wn = c0 * base * F;
        acc_w.add(wn);
        acc_fobs.add(base * F);
        R suf = R(1);
        R dwdf[NI + 1];
#pragma unroll
        for (int k = NI; k >= 0; --k) {
            dwdf[k] = c0 * base * pre[k] * suf * dfac[k];
            suf *= fac[k];
        }
        if constexpr (JVP) {
            // tangent: d w_n = sum_k dw/df_k df_k + (w_n / c0) U (U = dobs u_obs / scale)
            R dw = base * F * U;
#pragma unroll
            for (int k = 0; k <= NI; ++k) {
                R dfk;
                if (k == NI && !inside) {
                    dfk = dfdz * (below ? fma(dtb_lo, Ec, dta_lo) : fma(dtb_hi, Ec, dta_hi));
                } else {
                    const int sp = k < NI ? spc[k] : spcn;
                    const R* dc = s_dsp + sp * ncoef + 4 * jl[k];
                    const R t = tl[k];
                    dfk = fma(fma(fma(dc[3], t, dc[2]), t, dc[1]), t, dc[0]);
                }
                dw = fma(dwdf[k], dfk, dw);
            }
            acc_dw.add(dw);
        } else {
            const R dEterm = -wn * dEs;
            const R wsig = wn * sig_term;           // fractional width: same for every leg
            const R wme = wn * me_d;                // s-dependent |M|^2: every initial leg
#pragma unroll
            for (int j = 0; j < NI; ++j) {
                const R gE = fma(-wn, rE[j], fma(dEterm, sgnE[j], fma(inw[j], wme, wsig)));
                acc_m[j].add(gE * mass[j] * rE[j]);
            }
            const R gz = dwdf[NI] * dfdz;           // zero inside the grid
            const R gEc = fma(-wn, rEc, fma(dEterm, sgn_cons, fma(gz, below ? tlo_b : thi_b,
                                                                  fma(cons_inw, wme, wsig))));
            acc_mc.add(gEc * mass_c * rEc);
            acc_mobs.add(fma(-wn, inv_Eobs, fma(dEterm, s_obs, fma(obs_inw, wme, wsig))));
            if (below) { acc_tla.add(gz); acc_tlb.add(gz * Ec); }
            if (above) { acc_tha.add(gz); acc_thb.add(gz * Ec); }
            // spline coefficient gradients of this sample's lookups
#pragma unroll
            for (int k = 0; k <= NI; ++k) {
                if (k == NI && !inside) continue;
                const R gk = U * dwdf[k];
                if (gk != R(0)) {
                    const int sp = k < NI ? spc[k] : spcn;
                    if constexpr (F32) {
                        // FP32 shared-memory sums of this segment (one task: the
                        // contributions share a sign), moved into the FP64 array
                        // at the end of the segment
                        float* dst = s_dsp + sp * ncoef + 4 * jl[k];
                        const float t = tl[k];
                        const float g1 = gk * t, g2 = g1 * t;
                        atomicAdd(dst + 0, gk);
                        atomicAdd(dst + 1, g1);
                        atomicAdd(dst + 2, g2);
                        atomicAdd(dst + 3, g2 * t);
                    } else {
                        double* dst = s_gc + sp * ncoef + 4 * jl[k];
                        const double td_ = tl[k];
                        atomicAdd(dst + 0, gk);
                        atomicAdd(dst + 1, gk * td_);
                        atomicAdd(dst + 2, gk * td_ * td_);
                        atomicAdd(dst + 3, gk * td_ * td_ * td_);
                    }
                }
            }
        }
    };

    // FP32: samples with a non-zero kinematic part are queued per warp and
    // their statistical factors and derivatives evaluated 32 at a time (as in
    // the sample kernel); the warp runs the loop in step so that its votes
    // see all 32 lanes.  FP64: every sample is accumulated where it is drawn.
    constexpr int QW = vjp_queue_words(NLEG, JVP);
    float* q = F32 ? s_queue + (tid >> 5) * (kQueueSlots * QW) : nullptr;
    const int lane = tid & 31;
    const uint32_t lanes_below = (1u << lane) - 1u;
    int qn = 0;                                   // queued samples (warp-uniform)
    auto drain = [&](int slot) {
        R r[NI], rE[NI];
#pragma unroll
        for (int j = 0; j < NI; ++j) r[j] = q[(1 + j) * kQueueSlots + slot];
        if constexpr (JVP) {
#pragma unroll
            for (int j = 0; j < NI; ++j) rE[j] = R(0);
            accumulate(q[slot], r, rE, q[(1 + NI) * kQueueSlots + slot], q[(2 + NI) * kQueueSlots + slot], R(0),
                       R(0), R(0), R(0));
        } else {
#pragma unroll
            for (int j = 0; j < NI; ++j) rE[j] = q[(1 + NI + j) * kQueueSlots + slot];
            accumulate(q[slot], r, rE, q[(1 + 2 * NI) * kQueueSlots + slot], q[(2 + 2 * NI) * kQueueSlots + slot],
                       q[(3 + 2 * NI) * kQueueSlots + slot], q[(4 + 2 * NI) * kQueueSlots + slot],
                       q[(5 + 2 * NI) * kQueueSlots + slot], q[(6 + 2 * NI) * kQueueSlots + slot]);
        }
    };
    for (int32_t gb = static_cast<int32_t>(seg.g0) + (tid & ~31); gb < g1; gb += blockDim.x) {
        const int64_t grp = static_cast<int64_t>(gb) + lane;
        uint32_t uw[F32 ? SS::kUniforms : 1];
        R u[F32 ? 1 : SS::kUniforms];
        if constexpr (F32) group_words<D>(uw, static_cast<uint32_t>(grp), P.itn, ts.call, task, P.rk);
        else group_uniforms<D, F32, R>(u, grp, P.itn, ts.call, task, P.rk);
#pragma unroll
        for (int sgi = 0; sgi < G; ++sgi) {
            const bool valid = grp < g1 && grp * G + sgi < N;
            R y[D];
            R jac = R(1);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                int b;
                R fr;
                if constexpr (F32) {
                    const uint64_t m = static_cast<uint64_t>(uw[sgi * D + d]) * static_cast<uint32_t>(nb);
                    b = static_cast<int>(m >> 32);
                    fr = static_cast<float>(static_cast<uint32_t>(m)) * 2.3283064365386963e-10f;
                } else {
                    const R t = u[sgi * D + d] * nbR;
                    b = static_cast<int>(t);
                    b = b < nb - 1 ? b : nb - 1;
                    fr = t - static_cast<R>(b);
                }
                const Real2<R> e = s_map[d * nb + b];
                y[d] = fma(e.dy, fr, e.y0);
                jac *= e.dy;
            }
            R px = R(0), py = R(0), pz = pobs_sig;
            EBal<R> bal(sgn_obs_E);
            R Esum = e_obs;
            R Qx = R(0), Qy = R(0), Qz = obs_in_p, Ein = obs_in_E;
            R meas = jac;
            R rinv = R(1);
            bool cut = obs_cut;
            R r[NI], rE[NI];
#pragma unroll
            for (int j = 0; j < NI; ++j) {
                r[j] = y[3 * j];
                R st, ct, sp, cp;
                RMath<R>::sincos_(y[3 * j + 1], &st, &ct);
                RMath<R>::sincos_(y[3 * j + 2], &sp, &cp);
                const R p = r[j] * inv_a;
                const R ps = p * st;
                px = fma(-sig[j] * ps, cp, px);
                py = fma(-sig[j] * ps, sp, py);
                pz = fma(sig[j] * p, ct, pz);
                const R E2 = fma(p, p, m2[j]);
                const R rr = RMath<R>::rsqrt_(E2);
                const R E = E2 * rr;
                cut |= E < e_cut;
                bal.add(sgnE[j] * E);
                Esum += E;
                if (me_on) {
                    Qx = fma(-inw[j] * ps, cp, Qx);
                    Qy = fma(-inw[j] * ps, sp, Qy);
                    Qz = fma(inw[j] * p, ct, Qz);
                    Ein = fma(inw[j], E, Ein);
                }
                meas *= r[j] * r[j] * st;
                rinv *= rr;
                rE[j] = rr;
            }
            const R pc2 = fma(px, px, fma(py, py, pz * pz));
            const R Ec2 = pc2 + m2c;
            const R rEc = RMath<R>::rsqrt_(Ec2 > RMath<R>::kTiny ? Ec2 : R(1e-30));
            const R Ec = Ec2 * rEc;
            cut |= Ec < e_cut;
            bal.add(sgn_cons * Ec);
            const R dE = bal.value();
            const R qc = pc2 * (pc2 > RMath<R>::kTiny ? RMath<R>::rsqrt_(pc2) : R(0)) * a;
            // Gaussian and, for the adjoint, 1/sigma^2 and the derivative of
            // log(1/sigma) with exp(-dE^2 / 2 sigma^2) through sigma(E_k)
            R gs, inv_sig2, sig_term;
            if (frac) {
                Esum += Ec;
                const R iS = RMath<R>::rcp_(Esum);
                const R x = dE * iS;
                gs = RMath<R>::exp2_(gauss_k * x * x) * (R(2) * e_obs * iS);
                inv_sig2 = four_over_w2 * iS * iS;
                // d log g / d E_k from sigma: (dE^2 / sigma^2 - 1) / S for every leg
                sig_term = fma(dE * dE, inv_sig2, R(-1)) * iS;
            } else {
                gs = RMath<R>::exp2_(gauss_k * dE * dE);
                inv_sig2 = inv_sig2_abs;
                sig_term = R(0);
            }
            R base = meas * rinv * rEc * gs;
            base = (cut || !valid) ? R(0) : base;
            R me_d = R(0);          // d log P / d E_k of every initial leg: P'(s) / P(s) 2 E_in
            if (me_on) {
                const R qx = fma(cons_inw, px, Qx), qy = fma(cons_inw, py, Qy), qz = fma(cons_inw, pz, Qz);
                const R e = fma(cons_inw, Ec, Ein);
                const R sv = fma(e, e, -fma(qx, qx, fma(qy, qy, qz * qz)));
                const R Pv = fma(fma(fma(mec[3], sv, mec[2]), sv, mec[1]), sv, mec[0]);
                const R dP = fma(fma(R(3) * mec[3], sv, R(2) * mec[2]), sv, mec[1]);
                me_d = Pv != R(0) ? R(2) * e * dP * RMath<R>::rcp_(Pv) : R(0);
                base *= Pv;
            }
            const R dEs = dE * inv_sig2;
            if constexpr (F32) {
                const bool keep = base != R(0);
                const uint32_t vote = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int slot = qn + __popc(vote & lanes_below);     // < 2 * 32
                    q[slot] = base;
#pragma unroll
                    for (int j = 0; j < NI; ++j) q[(1 + j) * kQueueSlots + slot] = r[j];
                    if constexpr (JVP) {
                        q[(1 + NI) * kQueueSlots + slot] = qc;
                        q[(2 + NI) * kQueueSlots + slot] = Ec;
                    } else {
#pragma unroll
                        for (int j = 0; j < NI; ++j) q[(1 + NI + j) * kQueueSlots + slot] = rE[j];
                        q[(1 + 2 * NI) * kQueueSlots + slot] = qc;
                        q[(2 + 2 * NI) * kQueueSlots + slot] = Ec;
                        q[(3 + 2 * NI) * kQueueSlots + slot] = rEc;
                        q[(4 + 2 * NI) * kQueueSlots + slot] = dEs;
                        q[(5 + 2 * NI) * kQueueSlots + slot] = sig_term;
                        q[(6 + 2 * NI) * kQueueSlots + slot] = me_d;
                    }
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
            } else {
                accumulate(base, r, rE, qc, Ec, rEc, dEs, sig_term, me_d);
            }
        }
    }
    if constexpr (F32) {
        __syncwarp();
        if (lane < qn) drain(lane);
    }

    // ---- segment record: VJP [w, fobs, mobs, mc, tla, tlb, tha, thb, m_0 .. m_{NI-1}];
    //      JVP [w, dw] ----
    constexpr int NV = JVP ? 2 : 8 + NI;
    double vals[NV];
    if constexpr (JVP) {
        vals[0] = acc_w.value();
        vals[1] = acc_dw.value();
    } else {
        vals[0] = acc_w.value(); vals[1] = acc_fobs.value(); vals[2] = acc_mobs.value(); vals[3] = acc_mc.value();
        vals[4] = acc_tla.value(); vals[5] = acc_tlb.value(); vals[6] = acc_tha.value(); vals[7] = acc_thb.value();
#pragma unroll
        for (int j = 0; j < NI; ++j) vals[8 + j] = acc_m[j].value();
    }
    const int warp = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double v = vals[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[k * 8 + warp] = v;
    }
    __syncthreads();
    double* part = P.partials + seg.part;
    if (tid < NV) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += s_red[tid * 8 + w];
        part[tid] = v;
    }
    if constexpr (!JVP && F32) {
        // the segment's FP32 coefficient-gradient sums into the FP64 array
        const int ngc = g.n_species * ncoef;
        for (int k = tid; k < ngc; k += blockDim.x) {
            const float v = s_dsp[k];
            if (v != 0.0f) {
                s_gc[k] += static_cast<double>(v);
                s_dsp[k] = 0.0f;
            }
        }
    }
    __syncthreads();
}

template <typename R, int NMAX, bool JVP, bool ME = false>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) vjp_kernel(VjpParams V) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const EvalParams& P = V.E;
    R* s_spline = reinterpret_cast<R*>(smem_raw);
    const int nsp = P.smem_spline_elems;
    Real2<R>* s_map = reinterpret_cast<Real2<R>*>(s_spline + ((nsp + 3) & ~3));
    const int map_elems = kMaxDim * P.geo.nbins_max;
    const int ngc = 4 * (P.geo.n_grid - 1) * P.geo.n_species;
    double* s_gc = reinterpret_cast<double*>(s_map + map_elems);     // VJP: coefficient gradients
    double* s_red = s_gc + (JVP ? 0 : ngc);
    // JVP: tangent coefficients; FP32 VJP: the segment's coefficient-gradient sums
    R* s_dsp = reinterpret_cast<R*>(s_red + 12 * 8);
    // FP32: per-warp sample queues after the coefficient table
    float* s_queue = sizeof(R) == 4 ? reinterpret_cast<float*>(s_dsp + ngc) : nullptr;
    {
        const R* gc = static_cast<const R*>(P.coef);
        for (int k = threadIdx.x; k < ngc; k += blockDim.x) {
            s_spline[k] = gc[k];
            if constexpr (JVP) {
                s_dsp[k] = static_cast<const R*>(V.dcoef)[k];
            } else {
                s_gc[k] = 0.0;
                if constexpr (sizeof(R) == 4) s_dsp[k] = R(0);
            }
        }
        const R* gk = static_cast<const R*>(P.knots);
        for (int k = threadIdx.x; k < P.geo.n_grid; k += blockDim.x) s_spline[ngc + k] = gk[k];
    }
    // chunks of the partition, as in the sample kernel
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
                case 3: if constexpr (NMAX >= 3) vjp_segment<R, 3, JVP, ME>(V, seg, sd, td, tc, s_spline, s_map, s_gc, s_red, s_dsp, s_queue); break;
                case 4: if constexpr (NMAX >= 4) vjp_segment<R, 4, JVP, ME>(V, seg, sd, td, tc, s_spline, s_map, s_gc, s_red, s_dsp, s_queue); break;
                case 5: if constexpr (NMAX >= 5) vjp_segment<R, 5, JVP, ME>(V, seg, sd, td, tc, s_spline, s_map, s_gc, s_red, s_dsp, s_queue); break;
                case 6: if constexpr (NMAX >= 6) vjp_segment<R, 6, JVP, ME>(V, seg, sd, td, tc, s_spline, s_map, s_gc, s_red, s_dsp, s_queue); break;
                default: break;
            }
        }
        if (!P.chunk_counter) break;
    }
    if constexpr (!JVP) {
        __syncthreads();
        for (int k = threadIdx.x; k < ngc; k += blockDim.x) {
            const double v = s_gc[k];
            if (v != 0.0) atomicAdd(V.gcoef + k, v);
        }
    }
}

}  // namespace best
