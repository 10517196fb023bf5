"""Adjoint (best_collision_vjp) through the C ABI against the oracle's
autograd gradient of the same fixed-sample integral, against central
finite differences (h = 1e-4 relative) of the GPU's own fixed-sample C~, and
the exact coupling derivative."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle.tasks import side_integrals

pytestmark = pytest.mark.gpu


def _problem(kind):
    if kind == "mb22":
        return W.c1_maxwell_2to2(n=10, neval=3000, nitn=2), 0.0
    if kind == "be23":
        return W.c3_cannibal_2to3(n=8, neval=2000, nitn=2), 0.0
    if kind == "multi":
        return W.c4_multi_species(n=8, nmin=800, nmax=1500, nitn=2), 2.0
    return W.c5_2to4(n=6, neval=1000, nitn=2), 0.0


def _oracle_maps(col, prob):
    maps = col.maps()
    out = {}
    n = prob.grid.n
    for k, si in enumerate(side_integrals(prob)):
        nb = prob.processes[si.process].nbins
        for i in range(n):
            for term in (0, 1):
                tid = (k * n + i) * 2 + term
                out[tid] = maps[tid][: si.dim * (nb + 1)].reshape(si.dim, nb + 1)
    return out


def _run(kind, precision, refine_first):
    import torch
    from paper_2603_28848_gb300 import Collision
    (prob, f0), t = _problem(kind)
    col = Collision(prob, precision)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda")
    if refine_first:
        col.eval(f, t)                       # adapted maps, counter advanced
    rng = np.random.default_rng(7)
    v = torch.tensor(rng.normal(size=f0.shape), dtype=torch.float64, device="cuda")
    C, gf, gm, gl = [x.cpu().numpy() for x in col.vjp(f, v, t)]
    col.check()
    mode = "f32" if precision == W.PREC_FP32 else "f64"
    Co, gfo, gmo, glo = oadj.vjp(prob, f0, t, v.cpu().numpy(), _oracle_maps(col, prob), col.call_counter, mode)
    return col, f, v, (C, gf, gm, gl), (Co, gfo, gmo, glo), prob, t


def _close(a, b, rtol):
    scale = np.max(np.abs(b)) + 1e-300
    return np.max(np.abs(a - b)) <= rtol * scale


@pytest.mark.parametrize("kind", ["mb22", "be23", "multi", "2to4"])
def test_fp64_adjoint_matches_oracle_autograd(kind):
    col, f, v, g, o, prob, t = _run(kind, W.PREC_FP64, refine_first=kind != "2to4")
    for got, want, name in zip(g, o, ("C", "df", "dm", "dcoupling")):
        assert _close(got, want, 1e-8), (name, got, want)
    col.close()


@pytest.mark.parametrize("kind", ["mb22", "be23", "multi"])
def test_fp32_adjoint_matches_oracle_autograd(kind):
    """FP32 per-sample arithmetic (compensated energy balance) with FP64
    accumulation against the oracle's FP64 gradient of the same samples, over
    five seeds: the median over seeds of max |diff| / max |oracle| is below
    5e-4 for C~, dL/df and dL/dcoupling and below 1e-3 for dL/dm; every seed
    stays within 10 times that, dL/dm within 50 times.  What is left is the
    FP32 rounding of the sample coordinates (r, theta, phi) themselves, which
    moves E_in - E_out by about one FP32 ulp of the energies (3e-7 for
    energies of a few units); through the Gaussian of Eq. (11) a sample's
    weight moves by |dE| d(dE) / sigma^2, up to 13 d(dE) / sigma = 4e-4 at
    sigma = 0.01 for the samples in the Gaussian's tail, so no bound below
    that scale holds for every seed and map.  dL/dm, one number per species
    made of Gaussian derivatives dE / sigma^2 that nearly cancel over the
    shell, amplifies it most, and its relative error has a heavy tail over
    seeds (the MB 2 -> 2 problem's default seed: 8.5e-3)."""
    from dataclasses import replace
    base = _problem
    errs = []
    try:
        for seed in range(5):
            def seeded(k, seed=seed):
                (p, f0), t = base(k)
                return (replace(p, seed=p.seed + 7919 * seed), f0), t
            globals()["_problem"] = seeded
            col, f, v, g, o, prob, t = _run(kind, W.PREC_FP32, refine_first=True)
            errs.append([np.max(np.abs(a - b)) / np.max(np.abs(b)) for a, b in zip(g, o)])
            col.close()
    finally:
        globals()["_problem"] = base
    errs = np.array(errs)                                   # seeds x (C, df, dm, dcoupling)
    bound = np.array([5e-4, 5e-4, 1e-3, 5e-4])
    assert np.all(np.median(errs, axis=0) < bound), errs
    assert np.all(errs < np.array([10.0, 10.0, 50.0, 10.0]) * bound), errs


@pytest.mark.parametrize("kind,h,rtol", [("mb22", 1e-4, 1e-4), ("be23", 1e-4, 1e-4), ("2to4", 1e-4, 1e-4),
                                         ("multi", 1e-4, 3e-4), ("multi", 1e-5, 1e-4)])
def test_adjoint_passes_central_differences(kind, h, rtol):
    """dL/df_j against (L(f + h f_j e_j) - L(f - h f_j e_j)) / (2 h f_j), L =
    v . C~ from the GPU itself (FP64 path, same samples).  C~ is only
    piecewise smooth: samples whose spline value crosses a clamp (f >= 0, and
    f <= 1 for the FD species of the multi-species problem) within +-h give
    the difference quotient an O(h) error, so that problem is also checked
    at h = 1e-5."""
    import torch
    col, f, v, g, o, prob, t = _run(kind, W.PREC_FP64, refine_first=kind != "2to4")
    C, gf, gm, gl = g

    def L(ff):
        c = col.vjp(ff, v, t)[0]
        return float((c * v).sum())

    f0 = f.cpu().numpy()
    S, n = f0.shape
    checked = 0
    for s in range(S):
        for j in (1, n // 2, n - 2):
            if f0[s, j] < 1e-8 * f0.max():
                continue
            fp = f.clone(); fp[s, j] *= 1 + h
            fm = f.clone(); fm[s, j] *= 1 - h
            fd = (L(fp) - L(fm)) / (2 * h * f0[s, j])
            assert abs(fd - gf[s, j]) <= rtol * abs(gf[s, j]) + 1e-6 * np.max(np.abs(gf))
            checked += 1
    assert checked >= 3
    col.close()


def test_coupling_gradient_is_exact():
    import torch
    col, f, v, g, o, prob, t = _run("mb22", W.PREC_FP64, refine_first=True)
    C, gf, gm, gl = g
    lam = prob.processes[0].coupling
    assert np.isclose(gl[0], 2.0 * np.sum(v.cpu().numpy() * C) / lam, rtol=1e-12)
    col.close()


def test_autograd_function_backward_is_the_vjp():
    """torch.autograd through fixed_sample_collision gives the adjoint's
    gradients w.r.t. f, the masses and the couplings."""
    import torch
    from paper_2603_28848_gb300 import Collision, fixed_sample_collision
    (prob, f0), t = _problem("multi")
    col = Collision(prob, W.PREC_FP64)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda", requires_grad=True)
    m = torch.tensor([s.mass0 + s.mass1 * t for s in prob.species], dtype=torch.float64, device="cuda",
                     requires_grad=True)
    lam = torch.tensor([p.coupling for p in prob.processes], dtype=torch.float64, device="cuda", requires_grad=True)
    v = torch.tensor(np.random.default_rng(3).normal(size=f0.shape), dtype=torch.float64, device="cuda")
    C = fixed_sample_collision(col, f, t, m, lam)
    (C * v).sum().backward()
    C2, gf, gm, gl = col.vjp(f.detach(), v, t)
    assert torch.equal(C.detach(), C2)
    assert torch.allclose(f.grad, gf, rtol=1e-12, atol=0) and torch.allclose(m.grad, gm, rtol=1e-12, atol=0)
    assert torch.allclose(lam.grad, gl, rtol=1e-12, atol=0)
    col.close()
