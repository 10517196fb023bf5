"""Forward-mode tangent (best_collision_jvp) and the Newton-Krylov implicit
Euler step (best_step_implicit_euler) through the C ABI: the tangent
against the oracle's automatic differentiation of the same fixed-sample
integral and against the library's own adjoint (<v, J u> = <J^T v, u>); the
implicit step against the oracle's dense-Jacobian Newton solve on the same
maps and samples."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import implicit as oimp
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


def _close(a, b, rtol):
    scale = np.max(np.abs(b)) + 1e-300
    return np.max(np.abs(a - b)) <= rtol * scale


def _setup(kind, precision, refine_first=True):
    import torch
    from paper_2603_28848_gb300 import Collision
    (prob, f0), t = _problem(kind)
    col = Collision(prob, precision)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda")
    if refine_first:
        col.eval(f, t)
    return col, prob, f0, f, t


@pytest.mark.parametrize("kind", ["mb22", "be23", "multi", "2to4"])
def test_fp64_jvp_matches_oracle_autodiff(kind):
    import torch
    col, prob, f0, f, t = _setup(kind, W.PREC_FP64, refine_first=kind != "2to4")
    u0 = f0 * np.random.default_rng(3).normal(size=f0.shape)
    C, JU = [x.cpu().numpy() for x in col.jvp(f, torch.tensor(u0, device="cuda"), t)]
    col.check()
    Co, JUo = oadj.jvp(prob, f0, t, u0, _oracle_maps(col, prob), col.call_counter, "f64")
    assert _close(C, Co, 1e-8)
    assert _close(JU, JUo, 1e-8), np.max(np.abs(JU - JUo)) / np.max(np.abs(JUo))
    col.close()


@pytest.mark.parametrize("kind", ["mb22", "multi"])
def test_fp32_jvp_matches_oracle_autodiff(kind):
    """FP32 per-sample arithmetic, FP64 accumulation, same samples: within
    5e-4 of the largest component, as for the FP32 adjoint."""
    import torch
    col, prob, f0, f, t = _setup(kind, W.PREC_FP32)
    u0 = f0 * np.random.default_rng(3).normal(size=f0.shape)
    C, JU = [x.cpu().numpy() for x in col.jvp(f, torch.tensor(u0, device="cuda"), t)]
    col.check()
    Co, JUo = oadj.jvp(prob, f0, t, u0, _oracle_maps(col, prob), col.call_counter, "f32")
    assert _close(C, Co, 5e-4)
    assert _close(JU, JUo, 5e-4), np.max(np.abs(JU - JUo)) / np.max(np.abs(JUo))
    col.close()


@pytest.mark.parametrize("precision,rtol", [(W.PREC_FP64, 1e-11), (W.PREC_FP32, 2e-4)])
@pytest.mark.parametrize("kind", ["mb22", "be23", "multi", "2to4"])
def test_jvp_and_vjp_are_transposes(kind, precision, rtol):
    """<v, J u> from the tangent launch equals <J^T v, u> from the adjoint
    launch: two independent kernels' derivatives of the same C~."""
    import torch
    col, prob, f0, f, t = _setup(kind, precision)
    rng = np.random.default_rng(9)
    u0 = f0 * rng.normal(size=f0.shape)
    v0 = rng.normal(size=f0.shape)
    C1, JU = col.jvp(f, torch.tensor(u0, device="cuda"), t)
    C2, gf, _, _ = col.vjp(f, torch.tensor(v0, device="cuda"), t)
    lhs = float(np.sum(v0 * JU.cpu().numpy()))
    rhs = float(np.sum(gf.cpu().numpy() * u0))
    scale = float(np.sum(np.abs(v0 * JU.cpu().numpy())))
    assert abs(lhs - rhs) <= rtol * scale, (lhs, rhs, scale)
    # the two kernels sum the same samples in different orders: C~ agrees to
    # rounding relative to its largest value (a point where gain and loss
    # nearly cancel has no relative precision of its own in FP32)
    crtol = 1e-12 if precision == W.PREC_FP64 else 1e-6
    c1, c2 = C1.cpu().numpy(), C2.cpu().numpy()
    assert np.max(np.abs(c1 - c2)) <= crtol * np.max(np.abs(c2)), np.max(np.abs(c1 - c2)) / np.max(np.abs(c2))
    col.close()


def test_jvp_is_bitwise_repeatable_and_linear():
    import torch
    col, prob, f0, f, t = _setup("multi", W.PREC_FP64)
    u = torch.tensor(f0 * np.random.default_rng(4).normal(size=f0.shape), device="cuda")
    _, a = col.jvp(f, u, t)
    _, b = col.jvp(f, u, t)
    _, c = col.jvp(f, 2.5 * u, t)
    _, z = col.jvp(f, torch.zeros_like(u), t)
    assert torch.equal(a, b)
    assert torch.allclose(c, 2.5 * a, rtol=1e-12, atol=1e-300)
    assert torch.count_nonzero(z) == 0
    col.close()


@pytest.mark.parametrize("kind", ["mb22", "multi"])
def test_fp64_implicit_euler_matches_oracle_newton(kind):
    """Same maps, same samples (train=False): the Newton-Krylov root equals
    the oracle's dense-Newton root of the backward-Euler equation."""
    import torch
    col, prob, f0, f, t = _setup(kind, W.PREC_FP64)
    C, _ = col.jvp(f, torch.zeros_like(f), t)
    rate = float(np.max(np.abs(C.cpu().numpy() / f0)))
    dt = 0.2 / rate
    logf = torch.log(f).contiguous()
    info = col.step_implicit_euler(logf, t, dt, train=False, tol=1e-11)
    col.check()
    g = logf.cpu().numpy()
    go, it, rinf = oimp.collision_step(prob, np.log(f0), t, dt, _oracle_maps(col, prob), col.call_counter, tol=1e-12)
    assert rinf <= 1e-12
    assert np.max(np.abs(g - go)) <= 1e-9, (np.max(np.abs(g - go)), info)
    assert info["newton"] >= 1 and info["residual"] <= 1e-11
    col.close()


def test_fp32_implicit_euler_matches_oracle_newton():
    """FP32 samples (uniforms from one Philox word each, as the oracle's f32
    mode draws them), FP32 per-sample arithmetic: the root within 2e-4 in
    log f, i.e. dt (0.2 / max|C~/f|) times the 5e-4 FP32 level of C~."""
    import torch
    col, prob, f0, f, t = _setup("mb22", W.PREC_FP32)
    C, _ = col.jvp(f, torch.zeros_like(f), t)
    dt = 0.2 / float(np.max(np.abs(C.cpu().numpy() / f0)))
    logf = torch.log(f).contiguous()
    info = col.step_implicit_euler(logf, t, dt, train=False)
    assert info["residual"] <= 1e-6
    go, it, rinf = oimp.collision_step(prob, np.log(f0), t, dt, _oracle_maps(col, prob), col.call_counter,
                                       tol=1e-12, mode="f32")
    assert np.max(np.abs(logf.cpu().numpy() - go)) <= 2e-4
    col.close()


def test_implicit_euler_trains_maps_and_reports_failure():
    import torch
    from paper_2603_28848_gb300 import BestError
    col, prob, f0, f, t = _setup("mb22", W.PREC_FP64, refine_first=False)
    logf = torch.log(f).contiguous()
    c0 = col.call_counter
    info = col.step_implicit_euler(logf, t, 1e-3, train=True)
    assert col.call_counter > c0 and info["residual"] <= 1e-10
    # a tolerance Newton cannot meet in one iteration: error, logf untouched
    before = logf.clone()
    with pytest.raises(BestError):
        col.step_implicit_euler(logf, t, 10.0, train=False, tol=1e-300, max_newton=1)
    assert torch.equal(logf, before)
    col.close()
