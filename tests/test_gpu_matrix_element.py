"""s-dependent matrix element |M|^2 = coupling^2 P(s) through the C ABI
against the oracle: FP64 parity on identical samples (alone, with stratified
sampling, and in the multi-species FRW problem), FP32 within three standard
errors, and the adjoint (including the mass gradient through s) and tangent
against the oracle's automatic differentiation."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from tests.test_gpu_parity import _compare_fp32, _compare_fp64
from tests.test_gpu_vjp import _oracle_maps

pytestmark = pytest.mark.gpu

ME = (0.5, 0.3, 0.05, 0.002)


def _me(prob, which=None, **kw):
    return replace(prob, processes=tuple(replace(p, me_coef=ME, **kw) if which is None or k in which else p
                                         for k, p in enumerate(prob.processes)))


def test_me_maxwell_fp64():
    prob, f0 = W.c1_maxwell_2to2(n=12, neval=3001, nitn=2)
    _compare_fp64(_me(prob), f0, sweeps=2)


def test_me_multi_species_one_process_fp64():
    prob, f0 = W.c4_multi_species(n=8, nmin=500, nmax=3000, nitn=2)
    _compare_fp64(_me(prob, which=(1,)), f0, t=2.0)


def test_me_with_stratified_sampling_fp64():
    prob, f0 = W.c3_cannibal_2to3(n=6, neval=4000, nitn=2, with_2to2=True)
    _compare_fp64(_me(prob, strat=1), f0)


def test_me_fp32_within_three_sigma():
    prob, f0 = W.c3_cannibal_2to3(n=8, neval=4001, nitn=2)
    _compare_fp32(_me(prob), f0)


@pytest.mark.parametrize("kind", ["mb22", "multi"])
def test_me_adjoint_and_tangent_match_oracle(kind):
    import torch
    from paper_2603_28848_gb300 import Collision
    if kind == "mb22":
        (prob, f0), t = W.c1_maxwell_2to2(n=10, neval=3000, nitn=2), 0.0
        prob = _me(prob)
    else:
        (prob, f0), t = W.c4_multi_species(n=8, nmin=800, nmax=1500, nitn=2), 2.0
        prob = _me(prob, which=(0, 2))
    col = Collision(prob, W.PREC_FP64)
    f = torch.tensor(f0, dtype=torch.float64, device="cuda")
    col.eval(f, t)
    rng = np.random.default_rng(11)
    v = rng.normal(size=f0.shape)
    u = f0 * rng.normal(size=f0.shape)
    C, gf, gm, gl = [x.cpu().numpy() for x in col.vjp(f, torch.tensor(v, device="cuda"), t)]
    _, JU = [x.cpu().numpy() for x in col.jvp(f, torch.tensor(u, device="cuda"), t)]
    maps = _oracle_maps(col, prob)
    Co, gfo, gmo, glo = oadj.vjp(prob, f0, t, v, maps, col.call_counter, "f64")
    _, JUo = oadj.jvp(prob, f0, t, u, maps, col.call_counter, "f64")
    for got, want, name in ((C, Co, "C"), (gf, gfo, "df"), (gm, gmo, "dm"), (gl, glo, "dl"), (JU, JUo, "Ju")):
        assert np.max(np.abs(got - want)) <= 1e-8 * np.max(np.abs(want)), (name, got, want)
    col.close()


def test_all_zero_coefficients_are_rejected():
    from paper_2603_28848_gb300 import BestError, Collision
    prob, f0 = W.c1_maxwell_2to2(n=8, neval=1000, nitn=1)
    prob = replace(prob, processes=tuple(replace(p, me_coef=(0.0, 0.0, 0.0, 0.0)) for p in prob.processes))
    with pytest.raises(BestError):
        Collision(prob, W.PREC_FP32)
