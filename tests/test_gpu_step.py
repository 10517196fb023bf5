"""Euler and Heun steps (Eq. (14)-(16)) through the C ABI against the
oracle's steps on the same Philox samples (FP64), including a species whose
mass follows a knot table and changes between the two Heun stages, and the
library's m_s(t) against the oracle's."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import collision as ocol
from oracle import step as ostep

pytestmark = pytest.mark.gpu

# FP64, identical samples: the steps differ by rounding order only; the bar
# is 1e-5 of the largest change of log f (the parity bar of the integral).
TOL = 1e-5
RAMP = 1e-7
TABLE = ((1.0, 1.0), (2.0, 0.7), (2.0 + RAMP, 0.4), (3.0, 0.4))


def _multi_species_with_table():
    prob, f0 = W.c4_multi_species(n=8, nmin=500, nmax=3000, nitn=2)
    a = replace(prob.species[0], mass0=5.0, mass1=3.0, mass_table=TABLE)
    return replace(prob, species=(a, prob.species[1])), f0


def _run(prob, f0, t0, dt0, method):
    import torch
    from paper_2603_28848_gb300 import Collision
    col = Collision(prob, W.PREC_FP64)
    logf = torch.tensor(np.log(f0), dtype=torch.float64, device="cuda").contiguous()
    t = torch.tensor([t0], dtype=torch.float64, device="cuda")
    dt = torch.tensor([dt0], dtype=torch.float64, device="cuda")
    (col.step_heun if method == "heun" else col.step_euler)(logf, t, dt)
    col.check()
    out = logf.cpu().numpy(), t.item(), dt.item()
    col.close()
    st = ocol.State()
    ref = (ostep.heun_step if method == "heun" else ostep.euler_step)(prob, np.log(f0), t0, dt0, st)
    return out, ref


@pytest.mark.parametrize("method", ["euler", "heun"])
def test_step_with_mass_table(method):
    """From t0 just before a steep ramp of m_A (0.7 -> 0.4 over 1e-7): the
    step of Eq. (16) (about 2e-6 here) takes the Heun stage k2 past the ramp,
    so the two stages see different masses."""
    prob, f0 = _multi_species_with_table()
    prob = replace(prob, eps_dt=1.0)
    t0 = 2.0 - RAMP
    (lg, tg, dtg), ref = _run(prob, f0, t0, 0.3, method)
    lo, to, dto = ref[0], ref[1], ref[2]
    assert dto > 4 * RAMP and dtg == pytest.approx(dto, rel=1e-6)
    assert tg == pytest.approx(to, rel=1e-12)
    d = np.max(np.abs(lg - lo)) / np.max(np.abs(lo - np.log(f0)))
    assert d < TOL, d


@pytest.mark.parametrize("method", ["euler", "heun"])
def test_step_limited_by_eq16(method):
    """A requested dt far above the bound: both sides take dt = eps / max|C/f|."""
    prob, f0 = W.c1_maxwell_2to2(n=12, neval=2000, nitn=2)
    (lg, tg, dtg), ref = _run(prob, f0, 0.0, 1e6, method)
    lo, to, dto = ref[0], ref[1], ref[2]
    assert dto < 1e6 and dtg == pytest.approx(dto, rel=1e-6)
    d = np.max(np.abs(lg - lo)) / np.max(np.abs(lo - np.log(f0)))
    assert d < TOL, d


def test_species_masses_match_the_oracle():
    from paper_2603_28848_gb300 import Collision
    prob, _ = _multi_species_with_table()
    col = Collision(prob, W.PREC_FP64)
    for t in (0.0, 1.0, 1.5, 2.0, 2.02, 2.05, 2.5, 3.0, 9.0):
        assert np.allclose(col.species_masses(t), ocol.masses(prob, t), rtol=1e-15, atol=1e-15), t
    col.close()
