"""Density diagnostics (best_moments) against the oracle, and the chunked
thermalisation driver."""
import numpy as np
import pytest

import workloads as W
from oracle import moments as om

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["bose", "multi"])
def test_moments_match_oracle(kind):
    import torch
    from paper_2603_28848_gb300 import Collision
    if kind == "bose":
        (prob, f0), t = W.c2_bose_2to2(n=128, neval=1000, nitn=1), 0.0
    else:
        (prob, f0), t = W.c4_multi_species(n=64, nmin=200, nmax=400, nitn=1), 2.5
    col = Collision(prob, W.PREC_FP32)
    n, rho = col.moments(torch.tensor(f0, dtype=torch.float64, device="cuda"), t)
    no, ro = om.moments(prob, f0, t)
    assert np.allclose(n.cpu().numpy(), no, rtol=1e-12, atol=0)
    assert np.allclose(rho.cpu().numpy(), ro, rtol=1e-12, atol=0)
    col.close()


def test_thermalisation_driver_records_histories():
    from paper_2603_28848_gb300 import evolve
    prob, f0 = W.c1_maxwell_2to2(n=16, neval=4000, nitn=2)
    h = evolve.run(prob, f0, steps=6, every=2, precision=W.PREC_FP32, autotune=False)
    assert h["step"] == [0, 2, 4, 6]
    assert len(h["n"]) == 4 and len(h["rho"]) == 4
    assert np.all(np.diff(h["t"]) > 0)
    assert np.all(np.isfinite(h["n"])) and np.all(np.isfinite(h["rho"]))
    # MB 2 -> 2 conserves N and E up to the Monte Carlo error, the Gaussian
    # width and the grid truncation: a few percent over six short steps
    assert max(h["max_rel_change_n"]) < 0.05 and max(h["max_rel_change_rho"]) < 0.05
