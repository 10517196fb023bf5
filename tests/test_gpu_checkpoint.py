"""Checkpoint / resume through the C ABI: bitwise continuation."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_resume_is_bitwise(tmp_path):
    import torch
    from paper_2603_28848_gb300 import BestError, Collision, checkpoint
    prob, f0 = W.c4_multi_species(n=8, nmin=600, nmax=1500, nitn=2)

    def fresh():
        col = Collision(prob, W.PREC_FP32)
        logf = torch.tensor(np.log(f0), dtype=torch.float64, device="cuda").contiguous()
        t = torch.ones(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        return col, logf, t, dt

    a = fresh()
    a[0].evolve(a[1], a[2], a[3], 4, 0.05, "heun")
    b = fresh()
    b[0].evolve(b[1], b[2], b[3], 2, 0.05, "heun")
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, b[0], b[1], b[2], b[3])
    b[0].close()
    c = fresh()
    logf, t, dt = checkpoint.load(path, c[0])
    c[0].evolve(logf, t, dt, 2, 0.05, "heun")
    torch.cuda.synchronize()
    assert torch.equal(a[1], logf) and torch.equal(a[2], t)
    # a different configuration is refused
    other = Collision(W.c4_multi_species(n=9, nmin=600, nmax=1500, nitn=2)[0], W.PREC_FP32)
    with pytest.raises(BestError):
        other.load_state(np.load(path)["state"].tobytes())
    for x in (a[0], c[0], other):
        x.close()
