"""CUDA-graph evolution and the launch-shape autotuner, through the C ABI."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _state(prob, f0, precision):
    import torch
    from paper_2603_28848_gb300 import Collision
    col = Collision(prob, precision)
    logf = torch.tensor(np.log(f0), dtype=torch.float64, device="cuda").contiguous()
    t = torch.ones(1, dtype=torch.float64, device="cuda")      # a(t) = (t/t0)^(1/2) needs t > 0
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    return col, logf, t, dt


@pytest.mark.parametrize("method", ["euler", "heun"])
def test_graph_replay_equals_direct_steps(method):
    """n steps replayed from one captured graph are bitwise the n direct
    calls (all kernels are deterministic)."""
    import torch
    prob, f0 = W.c4_multi_species(n=10, nmin=800, nmax=2000, nitn=2)
    a = _state(prob, f0, W.PREC_FP32)
    b = _state(prob, f0, W.PREC_FP32)
    for _ in range(3):
        a[3].fill_(0.05)
        (a[0].step_heun if method == "heun" else a[0].step_euler)(a[1], a[2], a[3])
    b[0].evolve(b[1], b[2], b[3], 3, 0.05, method)
    torch.cuda.synchronize()
    a[0].check()
    b[0].check()
    assert torch.all(torch.isfinite(a[1]))
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])
    assert a[2].item() > 1.0
    # replaying again continues the evolution from the graph's state
    b[0].evolve(b[1], b[2], b[3], 2, 0.05, method)
    for _ in range(2):
        a[3].fill_(0.05)
        (a[0].step_heun if method == "heun" else a[0].step_euler)(a[1], a[2], a[3])
    torch.cuda.synchronize()
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    a[0].close()
    b[0].close()


def test_autotune_preserves_state_and_parity():
    import torch
    from oracle import collision as ocol
    from tests._helpers import task_arrays
    prob, f0 = W.c1_maxwell_2to2(n=16, neval=20000, nitn=3)
    col, logf, t, dt = _state(prob, f0, W.PREC_FP32)
    f = torch.exp(logf)
    col.eval(f, 0.0)
    maps0 = col.maps()
    call0 = col.call_counter
    mb = col.autotune(f, 0.0)
    assert mb in (3, 4, 5)
    assert np.array_equal(col.maps(), maps0) and col.call_counter == call0
    C, err = col.eval(f, 0.0)
    mean, terr = col.task_results()
    st = ocol.State()
    ocol.collision(prob, f0, 0.0, st, "f32")
    _, _, detail = ocol.collision(prob, f0, 0.0, st, "f32")
    om, oe = task_arrays(detail, col.n_tasks)
    z = np.abs(mean - om) / np.sqrt(terr ** 2 + oe ** 2)
    assert np.mean(z < 3) >= 0.95 and np.max(z) < 6
    col.close()


def test_profiling_inside_graph():
    """Timing events captured into the step graph report the sample-kernel
    launches of the last replayed step."""
    import torch
    prob, f0 = W.c1_maxwell_2to2(n=12, neval=5000, nitn=3)
    col, logf, t, dt = _state(prob, f0, W.PREC_FP32)
    col.profile(True)
    col.evolve(logf, t, dt, 2, 0.1, "heun")
    ms, n = col.profile_read()
    assert n == 2 * 3 and ms > 0
    col.profile(False)
    col.close()
