"""The Solver (the paper's set-up style) on the GPU: its steps equal direct
Collision steps on the same problem, its checkpoint resumes bit for bit, and
its densities come from the library."""
import numpy as np
import pytest

import workloads as W
from paper_2603_28848_gb300.solver import Solver

pytestmark = pytest.mark.gpu


def _solver():
    s = Solver(q_min=0.1, q_max=20.0, n_grid=24, seed=5)
    s.initialize_species("phi", lambda q: 1.0 / (1.0 + np.exp((q - 3.0) / 2.0)), stat="boson", mass=1.0)
    s.add_process("elastic", ["phi", "phi"], ["phi", "phi"], coupling=1.0, neval=4000, delta_width=0.01)
    return s


def test_solver_steps_equal_direct_steps():
    import torch
    from paper_2603_28848_gb300 import Collision
    s = _solver()
    for _ in range(3):
        s.evolve_step(0.5, "heun")
    got = s.distribution("phi")
    col = Collision(s.problem(), W.PREC_FP32)
    logf = torch.tensor(np.log(1.0 / (1.0 + np.exp((W.grid_points(s.grid) - 3.0) / 2.0))), device="cuda")[None]
    logf = logf.contiguous()
    t = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    dt = torch.tensor([0.0], dtype=torch.float64, device="cuda")
    for _ in range(3):
        dt.fill_(0.5)
        col.step_heun(logf, t, dt)
    assert np.array_equal(got, np.exp(logf[0].cpu().numpy()))
    assert s.current_time == float(t.item())
    n, rho = s.densities()["phi"]
    assert n > 0 and rho > n                       # m = 1: every E > 1, so rho > n
    col.close()
    s.close()


def test_solver_checkpoint_resumes_bitwise(tmp_path):
    s = _solver()
    s.evolve_step(0.5)
    s.evolve_step(0.5)
    path = str(tmp_path / "run.npz")
    history = {"t": [1.0, 1.5, 2.0], "n": np.array([0.2, 0.21, 0.22]), "note": "two Heun steps"}
    s.save_checkpoint(path, history=history)
    s.evolve_step(0.5)
    s.evolve_step(0.5)
    a = s.distribution("phi")
    s.close()
    r = Solver.load_checkpoint(path)
    assert r.history == {"t": [1.0, 1.5, 2.0], "n": [0.2, 0.21, 0.22], "note": "two Heun steps"}
    r.evolve_step(0.5)
    r.evolve_step(0.5)
    assert np.array_equal(a, r.distribution("phi"))
    r.close()


def test_solver_with_callable_matrix_element_and_mass_function():
    """A matrix element given as a callable of (momenta, coupling) and a mass
    given as a function of time run through the library: the Solver's steps
    equal direct steps on the problem with the fitted P(s) and the knot table,
    and the library's m(t) follows the table."""
    import torch
    from paper_2603_28848_gb300 import Collision

    def me(k, g):
        tot = k[0] + k[1]
        s2 = tot[0] ** 2 - tot[1] ** 2 - tot[2] ** 2 - tot[3] ** 2
        return g * g * (0.8 + 0.05 * s2)

    s = Solver(q_min=0.1, q_max=15.0, n_grid=20, seed=9)
    s.initialize_species("chi", lambda q: 0.3 * np.exp(-0.5 * (q - 2.0) ** 2) + 0.05, stat="boson", mass=1.0)
    s.add_process("chichi", ["chi", "chi"], ["chi", "chi"], me, coupling=0.9, neval=3000, delta_width=0.02)
    s.set_mass_func("chi", lambda t: 1.0 if t < 1.6 else 0.7, [1.0, 1.5, 1.6, 10.0])
    prob = s.problem()
    assert np.allclose(prob.processes[0].me_coef, (0.8, 0.05, 0.0, 0.0), rtol=1e-7, atol=1e-12)
    for _ in range(3):
        s.evolve_step(0.4, "heun")
    got = s.distribution("chi")
    col = Collision(prob, W.PREC_FP32)
    q = W.grid_points(s.grid)
    logf = torch.tensor(np.log(0.3 * np.exp(-0.5 * (q - 2.0) ** 2) + 0.05), device="cuda")[None].contiguous()
    t = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    dt = torch.tensor([0.0], dtype=torch.float64, device="cuda")
    for _ in range(3):
        dt.fill_(0.4)
        col.step_heun(logf, t, dt)
    assert np.array_equal(got, np.exp(logf[0].cpu().numpy()))
    assert np.allclose(col.species_masses(1.55), [0.85], rtol=1e-14)
    assert np.allclose(col.species_masses(2.0), [0.7], rtol=1e-14)
    col.close()
    s.close()
