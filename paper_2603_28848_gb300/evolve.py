"""Thermalisation runs with conservation diagnostics (Sec. 5C, Fig. 3).

Steps are replayed from the context's captured CUDA graph (best_evolve) in
chunks of ``every`` steps; between chunks the number and energy density of
every species are taken on the device (best_moments), so that a run records
how well N and E are conserved.  Every step of the path runs in libbest; this
module only sequences the calls and copies the small histories to the host.

    python -m paper_2603_28848_gb300.evolve --workload c2_bose_2to2 --steps 200 --every 20
    python -m paper_2603_28848_gb300.evolve --workload c3_cannibal_2to3 --n 64 --neval 1000000 \
        --nitn 4 --method euler --dt 1e9 --t0 0 --steps 300 --every 30
"""
import argparse
import json
import sys

import numpy as np


def equilibrium_fit(problem, f, t):
    """(T, mu) per species from the least-squares line of log(1/f + eta)
    against E(q/a) over the grid points with f > 1e-12: an equilibrium
    distribution 1/(exp((E - mu)/T) - eta) gives exactly y = (E - mu)/T.  A
    number-changing process drives mu to 0 (chemical equilibrium, Sec. 5D)."""
    g = problem.grid
    q = (np.geomspace(g.q_min, g.q_max, g.n) if g.log_spaced else np.linspace(g.q_min, g.q_max, g.n))
    a = 1.0 if problem.expansion is None else problem.expansion.a0 * np.sqrt(t / problem.expansion.t0)
    out = []
    for s, sp in enumerate(problem.species):
        eta = {0: 0.0, 1: 1.0, 2: -1.0}[sp.stat]
        if sp.mass_table is not None:
            m = float(np.interp(t, [k[0] for k in sp.mass_table], [k[1] for k in sp.mass_table]))
        else:
            m = sp.mass0 + sp.mass1 * t
        fs = np.asarray(f[s], dtype=np.float64)
        ok = fs > 1e-12
        E = np.sqrt((q[ok] / a) ** 2 + m * m)
        y = np.log(1.0 / fs[ok] + eta)
        slope, icpt = np.polyfit(E, y, 1)
        out.append((1.0 / slope, -icpt / slope))
    return out


def run(problem, f0, steps, every, precision=1, method="heun", t0=1.0, dt=1.0, autotune=True):
    """Evolve log f from f0 for ``steps`` steps (dt requested per step,
    bounded by Eq. (16)); returns a dict of histories: t, n[S], rho[S],
    the fitted temperature and chemical potential of every species, the
    widths of App. C and the final log f."""
    import torch

    from . import Collision
    col = Collision(problem, precision)
    try:
        f = torch.tensor(np.asarray(f0, dtype=np.float64), device="cuda").contiguous()
        if autotune:
            col.autotune(f, t0)
        logf = torch.log(f).contiguous()
        t = torch.tensor([t0], dtype=torch.float64, device="cuda")
        dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        hist = {"t": [], "n": [], "rho": [], "width": [], "step": [], "T": [], "mu": []}

        def record(k):
            n, rho = col.moments(torch.exp(logf), float(t.item()))
            fit = equilibrium_fit(problem, torch.exp(logf).cpu().numpy(), float(t.item()))
            hist["T"].append([x[0] for x in fit])
            hist["mu"].append([x[1] for x in fit])
            hist["t"].append(float(t.item()))
            hist["n"].append(n.cpu().numpy().tolist())
            hist["rho"].append(rho.cpu().numpy().tolist())
            hist["width"].append(col.widths()[0].tolist())
            hist["step"].append(k)

        record(0)
        logf0 = logf.clone()
        done = 0
        while done < steps:
            k = min(every, steps - done)
            col.evolve(logf, t, dtt, k, dt, method)
            done += k
            record(done)
        col.check()
        hist["logf"] = logf.cpu().numpy().tolist()
        # how far the distribution moved: conservation is only informative when it did
        hist["max_abs_dlogf"] = float((logf - logf0).abs().max().item())
        n = np.array(hist["n"])
        rho = np.array(hist["rho"])
        hist["max_rel_change_n"] = (np.max(np.abs(n / n[0] - 1.0), axis=0)).tolist()
        hist["max_rel_change_rho"] = (np.max(np.abs(rho / rho[0] - 1.0), axis=0)).tolist()
        hist["final_rel_change_n"] = (n[-1] / n[0] - 1.0).tolist()
        hist["final_rel_change_rho"] = (rho[-1] / rho[0] - 1.0).tolist()
        return hist
    finally:
        col.close()


def main(argv=None):
    import workloads as W
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c2_bose_2to2", choices=sorted(W.WORKLOADS))
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--dt", type=float, default=1.0, help="requested step (bounded by Eq. (16))")
    ap.add_argument("--t0", type=float, default=1.0)
    ap.add_argument("--method", default="heun", choices=["heun", "euler"])
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="grid points (default: the workload's)")
    ap.add_argument("--neval", type=int, default=None, help="samples per task per iteration")
    ap.add_argument("--nitn", type=int, default=None, help="VEGAS iterations per evaluation")
    ap.add_argument("--sides", type=int, default=0, choices=[0, 1, 2],
                    help="side integrals of every process: 0 all, 1 observed leg initial, 2 final")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    kw = {k: v for k, v in (("n", args.n), ("neval", args.neval), ("nitn", args.nitn)) if v is not None}
    prob, f0 = W.WORKLOADS[args.workload](**kw)
    if args.sides:
        from dataclasses import replace
        prob = replace(prob, processes=tuple(replace(p, sides=args.sides) for p in prob.processes))
    hist = run(prob, f0, args.steps, args.every, W.PREC_FP64 if args.fp64 else W.PREC_FP32, args.method,
               args.t0, args.dt)
    summary = {k: v for k, v in hist.items() if k != "logf"}
    text = json.dumps(summary)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")
    print(json.dumps({k: hist[k] for k in ("max_rel_change_n", "max_rel_change_rho", "final_rel_change_n",
                                           "final_rel_change_rho", "max_abs_dlogf")}
                     | {"t_final": hist["t"][-1], "T_final": hist["T"][-1], "mu_final": hist["mu"][-1]}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
