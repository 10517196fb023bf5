"""Checkpoint / resume of an evolution (the paper's Sec. 3F keeps f, the
grids and the integrator states in one file; here: an .npz with the
distribution, time, step and the library's state blob)."""
import numpy as np


def save(path, col, logf, t, dt, **extra):
    """Write log f, t, dt (device tensors) and the context state to `path`."""
    np.savez(path, logf=logf.detach().cpu().numpy(), t=t.detach().cpu().numpy(), dt=dt.detach().cpu().numpy(),
             state=np.frombuffer(col.save_state(), dtype=np.uint8), **extra)


def load(path, col, device="cuda"):
    """Restore the context state from `path`; returns (logf, t, dt) on `device`."""
    import torch
    z = np.load(path)
    col.load_state(z["state"].tobytes())
    to = lambda a: torch.tensor(a, dtype=torch.float64, device=device).contiguous()
    return to(z["logf"]), to(z["t"]), to(z["dt"])
