"""The C-ABI library builds for sm_103a, loads, exports every entry point the
header declares, and its structs have the layout the binding assumes.  No
compute calls: these run without a GPU."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "best.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2603_28848_gb300 import build, _lib
    build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(best_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("best_collision_init", "best_collision_eval", "best_step_euler",
                     "best_step_heun", "best_collision_destroy", "best_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2603_28848_gb300 import _lib
    nm = shutil.which("nm")
    names = declared_functions()
    if nm:
        out = subprocess.run([nm, "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
        exported = set(re.findall(r"\bT (best_[a-z0-9_]+)", out))
        assert set(names) <= exported, set(names) - exported
    for n in names:
        assert hasattr(lib, n)
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_struct_layout_matches_c(tmp_path):
    """Compile a C program against the header and compare sizes and offsets
    with the ctypes declarations."""
    from paper_2603_28848_gb300 import _lib
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc missing")
    fields = {
        "best_grid": ["n", "log_spaced", "q_min", "q_max"],
        "best_species": ["stat", "n_mass_knots", "mass0", "mass1", "mass_t", "mass_m"],
        "best_process": ["n_in", "n_out", "species", "coupling", "sigma_E", "neval", "neval_per_point",
                         "nitn", "nbins", "alpha", "width_mode", "width", "width_rel_lo", "width_rel_hi",
                         "width_factor", "width_min", "width_max", "strat", "strat_max_hcubes", "strat_beta",
                         "me_coef", "budget", "sides", "neval_min", "neval_max"],
        "best_config": ["grid", "n_species", "n_processes", "species", "processes", "precision",
                        "tail_points", "seed", "e_cut", "expansion", "a0", "t0", "eps_dt", "point_lo",
                        "point_hi"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in out:
        if not line:
            continue
        st, f, v = line.split()
        cls = getattr(_lib, st)
        want = ctypes.sizeof(cls) if f == "size" else getattr(cls, f).offset
        assert int(v) == want, (st, f)


def test_build_targets_sm103a():
    from paper_2603_28848_gb300 import buildlib as b
    assert "arch=compute_103a,code=sm_103a" in b.ARCH


def test_binding_rejects_tensors_the_library_cannot_take():
    """Device pointers go to the library unchecked, so the binding refuses
    host tensors, other dtypes, wrong sizes and non-scalar step times before
    any call (checked here without a GPU: every CPU tensor is refused)."""
    import torch
    from paper_2603_28848_gb300 import BestError, _require, _require_opt, _require_time
    with pytest.raises(BestError):
        _require(torch.zeros(4, dtype=torch.float64), 4, "f")
    with pytest.raises(BestError):
        _require(np.zeros(4), 4, "f")
    with pytest.raises(BestError):
        _require_time(torch.zeros(1, dtype=torch.float64), torch.zeros(1, dtype=torch.float64))
    with pytest.raises(BestError):
        _require_opt(torch.zeros(4, dtype=torch.float32), 4, "C")
    _require_opt(None, 4, "C")                       # None: the library's own buffer
