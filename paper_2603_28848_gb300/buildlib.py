"""Builds libbest.so in-tree with nvcc for sm_103a (no torch in the ABI)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libbest.so")
SOURCES = ["api.cu", "kernels.cu", "eval_f32.cu", "eval_f32_n6.cu", "eval_f64.cu", "variants.cu", "vjp.cu", "newton.cu", "noalloc.cu", "eval_strat.cu", "vjp_me.cu", "budget.cu", "eval_f32_b.cu", "eval_f32_n6_b.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def build(verbose=False, force=False, out=None, defines=()):
    """Compile every translation unit (in parallel) and link libbest.so
    (or `out`, with extra -D `defines`, for launch-shape experiments)."""
    lib = out or LIB
    bdir = os.path.join(HERE, "_build") if out is None else out + ".build"
    os.makedirs(bdir, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "best.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *[f"-D{d}" for d in defines], "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
