"""Builds libgsr.so (the CUDA kernels and the C ABI of include/gsr.h) in-tree
for sm_103a with nvcc.  Run `python -m paper_2411_17660_b300.build`; with
`--checked` it builds libgsr_checked.so instead, the same library with the
device-side index checks of GSR_CHECKED compiled in."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libgsr.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libgsr_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v", f"-I{INCLUDE}"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(args) -> tuple:
    src, checked = args
    obj_dir = os.path.join(OUT_DIR, "checked") if checked else OUT_DIR
    obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *(["-DGSR_CHECKED"] if checked else []), "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, p.returncode, p.stdout + p.stderr


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles every csrc/*.cu for sm_103a and links libgsr.so (or, checked,
    libgsr_checked.so); returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(checked):
        return lib
    os.makedirs(os.path.join(OUT_DIR, "checked") if checked else OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_compile, [(s, checked) for s in _sources()]))
    logs = []
    for src, obj, rc, log in results:
        logs.append(f"== {os.path.basename(src)}\n{log}")
        if rc != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{log}")
    if not checked:
        with open(os.path.join(OUT_DIR, "ptxas.log"), "w") as f:
            f.write("\n".join(logs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp] + [r[1] for r in results]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}{p.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("\n".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
