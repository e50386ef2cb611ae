"""Build libgdg.so in-tree for sm_103a (nvcc + g++, no cmake).

Usage: python -m paper_2105_01722_gb300.build [--checks]   (or __graft_entry__.build())
--checks builds libgdg_checks.so, the same sources with the trap-free index
checks compiled in (-DGDG_CHECKS=1, gdg_checks.cuh); the binding loads it
instead of libgdg.so when the environment has GDG_CHECKS=1.
"""
import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "libgdg.so")
OUT_CHECKS = os.path.join(PKG, "libgdg_checks.so")
BUILD = os.path.join(PKG, "_build", platform.machine())
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(cand, "bin", "nvcc") if cand else ""
        if p and os.path.exists(p):
            return p
    p = shutil.which("nvcc")
    if not p:
        raise RuntimeError("nvcc not found")
    return p


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _compile(src, nvcc, build_dir=BUILD, defines=()):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(
            os.path.getmtime(src), *(os.path.getmtime(os.path.join(CSRC, h)) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))),
            os.path.getmtime(os.path.join(ROOT, "include", "gdg.h"))):
        return obj
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *defines,
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj


def build(verbose=True, checks=False):
    nvcc = nvcc_path()
    build_dir = BUILD + ("_checks" if checks else "")
    out = OUT_CHECKS if checks else OUT
    defines = ("-DGDG_CHECKS=1",) if checks else ()
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, build_dir, defines), srcs))
    cmd = [nvcc, *ARCH, "-shared", "-o", out, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    if verbose:
        print("built", out)
    return out


if __name__ == "__main__":
    build(checks="--checks" in sys.argv[1:])
    sys.exit(0)
