"""Build the lbsc C-ABI shared library (CUDA for sm_103a) in-tree.

    python -m paper_0910_3915_gb300.build [--verbose] [--debug-bounds]

Compiles csrc/*.cu in parallel with nvcc into _build/ and links
paper_0910_3915_gb300/liblbsc.so against the shared CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "liblbsc.so")
BUILD = os.path.join(ROOT, "_build", "lbsc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


DEBUG_OUT = os.path.join(PKG, "liblbsc_debug.so")


def build(verbose: bool = False, force: bool = False, debug_bounds: bool = False) -> str:
    """Build liblbsc.so, or with debug_bounds liblbsc_debug.so, whose step
    kernels check every population index (LBSC_DEBUG_BOUNDS)."""
    out_path = DEBUG_OUT if debug_bounds else OUT
    build_dir = BUILD + ("_debug" if debug_bounds else "")
    extra = ["-DLBSC_DEBUG_BOUNDS"] if debug_bounds else []
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    deps.append(os.path.join(ROOT, "include", "lbsc.h"))
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(out_path) and os.path.getmtime(out_path) >= newest:
        return out_path
    cc = nvcc()
    procs, objs = [], []
    for s in srcs:
        o = os.path.join(build_dir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = False
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out)
        failed |= p.returncode != 0
    if failed:
        raise RuntimeError("nvcc failed")
    cudalib = os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")
    tmp = out_path + f".tmp{os.getpid()}"
    subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                    "-Xlinker", f"-rpath,{cudalib}"], check=True)
    os.replace(tmp, out_path)
    return out_path


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, force=True, debug_bounds="--debug-bounds" in sys.argv))
