"""Build the CUDA library libceleris_gb.so in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libceleris_gb.so")
SOURCES = ["celeris_kernels.cu", "celeris_api.cu", "celeris_render.cu", "celeris_adjoint.cu"]
# the renderer's bytes must not depend on fast-math choices: IEEE division and
# square root, no contraction into FMA, denormals kept (its arithmetic also
# spells out each rounding)
SOURCE_FLAGS = {"celeris_render.cu": ["-ftz=false", "-prec-div=true", "-prec-sqrt=true", "-fmad=false"]}
HEADERS = [os.path.join(CSRC, "celeris_internal.cuh"), os.path.join(CSRC, "celeris_physics.cuh"),
           os.path.join(CSRC, "celeris_adjoint.cuh"),
           os.path.join(INCLUDE, "celeris_gb.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 division and square root use the fast reciprocal / reciprocal-square-root
# paths (about 2 ulp); FP64 arithmetic is unaffected by these flags.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
         "-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile both translation units in parallel, then link the shared library."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        nvcc = _nvcc()
        procs, objs = [], []
        for src in SOURCES:
            obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
            objs.append(obj)
            flags = [f for f in FLAGS if not any(f.split("=")[0] == o.split("=")[0] for o in SOURCE_FLAGS.get(src, []))]
            cmd = [nvcc, *ARCH, *flags, *SOURCE_FLAGS.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode != 0:
                sys.stderr.write(out.decode(errors="replace"))
            if p.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
