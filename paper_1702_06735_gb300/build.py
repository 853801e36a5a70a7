"""Builds the CUDA library libtdmix.so in-tree for sm_103a.

Steps: compile the model compiler as a host tool (shapegen), generate the
header of compile-time model structures from the shipped amplitude-model
files, then compile the kernels and the C ABI with nvcc (translation units in
parallel) and link one shared library next to this file.
Run:  python -m paper_1702_06735_gb300.build  [--verbose]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
MODELS = os.path.join(HERE, "amplitude_models")
LIB = os.path.join(HERE, "libtdmix.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd, verbose=False):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout, r.stderr, flush=True)
    return r


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    gen = os.path.join(BUILD, "shapegen")
    _run(["g++", "-O1", "-std=c++17", "-o", gen, os.path.join(CSRC, "shapegen.cpp"),
          os.path.join(CSRC, "model.cpp"), os.path.join(CSRC, "json.cpp")], verbose)
    models = sorted(glob.glob(os.path.join(MODELS, "*.json")))
    _run([gen, os.path.join(BUILD, "shapes_gen.h")] + models, verbose)

    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-I", CSRC, "-I", BUILD, "-I", INCLUDE]
    if ptxas_info:
        common += ["-Xptxas", "-v"]
    units = [
        ("kernels.cu", "kernels.o", []),
        ("eval_inst.cu", "eval_f64.o", ["-DTDMIX_PREC_F32=0"]),
        ("eval_inst.cu", "eval_f32.o", ["-DTDMIX_PREC_F32=1"]),
        ("capi.cu", "capi.o", []),
        ("noalloc.cu", "noalloc.o", []),
        ("generic.cu", "generic.o", []),
        ("selftest.cu", "selftest.o", []),
        ("serve.cu", "serve.o", []),
        ("model.cpp", "model.o", []),
        ("json.cpp", "json.o", []),
    ]

    def compile_one(u):
        src, obj, extra = u
        out = os.path.join(BUILD, obj)
        cmd = [nvcc] + common + extra + ["-c", os.path.join(CSRC, src), "-o", out]
        return _run(cmd, verbose), out

    objs = []
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        for r, out in ex.map(compile_one, units):
            objs.append(out)
            if ptxas_info:
                sys.stdout.write(r.stderr)
    tmp = LIB + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, verbose)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="--verbose" in sys.argv, ptxas_info="--ptxas" in sys.argv))
