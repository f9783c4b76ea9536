"""Build libdfmm.so in-tree with nvcc for sm_103a (one nvcc per translation
unit, in parallel, then one link)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdfmm.so")

SOURCES = ["sort.cu", "tree.cu", "operators.cu", "apply.cu", "apply64.cu", "skeleton_gpu.cu", "validate.cu", "m2l_tc.cu", "m2l_cx.cu", "noalloc.cu", "probes.cu", "skeleton.cpp", "dfmm.cpp",
           "serve.cpp", "solve.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _flags(src: str) -> list[str]:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if os.environ.get("DFMM_CHECK") == "1":   # bounds-checking build: dfmm_plan validates every plan
        f += ["-DDFMM_CHECK"]
    if src.endswith(".cu"):
        f += ARCH + ["--expt-relaxed-constexpr", "-Xptxas", "-v"] if os.environ.get("DFMM_PTXAS_V") else ARCH
        if src == "apply.cu":
            # FP32 kernels whose values never come near the denormal range: the
            # special-function approximations (rsqrt, sin, cos) skip the
            # subnormal-input handling
            f += ["-ftz=true"]
    else:
        # host code: no FMA contraction, so the skeleton arithmetic is reproducible
        f += ["-x", "cu", "-Xcompiler", "-ffp-contract=off"] + ARCH
    return f


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    objs = []
    cmds = []
    for s in srcs:
        o = os.path.join(BUILD, s + (".check" if os.environ.get("DFMM_CHECK") == "1" else "") + ".o")
        objs.append(o)
        src = os.path.join(CSRC, s)
        deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")]
        deps.append(os.path.join(INCLUDE, "dfmm.h"))
        if os.path.exists(o) and all(os.path.getmtime(o) >= os.path.getmtime(d) for d in deps):
            continue
        cmds.append([nvcc(), "-c", src, "-o", o] + _flags(s))
    errs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(cmds)))) as ex:
        for cmd, res in zip(cmds, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds)):
            if verbose or res.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
            if res.returncode != 0:
                errs.append(cmd[2])
    if errs:
        raise RuntimeError("nvcc failed for: " + ", ".join(errs))
    # the objects of the last link (the bounds-checking build links other objects)
    stamp = os.path.join(BUILD, "libdfmm.objs")
    linked = open(stamp).read() if os.path.exists(stamp) else ""
    if cmds or not os.path.exists(LIB) or linked != "\n".join(objs) or \
            any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        link = [nvcc(), "-shared", "-o", LIB] + objs + ARCH + ["-lcublas", "-lcudart"]
        res = subprocess.run(link, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n" + res.stdout + res.stderr)
        with open(stamp, "w") as fh:
            fh.write("\n".join(objs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
