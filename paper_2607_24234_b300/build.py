"""Build libqs.so (the sm_103a CUDA library) in-tree with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "libqs.so")
SRCS = [os.path.join(HERE, "csrc", "qs_runtime.cu"), os.path.join(HERE, "csrc", "qs_noalloc.cu"),
        os.path.join(HERE, "csrc", "qs_probe.cu"),
        os.path.join(HERE, "csrc", "qs_mlp.cu"),
        os.path.join(HERE, "csrc", "qs_real2.cu")]
DEPS = SRCS + [os.path.join(HERE, "csrc", f) for f in ("qs_kernels.cuh", "qs_resident.cuh", "qs_tune.inc", "qs_green.inc", "qs_surdata.inc")] + \
    [os.path.join(ROOT, "include", "qs.h"), os.path.abspath(__file__)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_cmd(out: str, extra=()):
    return ["nvcc", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-shared",
            "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
            "-I", os.path.join(HERE, "csrc"), *extra, *SRCS, "-o", out, "-cudart", "static"]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(SO):
        t = os.path.getmtime(SO)
        if all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d)):
            return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = nvcc_cmd(tmp, ("-Xptxas", "-v") if verbose else ())
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(SO)
