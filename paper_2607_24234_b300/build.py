"""Build the sm_103a CUDA library in-tree with nvcc: libqs.so, and the
bounds-checked variant libqs_checked.so (-DQS_CHECK_BOUNDS).  Every source
is compiled to an object in parallel, then each variant is linked."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "libqs.so")
SO_CHECKED = os.path.join(HERE, "libqs_checked.so")
OBJ = os.path.join(HERE, "_build")
SRCS = [os.path.join(HERE, "csrc", f) for f in
        ("qs_runtime.cu", "qs_noalloc.cu", "qs_probe.cu", "qs_mlp.cu", "qs_real2.cu")]
DEPS = SRCS + [os.path.join(HERE, "csrc", f) for f in ("qs_kernels.cuh", "qs_resident.cuh", "qs_problem.h", "qs_nvtx.h",
                                                       "qs_tune.inc", "qs_green.inc", "qs_surdata.inc")] + \
    [os.path.join(ROOT, "include", "qs.h"), os.path.abspath(__file__)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
VARIANTS = {SO: (), SO_CHECKED: ("-DQS_CHECK_BOUNDS",)}


def compile_cmd(src: str, obj: str, extra=()):
    return ["nvcc", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-c", "-Xcompiler", "-fPIC,-ffp-contract=off",
            "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc"), *extra, src, "-o", obj]


def link_cmd(objs, out: str):
    return ["nvcc", "-shared", *ARCH, *objs, "-o", out, "-cudart", "static"]


def source_hash() -> str:
    """Hash of every source the library is built from (written beside each
    built library; the binding refuses a library whose sources changed)."""
    import hashlib
    h = hashlib.sha256()
    for d in DEPS[:-1]:   # the sources and headers (not this script)
        with open(d, "rb") as f:
            h.update(os.path.basename(d).encode() + b"\0" + f.read())
    return h.hexdigest()


def _fresh(target: str) -> bool:
    if not os.path.exists(target) or not os.path.exists(target + ".srchash"):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    todo = [so for so in VARIANTS if force or not _fresh(so)]
    if not todo:
        return SO
    os.makedirs(OBJ, exist_ok=True)
    jobs = []
    for so in todo:
        tag = os.path.splitext(os.path.basename(so))[0]
        for src in SRCS:
            obj = os.path.join(OBJ, f"{tag}_{os.path.splitext(os.path.basename(src))[0]}.o")
            extra = VARIANTS[so] + (("-Xptxas", "-v") if verbose and so == SO else ())
            jobs.append((so, obj, compile_cmd(src, obj, extra)))
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(subprocess.check_call, cmd) for _, _, cmd in jobs]:
            f.result()
    digest = source_hash()
    for so in todo:
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(link_cmd([o for s, o, _ in jobs if s == so], tmp))
        os.replace(tmp, so)
        with open(so + ".srchash", "w") as f:
            f.write(digest + "\n")
    return SO


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(SO, SO_CHECKED)
