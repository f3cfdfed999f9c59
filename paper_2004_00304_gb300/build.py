"""Build liblbmpcd.so in-tree with nvcc for sm_103a (no torch extension machinery).

Each translation unit is compiled in parallel.  Particle streaming and
binning spell out their binary64 operations with non-contractible
intrinsics, so no translation unit needs -fmad=false.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbmpcd.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                 "-Xptxas", "-warn-spills"]
SOURCES = {
    "lbmpcd_api.cu": [],
    "lb.cu": [],
    "mpcd.cu": [],
    "closure.cu": [],
    "closure_coupling.cu": [],
}
HEADERS = ["common.cuh", "kernels.h", "tc_gemm.cuh", "net_fused.cuh", "lb_core.cuh", "cell_core.cuh"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "lbmpcd.h")]
    jobs = []
    objs = []
    for src, extra in SOURCES.items():
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc] + COMMON + extra + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64") if os.path.isabs(nvcc) else ""
        rpath = ["-Xlinker", "-rpath=" + cuda_lib] if cuda_lib else []
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"] + rpath)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
