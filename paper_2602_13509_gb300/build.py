"""Build the hsad CUDA library in-tree for sm_103a (GB300).

Compiles every ``csrc/*.cu`` to an object in parallel with nvcc and links
``libhsad.so`` next to this file. Objects go to ``_build/``. Rebuilds only what
changed (source or header newer than its object). Usage::

    python -m paper_2602_13509_gb300.build [--force]
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libhsad.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + CSRC, "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the hsad CUDA library cannot be built")


# Sources compiled more than once, with different macro definitions: the factor kernel,
# once per arithmetic (0 float-float, 1 FP64) and working precision (0..4), so that its
# instances compile in parallel.
VARIANTS = {
    "k_factor_inst.cu": [(f"k_factor_inst_a{a}_p{p}", [f"-DHSAD_FI_AR={a}", f"-DHSAD_FI_PREC={p}"])
                         for a in (0, 1) for p in range(5)],
}


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = _headers()
    cc = nvcc()
    jobs = []
    objs = []
    for s in srcs:
        base = os.path.basename(s)
        for name, defs in VARIANTS.get(base, [(base[:-3], [])]):
            o = os.path.join(BUILD, name + ".o")
            objs.append(o)
            if force or _stale(o, [s] + hdrs):
                jobs.append([cc, *ARCH, *NVCC_FLAGS, *defs, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    # stale objects of sources or variants that no longer exist must not be linked
    for o in glob.glob(os.path.join(BUILD, "*.o")):
        if o not in objs:
            os.remove(o)
    if jobs:
        jobs.sort(key=lambda c: "k_factor_inst" not in c[-3])  # longest first
        with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            list(ex.map(run, jobs))
    if jobs or force or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


GEN_CSRC = os.path.join(os.path.dirname(HERE), "gen", "csrc")
GEN_LIB = os.path.join(os.path.dirname(HERE), "gen", "libhsadgen.so")


def build_gen(force: bool = False) -> str:
    """Synthetic-input generator for large device-resident cubes (gen/csrc -> gen/libhsadgen.so)."""
    srcs = sorted(glob.glob(os.path.join(GEN_CSRC, "*.cu")))
    if not srcs:
        return ""
    if force or _stale(GEN_LIB, srcs):
        tmp = GEN_LIB + ".tmp"
        cmd = [nvcc(), *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, *srcs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        os.replace(tmp, GEN_LIB)
    return GEN_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(build_gen(force="--force" in sys.argv))
