"""Builds libkns.so in-tree: every csrc/*.cu compiled for sm_103a in parallel, then linked.

No cmake: one nvcc per translation unit, a thread pool, and an mtime check so an
unchanged tree rebuilds nothing.
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
LIB = os.path.join(HERE, "libkns.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC] + ARCH


# Grid configurations (sdf_width, sdf_hidden, pe_pos_L, pe_dir_L) compiled into the library.
# Sources marked "kns:instantiate" are compiled once per configuration.
CONFIGS = [(32, 2, 4, 2), (32, 3, 4, 2), (64, 2, 4, 2), (64, 3, 4, 2),
           (32, 2, 6, 4), (32, 3, 6, 4), (64, 2, 6, 4), (64, 3, 6, 4)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_info: bool = False, jobs: int = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                     + glob.glob(os.path.join(INCLUDE, "*.h")))
    exe = nvcc()
    objs = []
    todo = []
    for s in srcs:
        with open(s) as f:
            inst = "kns:instantiate" in f.read(4096)
        variants = [("_w%dh%dl%dd%d" % c, ["-DKNS_W=%d" % c[0], "-DKNS_H=%d" % c[1], "-DKNS_L=%d" % c[2],
                                             "-DKNS_LD=%d" % c[3]]) for c in CONFIGS] if inst else [("", [])]
        for suffix, defs in variants:
            o = os.path.join(BUILD, os.path.basename(s)[:-3] + suffix + ".o")
            objs.append(o)
            if ptxas_info or _stale(o, [s] + headers + [__file__]):
                cmd = [exe] + NVCC_FLAGS + defs + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", s, "-o", o]
                todo.append(cmd)

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    failed = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for cmd, p in ex.map(run, todo):
                if verbose or ptxas_info or p.returncode:
                    sys.stderr.write(" ".join(cmd) + "\n" + p.stdout + p.stderr)
                if p.returncode:
                    failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    if _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        # export only the C ABI (kns_*): the statically linked CUDA runtime stays private and
        # binds locally, so it cannot interpose on (or be interposed by) another runtime in the process
        vs = os.path.join(BUILD, "exports.map")
        with open(vs, "w") as f:
            f.write("{ global: kns_*; local: *; };\n")
        cmd = [exe, "-shared", "-o", tmp] + objs + ARCH + ["-Xlinker", "--version-script=" + vs]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode:
            raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
