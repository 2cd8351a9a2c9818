"""Build the fastpod shared library in-tree for sm_103a.

Compiles every CUDA translation unit of ``csrc/`` with nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``) and links them into
``_lib/libfastpod.so``.  Regenerates ``csrc/contract_gen.cuh`` first.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libfastpod.so")
SOURCES = ["pod_api.cu", "neigh.cu", "atom_f32.cu", "atom_f64.cu", "atom_emb_f32.cu", "atom_emb_f64.cu", "gather.cu", "batch.cu", "fit.cu", "static_desc.cu", "peak.cu", "adjoint_f32.cu", "qr.cu", "halo.cu", "model_grad.cu",
           "model_io.cu", "gram_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wno-deprecated-declarations"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the fastpod CUDA library cannot be built")


def _deps_mtime() -> float:
    m = 0.0
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h", ".py")):
            m = max(m, os.path.getmtime(os.path.join(CSRC, f)))
    m = max(m, os.path.getmtime(os.path.join(HERE, "..", "include", "pod.h")))
    return m


def build(force: bool = False, verbose: bool = False) -> str:
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_contract.py"), "4",
                    os.path.join(CSRC, "contract_gen.cuh")], check=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OBJ, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
