"""Build libfe_ks.so in-tree with nvcc for sm_103a (no CMake).

The translation units compile in parallel: the C-ABI / setup, the host 1D
tables, the nonlocal kernels, and one object per FE degree of the fused local
kernel (and per quadrature order n_q = n_p, n_p + 2).  Objects go to ``_build/`` beside this file; the shared library to
``libfe_ks.so``.  A rebuild happens only when a source is newer than the
library.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfe_ks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
DEGREES = range(1, 9)
NQ_OFFSETS = (0, 2)   # n_q - n_p
BATCH_THREADS = (256, 384, 512, 672)   # block sizes of the batched persistent kernel


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfe_ks.so")
    return cand


def _units():
    units = []
    for name in ("fe_ks_api.cu", "fe_ks_tables.cu", "fe_ks_nonlocal.cu", "fe_ks_probe.cu", "fe_ks_cheb.cu", "fe_ks_static.cu", "fe_ks_batched.cu", "fe_ks_gemm.cu", "fe_ks_ffgemm.cu", "fe_ks_tc.cu", "fe_ks_cm.cu", "fe_ks_rr.cu", "fe_ks_tcgram.cu", "fe_ks_tc5.cu"):
        units.append((os.path.join(CSRC, name), os.path.join(BUILD, name + ".o"), []))
    for nt in BATCH_THREADS:
        units.append((os.path.join(CSRC, "fe_ks_batched_k.cu"),
                      os.path.join(BUILD, f"fe_ks_batched_k{nt}.o"), [f"-DFEKS_BNT={nt}"]))
    for p in DEGREES:
        for nqx in NQ_OFFSETS:
            units.append((os.path.join(CSRC, "fe_ks_local_deg.cu"),
                          os.path.join(BUILD, f"fe_ks_local_p{p}_q{nqx}.o"), [f"-DFEKS_P={p}", f"-DFEKS_NQX={nqx}"]))
    return units


def _sources():
    out = []
    for root in (CSRC, INCLUDE):
        for f in os.listdir(root):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(root, f))
    return out


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False, jobs=None):
    """Compile every CUDA unit for sm_103a and link libfe_ks.so; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(u):
        src, obj, extra = u
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    jobs = jobs or max(1, min(len(_units()), os.cpu_count() or 1))
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, _units()))
    tmp = LIB + ".tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcublas", "-lcusolver", "-Xlinker", "-rpath", "-Xlinker", cuda_lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
