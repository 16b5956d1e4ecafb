"""Build the gbfmm CUDA library in-tree for sm_103a.

Steps: generate the swap-matrix table (``csrc/gen_swap.py``), compile every
``csrc/*.cu`` translation unit in parallel with nvcc, link
``_lib/libgbfmm.so``. The translation units that evaluate the tree geometry,
the MAC and the scalar-force estimate are compiled with -fmad=false.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
GEN = os.path.join(LIBDIR, "gen")
LIB = os.path.join(LIBDIR, "libgbfmm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NO_FMA = {"tree.cu", "walk.cu", "noalloc.cu", "timestep.cu", "hold.cu"}
# FP32 kernels flush denormals: the hat scale floor keeps every coefficient
# that matters far above the denormal range
FTZ = {"p2p.cu", "m2l.cu"}
M2L32_ORDERS = [4, 6, 8, 10, 12, 14]  # orders of the FP32 register M2L kernel
EXTRA_FLAGS = os.environ.get("GBFMM_NVCC_FLAGS", "").split()  # extra nvcc flags for experiments
SOURCES = ["api.cu", "sort.cu", "tree.cu", "walk.cu", "expansions.cu", "m2l.cu", "translate.cu", "p2p.cu", "noalloc.cu",
           "timestep.cu", "hold.cu", "peaks.cu"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs_digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/gbfmm.h", "../build_lib.py"]:
        path = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(path):
            with open(path, "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(GEN, exist_ok=True)
    stamp = os.path.join(LIBDIR, "stamp")
    digest = _inputs_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return LIB
    table = os.path.join(GEN, "swap_table.inc")
    with open(table + ".tmp", "w") as fh:
        subprocess.run([sys.executable, os.path.join(CSRC, "gen_swap.py")], stdout=fh, check=True)
    os.replace(table + ".tmp", table)
    m2l_gen = os.path.join(GEN, "m2l_gen.inc")
    with open(m2l_gen + ".tmp", "w") as fh:
        subprocess.run([sys.executable, os.path.join(CSRC, "gen_m2l.py")] + [str(p) for p in M2L32_ORDERS],
                       stdout=fh, check=True)
    os.replace(m2l_gen + ".tmp", m2l_gen)
    common = ARCH + EXTRA_FLAGS + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-I", os.path.join(ROOT, "include"), "-I", GEN, "-I", CSRC]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(LIBDIR, src.replace(".cu", ".o"))
        flags = list(common) + (["-fmad=false"] if src in NO_FMA else []) + (["-ftz=true"] if src in FTZ else [])
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for obj, err in results:
            print(os.path.basename(obj), err)
    objs = [o for o, _ in results]
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([nvcc(), "-shared", "-o", tmp] + objs + ARCH, check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
