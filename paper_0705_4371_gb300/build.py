"""Build liblbm.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc and linked into one
shared library next to this file.  Nothing here needs a GPU.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ROOT = os.path.dirname(HERE)
HEADERS = [os.path.join(ROOT, "include", "lbm.h")]

SOURCES = ["lbm_kernels_f64.cu", "lbm_kernels_f32.cu", "lbm_kernels_f16.cu", "lbm_kernels_f32p.cu",
           "lbm_energy_f64.cu", "lbm_energy_f32.cu", "lbm_energy_f16.cu", "lbm_energy_f32p.cu",
           "lbm_api.cu", "lbm_noalloc.cu", "lbm_mlp.cu",
           "lbm_batch.cu", "lbm_batch_f64.cu", "lbm_batch_f32.cu", "lbm_batch_f16.cu",
           "lbm_batch_f32p.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false (device) and -ffp-contract=off (host): no automatic multiply-add
# contraction; the code writes its fused multiply-adds explicitly, so every
# kernel, and the host's FP64 boundary values, round the same way on every
# machine.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-fmad=false"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + HEADERS
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [NVCC] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
