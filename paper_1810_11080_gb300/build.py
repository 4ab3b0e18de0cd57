"""Build libsnsweep.so in-tree for sm_103a (nvcc for the CUDA units, g++ for host C++).

graph.cu is compiled with -fmad=false and the host C++ with -ffp-contract=off: the graph
stage reproduces a fixed operation order bit for bit.  The other CUDA units may contract
multiply-adds.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsnsweep.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose=False, extra_nvcc=()):
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    common = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-lineinfo", "-I", os.path.join(ROOT, "include")] + ARCH
    cu = {
        "geom.cu": [],
        "graph.cu": ["-fmad=false"],
        "scc.cu": ["-fmad=false"],
        "dsa.cu": [],
        "sweep.cu": [],
        "sweep_inv.cu": [],
        "noalloc.cu": [],
        "batch.cu": [],
        "mlp.cu": [],
    }
    cpp = ["api.cpp", "batch_api.cpp", "predictor.cpp", "tables.cpp", "quadrature.cpp"]
    jobs = []
    for src, flags in cu.items():
        obj = os.path.join(BUILD, src + ".o")
        jobs.append([nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + common + flags + list(extra_nvcc))
    for src in cpp:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(["g++", "-c", os.path.join(CSRC, src), "-o", obj, "-std=c++17", "-O2", "-fPIC",
                     "-ffp-contract=off", "-I", os.path.join(cuda, "include"), "-I", os.path.join(ROOT, "include")])
    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, s + ".o") for s in list(cu) + cpp]
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-Xlinker",
                                                       "-rpath=" + os.path.join(cuda, "lib64")])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(LIB)
