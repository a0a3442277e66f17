"""Build libygm.so in-tree for sm_103a (nvcc, parallel compile of the three translation units)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libygm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libygm.so")


def build(verbose=False, force=False):
    srcs = [os.path.join(CSRC, f) for f in ("builder.cpp", "ygm.cu", "yee.cu", "builder.h")]
    srcs.append(os.path.join(os.path.dirname(HERE), "include", "ygm.h"))
    if not force and os.path.exists(OUT) and all(os.path.getmtime(OUT) >= os.path.getmtime(s) for s in srcs):
        return OUT
    nvcc = _nvcc()
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-pthread", "-lineinfo"]
    jobs = [
        [nvcc, "-x", "c++", *common, "-c", os.path.join(CSRC, "builder.cpp"), "-o", os.path.join(bdir, "builder.o")],
        [nvcc, *ARCH, *common, "-Xptxas", "-O3", "-c", os.path.join(CSRC, "ygm.cu"), "-o", os.path.join(bdir, "ygm.o")],
        [nvcc, *ARCH, *common, "-Xptxas", "-O3", "-c", os.path.join(CSRC, "yee.cu"), "-o", os.path.join(bdir, "yee.o")],
    ]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with ThreadPoolExecutor(3) as ex:
        list(ex.map(run, jobs))
    tmp = OUT + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, os.path.join(bdir, "builder.o"), os.path.join(bdir, "ygm.o"),
         os.path.join(bdir, "yee.o"),
         "-Xcompiler", "-pthread"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
