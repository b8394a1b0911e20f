"""Build the CUDA library libfem_b300.so in-tree (nvcc, sm_103a).

    python paper_2103_16747_b300/build.py [-v] [--checked]    (or build() from Python)

Run it by path: importing the package loads the library this script builds.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfem_b300.so")
LIB_CHECKED = os.path.join(HERE, "libfem_b300_checked.so")   # FEM_CHECKED: bounds- and NaN-checked kernels
SOURCES = ["fem_solve.cu", "fem_stress.cu", "fem_api.cpp", "fem_batch.cpp", "fem_server.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(verbose: bool = False, force: bool = False, extra=(), checked: bool = False) -> str:
    """Build the production library, or with checked=True the FEM_CHECKED
    variant (same sources, every kernel index bounded and element values
    NaN-checked; selected at import with FEM_B300_CHECKED=1)."""
    lib = LIB_CHECKED if checked else LIB
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "fem.h"))
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib
    cmd = [nvcc(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "include"), "-o", lib + ".tmp", *srcs, "-cudart=static", "-Xcompiler", "-pthread",
           *(["-DFEM_CHECKED"] if checked else []), *extra]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True, checked="--checked" in sys.argv))
