"""Build the in-tree CUDA library ``libaim.so`` for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared object next to this file.  No cmake, no torch extension machinery.
Usage: ``python -m paper_1010_1456_gb300.build [--force] [--check]`` (or ``build()``).
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libaim.so")
LIB_CHECK = os.path.join(HERE, "libaim_check.so")
SOURCES = ["api.cu", "setup.cu", "setup_dev.cu", "fft.cu", "matvec.cu", "krylov.cu", "rcs.cu", "rcs_ref.cu", "probe.cu", "profile.cu", "noalloc.cu", "autotune.cu", "nearfill.cu", "pack.cu", "fft4_p32.cu",
           "fft4_p64.cu", "fft4_pff.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = [
    "-O3",
    "-std=c++17",
    "--expt-relaxed-constexpr",
    "-lineinfo",
    "-Xcompiler",
    "-fPIC,-ffp-contract=off,-O3",
    "-Xptxas",
    "-O3",
]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def build(verbose=False, force=False, check=False):
    """Compile the library (check=True: the index-checking debug build
    ``libaim_check.so``, compiled with -DAIM_CHECK into its own object folder)."""
    out_dir = OUT_DIR + ("_check" if check else "")
    lib = LIB_CHECK if check else LIB
    flags = FLAGS + (["-DAIM_CHECK"] if check else [])
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "aim.h"))
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _newer([s] + headers, o):
            jobs.append([nvcc(), *ARCH, *flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4) or 1) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _newer(objs, lib):
        run([nvcc(), *ARCH, "-shared", "-o", lib, *objs, "-lpthread"])
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, check="--check" in sys.argv))
