"""Build ``libhubhmc.so`` (the C-ABI CUDA library) in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked with the static CUDA
runtime, so the library depends only on the NVIDIA driver.  The output goes to
``paper_1007_3432_gb300/lib/``.  ``build(bounds_check=True)`` builds the debug
variant ``libhubhmc_check.so`` (compiled with ``-DHH_BOUNDS_CHECK``: index
checks that record the first bad index instead of accessing it), which the
binding loads when ``HH_BOUNDS_CHECK=1``.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libhubhmc.so")
LIB_CHECK = os.path.join(LIBDIR, "libhubhmc_check.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), bounds_check: bool = False) -> str:
    lib = LIB_CHECK if bounds_check else LIB
    if not force and up_to_date(lib):
        return lib
    objdir = os.path.join(LIBDIR, "obj_check" if bounds_check else "obj")
    os.makedirs(objdir, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(objdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    flags = FLAGS + (["-DHH_BOUNDS_CHECK"] if bounds_check else [])

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc()] + ARCH + flags + list(extra) + ["-I", INCLUDE, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(compile_one, zip(srcs, objs)))
    failed = [(s, out) for s, rc, out in results if rc != 0]
    for s, rc, out in results:
        if verbose and out.strip():
            sys.stderr.write(out)
    if failed:
        msg = "\n".join("%s:\n%s" % (s, out) for s, out in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                bounds_check="--bounds-check" in sys.argv))
