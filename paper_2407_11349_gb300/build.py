"""Build libhawkes.so (sm_103a) in-tree: paper_2407_11349_gb300/lib/libhawkes.so.

nvcc compiles each CUDA translation unit in parallel for
``-gencode arch=compute_103a,code=sm_103a``; the shared library links the CUDA
runtime statically so it loads next to any PyTorch build.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libhawkes.so")
LIB_DEBUG = os.path.join(LIBDIR, "libhawkes_debug.so")  # -DHAWKES_DEBUG: device index checks
SOURCES = ["sweep.cu", "sweep_bgt.cu", "sweep_ll.cu", "sweep_spatial.cu", "sweep_group.cu", "api.cu", "kernels.cu",
           "batch.cu", "mlp.cu", "noalloc.cu", "tune_cache.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhawkes")


def _flags(verbose, debug=False):
    f = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
         "--expt-relaxed-constexpr"]
    if debug:
        f += ["-DHAWKES_DEBUG"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "hawkes.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, debug=False):
    """Compile (if sources changed) and return the path of libhawkes.so, or of
    libhawkes_debug.so (device index checks, HAWKES_DEBUG) with debug=True."""
    lib = LIB_DEBUG if debug else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = os.path.join(LIBDIR, "obj_debug" if debug else "obj")
    os.makedirs(tmp, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(tmp, src.replace(".cu", ".o"))
        cmd = [cc, *_flags(verbose, debug), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    out = lib + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "static", "-o", out,
                        *[o for o, _ in results]], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(out, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
