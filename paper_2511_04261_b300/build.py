"""Build libdppix.so in-tree for sm_103a (B300) with nvcc.

The library is plain CUDA C++ with a C ABI (include/dppix.h); it links the CUDA runtime statically and
has no torch dependency.  `build()` is idempotent: it rebuilds only when a source is newer than the
library.
"""
import concurrent.futures
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libdppix.so")
OBJDIR = os.path.join(PKG, "_build")
# the bounds-checked build (DPPIX_CHECKED): same sources, every checked access tested against its buffer
LIB_CHECKED = os.path.join(PKG, "libdppix_checked.so")
OBJDIR_CHECKED = os.path.join(PKG, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles each stale source to an object under _build/ (one nvcc per file, in parallel), then links the
    shared library.  An object is stale when it is older than its source, a header, or this file.  checked:
    the bounds-checked library (objects under _build_checked/, -DDPPIX_CHECKED)."""
    lib_path, objdir = (LIB_CHECKED, OBJDIR_CHECKED) if checked else (LIB, OBJDIR)
    if not force and not _stale(lib_path):
        return lib_path
    nvcc = os.environ.get("NVCC", "nvcc")
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "-I", INCLUDE]
    if checked:
        flags.append("-DDPPIX_CHECKED")
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    os.makedirs(objdir, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]
    newest_header = max(os.path.getmtime(h) for h in headers)
    objs, todo = [], []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or verbose or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_header):
            todo.append((src, obj))
    jobs = max(1, min(len(todo), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as pool:
        futs = [pool.submit(subprocess.run, [nvcc, *flags, "-c", src, "-o", obj + ".tmp"], check=True)
                for src, obj in todo]
        for fut in futs:
            fut.result()
    for _, obj in todo:
        os.replace(obj + ".tmp", obj)
    tmp = lib_path + ".tmp%d" % os.getpid()
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
