"""Build libnufft.so in-tree from csrc/ with nvcc (sm_103a), in parallel.

    python -m paper_1701_04492_gb300.build          # incremental
    python -m paper_1701_04492_gb300.build --force

Objects go to paper_1701_04492_gb300/_build/, the library to
paper_1701_04492_gb300/libnufft.so.  Each translation unit is rebuilt when it or
any header in csrc/ (or include/) is newer than its object.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libnufft.so")
# the checked variant: every data-dependent index checked, a failure recorded in the
# error word (NUFFT_ECHECK from nufft2_check) and the access skipped
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(PKG, "libnufft_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnufft.so")
    return exe


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(CSRC, "*.inc")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def sources():
    """Translation units, the slowest to compile (the FP32 row and batched passes) first."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    order = ("inst_rows_f32", "inst_many_f32", "inst_cols_f32", "inst_many_cols", "inst_rows_f64")

    def rank(path):
        name = os.path.basename(path)
        return next((i for i, pre in enumerate(order) if name.startswith(pre)), len(order))
    return sorted(srcs, key=rank)


def _compile(src, force, hdr_mtime, bdir=BUILD, extra=()):
    obj = os.path.join(bdir, os.path.basename(src) + ".o")
    if not force and os.path.exists(obj):
        if os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_mtime):
            return obj, False
    cmd = [_nvcc()] + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-x", "c++",
               "-I" + os.path.join(ROOT, "include"), "-c", src, "-o", obj + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), res.stdout, res.stderr))
    os.replace(obj + ".tmp", obj)
    return obj, True


def _stamp_ok(bdir=BUILD):
    """Objects are only reused on the machine type that built them."""
    stamp = os.path.join(bdir, "machine")
    me = platform.machine()
    ok = os.path.exists(stamp) and open(stamp).read().strip() == me
    if not ok:
        with open(stamp, "w") as fh:
            fh.write(me)
    return ok


def build(force=False, jobs=None, verbose=False, check=False):
    """Compile every translation unit of csrc/ and link libnufft.so.  Returns its path.

    check=True builds the checked variant instead (libnufft_check.so, objects in their
    own folder, -DNUFFT_CHECK): same entry points, every data-dependent index tested."""
    bdir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    extra = ["-DNUFFT_CHECK"] if check else []
    os.makedirs(bdir, exist_ok=True)
    if not _stamp_ok(bdir):
        force = True
    srcs = sources()
    hdr_mtime = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    jobs = jobs or max(1, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, force, hdr_mtime, bdir, extra), srcs))
    objs = [o for o, _ in results]
    rebuilt = any(r for _, r in results)
    if rebuilt or force or not os.path.exists(lib) or \
            os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".%d.tmp" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed: %s\n%s" % (res.stdout, res.stderr))
        os.replace(tmp, lib)
        if verbose:
            print("linked", lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv)
