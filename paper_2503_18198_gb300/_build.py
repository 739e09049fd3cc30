"""Compile the CUDA library (csrc/*.cu) for sm_103a into _lib/libspmttkrp.so.

The translation units are compiled in parallel with nvcc, then linked into
one shared library with the C ABI of include/spmttkrp.h.  The library is
built in-tree so that the process loading it can be seen to use it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
SO_NAME = "libspmttkrp.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fno-ipa-icf: no identical-code folding of host functions, so that no two
# kernel launch stubs (one per template instantiation) are ever merged.  (The
# ALS device bodies shared by the batched and single-tensor sweeps write every
# rounding explicitly, so their bits do not depend on FMA contraction.)
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-fno-ipa-icf",
              "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest(extra_flags) -> str:
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(CSRC, "*"))) + [
            os.path.join(ROOT, "include", "spmttkrp.h")]:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra_flags)).encode())
    return h.hexdigest()


def so_path() -> str:
    return os.path.join(OUT_DIR, SO_NAME)


def build(force: bool = False, extra_flags=(), verbose: bool = False) -> str:
    """Build (if sources changed) and return the path of libspmttkrp.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "stamp.txt")
    digest = _digest(extra_flags)
    so = so_path()
    if not force and os.path.exists(so) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return so
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = so + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{res.stderr}")
    os.replace(tmp, so)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return so


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
