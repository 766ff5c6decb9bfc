"""Build libgbnfft.so (the CUDA library) in-tree with nvcc for sm_103a.

Each translation unit compiles in its own nvcc process (in parallel), then one
link step produces ``paper_1605_01244_gb300/_build/libgbnfft.so``.  No cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
SO = os.path.join(BUILD, "libgbnfft.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(os.path.realpath(nv)))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(extra_flags) -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(ROOT, "include", "gbnfft.h"))
    deps.append(os.path.abspath(__file__))
    flag_file = os.path.join(BUILD, "flags.txt")
    if not os.path.exists(flag_file) or open(flag_file).read() != " ".join(extra_flags):
        return True
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, extra_flags: tuple[str, ...] = (), verbose: bool = False) -> str:
    """Compile and link the library if any input changed; returns the .so path."""
    extra_flags = tuple(extra_flags)
    if not force and not _stale(extra_flags):
        return SO
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    # host code: no FMA contraction, so the host-side window checks round the
    # same way on x86 and Arm
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                     "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra_flags]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = SO + ".tmp%d" % os.getpid()
    lib = os.path.join(home, "lib64")
    cmd = [nvcc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs,
           "-L", lib, "-lcufft", "-Xlinker", "-rpath=" + lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, SO)
    with open(os.path.join(BUILD, "flags.txt"), "w") as fh:
        fh.write(" ".join(extra_flags))
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
