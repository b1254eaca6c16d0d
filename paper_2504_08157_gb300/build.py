"""In-tree build of the CUDA library ``libxg.so`` (sm_103a only).

Six translation units (the C ABI with the line kernels for orders 1-8,
the allocation-free right-hand side, the batched persistent form, the
learned closure, hyper-diffusion / sponge / RI velocity, and IMEX),
compiled in parallel with nvcc for ``-gencode arch=compute_103a,code=sm_103a``
and linked as a shared library next to this file.  The CUDA runtime is
linked statically so the library loads without the toolkit's library path.
"""

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libxg.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("xg_api.cu", "xg_noalloc.cu", "xg_batch.cu",
                                                         "xg_closure.cu", "xg_dynamics.cu",
                                                         "xg_imex.cu")]
DEPENDS = SOURCES + [os.path.join(HERE, "csrc", f) for f in
                     ("xg_kernels.cuh", "xg_setup.h", "xg_df.cuh", "xg_kernels_df.cuh",
                      "xg_kernels_f32.cuh", "xg_plane_f32.cuh", "xg_tc.cuh", "xg_plane_tc.cuh", "xg_plane_h16.cuh",
                      "xg_column_f32.cuh", "xg_tma.cuh", "xg_ctx.h")] + [
                     os.path.join(ROOT, "include", f) for f in ("xg.h", "xg_batch.h", "xg_closure.h",
                                                               "xg_dynamics.h", "xg_imex.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: set NVCC or put the CUDA toolkit on PATH")


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPENDS)


def build(force=False, verbose=False):
    """Compile libxg.so if any source is newer than it; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    tag = "%d" % os.getpid()
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, "%s.%s.o" % (os.path.basename(src)[:-3], tag))
        cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    try:
        for cmd, p in procs:
            if p.wait() != 0:
                raise subprocess.CalledProcessError(p.returncode, cmd)
        tmp = LIB + ".tmp" + tag
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    finally:
        for cmd, p in procs:
            if p.poll() is None:
                p.kill()
                p.wait()
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
