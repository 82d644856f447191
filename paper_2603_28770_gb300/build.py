"""Build ``libzeus.so`` (the C-ABI library of include/zeus.h) for sm_103a.

Each CUDA translation unit is compiled by nvcc in parallel, then linked into
one shared library inside the package (``_build/libzeus.so``).  No cmake,
no torch extension machinery: the library exports plain C symbols.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libzeus.so")

# (source, extra defines): the kernels of each (gradient mode, precision)
# pair are compiled as translation units of their own, in parallel
_PAIRS = [("-DZEUS_KGRAD=%d" % g, "-DZEUS_KF32=%d" % f) for g in (0, 1) for f in (0, 1)]
SOURCES = ([(s, ()) for s in ("zeus_capi.cu", "zeus_pso.cu", "zeus_bfgs.cu", "zeus_objective.cu",
                              "zeus_noalloc.cu", "zeus_stream.cu", "zeus_batch.cu", "zeus_cluster.cu")]
           + [("zeus_bfgs_kernels.cu", d) for d in _PAIRS]
           + [("zeus_batch_kernels.cu", d) for d in _PAIRS]
           + [("zeus_batch_kernels.cu", ("-DZEUS_KGRAD=0", "-DZEUS_KF32=%d" % f, "-DZEUS_KUSER=1"))
              for f in (0, 1)])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the Zeus CUDA library cannot be built")


def _flags(extra=()):
    # --fmad=false: every product and sum is rounded on its own, as in the
    # FP64 oracle, so rational-operation objectives reproduce it bit for bit
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-I", CSRC, *extra]


STAMP = os.path.join(BUILD, "user_plugin.txt")


def user_plugin(path: str | None = None) -> str:
    """The plug-in header of user objectives compiled into the library
    (contract in include/zeus_user.cuh): ``path``, else the environment's
    ZEUS_USER_OBJECTIVES, else the package's default plug-in."""
    p = path or os.environ.get("ZEUS_USER_OBJECTIVES")
    return os.path.abspath(p) if p else os.path.join(CSRC, "zeus_user_objectives.cuh")


def _deps(plugin: str):
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in ("zeus.h", "zeus_user.cuh")]
    files += [os.path.abspath(__file__), plugin]
    return max(os.path.getmtime(f) for f in files)


def _stamp() -> str:
    try:
        with open(STAMP) as fh:
            return fh.read().strip()
    except OSError:
        return ""


def _obj_name(src: str, defines) -> str:
    tag = "".join("_" + d.split("=")[-1] for d in defines)
    return os.path.join(BUILD, src.replace(".cu", tag + ".o"))


def _compile(src: str, obj: str, extra=()) -> None:
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, *_flags(extra)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")


def build(force: bool = False, verbose: bool = False, extra=(), user_objectives: str | None = None) -> str:
    """Compile and link libzeus.so if any source changed (or another plug-in
    of user objectives is asked for); return its path."""
    plugin = user_plugin(user_objectives)
    if not os.path.exists(plugin):
        raise FileNotFoundError(f"user-objective plug-in {plugin} not found")
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps(plugin)
            and _stamp() == plugin):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = (*extra, f'-DZEUS_USER_PLUGIN="{plugin}"')
    objs = [_obj_name(s, d) for s, d in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        futs = [ex.submit(_compile, s, o, (*d, *extra)) for (s, d), o in zip(SOURCES, objs)]
        for f in futs:
            f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(plugin + "\n")
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
