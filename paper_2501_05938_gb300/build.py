"""Build the in-tree CUDA libraries for sm_103a with plain nvcc.

  libtps.so       the solver (csrc/*.cu) behind the C ABI of include/tps.h
  libtpssynth.so  the seeded input generator kernel (synth/synth.cu)

Each translation unit compiles to an object in parallel, then one link.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]

LIBTPS = os.path.join(HERE, "libtps.so")
LIBSYNTH = os.path.join(HERE, "synth", "libtpssynth.so")


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libtps")
    return p


def _newer(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _compile(src, obj, extra=()):
    cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> None:
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(
        os.path.join(HERE, "csrc", "*.h")) + [os.path.join(ROOT, "include", "tps.h")]
    srcs = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
    synth_src = os.path.join(HERE, "synth", "synth.cu")
    jobs = []
    if force or _newer(LIBTPS, srcs + headers):
        objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
            list(ex.map(lambda so: _compile(*so), zip(srcs, objs)))
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIBTPS + ".tmp", *objs, "-lcudart", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIBTPS + ".tmp", LIBTPS)
        jobs.append(LIBTPS)
    if os.path.exists(synth_src) and (force or _newer(LIBSYNTH, [synth_src])):
        obj = os.path.join(BUILD, "synth.o")
        _compile(synth_src, obj)
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIBSYNTH + ".tmp", obj, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIBSYNTH + ".tmp", LIBSYNTH)
        jobs.append(LIBSYNTH)
    if verbose:
        print("built:", jobs or "up to date")


if __name__ == "__main__":
    build(force=True, verbose=True)
