"""In-tree build of the native library ``libpcband.so`` (sm_103a) and of the
host-side kernel emulator used by the CPU tests.

Each CUDA translation unit is compiled by its own nvcc process (in parallel),
then linked with cuFFT.  A rebuild happens only when a source or
header is newer than the library.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpcband.so")
EMU = os.path.join(BUILD, "libpcband_emu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(os.path.dirname(PKG), "include", "*.h")))


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every CUDA source for sm_103a and link ``libpcband.so``; return its path."""
    srcs = _sources()
    hdr_time = _newest(_headers())
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(_newest(srcs), hdr_time)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time)):
            return obj
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj + ".tmp"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))
        if verbose and res.stderr:
            print(res.stderr)
        os.replace(obj + ".tmp", obj)
        return obj

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcufft", "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
    os.replace(tmp, LIB)
    return LIB


def build_emulator(force: bool = False) -> str:
    """Host-only build (g++) of the kernel-tile emulator ``_build/libpcband_emu.so``."""
    src = os.path.join(CSRC, "emu", "pc_emu.cu")
    deps = [src] + _headers()
    if not force and os.path.exists(EMU) and os.path.getmtime(EMU) >= _newest(deps):
        return EMU
    os.makedirs(BUILD, exist_ok=True)
    inc = os.path.join(_cuda_home(), "include")
    tmp = EMU + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-x", "c++", "-std=c++17", "-O1", "-fPIC", "-shared", "-I", inc, src, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, EMU)
    return EMU


if __name__ == "__main__":
    print(build(verbose=True))
