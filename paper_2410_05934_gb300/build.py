"""Builds the native libraries of the package in-tree.

  _lib/libntt_gb300.so      the product: sm_103a kernels + C ABI (nvcc)
  _lib/libntt_gb300_emu.so  host emulation of the same kernel phases (g++),
                            loaded only by the CPU test suite

Every translation unit is compiled in parallel; a stamp of the sources and
flags skips the build when nothing changed.  No cmake, no torch extension
machinery: plain nvcc / g++ so the same step works on x86_64 and aarch64.
"""
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIB_DIR, "libntt_gb300.so")
EMU_LIB = os.path.join(LIB_DIR, "libntt_gb300_emu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function",
             "-I", INCLUDE, "-I", CSRC]

PRODUCT_SOURCES = ["capi.cu", "kernels_small.cu", "kernels_mid.cu", "kernels_large.cu", "kernels_huge.cu",
                   "kernels_otf.cu",
                   "kernels_misc.cu", "batch.cu", "grouped.cu", "costmodel.cu", "tfhe.cu", "rns.cu", "ntt32.cu",
                   "plan_host.cpp"]
EMU_SOURCES = ["plan_host.cpp", "emulate.cpp"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libntt_gb300")


def _stamp(kind, flags):
    h = hashlib.sha256()
    h.update(kind.encode())
    h.update(" ".join(flags).encode())
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    return h.hexdigest()


TILE_KERNEL_SOURCES = ["ntt_arith.cuh", "ntt_tile.cuh", "ntt_kernels.cuh", "ntt_schedules.h",
                       "kernels_small.cu", "kernels_mid.cu", "kernels_large.cu", "kernels_huge.cu",
                       "kernels_otf.cu", "kernels_misc.cu"]


def kernel_stamp():
    """Hash of the transform kernels' sources: identifies the kernels that a
    hardware-counter capture (profiles/) was taken on."""
    h = hashlib.sha256()
    for name in TILE_KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _up_to_date(lib, stamp):
    sp = lib + ".stamp"
    return os.path.exists(lib) and os.path.exists(sp) and open(sp).read().strip() == stamp


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n%s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def build_product(force=False, verbose=False, extra_flags=()):
    """Compiles the sm_103a library; returns its path."""
    flags = NVCC_FLAGS + list(extra_flags)
    stamp = _stamp("product", flags)
    if not force and _up_to_date(LIB, stamp):
        return LIB
    os.makedirs(LIB_DIR, exist_ok=True)
    obj_dir = os.path.join(LIB_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    nv = nvcc()
    jobs = []
    for src in PRODUCT_SOURCES:
        obj = os.path.join(obj_dir, src + ".o")
        cmd = [nv] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp.%d" % os.getpid()
    _run([nv] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + [o for _, o in jobs])
    os.replace(tmp, LIB)
    with open(LIB + ".stamp", "w") as f:
        f.write(stamp)
    return LIB


def build_emulation(force=False):
    """Compiles the host emulation library (no CUDA needed); returns its path."""
    stamp = _stamp("emu", CXX_FLAGS)
    if not force and _up_to_date(EMU_LIB, stamp):
        return EMU_LIB
    os.makedirs(LIB_DIR, exist_ok=True)
    cxx = os.environ.get("CXX", "g++")
    tmp = EMU_LIB + ".tmp.%d" % os.getpid()
    _run([cxx] + CXX_FLAGS + ["-shared", "-o", tmp] + [os.path.join(CSRC, s) for s in EMU_SOURCES])
    os.replace(tmp, EMU_LIB)
    with open(EMU_LIB + ".stamp", "w") as f:
        f.write(stamp)
    return EMU_LIB


def build(force=False, verbose=False):
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build_product, force, verbose)
        b = ex.submit(build_emulation, force)
        return a.result(), b.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
