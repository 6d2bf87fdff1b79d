"""Compile the CUDA library libcplbm.so in-tree for sm_103a with nvcc.

Translation units compile in parallel; the result lands next to this file.
The build is skipped when the library is newer than every source.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcplbm.so")
# Library variants: the product, and a bounds-checked debug build in which
# every global access of the step and field kernels is checked against its
# buffer (CPLBM_CHECK_BOUNDS in csrc/device_common.cuh), built only on
# request (tests/test_gpu_bounds.py).
VARIANT_FLAGS = {"": [], "checked": ["-DCPLBM_CHECK_BOUNDS"]}


def lib_path(variant: str = "") -> str:
    return LIB if not variant else os.path.join(HERE, "libcplbm_%s.so" % variant)


def build_dir(variant: str = "") -> str:
    return BUILD if not variant else BUILD + "_" + variant

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + INCLUDE, "-I" + CSRC, "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required")
    return path


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, variant: str = "") -> str:
    if variant not in VARIANT_FLAGS:
        raise ValueError("unknown library variant %r" % variant)
    lib = lib_path(variant)
    if not force and not _stale(lib):
        return lib
    bdir = build_dir(variant)
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *VARIANT_FLAGS[variant], "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, res.stderr))
        return obj, res.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, len(sources()))) as ex:
        results = list(ex.map(compile_one, sources()))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = lib + ".tmp%d" % os.getpid()
    # -ldl: NVTX (csrc/trace.h) looks up a profiler's library at run time
    cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results] + ["-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s" % res.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                variant="checked" if "--checked" in sys.argv else ""))
