"""Build libpicgb.so in-tree: every CUDA source compiled for sm_103a, in parallel.

    python -m paper_1608_01009_gb300.build [--force] [--verbose] [--debug]

--debug builds libpicgb_debug.so instead: the same sources with PICGB_DEBUG=1,
whose kernels check every array index they use (see pic_selftest_index_check).
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpicgb.so")
LIB_DEBUG = os.path.join(HERE, "libpicgb_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"] + ARCH


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "pic.h")]


def build(force: bool = False, verbose: bool = False, out: str = None, defines=(), debug: bool = False) -> str:
    """Compile every CUDA source for sm_103a into `out` (default: the in-tree
    libpicgb.so, or libpicgb_debug.so with `debug`).  `defines` are extra -D
    macros (launch-shape experiments)."""
    lib = out or (LIB_DEBUG if debug else LIB)
    if not force and not defines and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(p) <= t for p in _deps()):
            return lib
    bdir = BUILD if not defines else BUILD + "_" + "_".join(d.replace("=", "") for d in defines)
    if debug:
        defines = tuple(defines) + ("PICGB_DEBUG=1",)
        bdir = BUILD + "_debug"
    os.makedirs(bdir, exist_ok=True)
    extra = (["-Xptxas", "-v"] if verbose else []) + ["-D" + d for d in defines]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [NVCC] + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, "-shared"] + ARCH + ["-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
