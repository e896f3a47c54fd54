"""Build the CUDA library ``liblbm_gb300.so`` in-tree for sm_103a (GB300).

Every translation unit under ``csrc`` is compiled in parallel with nvcc and linked into
one shared object next to this file.  No CMake, no PyTorch extension machinery: the
library has a plain C ABI (``include/lbm.h``) and is loaded with ctypes.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm_gb300.so")
CHECK_LIB = os.path.join(HERE, "liblbm_gb300_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith(".cu") or f.endswith(".cpp"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    inc = os.path.join(os.path.dirname(HERE), "include")
    hs += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    return hs


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Compile (only what changed) and link; returns the library path.  check=True builds
    the bounds-check variant (kernels compiled with -DLBM_BOUNDS_CHECK: every global and
    shared-memory access of the step kernels is index-checked and a failure is reported as
    LBM_ECORRUPT) into liblbm_gb300_check.so, beside the normal library."""
    build_dir = BUILD + ("_check" if check else "")
    lib = CHECK_LIB if check else LIB
    flags = NVCC_FLAGS + (["-DLBM_BOUNDS_CHECK"] if check else [])
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    hdrs = _headers()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [cc] + ARCH + flags + ["-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [cc] + flags + ["-x", "c++", "-c", src, "-o", obj]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(subprocess.run, cmd, capture_output=True, text=True) for cmd in jobs]
            for cmd, fut in zip(jobs, futs):
                res = fut.result()
                if verbose or res.returncode != 0:
                    print(" ".join(cmd))
                    print(res.stdout + res.stderr)
                if res.returncode != 0:
                    raise RuntimeError("nvcc failed on %s" % cmd[-3])
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static"],
                       check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose=True, check="--check" in sys.argv[1:]))
