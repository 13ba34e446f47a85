"""Build libsuperdc.so (sm_103a) in-tree with nvcc.

Every translation unit under ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_2108_04209_gb300/_lib/libsuperdc.so``.  No cmake, no torch types.
"""
import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libsuperdc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stamp():
    h = hashlib.sha1()
    for f in _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INC, "superdc.h")]:
        h.update(f.encode())
        h.update(open(f, "rb").read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra=(), check: bool = False) -> str:
    """Compile and link the library; check=True makes the checked variant
    _lib/libsuperdc_check.so (-DSUPERDC_CHECK: data-dependent indexes are
    tested and latch SUPERDC_DEV_INDEX instead of being used out of range)."""
    out = os.path.join(OUT, "check") if check else OUT
    lib_path = os.path.join(OUT, "libsuperdc_check.so") if check else LIB
    os.makedirs(out, exist_ok=True)
    stamp = _stamp() + (" check" if check else "")
    sf = os.path.join(out, "stamp")
    if not force and os.path.exists(lib_path) and os.path.exists(sf) and open(sf).read() == stamp:
        return lib_path
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
                    "--expt-relaxed-constexpr"] + (["-DSUPERDC_CHECK"] if check else []) + list(extra)
    objs = []

    def comp(src):
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc(), "-c", src, "-o", obj] + flags
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            print(r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(comp, _sources()))
    tmp = lib_path + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    open(sf, "w").write(stamp)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], check="--check" in sys.argv))
