"""The checked build (-DSUPERDC_CHECK): its index guard, compiled for the
host from the same header the kernels use, and the checked translation units
cross-compiled for sm_103a.  (No GPU.)"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")
CSRC = os.path.join(ROOT, "paper_2108_04209_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include "check.cuh"
#include <cstdio>
int main()
{
    int32_t w = 0;
    // in range: returned unchanged, nothing latched
    long a = (long)sdc_check::guard(0, 1, &w), b = (long)sdc_check::guard(9, 10, &w);
    printf("%ld %ld %d\n", a, b, w);
    // one past the end, negative, huge: 0 and the index bit
    long c = (long)sdc_check::guard(10, 10, &w);
    printf("%ld %d\n", c, w);
    w = 0;
    long d = (long)sdc_check::guard(-1, 10, &w);
    printf("%ld %d\n", d, w);
    w = 1;                                       // other bits are kept
    long e = (long)sdc_check::guard(1LL << 40, 10, &w);
    printf("%ld %d\n", e, w);
    long f = (long)sdc_check::guard(-5, 3, nullptr);  // no word: still clamped
    printf("%ld\n", f);
    int x = 7;
    int y = SDC_IDX(x, 4, &w);                    // the macro form
    printf("%d %d\n", y, w);
    return 0;
}
"""


def _gxx(tmp_path, defines):
    gxx = shutil.which("g++")
    if not gxx or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are missing")
    src = tmp_path / "h.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / ("h" + "".join(d.replace("-D", "_") for d in defines))
    subprocess.run([gxx, "-std=c++17", "-I", INC, "-I", CSRC, "-I", CUDA_INC] + defines + [str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")


def test_guard_logic_checked(tmp_path):
    out = _gxx(tmp_path, ["-DSUPERDC_CHECK"])
    assert out[0] == "0 9 0"
    assert out[1] == "0 4"
    assert out[2] == "0 4"
    assert out[3] == "0 5"
    assert out[4] == "0"
    assert out[5] == "0 5"          # 7 outside [0, 4): replaced by 0, bit latched


def test_guard_macro_is_identity_unchecked(tmp_path):
    out = _gxx(tmp_path, [])
    assert out[5] == "7 5"          # the default build uses the index as it is


@pytest.mark.parametrize("unit", ["rank1.cu", "fmm32.cu", "cauchy.cu"])
def test_checked_units_compile(tmp_path, unit):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc missing")
    cmd = [nvcc, "-c", os.path.join(CSRC, unit), "-o", str(tmp_path / "u.o"),
           "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", INC, "-I", CSRC, "--expt-relaxed-constexpr", "-DSUPERDC_CHECK"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
