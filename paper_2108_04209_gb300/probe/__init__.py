"""FP64 peak probe (roofline denominator for the FP64-bound kernels).

``python -m paper_2108_04209_gb300.probe`` compiles ``fp64_peak.cu`` for
sm_103a and prints one JSON line: DFMA throughput (TFLOP/s, FMA = 2 flops),
DFMA per clock per SM, and FP64 division throughput.
"""
import os
import subprocess
import sys

from ..build import ARCH, OUT, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def build_probe():
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "fp64_peak")
    src = os.path.join(HERE, "fp64_peak.cu")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        subprocess.check_call([nvcc(), src, "-o", exe, "-O3"] + ARCH)
    return exe


def main():
    exe = build_probe()
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    sys.stderr.write(r.stderr)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
