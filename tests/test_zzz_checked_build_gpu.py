"""The checked build (-DSUPERDC_CHECK, _lib/libsuperdc_check.so) on the GPU.

A child process with SUPERDC_CHECKED=1 loads the checked library and runs
the FMM batch of test_gpu_fmm (near lists of every shape, including the
all-near fallback and chains of one-point boxes) against the oracle, and an
eigendecomposition whose Q and Q^T go through the FMM Cauchy-like kernels
(the guarded permutation rows).  No index guard may fire: every call returns
SUPERDC_OK and the results keep their parity.  Runs last (its first call
compiles the checked library)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os
import numpy as np
import torch
import paper_2108_04209_gb300 as sdc
from paper_2108_04209_gb300 import _lib, inputs
from tests import parity as P
from tests.test_gpu_fmm import fmm_batch, FMM_ON
from tests.test_gpu_secular import run_batch

assert os.path.basename(_lib.lib()._name) == "libsuperdc_check.so", _lib.lib()._name
b = fmm_batch()
out = run_batch(b, 1e-12, fmm_min_m=FMM_ON)
for p in range(b.nprob):
    d, z = b.problem(p)
    P.compare_problem(P.gpu_problem(out, b.offsets, p), d, z, 1e-12, mode=0)
h = inputs.hss_random(4096, 64, 6, seed=31)
lam, F = sdc.HSSMatrix(h).eig(sdc.default_opts(tau=1e-10, fmm_min_m=256))
X = torch.from_numpy(inputs.normal_block(4096, 8, seed=1)).cuda()
Y = F.apply_Q(F.apply_Q(X, trans=True))
err = (Y - X).abs().max().item()
assert err < 1e-11, err
print("CHECKED_OK", flush=True)
"""


def test_checked_build_runs_clean():
    env = dict(os.environ)
    env["SUPERDC_CHECKED"] = "1"
    env["PYTHONPATH"] = ROOT + (os.pathsep + env["PYTHONPATH"] if env.get("PYTHONPATH") else "")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "CHECKED_OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
