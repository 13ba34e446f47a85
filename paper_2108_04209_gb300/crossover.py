"""Direct tiled evaluator vs triangular FMM: the measured crossover.

    python -m paper_2108_04209_gb300.crossover [--sizes 256,512,...] [--reps 3]

For each size m, a batch of rank-one problems drawn like the batched secular
workload (poles U[0,1] with 10 % in clusters of width 1e-10, z ~ N(0,1),
rho = 1, tau = 1e-12), min(2^21 / m, 2^30 / m^2) problems (at least one; the
second bound keeps the direct runs of the largest sizes to seconds), is
run through
  * the whole batched rank-one step (superdc_secular_batched: deflation,
    roots, zhat, b, merge) with opts.fmm_min_m = -1 (direct) and = 256 (FMM);
  * the Cauchy-like application Qhat^T X (superdc_rank1_apply) with
    c = 1, 19, 64 columns, direct and FMM,
timed with CUDA events on the launching stream (best of --reps, after one
warm-up).  Prints one JSON line per size.
"""
import argparse
import json

import numpy as np
import torch

import paper_2108_04209_gb300 as sdc
from paper_2108_04209_gb300 import inputs

DIRECT, FMM = -1, 256


def timed(fn, reps):
    st = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default=",".join(str(1 << k) for k in range(8, 18)))
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--cols", default="1,19,64")
    args = ap.parse_args()
    dev = torch.device("cuda")
    cols = [int(c) for c in args.cols.split(",")]
    for m in (int(s) for s in args.sizes.split(",")):
        nprob = max(1, min((1 << 21) // m, (1 << 30) // (m * m)))
        b = inputs.secular_batch(nprob, m, m, seed=5)
        offs, d, z = (torch.from_numpy(x).to(dev) for x in (b.offsets, b.d, b.z))
        total = int(b.offsets[-1])
        row = {"m": m, "nprob": nprob}
        outs = {}
        for mode, tag in ((DIRECT, "direct"), (FMM, "fmm")):
            o = sdc.default_opts(tau=1e-12, fmm_min_m=mode)
            out = sdc.secular_batched(offs, d, z, opts=o)
            row["step_ms_" + tag] = timed(lambda: sdc.secular_batched(offs, d, z, opts=o, out=out, check=False),
                                          args.reps)
            outs[tag] = out
        row["fmm_problems"] = int(outs["fmm"]["fmm"][:nprob].sum().item())
        for c in cols:
            X = torch.from_numpy(inputs.normal_block(total, c, seed=9)).to(dev)
            for mode, tag in ((DIRECT, "direct"), (FMM, "fmm")):
                o = sdc.default_opts(fmm_min_m=mode)
                row["apply%d_ms_%s" % (c, tag)] = timed(
                    lambda: sdc.apply_rank1(offs, outs["fmm"], X, trans=True, opts=o), args.reps)
        print(json.dumps(row), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
