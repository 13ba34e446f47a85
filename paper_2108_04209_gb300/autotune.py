"""Autotuners for the schedule of the batched rank-one step and of the whole
eigendecomposition.

Stage 1, the direct secular kernel: per-warp root pools (sched=1) with
256..2048 roots per work unit, and the pole-split schedule (sched=2) with
64..256 roots per work unit.  Stage 2, with the stage-1 winner: the kept
problem size from which the triangular FMM takes over (opts.fmm_min_m; the
crossover depends on the batch, not only on m).  Each candidate is timed with
CUDA events on the caller's batch (device tensors, the same call the user
makes); the fastest is cached per (device, problem-count bucket, root-count
bucket) in a JSON file so later calls skip the search.
"""
import json
import os

import torch

from . import _lib as L

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "superdc_gb300", "tune.json")
CANDIDATES = [(1, t) for t in (2048, 1024, 512, 256)] + [(2, t) for t in (64, 128, 256)]
FMM_CANDIDATES = (512, 1024, 2048, -1)     # -1: direct evaluator only


def _key(nprob, total):
    b = lambda x: 1 << max(0, int(x).bit_length() - 1)
    return "%s|p%d|t%d" % (torch.cuda.get_device_name(), b(nprob), b(total))


def _load():
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _save(tab):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        json.dump(tab, open(CACHE, "w"), indent=1)
    except OSError:
        pass


def tune_secular(offsets, d, z, rho=1.0, tau=1e-12, reps=2, use_cache=True):
    """Return (opts, table of measured ms per candidate) for this batch."""
    from . import secular_batched, alloc_rank1_out, default_opts
    nprob, total = offsets.numel() - 1, d.numel()
    key = _key(nprob, total)
    tab = _load() if use_cache else {}
    if use_cache and key in tab and len(tab[key].get("best", [])) == 3:
        s, t, f = tab[key]["best"]
        return default_opts(tau=tau, sched=s, tile_roots=t, fmm_min_m=f), tab[key]["ms"]
    out = alloc_rank1_out(nprob, total, d.device)

    def measure(o):
        secular_batched(offsets, d, z, rho, o, out=out, check=False)      # warm-up
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            secular_batched(offsets, d, z, rho, o, out=out, check=False)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    ms = {}
    for s, t in CANDIDATES:
        ms["%d/%d" % (s, t)] = measure(default_opts(tau=tau, sched=s, tile_roots=t))
    s, t = min(CANDIDATES, key=lambda c: ms["%d/%d" % c])
    for f in FMM_CANDIDATES:
        ms["%d/%d/fmm%d" % (s, t, f)] = measure(default_opts(tau=tau, sched=s, tile_roots=t, fmm_min_m=f))
    f = min(FMM_CANDIDATES, key=lambda c: ms["%d/%d/fmm%d" % (s, t, c)])
    tab[key] = {"best": [s, t, f], "ms": ms}
    if use_cache:
        _save(tab)
    return default_opts(tau=tau, sched=s, tile_roots=t, fmm_min_m=f), ms


EIG_FMM_CANDIDATES = (256, 512, 1024)
EIG_SCHED_CANDIDATES = (1, 2)


def tune_eig(H, tau=1e-10, reps=1, use_cache=True):
    """Schedule of the whole eigendecomposition of the HSS handle H: stage 1
    the FMM threshold (256 / 512 / 1024 kept poles) with the automatic secular
    schedule, stage 2 the winner with the schedule forced to whole problems
    per CTA (sched=1) or to the pole split (sched=2).  Each candidate is one
    superdc_eig on H timed with CUDA events after one untimed run.  Returns
    (opts, table of measured ms); cached per (device, n, rank)."""
    from . import default_opts
    key = "%s|eig|n%d|r%d" % (torch.cuda.get_device_name(), H.n, H.rank)
    tab = _load() if use_cache else {}
    if use_cache and key in tab and len(tab[key].get("best", [])) == 2:
        s, f = tab[key]["best"]
        return default_opts(tau=tau, sched=s, fmm_min_m=f), tab[key]["ms"]

    def measure(o):
        H.eig(o)
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            H.eig(o)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    ms = {}
    for f in EIG_FMM_CANDIDATES:
        ms["0/fmm%d" % f] = measure(default_opts(tau=tau, fmm_min_m=f))
    f = min(EIG_FMM_CANDIDATES, key=lambda c: ms["0/fmm%d" % c])
    for s in EIG_SCHED_CANDIDATES:
        ms["%d/fmm%d" % (s, f)] = measure(default_opts(tau=tau, sched=s, fmm_min_m=f))
    s = min((0,) + EIG_SCHED_CANDIDATES, key=lambda c: ms["%d/fmm%d" % (c, f)])
    tab[key] = {"best": [s, f], "ms": ms}
    if use_cache:
        _save(tab)
    return default_opts(tau=tau, sched=s, fmm_min_m=f), ms
