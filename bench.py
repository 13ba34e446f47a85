#!/usr/bin/env python3
"""Benchmark of the SuperDC conquering-stage hot path on GB300.

Workload (one "step"): the batched secular solve of 4096 independent
rank-one problems diag(d) + z z^T, m ~ U{32..2048}, poles U[0,1] with 10% in
clusters of width 1e-10, z ~ N(0,1), rho = 1, tau = 1e-12: deflation, all
shifted secular roots, Loewner zhat, b and the sorted eigenvalues -- the
whole rank-one pipeline of the conquering stage, in one C-ABI call.

Metric: secular roots per second (all roots of the batch / device time of
the step).  Inputs are resident in HBM when the timed region starts; the L2
is flushed (256 MiB write) before every timed step.  ``e2e`` repeats the
measurement through the C-ABI host-buffer entry point
superdc_secular_batched_host (pinned host -> device copies of the inputs and
device -> host copies of the results inside the timed region).

Multi-GPU: the path has no exchange step; N ranks run N independent replicas
(weak scaling), ``value`` = roots of all ranks / max-over-ranks time.

Beside the batched step (single-GPU runs only; --no-eig skips them):
``hss_eig_131072`` times superdc_eig on the n=131072, leaf 128, rank 10 HSS
matrix (median of 3 after a warm-up, wall and CUDA-event time, clocks), Q^T X
on a 131072 x 64 block through superdc_apply_Q (time, HBM GB/s of its
algorithmic bytes, FP64 fraction of its algorithmic flops), the direct-only
eigendecomposition once (--no-direct skips it) and Table 5's statistic;
``hss_eig_16384`` times the clustered n=16384 problem level-batched and one
node at a time, and the oracle on the same problem on the host cores;
``example1_262144`` runs the paper's Example 1 at its largest size with its
leaf size 2048 against the closed-form spectrum.

``--impl reference`` times the CPU oracle (plain C + OpenMP, FP64) on a
bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HSS eigendecomp time at n=131072; secular roots/s; FP64-pipe % of peak"
WORKLOAD = ("batched secular solve: 4096 independent rank-one problems, m~U{32..2048}, "
            "poles U[0,1] with 10% in clusters of width 1e-10, z~N(0,1), rho=1, tau=1e-12; "
            "deflation + shifted roots + Loewner zhat + b + sorted eigenvalues")
FP64_NOMINAL_TFLOPS = 1.25     # GB300 nominal FP64 (no measured figure in the peaks file)
SECULAR_FLOPS_PER_INTERACTION = 7.0   # 2 sub, 1 recip, 1 mul, 1 add, 1 fma (2)
FMM_P = 22                              # Chebyshev order of the FMM expansions
FMM_FAR_FLOPS = 4 * (FMM_P - 1) * 3     # per root and sweep: four Clenshaw sums (fma + sub per step)


def _code_sha1(text):
    """sha1 of a C/CUDA source without its comments and blank space (the code
    the counters were taken on, unchanged by edits to comments)."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [ln for ln in (re.sub(r"//.*$", "", ln).strip() for ln in text.splitlines()) if ln]
    return hashlib.sha1("\n".join(lines).encode()).hexdigest()


def _profiled(name, src):
    """Numbers of a committed ncu summary, if it was taken on the current kernel code."""
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        code = _code_sha1(open(os.path.join(ROOT, src)).read())
        if ("code sha1: %s" % code) not in txt:
            return None
        return {k: float(v) for k, v in re.findall(r"^(\w+): ([0-9.]+)$", txt, re.M)}
    except OSError:
        return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _fp64_peak():
    """FP64 peak: the peaks file if it has one, else the DFMA probe run live on
    this GPU (paper_2108_04209_gb300.probe), else the nominal figure."""
    pk = _peaks()
    if "fp64_tflops" in pk:
        return float(pk["fp64_tflops"]), "measured (MEASURED_PEAKS.json fp64_tflops)"
    try:
        from paper_2108_04209_gb300.probe import build_probe
        r = subprocess.run([build_probe()], capture_output=True, text=True, timeout=120)
        v = json.loads(r.stdout.strip().splitlines()[-1])
        return float(v["fp64_tflops"]), "measured: DFMA probe run live by bench.py (%.3f DFMA/clk/SM)" % (
            v["dfma_per_clk_per_sm"])
    except Exception:
        return FP64_NOMINAL_TFLOPS, "nominal GB300 FP64 (1.25 TFLOP/s)"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(batch, budget_s=20.0, tau=1e-12):
    """The oracle, as it stands, on a bounded prefix of the workload's problems."""
    from oracle import rank1 as r1
    t0 = time.perf_counter()
    roots = 0
    nprob = 0
    for p in range(batch.nprob):
        d, z = batch.problem(p)
        r1.rank1_step(d, z, tau, mode=1)
        roots += len(d)
        nprob += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    return {"value": roots / dt, "unit": "roots/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of the 4096 problems (%d roots), oracle newton mode, %.1f s" % (nprob, roots, dt)}


def max_over_ranks(vals, pg, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the job
    time); identity without a process group."""
    if pg is None:
        return [float(v) for v in vals]
    import torch
    tt = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    pg.all_reduce(tt, op=pg.ReduceOp.MAX)
    return [float(v) for v in tt.cpu()]


def job_throughput(units_per_rank_step, steps, ws, tmax_ms):
    """Whole-job units and units/s: every rank processes units_per_rank_step
    per step (replicas), the job takes the slowest rank's time."""
    units = float(units_per_rank_step) * steps * ws
    return units, units / (tmax_ms * 1e-3)


def _median(v):
    return float(np.median(np.asarray(v, dtype=np.float64)))


def _timed(fn, reps):
    """(median wall s, median CUDA-event ms, last result) of reps calls after
    the caller's warm-up; the events bracket the call on the current stream."""
    import torch
    walls, evs, res = [], [], None
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        res = fn()
        e1.record()
        e1.synchronize()
        walls.append(time.perf_counter() - t0)
        evs.append(e0.elapsed_time(e1))
    return _median(walls), _median(evs), res


def apply_q_work(F, ncols, fmm_min_m=512):
    """Algorithmic bytes and flops of Q^T X for the direct part (the FMM part's
    flops come from the device counter): per rank-one factor the block is read
    and written once and the factor vectors (dk, eta, d_K, vhat, b: doubles;
    src, pinv: int32) read once; per level one permutation pass; the leaves
    read the block, their dense Q and write the result.  Direct Cauchy-like
    terms: difference, reciprocal and one FMA per column of each 32-column
    chunk, over every (target, source) pair of the nodes below the FMM
    threshold."""
    n = F.n
    blk = 2.0 * n * ncols * 8
    nbytes = F.lmax * F.rank * (blk + n * (5 * 8 + 2 * 4)) + F.lmax * blk + blk + n * 128 * 8
    chunks = [min(32, ncols - c0) for c0 in range(0, ncols, 32)]
    per_pair = sum(3 + 2 * c for c in chunks)
    dflops = 0.0
    for lev in range(F.lmax):
        for j in range(F.rank):
            mk = F.get(lev, j, "mk").astype(np.float64)
            dmk = mk[mk < fmm_min_m]
            dflops += per_pair * float(np.sum(dmk * dmk))
    return nbytes, dflops


def eig_graph(H, opts, reps=3):
    """superdc_eig_plan once, superdc_eig_run captured into one CUDA graph,
    the replay timed (median of reps CUDA-event times after one replay)."""
    import torch
    F = H.eig_plan(opts)
    lam = torch.empty(H.n, dtype=torch.float64, device="cuda")
    F.run(lam)
    torch.cuda.synchronize()
    F.sync_status()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.run(lam)
    g.replay()
    torch.cuda.synchronize()
    _, ev, _ = _timed(g.replay, reps)
    F.sync_status()
    del g
    return ev * 1e-3


def eig_headline(dev, peak, peak_src, direct=True, reps=3):
    """HSS eigendecomposition at n=131072 (leaf 128, rank 10, seed 4) and
    Q^T X on a 131072 x 64 N(0,1) block: median of reps after one warm-up,
    wall time around the C-ABI call (which synchronises) and CUDA-event time,
    the clocks during the runs; the direct-only time once; Table 5's statistic
    over the root node's r secular equations."""
    import ctypes
    import torch
    import paper_2108_04209_gb300 as sdc
    from paper_2108_04209_gb300 import _lib as L, inputs
    lib = L.lib()
    from paper_2108_04209_gb300.autotune import tune_eig
    h = inputs.cfg_large_131072()
    H = sdc.HSSMatrix(h)
    opts, tune_ms = tune_eig(H, use_cache=False)
    clk = Clocks(dev.index or 0)
    lam, F = H.eig(opts)                       # warm-up
    del F
    clk.start()
    wall, ev, (lam, F) = _timed(lambda: H.eig(opts), reps)
    n = F.n
    X = torch.from_numpy(inputs.normal_block(n, 64, seed=104)).to(dev)
    F.apply_Q(X, trans=True)                   # warm-up
    awall, aev, Y = _timed(lambda: F.apply_Q(X, trans=True), reps)
    # the device flop counter of the FMM part, one more call
    lib.superdc_profile_reset()
    lib.superdc_profile_enable(1)
    F.apply_Q(X, trans=True)
    torch.cuda.synchronize()
    lib.superdc_profile_enable(0)
    c = ctypes.c_int64(0)
    lib.superdc_profile_counter(b"fmm_flops", ctypes.byref(c))
    nbytes, dflops = apply_q_work(F, 64)
    aflops = float(c.value) + dflops
    graph_s = eig_graph(H, opts, reps)
    clocks = clk.stop()
    st = F.stats()
    mus = []
    for j in range(F.rank):
        swj = F.get(0, j, "sweeps")[:int(F.get(0, j, "mk")[0])]
        mus.append(float(np.mean(swj - 1 > 5)))
    out = {
        "workload": "HSS n=131072, leaf 128, rank 10, seed 4 (U orthonormal from QR of N(0,1), B = N(0,1) diag(2^-k)), "
                    "tau=1e-10; apply: Q^T X, X 131072 x 64 N(0,1) seed 104",
        "eig_s": {"wall_median": wall, "device_median": ev * 1e-3, "reps": reps,
                  "graph_replay_median": graph_s},
        "schedule": {"autotuned": "sched=%d fmm_min_m=%d" % (opts.sched, opts.fmm_min_m),
                     "candidates_ms": tune_ms},
        "apply_QT_64": {"wall_median_s": awall, "device_median_s": aev * 1e-3,
                        "hbm_gbs": nbytes / (aev * 1e-3) / 1e9, "algorithmic_bytes": nbytes,
                        "fp64_tflops": aflops / (aev * 1e-3) / 1e12, "fp64_frac": aflops / (aev * 1e-3) / 1e12 / peak,
                        "algorithmic_flops": aflops, "hbm_of": "measured copy bandwidth %.0f GB/s" % _peaks().get(
                            "hbm_gbs", 0.0), "fp64_of": peak_src},
        "stats": st,
        "mu_table5_root": {"max_over_steps": max(mus), "per_step": mus,
                           "note": "fraction of the root node's roots needing more than 5 iterations after the "
                                   "midpoint sweep (Section 5, Table 5)"},
        "clocks": clocks,
    }
    if direct:
        del F
        lam0, F0 = H.eig(sdc.default_opts(fmm_min_m=-1))
        torch.cuda.synchronize()
        dw, dev_ms, _ = _timed(lambda: H.eig(sdc.default_opts(fmm_min_m=-1)), 1)
        out["eig_direct_only_s"] = {"wall": dw, "device": dev_ms * 1e-3}
    out["cpu_oracle"] = "not run at n=131072: the oracle needs ~5 min on 16 cores per run (direct O(n^2) sweeps " \
                        "at the top levels); timed at n=16384 in hss_eig_16384"
    return out


def table1_metrics(n, leaf, nprobe=64):
    """Table 1's accuracy measures for Example 1 at size n (leaves of
    ``leaf``): delta = ||lambda - lambda*||_2 / (n ||lambda*||_2) against the
    closed form 3 - 2 cos(k pi/(n+1)); gamma = max_k ||A q_k - lambda_k q_k||
    / (n ||A||_2) and theta = max_k ||Q^T q_k - e_k|| / n over nprobe
    eigenvectors q_k (columns of Q read through superdc_apply_Q at evenly
    spread k; A q by the tridiagonal stencil)."""
    import torch
    import paper_2108_04209_gb300 as sdc
    from paper_2108_04209_gb300 import inputs
    H = sdc.HSSMatrix(inputs.hss_tridiag(n, leaf))
    lam, F = H.eig(sdc.default_opts(tau=1e-10))
    k = np.arange(1, n + 1)
    exact = np.sort(3.0 - 2.0 * np.cos(k * np.pi / (n + 1)))
    ln = lam.cpu().numpy()
    delta = float(np.linalg.norm(ln - exact) / (n * np.linalg.norm(exact)))
    idx = np.unique(np.linspace(0, n - 1, nprobe).astype(np.int64))
    E = torch.zeros((n, len(idx)), dtype=torch.float64, device="cuda")
    E[torch.from_numpy(idx).cuda(), torch.arange(len(idx), device="cuda")] = 1.0
    Qk = F.apply_Q(E)
    AQ = 3.0 * Qk
    AQ[1:] -= Qk[:-1]
    AQ[:-1] -= Qk[1:]
    lk = lam[torch.from_numpy(idx).cuda()]
    anorm = 3.0 + 2.0 * np.cos(np.pi / (n + 1))
    gamma = float(torch.linalg.vector_norm(AQ - Qk * lk[None, :], dim=0).max()) / (n * anorm)
    theta = float(torch.linalg.vector_norm(F.apply_Q(Qk, trans=True) - E, dim=0).max()) / n
    return {"n": n, "gamma": gamma, "delta": delta, "theta": theta, "probes": int(len(idx))}


def example1(dev, n=262144, leaf=2048, reps=3, oracle=True):
    """Section 5, Example 1 at the paper's largest size and leaf size: the
    tridiagonal matrix (3 on the diagonal, -1 off it) in its explicit rank-2
    HSS form with leaves of 2048 (refined by the library into subtrees of
    128-row leaves), tau = 1e-10; every eigenvalue against 3 - 2 cos(k pi/(n+1));
    beside the paper's 383.4 s (Matlab, 4 cores, same n, leaf and tau); and
    Table 1's gamma, delta, theta at n = 8192 ... 131072 and n."""
    import torch
    import paper_2108_04209_gb300 as sdc
    from paper_2108_04209_gb300 import inputs
    h = inputs.hss_tridiag(n, leaf)
    t0 = time.perf_counter()
    H = sdc.HSSMatrix(h)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del h
    opts = sdc.default_opts(tau=1e-10)
    H.eig(opts)
    wall, ev, (lam, F) = _timed(lambda: H.eig(opts), reps)
    k = np.arange(1, n + 1)
    exact = np.sort(3.0 - 2.0 * np.cos(k * np.pi / (n + 1)))
    rel = float(np.max(np.abs(lam.cpu().numpy() - exact) / exact))
    out = {"workload": "Example 1: tridiagonal (3, -1), n=%d, explicit rank-2 HSS form with leaves of %d "
                       "(refined to %d-row leaves), tau=1e-10" % (n, leaf, n >> F.lmax),
           "build_s": build_s, "eig_s": {"wall_median": wall, "device_median": ev * 1e-3},
           "max_rel_error_vs_closed_form": rel, "deflated": F.stats()["deflated"],
           "paper_s": {"total": 383.4, "dividing": 16.1, "hardware": "Matlab, 4 x 2.6 GHz CPU cores, FP64",
                       "source": "Section 5, Example 1"}}
    del F, H
    out["table1"] = [table1_metrics(nn, leaf) for nn in (8192, 16384, 32768, 65536, 131072, n)]
    if oracle:
        from oracle import superdc as osd
        hs = inputs.hss_tridiag(8192, 128)
        t0 = time.perf_counter()
        osd.superdc(hs, tau=1e-10, mode=1)
        out["cpu_oracle_n8192_s"] = {"s": time.perf_counter() - t0, "cores": len(os.sched_getaffinity(0)),
                                     "note": "the oracle at n=8192, leaf 128 (n=262144 with leaves of 2048 "
                                             "would take hours: its leaf solver is cyclic Jacobi)"}
    return out


def eig_clustered(dev, oracle=True, reps=3):
    """n=16384, leaf 64, rank 8, clustered leaf spectra (seed 2): level-batched
    launches vs one launch sequence per node (opts.batching = 0), and the
    oracle on the host cores (middle-way mode) for the same problem."""
    import torch
    import paper_2108_04209_gb300 as sdc
    from paper_2108_04209_gb300 import inputs
    h = inputs.cfg_clustered_16384()
    H = sdc.HSSMatrix(h)
    H.eig()
    bw, bev, (lam, F) = _timed(lambda: H.eig(), reps)
    H.eig(sdc.default_opts(batching=0))
    uw, uev, _ = _timed(lambda: H.eig(sdc.default_opts(batching=0)), 1)
    gs = eig_graph(H, sdc.default_opts(), reps)
    out = {"workload": "HSS n=16384, leaf 64, rank 8, clustered leaf spectra, seed 2, tau=1e-10",
           "batched_s": {"wall_median": bw, "device_median": bev * 1e-3, "graph_replay_median": gs},
           "per_node_s": {"wall": uw, "device": uev * 1e-3},
           "batched_speedup": uev / bev, "deflated": F.stats()["deflated"]}
    if oracle:
        from oracle import superdc as osd
        t0 = time.perf_counter()
        osd.superdc(h, tau=1e-10, mode=1)
        out["cpu_oracle"] = {"s": time.perf_counter() - t0, "cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle (middle-way mode), same box"}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2108_04209_gb300 import inputs
    batch = inputs.cfg_secular_4096()
    from oracle import rank1 as r1
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    nsample = 48
    vals, times = [], []

    def step(off):
        roots = 0
        t0 = time.perf_counter()
        for p in range(off, off + nsample):
            d, z = batch.problem(p % batch.nprob)
            r1.rank1_step(d, z, 1e-12, mode=1)
            roots += len(d)
        return roots, time.perf_counter() - t0

    for w in range(args.warmup):
        step(w * nsample)
    tot_r, tot_t = 0, 0.0
    for s in range(args.steps):
        r, t = step((args.warmup + s) * nsample)
        tot_r += r
        tot_t += t
    v = tot_r / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "roots/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "roots/s", "cores": cores, "kind": "oracle",
                             "sample": "%d consecutive problems per step of the 4096-problem workload" % nsample},
            "e2e": {"value": v, "unit": "roots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-eig", action="store_true", help="skip the HSS eigendecomposition blocks")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-only n=131072 run (~50 s)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2108_04209_gb300 as sdc
    from paper_2108_04209_gb300 import _lib as L, inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    batch = inputs.cfg_secular_4096()
    total = int(batch.offsets[-1])
    offs = torch.from_numpy(batch.offsets).to(dev)
    d = torch.from_numpy(batch.d).to(dev)
    z = torch.from_numpy(batch.z).to(dev)
    from paper_2108_04209_gb300.autotune import tune_secular
    opts, tune_ms = tune_secular(offs, d, z, 1.0, tau=1e-12, use_cache=False)
    out = sdc.alloc_rank1_out(batch.nprob, total, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lib = L.lib()

    for _ in range(max(3, args.warmup)):
        sdc.secular_batched(offs, d, z, 1.0, opts, out=out, check=False)
    sdc.check_status(out["status"], "warmup")
    torch.cuda.synchronize()

    clk = Clocks(local)
    lib.superdc_profile_reset()
    lib.superdc_profile_enable(1)
    st = torch.cuda.current_stream()
    evs = []
    barrier()
    clk.start()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sdc.secular_batched(offs, d, z, 1.0, opts, out=out, check=False)
        e1.record(st)
        evs.append((e0, e1))
    barrier()
    clocks = clk.stop()
    lib.superdc_profile_enable(0)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    sdc.check_status(out["status"], "timed")
    kern = {}
    import ctypes
    for name in ("deflate", "tiles", "units", "secular", "lowner", "bnorm", "merge", "fmm_plan", "fmm_tree",
                 "fmm_up", "fmm_m2l", "fmm_l2l", "fmm_secular", "fmm_secular_last", "fmm_lowner",
                 "fmm_bnorm"):
        n_ = ctypes.c_int64(0)
        t_ = ctypes.c_double(0.0)
        lib.superdc_profile_read(name.encode(), ctypes.byref(n_), ctypes.byref(t_))
        kern[name] = (n_.value, t_.value)
    launches = sum(v[0] for v in kern.values())

    # the same step captured once into a CUDA graph and replayed
    graph_ms = None
    try:
        g = torch.cuda.CUDAGraph()
        sdc.secular_batched(offs, d, z, 1.0, opts, out=out, check=False)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            sdc.secular_batched(offs, d, z, 1.0, opts, out=out, check=False)
        g.replay()
        torch.cuda.synchronize()
        gt = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            gt += e0.elapsed_time(e1)
        sdc.check_status(out["status"], "graph replay")
        graph_ms = gt / args.steps
        del g
    except Exception as ex:      # report, do not hide
        graph_ms = "capture failed: %s" % ex

    # unbatched baseline: the first problems launched one at a time
    nsample = 256
    singles = []
    for p in range(nsample):
        a_, b_ = int(batch.offsets[p]), int(batch.offsets[p + 1])
        singles.append((torch.tensor([0, b_ - a_], dtype=torch.int64, device=dev), d[a_:b_], z[a_:b_]))
    for o_, dd_, zz_ in singles[:8]:
        sdc.secular_batched(o_, dd_, zz_, 1.0, opts, check=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for o_, dd_, zz_ in singles:
        sdc.secular_batched(o_, dd_, zz_, 1.0, opts, check=False)
    e1.record()
    e1.synchronize()
    unb_roots = int(batch.offsets[nsample])
    unbatched_rps = unb_roots / (e0.elapsed_time(e1) * 1e-3)

    # algorithmic work of the secular kernels, from the run's own counts: the
    # direct kernel evaluates every (root, pole) pair of a sweep, the FMM
    # kernels the near-field pairs (counted on the device) plus four Clenshaw
    # sums per root and sweep
    mk = out["mk"].cpu().numpy().astype(np.float64)
    sw = out["sweeps"].cpu().numpy().astype(np.float64)
    fm = out["fmm"].cpu().numpy()[:batch.nprob] != 0
    per_prob_sweeps = np.add.reduceat(sw, batch.offsets[:-1]) if total else np.zeros(0)
    kept_sw = sw[sw > 0]
    mu = float(np.mean(kept_sw - 1 > 5)) if kept_sw.size else 0.0
    interactions = float(np.sum((mk * per_prob_sweeps)[~fm]))
    last_sweeps = np.array([sw[int(batch.offsets[p]) + int(mk[p]) - 1] if fm[p] else 0.0
                            for p in range(batch.nprob)])
    fmm_root_sweeps = float(np.sum(per_prob_sweeps[fm]) - last_sweeps.sum())   # tree roots only
    terms = ctypes.c_int64(0)
    lib.superdc_profile_counter(b"fmm_secular_terms", ctypes.byref(terms))
    fmm_terms = float(terms.value) / max(1, args.steps)
    fl_ctr = ctypes.c_int64(0)
    lib.superdc_profile_counter(b"fmm_flops", ctypes.byref(fl_ctr))
    fmm_other_flops = float(fl_ctr.value) / max(1, args.steps)
    peak, peak_src = _fp64_peak()
    sec_ms = kern["secular"][1] / max(1, kern["secular"][0])
    fsec_ms = kern["fmm_secular"][1] / max(1, args.steps)
    rl = {}
    if interactions > 0:
        a_ = SECULAR_FLOPS_PER_INTERACTION * interactions / (sec_ms * 1e-3) / 1e12
        rl["k_secular"] = {"achieved": a_, "ms": sec_ms, "flops": SECULAR_FLOPS_PER_INTERACTION * interactions,
                           "algorithmic": "%.0f flops/interaction x %.4g (root, pole) interactions per launch" % (
                               SECULAR_FLOPS_PER_INTERACTION, interactions)}
    if fmm_root_sweeps > 0 and fsec_ms > 0:
        fl = SECULAR_FLOPS_PER_INTERACTION * fmm_terms + FMM_FAR_FLOPS * fmm_root_sweeps
        rl["fmm_secular"] = {"achieved": fl / (fsec_ms * 1e-3) / 1e12, "ms": fsec_ms, "flops": fl,
                             "algorithmic": "%.0f flops x %.4g near-field terms + %d flops x %.4g root sweeps" % (
                                 SECULAR_FLOPS_PER_INTERACTION, fmm_terms, FMM_FAR_FLOPS, fmm_root_sweeps)}
    # whole step: every kernel's algorithmic work (direct secular, Loewner 5 and
    # b 6 flops per (target, source) pair of the direct problems, FMM secular
    # near terms and far-field sweeps, and the device-counted far fields and
    # Loewner / b consumers of the FMM problems) over the step time
    direct_pairs = float(np.sum((mk * mk)[~fm]))
    step_flops = (SECULAR_FLOPS_PER_INTERACTION * interactions + 11.0 * direct_pairs +
                  SECULAR_FLOPS_PER_INTERACTION * fmm_terms + FMM_FAR_FLOPS * fmm_root_sweeps + fmm_other_flops)
    dom = max(rl, key=lambda k: rl[k]["ms"]) if rl else "k_secular"
    prof = _profiled("k_secular_batched4096_dram.md", "paper_2108_04209_gb300/csrc/rank1.cu") \
        if dom == "k_secular" else _profiled("fmm_secular_batched4096_dram.md",
                                             "paper_2108_04209_gb300/csrc/fmm_impl.cuh")
    achieved = rl[dom]["achieved"] if rl else 0.0

    # e2e: the C-ABI host-buffer entry point (superdc_secular_batched_host):
    # pinned host inputs in, host results out, copies inside the timed region
    h_off = torch.from_numpy(batch.offsets).pin_memory()
    h_d = torch.from_numpy(batch.d).pin_memory()
    h_z = torch.from_numpy(batch.z).pin_memory()
    fields = ("lam", "eta", "org", "vhat", "bnorm")
    res = sdc.secular_batched_host(h_off, h_d, h_z, 1.0, opts, fields=fields)
    hout = dict(res)
    hout["status"] = torch.zeros(1, dtype=torch.int32).pin_memory()
    sdc.secular_batched_host(h_off, h_d, h_z, 1.0, opts, fields=fields, out=hout)
    barrier()
    e2e_t = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = sdc.secular_batched_host(h_off, h_d, h_z, 1.0, opts, fields=fields, out=hout)
        e2e_t += time.perf_counter() - t0
    h2d = h_off.numel() * 8 + h_d.numel() * 8 + h_z.numel() * 8
    d2h = sum(v.numel() * v.element_size() for v in res.values()) + 4

    # max over ranks; every rank solves the whole workload (replicas, weak scaling)
    tmax, e2e_max = max_over_ranks([ms, e2e_t], pg, dev)
    roots_all, value = job_throughput(total, args.steps, ws, tmax)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "roots/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nprob": batch.nprob, "total_roots": total,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "gpu_launches": int(launches),
            "kernels_ms_per_step": {k: v[1] / max(1, args.steps) for k, v in kern.items()},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "dtype": "fp64", "frac": achieved / peak,
                         "traffic": (prof or {}).get("traffic_bytes"),
                         "fp64_pipe_pct_ncu": (prof or {}).get("fp64_pipe_pct"),
                         "peak_source": peak_src,
                         "algorithmic": rl.get(dom, {}).get("algorithmic"),
                         "other": {k: {"achieved": v["achieved"], "frac": v["achieved"] / peak, "ms": v["ms"]}
                                   for k, v in rl.items() if k != dom}},
            "whole_step": {"flops": step_flops, "achieved_tflops": step_flops / (tmax / args.steps * 1e-3) / 1e12,
                           "frac": step_flops / (tmax / args.steps * 1e-3) / 1e12 / peak,
                           "of": "measured FP64 peak (DFMA probe)",
                           "algorithmic": "direct secular 7/pair-sweep, direct Loewner 5 + b 6 per pair, FMM secular "
                                          "7/near term + %d/root sweep, FMM far fields and consumers counted on the "
                                          "device (FMA 2, other operations 1)" % FMM_FAR_FLOPS},
            "mu_table5": {"value": mu, "unit": "fraction of roots not converged after 5 iterations",
                          "note": "iterations = sweeps after the midpoint sweep (Section 5, Table 5's statistic)"},
            "fmm": {"threshold": "opts.fmm_min_m=%d (0 = library default)" % opts.fmm_min_m,
                    "problems": int(fm.sum()), "roots": int(mk[fm].sum()),
                    "direct_problems": int((~fm).sum()), "direct_roots": int(mk[~fm].sum())},
            "secular_sweeps_mean": float(sw[sw > 0].mean()) if np.any(sw > 0) else 0.0,
            "schedule": {"autotuned": "sched=%d tile_roots=%d fmm_min_m=%d" % (opts.sched, opts.tile_roots,
                                                                             opts.fmm_min_m),
                         "candidates_ms": tune_ms},
            "graph_replay_ms_per_step": graph_ms,
            "unbatched": {"value": unbatched_rps, "unit": "roots/s",
                          "sample": "first %d problems, one launch sequence each" % nsample},
            "e2e": {"value": roots_all / e2e_max, "unit": "roots/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "clocks": clocks,
        }
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(batch, budget_s=args.cpu_budget)
        if not args.no_eig and ws == 1:
            del out, flush
            torch.cuda.empty_cache()
            line["hss_eig_131072"] = eig_headline(dev, peak, peak_src, direct=not args.no_direct)
            line["hss_eig_16384"] = eig_clustered(dev, oracle=(ws == 1 and not args.no_cpu_baseline))
            line["example1_262144"] = example1(dev, oracle=not args.no_cpu_baseline)
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
