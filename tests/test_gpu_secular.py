"""GPU parity of the batched rank-one step (C-ABI superdc_secular_batched)
against the CPU oracle, element by element, on seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_04209_gb300 import inputs  # noqa: E402
import paper_2108_04209_gb300 as sdc  # noqa: E402
from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu


def run_batch(b, tau, **kw):
    dev = torch.device("cuda")
    offs = torch.from_numpy(b.offsets).to(dev)
    d = torch.from_numpy(b.d).to(dev)
    z = torch.from_numpy(b.z).to(dev)
    out = sdc.secular_batched(offs, d, z, rho=b.rho, opts=sdc.default_opts(tau=tau, **kw))
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def edge_batch():
    """Ragged sizes spanning several tiles plus the degenerate cases."""
    rng = np.random.default_rng(42)
    probs = []
    probs.append((np.array([]), np.array([])))                          # empty problem
    probs.append((np.array([0.5]), np.array([0.3])))                    # m = 1
    probs.append((np.array([0.1, 0.5]), np.array([0.3, -0.4])))         # m = 2
    probs.append((np.linspace(0, 1, 17), np.zeros(17)))                 # z = 0: all deflated
    e = np.zeros(33)
    e[7] = 1.0
    probs.append((np.linspace(-1, 1, 33), e))                           # z = e_k
    dd = np.sort(rng.uniform(0, 1, 300))
    dd[100:108] = dd[100] + np.sort(rng.uniform(0, 1e-10, 8))           # tight cluster
    probs.append((np.sort(dd), rng.standard_normal(300)))
    d2 = np.sort(rng.uniform(0, 1, 129))
    d2[50] = d2[49] + 1e-13                                             # a Givens pair
    probs.append((np.sort(d2), rng.standard_normal(129)))
    for m in (31, 32, 33, 127, 128, 129, 255, 257, 1000, 2048, 2049, 4500):   # tile and chunk edges
        probs.append((np.sort(rng.uniform(-2, 3, m)), rng.standard_normal(m)))
    # exactly repeated poles (Givens deflation of equal d), small and FMM-sized
    probs.append((np.array([0.1, 0.2, 0.2, 0.2, 0.5, 0.7, 0.7]), rng.standard_normal(7)))
    dr = np.sort(rng.uniform(0, 1, 700))
    dr[200:210] = dr[200]
    dr[400:403] = dr[400]
    probs.append((dr, rng.standard_normal(700)))
    offs = np.zeros(len(probs) + 1, np.int64)
    offs[1:] = np.cumsum([len(p[0]) for p in probs])
    d = np.concatenate([p[0] for p in probs]).astype(np.float64)
    z = np.concatenate([p[1] for p in probs]).astype(np.float64)
    return inputs.SecularBatch(offs, d, z, 1.0)


@pytest.mark.parametrize("tau", [1e-12, 1e-10])
def test_edge_cases_vs_oracle(tau):
    b = edge_batch()
    out = run_batch(b, tau)
    for p in range(b.nprob):
        d, z = b.problem(p)
        if len(d) == 0:
            continue
        g = P.gpu_problem(out, b.offsets, p)
        P.compare_problem(g, d, z, tau, mode=0)


def test_small_config_distribution_all_problems():
    b = inputs.secular_batch(48, 32, 400, seed=3)
    out = run_batch(b, 1e-12)
    for p in range(b.nprob):
        d, z = b.problem(p)
        g = P.gpu_problem(out, b.offsets, p)
        P.compare_problem(g, d, z, 1e-12, mode=0)


def test_dense_eigenvectors_orthogonal_and_residual():
    b = inputs.secular_batch(8, 100, 700, seed=4)
    out = run_batch(b, 1e-12)
    for p in range(b.nprob):
        d, z = b.problem(p)
        g = P.gpu_problem(out, b.offsets, p)
        Q = P.dense_qhat(g)
        m = len(d)
        M = np.diag(d) + np.outer(z, z)
        lam = g["lam"]
        orth = np.abs(Q.T @ Q - np.eye(m)).max()
        res = np.abs(M @ Q - Q * lam).max() / np.abs(lam).max()
        ndefl = m - g["mk"]
        assert orth <= 1e-12, orth
        assert res <= 1e-12 + 4e-12 * ndefl, res


def test_full_size_4096_every_problem_vs_oracle():
    """The 4096-problem workload in the launch configuration the benchmark
    times (autotuned schedule and FMM threshold): every problem against the
    oracle's middle-way mode element by element, 32 sampled problems against
    its bisection to adjacent doubles, and invariants on every problem."""
    from paper_2108_04209_gb300.autotune import tune_secular
    b = inputs.cfg_secular_4096()
    dev = torch.device("cuda")
    offs = torch.from_numpy(b.offsets).to(dev)
    d = torch.from_numpy(b.d).to(dev)
    z = torch.from_numpy(b.z).to(dev)
    opts, _ = tune_secular(offs, d, z, 1.0, tau=1e-12, use_cache=False)
    out = sdc.secular_batched(offs, d, z, rho=1.0, opts=opts)
    out = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    assert out["status"][0] == 0
    print("problems on the FMM path:", int(out["fmm"][:b.nprob].sum()), "of", b.nprob)
    rng = np.random.default_rng(0)
    exact = set(rng.choice(b.nprob, 32, replace=False).tolist())
    for p in range(b.nprob):
        d_, z_ = b.problem(p)
        g = P.gpu_problem(out, b.offsets, p)
        P.compare_problem(g, d_, z_, 1e-12, mode=0 if p in exact else 1)
    # invariants on all problems: trace and order of the new eigenvalues
    lam = out["lam"]
    for p in range(b.nprob):
        a, e = int(b.offsets[p]), int(b.offsets[p + 1])
        d_, z_ = b.d[a:e], b.z[a:e]
        tr = d_.sum() + z_ @ z_
        assert abs(lam[a:e].sum() - tr) <= 1e-12 * (np.abs(d_).sum() + z_ @ z_) * (e - a)
        assert np.all(np.diff(lam[a:e]) >= 0)


@pytest.mark.parametrize("sched", [0, 2])
def test_host_entry_pipeline_matches_device_entry(sched):
    """The host-buffer entry point splits a batch of 2^20 roots or more into
    four chunks on two streams (copies of one chunk overlap the kernels of
    another), with the whole batch's schedule: every output it copies back is
    bit-identical to one device call over the whole 4096-problem batch."""
    torch = pytest.importorskip("torch")
    b = inputs.cfg_secular_4096()
    assert b.offsets[-1] >= (1 << 20)
    opts = sdc.default_opts(tau=1e-12, sched=sched)
    dev = torch.device("cuda")
    ref = sdc.secular_batched(torch.from_numpy(b.offsets).to(dev), torch.from_numpy(b.d).to(dev),
                              torch.from_numpy(b.z).to(dev), 1.0, opts)
    ref = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
    fields = ("lam", "dk", "zk", "eta", "vhat", "bnorm", "org", "src", "perm", "mk", "ngiv", "sweeps", "fmm")
    host = sdc.secular_batched_host(torch.from_numpy(b.offsets).pin_memory(), torch.from_numpy(b.d).pin_memory(),
                                    torch.from_numpy(b.z).pin_memory(), 1.0, opts, fields=fields)
    host = {k: v.numpy() for k, v in host.items()}
    for k in ("lam", "dk", "zk", "src", "perm", "mk", "ngiv", "fmm"):
        assert np.array_equal(host[k], ref[k]), k
    kept = np.zeros(len(host["lam"]), bool)          # per-root fields are written for kept roots only
    for p in range(b.nprob):
        kept[b.offsets[p]:b.offsets[p] + host["mk"][p]] = True
    for k in ("eta", "vhat", "bnorm", "org", "sweeps"):
        assert np.array_equal(host[k][kept], ref[k][kept]), k
