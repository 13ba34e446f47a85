"""GPU parity of the triangular FMM path (opts.fmm_min_m; Sections 4.1.2,
4.2.2, 4.3) against the CPU oracle and against the direct tiled evaluator.

The FMM replaces far-field sums by Chebyshev expansions (order 22, boxes of
32 or 64 indices, admissible when the gap is at least 0.75 x the larger box
width), whose relative error is ~1e-14 per far box: well below the stopping
tolerance of eq. (4.12), so roots, zhat and b keep the direct path's
tolerances against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import inputs  # noqa: E402
from oracle import dense, superdc as osd  # noqa: E402
from tests import parity as P  # noqa: E402
from tests.test_gpu_secular import run_batch  # noqa: E402

pytestmark = pytest.mark.gpu

FMM_ON = 256     # every problem with at least four leaf boxes takes the FMM path
FMM_OFF = -1


def fmm_batch():
    """Problem shapes that stress the box tree: uniform, clustered, graded
    (geometric), two far groups (a box straddling a wide gap), one dominant
    z (the last eigenvalue far to the right), an ultra-graded spectrum whose
    near lists exhaust the pool, sizes across box edges, the last pole alone
    in a chain of boxes of one point."""
    rng = np.random.default_rng(7)
    probs = []
    for m in (256, 300, 511, 777, 1025, 2049, 4500):
        probs.append((np.sort(rng.uniform(-2, 3, m)), rng.standard_normal(m)))
    b = inputs.secular_batch(6, 600, 3000, seed=11)
    for p in range(b.nprob):
        probs.append(b.problem(p))
    probs.append((np.geomspace(1e-8, 1.0, 3000), rng.standard_normal(3000)))
    d = np.sort(np.concatenate([rng.uniform(0, 1, 1500), rng.uniform(1000, 1001, 1500)]))
    probs.append((d, rng.standard_normal(3000)))
    z = rng.standard_normal(2000) * 1e-3
    z[5] = 30.0
    probs.append((np.sort(rng.uniform(0, 1, 2000)), z))
    # 30 decades: every box is wider than all boxes to its left together, so
    # near lists grow with the index until the list pool runs out and leaves
    # fall back to direct sums over every source
    probs.append((np.geomspace(1e-10, 1e20, 4096), rng.standard_normal(4096)))
    # the last pole alone beyond a wide gap, m = 3 * 1024 + 1 and 8 * 1024 + 1:
    # its leaf box and five or more ancestors hold that one point (boxes of
    # zero width, whose far field passes from level to level on the nodes)
    for m in (3073, 8193):
        d = np.append(np.sort(rng.uniform(-8.6, 5.2, m - 1)), 5.81)
        probs.append((d, rng.standard_normal(m)))
    offs = np.zeros(len(probs) + 1, np.int64)
    offs[1:] = np.cumsum([len(p[0]) for p in probs])
    d = np.concatenate([p[0] for p in probs]).astype(np.float64)
    z = np.concatenate([p[1] for p in probs]).astype(np.float64)
    return inputs.SecularBatch(offs, d, z, 1.0)


def test_fmm_secular_vs_oracle():
    b = fmm_batch()
    out = run_batch(b, 1e-12, fmm_min_m=FMM_ON)
    for p in range(b.nprob):
        d, z = b.problem(p)
        g = P.gpu_problem(out, b.offsets, p)
        assert out["fmm"][p] == (1 if g["mk"] >= FMM_ON else 0), (p, g["mk"], out["fmm"][p])
        P.compare_problem(g, d, z, 1e-12, mode=0)


def test_fmm_results_are_reproducible():
    """The tail pass takes straggler roots in whatever order its warps claim
    them, and the upward pass computes each parent box in whichever CTA
    finishes its second child last (leaf boxes claimed from a queue); every
    root's and every box's arithmetic is independent of that order, so two
    runs agree bit for bit (three far fields per plan, so the arrival counters
    and the queue reset themselves between launches)."""
    b = fmm_batch()
    o1 = run_batch(b, 1e-12, fmm_min_m=FMM_ON)
    o2 = run_batch(b, 1e-12, fmm_min_m=FMM_ON)
    assert np.array_equal(o1["lam"], o2["lam"])
    assert np.array_equal(o1["mk"], o2["mk"])
    kept = np.zeros(len(o1["lam"]), bool)            # slots of kept roots (the rest is not written)
    for p in range(b.nprob):
        kept[b.offsets[p]:b.offsets[p] + o1["mk"][p]] = True
    for key in ("eta", "org", "vhat", "bnorm", "sweeps"):
        assert np.array_equal(o1[key][kept], o2[key][kept]), key


def test_fmm_matches_direct_evaluator():
    """Same batch through both evaluators: eigenvalues to 1e-12 of the scale,
    gaps, zhat and b to the tolerances of two independently converged runs."""
    b = fmm_batch()
    of = run_batch(b, 1e-12, fmm_min_m=FMM_ON)
    od = run_batch(b, 1e-12, fmm_min_m=FMM_OFF)
    assert of["fmm"][:b.nprob].sum() > 0 and od["fmm"][:b.nprob].sum() == 0
    for p in range(b.nprob):
        gf, gd = P.gpu_problem(of, b.offsets, p), P.gpu_problem(od, b.offsets, p)
        mk = gf["mk"]
        assert mk == gd["mk"]
        scale = np.abs(gd["lam"]).max()
        assert np.abs(gf["lam"] - gd["lam"]).max() <= 1e-12 * scale, p
        same = gf["org"][:mk] == gd["org"][:mk]
        assert same.mean() >= 0.99
        ef, ed = gf["eta"][:mk][same], gd["eta"][:mk][same]
        assert np.all(np.abs(ef - ed) <= P.ETA_RTOL * np.abs(ed)), p
        # zhat and b of two root sets that agree to ETA_RTOL: each root moves
        # zhat_i by its gap error over (lambda_j - d_i), up to ~1e-9 relative
        assert np.all(np.abs(gf["vhat"][:mk] - gd["vhat"][:mk]) <= 1e-8 * np.abs(gd["vhat"][:mk])), p
        assert np.all(np.abs(gf["bnorm"][:mk] - gd["bnorm"][:mk]) <= 1e-8 * np.abs(gd["bnorm"][:mk])), p


def test_fmm_eig_small_vs_oracle_and_dense():
    """n=2048 (leaf 32, rank 4) with every node of at least 256 kept entries on
    the FMM path: eigenvalues vs the oracle and eigh, dense Q residual and
    orthogonality at the paper's metrics."""
    h = inputs.hss_random(2048, 32, 4, seed=21)
    A = dense.dense_from_hss(h)
    H = sdc.HSSMatrix(h)
    lam, F = H.eig(sdc.default_opts(tau=1e-10, fmm_min_m=FMM_ON))
    lam = lam.cpu().numpy()
    assert F.get(0, 0, "fmm")[0] == 1
    O = osd.superdc(h, tau=1e-10, mode=0)
    an = np.linalg.norm(A, 2)
    assert np.all(np.abs(lam - O.eigenvalues) <= 1e-10 * an)
    assert np.all(np.abs(lam - np.linalg.eigvalsh(A)) <= 1e-10 * an)
    n = h.tree.n
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    Q = F.apply_Q(I).cpu().numpy()
    QT = F.apply_Q(I, trans=True).cpu().numpy()
    assert np.abs(QT - Q.T).max() < 1e-12
    assert dense.gamma(A, lam, Q) <= 1e-12
    assert dense.theta(Q) <= 1e-12
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-11


def test_fmm_apply_matches_direct_on_same_factor():
    """One factorisation, Q X and Q^T X through the FMM and the direct
    Cauchy kernels: agreement to 1e-12 of the block's scale."""
    h = inputs.hss_random(8192, 64, 6, seed=22)
    H = sdc.HSSMatrix(h)
    lam, F = H.eig(sdc.default_opts(tau=1e-10, fmm_min_m=FMM_ON))
    n = h.tree.n
    X = torch.from_numpy(inputs.normal_block(n, 37, seed=5)).cuda()
    out = {}
    for mode in (FMM_ON, FMM_OFF):
        F.set_fmm_min_m(mode)
        out[mode] = (F.apply_Q(X), F.apply_Q(X, trans=True))
    s = X.abs().max().item()
    assert (out[FMM_ON][0] - out[FMM_OFF][0]).abs().max().item() <= 1e-12 * s * np.sqrt(n)
    assert (out[FMM_ON][1] - out[FMM_OFF][1]).abs().max().item() <= 1e-12 * s * np.sqrt(n)


def test_fmm_eig_matches_direct_eig_16384_clustered():
    """Clustered spectra (config n=16384): the default threshold puts the top
    levels on the FMM path; eigenvalues agree with the direct-only run to
    1e-10 ||A|| and the factor stays orthogonal on probes."""
    h = inputs.cfg_clustered_16384()
    H = sdc.HSSMatrix(h)
    lf, Ff = H.eig(sdc.default_opts(tau=1e-10))
    ld, Fd = H.eig(sdc.default_opts(tau=1e-10, fmm_min_m=FMM_OFF))
    assert Ff.get(0, 0, "fmm")[0] == 1 and Fd.get(0, 0, "fmm")[0] == 0
    lf, ld = lf.cpu().numpy(), ld.cpu().numpy()
    an = np.abs(ld).max()
    assert np.abs(lf - ld).max() <= 1e-10 * an
    n = h.tree.n
    Xn = inputs.normal_block(n, 16, seed=8)
    X = torch.from_numpy(Xn).cuda()
    back = Ff.apply_Q(Ff.apply_Q(X), trans=True).cpu().numpy()
    assert np.linalg.norm(back - Xn) / np.linalg.norm(Xn) < 1e-12 * np.sqrt(n)
