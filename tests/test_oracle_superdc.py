"""Pins of the CPU oracle's dividing and conquering stages (Algorithms 1, 3, 4)
against dense eigensolvers, closed forms and invariants.  (No GPU.)"""
import json
import os

import numpy as np
import pytest

from oracle import dense, superdc as sd
from paper_2108_04209_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_jacobi_vs_numpy():
    rng = np.random.default_rng(0)
    G = rng.standard_normal((40, 40))
    A = (G + G.T) / 2
    lam, V = sd.jacobi_eig(A)
    tol = 64 * np.finfo(float).eps * np.linalg.norm(A, 2)   # backward-stable level
    assert np.abs(lam - np.linalg.eigvalsh(A)).max() < tol
    assert np.abs(V.T @ V - np.eye(40)).max() < 1e-13
    assert np.abs(A @ V - V * lam).max() < tol


def test_dense_assembly_matches_generators():
    h = inputs.hss_random(256, 32, 4, seed=9)
    A = dense.dense_from_hss(h)
    assert np.allclose(A, A.T)
    assert abs(np.trace(A) - dense.trace_from_generators(h)) < 1e-12
    assert abs((A ** 2).sum() - dense.fro2_from_generators(h)) < 1e-10 * (A ** 2).sum()


def _reassemble(h, dv):
    """diag(Dhat_leaves) + sum over nodes of the Z_p Z_p^T blocks (eq. (2.4) applied recursively)."""
    t = h.tree
    A = np.zeros((t.n, t.n))
    for i in t.leaves:
        o, m = int(t.offset[i]), int(t.leaf_size[i])
        A[o:o + m, o:o + m] = dv.Dhat[i]
    for i, Z in dv.Z.items():
        o, m = int(t.offset[i]), int(t.leaf_size[i])
        A[o:o + m, o:o + m] += Z @ Z.T
    return A


@pytest.mark.parametrize("bscale", [1.0, 1e3])
def test_dividing_reassembles_A(bscale):
    h = inputs.hss_random(512, 32, 4, seed=0, bscale=bscale)
    A = dense.dense_from_hss(h)
    dv = sd.divide(h)
    err = np.abs(_reassemble(h, dv) - A).max()
    assert err < 1e-14 * np.abs(A).max() * 64


def test_prop32_norm_bound():
    # Proposition 3.2, eq. (3.13): after balanced dividing ||B~_k|| <= 2^l beta
    h = inputs.hss_random(1024, 32, 4, seed=1, bscale=1e3)
    beta = max(np.linalg.norm(h.B[i], 2) for i in range(h.tree.nnodes))
    dv = sd.divide(h)
    t = h.tree
    for i in range(t.nnodes):
        if t.lchild[i] >= 0:
            c1 = int(t.lchild[i])
            lev = int(t.level[c1])
            assert np.linalg.norm(dv.Bt[c1], 2) <= (2 ** lev) * beta * (1 + 1e-12)


@pytest.mark.parametrize("mode", [0, 1])
def test_small_hss_vs_dense(mode):
    h = inputs.cfg_small_hss()
    A = dense.dense_from_hss(h)
    F = sd.superdc(h, tau=1e-10, mode=mode)
    lam = F.eigenvalues
    ev = np.linalg.eigvalsh(A)
    assert np.abs(lam - ev).max() <= 1e-10 * np.abs(ev).max()
    Q = sd.superdcmv(F, h.tree.root, np.eye(h.tree.n), 0)
    QT = sd.superdcmv(F, h.tree.root, np.eye(h.tree.n), 1)
    assert np.abs(QT - Q.T).max() < 1e-13
    assert dense.gamma(A, lam, Q) < 1e-15
    assert dense.theta(Q) < 1e-15
    assert abs(lam.sum() - dense.trace_from_generators(h)) < 1e-11 * np.abs(lam).sum()


def test_brute_force_dense_jacobi():
    """Full SuperDC vs a brute-force dense cyclic Jacobi of the assembled matrix."""
    h = inputs.hss_random(128, 16, 3, seed=12)
    A = dense.dense_from_hss(h)
    lj, _ = sd.jacobi_eig(A)
    F = sd.superdc(h, tau=1e-10, mode=0)
    assert np.abs(F.eigenvalues - lj).max() <= 1e-12 * np.abs(lj).max()


def test_tridiagonal_closed_form_and_table1():
    g = json.load(open(os.path.join(GOLDEN, "example1_table1.json")))
    n = g["table1"]["n"][0]          # 8192
    h = inputs.hss_tridiag(n, 256, g["matrix"]["diag"], g["matrix"]["offdiag"])
    F = sd.superdc(h, tau=g["matrix"]["tau"], mode=1)
    k = np.arange(1, n + 1)
    exact = np.sort(3.0 - 2.0 * np.cos(k * np.pi / (n + 1)))
    lam = F.eigenvalues
    assert np.abs(lam - exact).max() < 1e-12
    # relative error delta of Section 5 against the closed form: the paper
    # reports 1.6e-18 at this n (Table 1); allow one order of magnitude
    assert dense.delta(lam, exact) <= 10 * g["table1"]["delta"][0]


def test_tridiagonal_small_full_metrics():
    n = 1024
    h = inputs.hss_tridiag(n, 64)
    A = dense.dense_from_hss(h)
    F = sd.superdc(h, tau=1e-10, mode=0)
    Q = sd.superdcmv(F, h.tree.root, np.eye(n), 0)
    # Table 1 reports gamma, theta of a few 1e-16; ours must be of that order
    assert dense.gamma(A, F.eigenvalues, Q) < 1e-15
    assert dense.theta(Q) < 1e-15


def test_clustered_leaves_deflate():
    h = inputs.hss_random(1024, 64, 8, seed=2, clustered=True)
    A = dense.dense_from_hss(h)
    F = sd.superdc(h, tau=1e-10, mode=1)
    ev = np.linalg.eigvalsh(A)
    assert np.abs(F.eigenvalues - ev).max() < 1e-9 * np.abs(ev).max() + 1e-8
    _, nbad, ndefl = F.stats()
    assert nbad == 0
    Q = sd.superdcmv(F, h.tree.root, np.eye(1024), 0)
    assert dense.theta(Q) < 1e-15
    assert dense.gamma(A, F.eigenvalues, Q) < 1e-12


def test_hss_matvec_vs_dense():
    for h in (inputs.hss_random(512, 32, 4, seed=0), inputs.hss_tridiag(256, 16)):
        A = dense.dense_from_hss(h)
        X = np.random.default_rng(1).standard_normal((h.tree.n, 3))
        assert np.abs(dense.hss_matvec(h, X) - A @ X).max() < 1e-13 * np.abs(A).max() * 10


@pytest.mark.parametrize("sizes,rank", [([1, 7, 128, 33, 2, 64, 100, 5], 4), ([37], 3), ([3, 1], 5),
                                        ([16] * 7 + [9], 2)])
def test_ragged_leaves_and_single_leaf_vs_dense(sizes, rank):
    """Perfect trees with ragged leaf sizes (1 to 128 rows, leaves smaller
    than the rank), a single-leaf tree and a two-leaf tree whose size is below
    the rank: eigenvalues against numpy's eigvalsh of the assembled matrix,
    the dense Q against the paper's metrics."""
    h = inputs.hss_random_sizes(sizes, rank, seed=3)
    A = dense.dense_from_hss(h)
    F = sd.superdc(h, tau=1e-14, mode=0)
    lam = F.eigenvalues
    ev = np.linalg.eigvalsh(A)
    an = np.abs(ev).max()
    assert np.abs(lam - ev).max() <= 1e-12 * an
    n = h.tree.n
    Q = sd.superdcmv(F, h.tree.root, np.eye(n), 0)
    assert dense.gamma(A, lam, Q) < 1e-14
    assert dense.theta(Q) < 1e-14
