"""Pins of the oracle functions added for the parity tests at full size and
for the extension rows (partial root sets, secular function values, the
original dividing, complex Hermitian assembly, kernel matrices) against
mathematics that does not go through the oracle: mpmath roots, numpy's dense
eigenvectors, closed forms, hand-computed values, reassembly of A.  (No GPU.)"""
import numpy as np
import pytest

from oracle import dense, rank1 as r1, superdc as sd
from paper_2108_04209_gb300 import inputs
from tests.test_oracle_rank1 import mp_roots, rand_problem

mpmath = pytest.importorskip("mpmath")


@pytest.mark.parametrize("mode", [0, 1])
def test_secular_some_vs_mpmath(mode):
    """Roots of a chosen subset (first, middle, clustered, last) of a kept
    problem: each gap d_K + eta - d_K against the 50-digit root (Section 4.2's
    relative gap accuracy), and the same values as the all-roots routine."""
    d, z = rand_problem(30, 7, cluster=True)
    f = r1.rank1_step(d, z, tau=1e-14, mode=mode)
    assert f.mk == 30
    ks = np.array([0, 9, 10, 11, 12, 17, 29], np.int32)
    K, eta, it, bad = r1.secular_some(f.dk, f.zk, ks, mode=mode)
    assert bad == 0 and np.all(it >= 1)
    lam_star = mp_roots(f.dk, f.zk)
    for t, k in enumerate(ks):
        eta_star = lam_star[k] - mpmath.mpf(float(f.dk[K[t]]))
        tol = (1e-12 if mode == 0 else 1e-9) * abs(eta_star)
        assert abs(mpmath.mpf(float(eta[t])) - eta_star) <= tol, (k, float(eta_star))
    assert np.array_equal(K, f.K[ks]) and np.array_equal(eta, f.eta[ks])
    K0, eta0, it0, bad0 = r1.secular_some(f.dk, f.zk, np.zeros(0, np.int32))
    assert len(K0) == 0 and bad0 == 0


def test_secular_eval_closed_form_m1():
    """m = 1: f(lambda) = 1 + z^2/(d - lambda), root d + z^2, so with origin 0
    and gap y = z^2: f = 0, psi = -1, phi = 0, f' = z^2/y^2 = 1/z^2."""
    z = 0.75
    f, psi, phi, df = r1.secular_eval(np.array([0.5]), np.array([z]), [0], [0], [z * z])
    assert abs(f[0]) <= 1e-15 and abs(psi[0] + 1) <= 1e-15 and phi[0] == 0.0
    assert abs(df[0] - 1 / z ** 2) <= 1e-15 / z ** 2


def test_secular_eval_at_exact_roots_and_eigenvectors():
    """At the 50-digit roots (rounded to doubles, expressed as origin + gap):
    f vanishes to rounding, psi < 0 < phi (the split of eqs. (4.7)/(4.8) at
    root k), and f' fixes the eigenvector's normalisation: the eigenvector of
    D + z z^T for lambda_k has squared entries z_j^2/(d_j - lambda_k)^2 / f',
    checked against numpy's eigh of the dense matrix."""
    d, z = rand_problem(20, 11)
    m = len(d)
    lam_star = mp_roots(d, z)
    ks = np.arange(m, dtype=np.int32)
    Ks = np.array([k if (k + 1 == m or lam_star[k] - d[k] <= d[k + 1] - lam_star[k]) else k + 1
                   for k in range(m)], np.int32)
    ys = np.array([float(lam_star[k] - mpmath.mpf(float(d[Ks[k]]))) for k in range(m)])
    f, psi, phi, df = r1.secular_eval(d, z, ks, Ks, ys)
    assert np.all(np.abs(f) <= 64 * m * np.finfo(float).eps * (1 + np.abs(psi) + np.abs(phi)))
    assert np.all(psi < 0) and np.all(phi[:-1] > 0) and phi[-1] == 0.0
    w, V = np.linalg.eigh(np.diag(d) + np.outer(z, z))
    for k in range(m):
        gap = (d - d[Ks[k]]) - ys[k]
        v2 = z ** 2 / gap ** 2 / df[k]
        assert abs(w[k] - float(lam_star[k])) <= 1e-13
        assert np.abs(v2 - V[:, k] ** 2).max() <= 1e-10, k


@pytest.mark.parametrize("bscale", [1.0, 3.0])
def test_original_dividing_reassembles_A(bscale):
    """Eqs. (2.4)/(2.5) with scale 1: the leaf blocks D - U (B B^T) U^T (or
    D - U U^T) and the unscaled Z_p = [U B; U] still sum back to A."""
    h = inputs.hss_random(512, 32, 4, seed=0, bscale=bscale)
    A = dense.dense_from_hss(h)
    dv = sd.divide(h, balanced=False)
    t = h.tree
    R = np.zeros_like(A)
    for i in t.leaves:
        o, m = int(t.offset[i]), int(t.leaf_size[i])
        R[o:o + m, o:o + m] = dv.Dhat[i]
    for i, Z in dv.Z.items():
        o, m = int(t.offset[i]), int(t.leaf_size[i])
        R[o:o + m, o:o + m] += Z @ Z.T
    scale = max(np.abs(A).max(), max(np.abs(dv.Dhat[i]).max() for i in t.leaves))
    assert np.abs(R - A).max() < 1e-14 * scale * 64
    # the unbalanced Z of a node is [U_c1 B~; U_c2] (or its swap): its second block has unit scale
    # (the nested U of hss_random are orthonormal, so that block's Gram matrix is I)
    root = t.root
    assert not dv.swapped[root]
    Z2 = dv.Z[root][int(t.leaf_size[int(t.lchild[root])]):, :]
    assert np.abs(Z2.T @ Z2 - np.eye(4)).max() <= 1e-12


def test_original_dividing_norm_growth():
    """Proposition 3.1: with ||B|| = beta > 1 the original dividing's updated
    generators grow doubly exponentially with depth; the balanced ones stay
    within Proposition 3.2's 2^l beta."""
    h = inputs.hss_random(256, 32, 3, seed=5, bscale=10.0)
    t = h.tree
    beta = max(np.linalg.norm(h.B[i], 2) for i in range(t.nnodes) if i != t.root)
    orig = sd.divide(h, balanced=False)
    bal = sd.divide(h, balanced=True)
    lmax = int(t.level.max())
    assert max(orig.beta.values()) >= beta ** 2
    assert max(bal.beta.values()) <= 2 ** lmax * beta * (1 + 1e-12)


def test_hermitian_assembly_brute_force():
    """Two levels written out by hand: A = [[A11, A12], [A12^H, A22]] with
    A11 = [[D1, U1 B1 U2^H], [.^H, D2]], A12 = [U1 R1; U2 R2] B3 [U4 R4; U5 R5]^H
    (postorder 0,1 | 2 ; 3,4 | 5 ; 6); Hermitian; real generators give the
    real assembly."""
    h = inputs.hss_random_hermitian(64, 16, 3, seed=4)
    t = h.tree
    assert t.nnodes == 7 and t.root == 6
    A = dense.dense_from_hss_hermitian(h)
    D = [h.leaf_D(i) for i in (0, 1, 3, 4)]
    U = [h.leaf_U(i) for i in (0, 1, 3, 4)]
    H = lambda M: M.conj().T  # noqa: E731
    E = np.zeros((64, 64), np.complex128)
    for q, o in enumerate((0, 16, 32, 48)):
        E[o:o + 16, o:o + 16] = D[q]
    for (a, b, oa, ob, Bi) in ((0, 1, 0, 16, h.B[0]), (2, 3, 32, 48, h.B[3])):
        E[oa:oa + 16, ob:ob + 16] = U[a] @ Bi @ H(U[b])
        E[ob:ob + 16, oa:oa + 16] = H(U[a] @ Bi @ H(U[b]))
    L = np.vstack([U[0] @ h.R[0], U[1] @ h.R[1]])
    Rt = np.vstack([U[2] @ h.R[3], U[3] @ h.R[4]])
    E[0:32, 32:64] = L @ h.B[2] @ H(Rt)
    E[32:64, 0:32] = H(E[0:32, 32:64])
    assert np.abs(A - E).max() <= 1e-13
    assert np.abs(A - H(A)).max() <= 1e-13
    hr = inputs.hss_random(64, 16, 3, seed=4)
    assert np.abs(dense.dense_from_hss_hermitian(hr) - dense.dense_from_hss(hr)).max() <= 1e-14


def test_kernel_matrix_values():
    """sqrt|x_i - x_j| at x = (0, 1, 4) by hand; exp(-|x_i - x_j|/2) likewise;
    Chebyshev points cos((2i-1)pi/(2n)) for n = 2 are +-1/sqrt(2)."""
    K = dense.kernel_matrix(np.array([0.0, 1.0, 4.0]))
    E = np.array([[0, 1, 2], [1, 0, np.sqrt(3)], [2, np.sqrt(3), 0]])
    assert np.abs(K - E).max() <= 1e-15
    K2 = dense.kernel_matrix(np.array([0.0, 1.0, 4.0]), "exp", 2.0)
    E2 = np.exp(-np.array([[0, 1, 4], [1, 0, 3], [4, 3, 0]]) / 2.0)
    assert np.abs(K2 - E2).max() <= 1e-15
    x = inputs.chebyshev_points(2)
    assert np.abs(x - np.array([1, -1]) / np.sqrt(2)).max() <= 1e-15
