"""Pins of the CPU oracle's rank-one step against mathematics, independent of
the oracle itself: mpmath at 50 digits, closed forms, dense eigensolvers,
invariants.  (Test infrastructure; no GPU.)"""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

from oracle import rank1 as r1  # noqa: E402
from paper_2108_04209_gb300 import inputs  # noqa: E402

mp = mpmath.mp


def mp_roots(d, z):
    """All roots of 1 + sum z_j^2/(d_j - x) (distinct d, z != 0) by bisection at 50 digits."""
    mp.dps = 50
    dm = [mpmath.mpf(float(x)) for x in d]
    wm = [mpmath.mpf(float(x)) ** 2 for x in z]
    m = len(d)

    def f(x):
        return 1 + mpmath.fsum(wm[j] / (dm[j] - x) for j in range(m))

    out = []
    W = mpmath.fsum(wm)
    for k in range(m):
        lo = dm[k]
        hi = dm[k + 1] if k + 1 < m else dm[k] + W
        for _ in range(200):
            mid = (lo + hi) / 2
            if f(mid) < 0:
                lo = mid
            else:
                hi = mid
        out.append((lo + hi) / 2)
    return out


def rand_problem(m, seed, cluster=False):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(0, 1, m))
    if cluster:
        s = m // 3
        d[s:s + 5] = d[s] + rng.uniform(0, 1e-10, 5)
        d.sort()
    z = rng.standard_normal(m)
    return d, z


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed,cluster", [(1, False), (2, False), (3, True), (4, True)])
def test_roots_gaps_vs_mpmath(mode, seed, cluster):
    d, z = rand_problem(24, seed, cluster)
    f = r1.rank1_step(d, z, tau=1e-14, mode=mode)
    assert f.mk == 24 and f.nbad == 0
    lam_star = mp_roots(f.dk, f.zk)
    for k in range(f.mk):
        eta_star = lam_star[k] - mpmath.mpf(float(f.dk[f.K[k]]))
        err = abs(mpmath.mpf(float(f.eta[k])) - eta_star)
        # gap accuracy relative to the gap itself (local shifting, Section 4.2)
        tol = (1e-12 if mode == 0 else 1e-9) * abs(eta_star)
        assert err <= tol, (k, float(err), float(eta_star))
        # interlacing d_k < lambda_k < d_{k+1} (eq. (4.4))
        assert lam_star[k] > f.dk[k]
        if k + 1 < f.mk:
            assert lam_star[k] < f.dk[k + 1]
        # the origin is the nearer pole (Section 4.2.1)
        if k + 1 < f.mk:
            mid = (mpmath.mpf(float(f.dk[k])) + mpmath.mpf(float(f.dk[k + 1]))) / 2
            assert (f.K[k] == k) == (lam_star[k] <= mid) or abs(lam_star[k] - mid) < 1e-15


def test_exact_mode_backward_error():
    """Bisection to adjacent doubles: at the returned gap the true g_K (50
    digits) is within the rounding level of one FP64 evaluation, i.e. well
    inside the stopping test of eq. (4.12)."""
    d, z = rand_problem(40, 7, cluster=True)
    f = r1.rank1_step(d, z, tau=1e-14, mode=0)
    w = f.zk ** 2
    mp.dps = 40
    eps = np.finfo(float).eps
    for k in range(0, f.mk, 3):
        y = mpmath.mpf(float(f.eta[k]))
        dK = mpmath.mpf(float(f.dk[f.K[k]]))
        terms = [mpmath.mpf(float(w[j])) / ((mpmath.mpf(float(f.dk[j])) - dK) - y) for j in range(f.mk)]
        g = 1 + mpmath.fsum(terms)
        scale = 1 + mpmath.fsum(abs(t) for t in terms)
        assert abs(g) <= 2 * f.mk * eps * scale, (k, float(g), float(scale))


@pytest.mark.parametrize("mode", [0, 1])
def test_zhat_and_b_vs_mpmath(mode):
    d, z = rand_problem(20, 11)
    f = r1.rank1_step(d, z, tau=1e-14, mode=mode)
    # Loewner's formula reproduces |z| when the roots are exact (eq. (4.23))
    assert np.allclose(np.abs(f.vhat), np.abs(f.zk), rtol=1e-10, atol=0)
    assert np.all(np.sign(f.vhat) == np.sign(f.zk))
    lam_star = mp_roots(f.dk, f.zk)
    for j in range(f.mk):
        s = mpmath.fsum((mpmath.mpf(float(f.zk[i])) ** 2) / (mpmath.mpf(float(f.dk[i])) - lam_star[j]) ** 2
                        for i in range(f.mk))
        bstar = 1 / mpmath.sqrt(s)
        assert abs(f.b[j] - bstar) <= 1e-10 * bstar


@pytest.mark.parametrize("mode,rtol", [(0, 1e-12), (1, 1e-10)])
def test_zhat_and_b_isolated_last_pole_and_close_pair(mode, rtol):
    """The structure of a large merge whose last pole sits alone beyond a
    wide gap, with a pair of poles 1e-9 apart inside: zhat from Loewner's
    formula still reproduces |z| and b matches the 50-digit value (eqs.
    (4.23), (4.27)); the last root lies right of d_{m-1} within sum z^2."""
    rng = np.random.default_rng(17)
    m = 40
    d = np.sort(rng.uniform(0, 1, m - 1))
    d[10:12] = d[10] + np.array([0.0, 1e-9])
    d = np.append(np.sort(d), 3.0)
    z = rng.standard_normal(m)
    f = r1.rank1_step(d, z, tau=1e-14, mode=mode)
    assert f.mk == m
    assert np.all(np.abs(np.abs(f.vhat) - np.abs(f.zk)) <= rtol * np.abs(f.zk))
    lam_star = mp_roots(f.dk, f.zk)
    assert lam_star[-1] > f.dk[-1] and lam_star[-1] < f.dk[-1] + mpmath.fsum(mpmath.mpf(float(x)) ** 2 for x in f.zk)
    for j in range(f.mk):
        s = mpmath.fsum((mpmath.mpf(float(f.zk[i])) ** 2) / (mpmath.mpf(float(f.dk[i])) - lam_star[j]) ** 2
                        for i in range(f.mk))
        bstar = 1 / mpmath.sqrt(s)
        assert abs(f.b[j] - bstar) <= rtol * bstar, j


@pytest.mark.parametrize("m,seed,cluster,tau", [(30, 1, False, 1e-12), (64, 5, True, 1e-12),
                                                (64, 6, True, 1e-10), (200, 8, True, 1e-9)])
def test_factor_diagonalises(m, seed, cluster, tau):
    d, z = rand_problem(m, seed, cluster)
    M = np.diag(d) + np.outer(z, z)
    f = r1.rank1_step(d, z, tau=tau, mode=0)
    Q = f.dense()
    assert np.abs(Q.T @ Q - np.eye(m)).max() < 1e-13
    # eigenpairs up to the deflation perturbation (Remark 4.1: dropped entries < tau)
    res = np.abs(M @ Q - Q * f.lam).max()
    assert res < 1e-13 + 4 * tau * max(1, f.m - f.mk)
    ev = np.linalg.eigvalsh(M)
    assert np.abs(np.sort(f.lam) - ev).max() < 1e-14 * np.abs(ev).max() + 4 * tau * (m - f.mk + 1)
    # lam ascending, and the kept roots interlace the kept poles
    assert np.all(np.diff(f.lam) >= 0)
    lk = f.lam_kept
    assert np.all(lk > f.dk)
    assert np.all(lk[:-1] < f.dk[1:])


def test_invariants_trace_and_squares():
    d, z = rand_problem(100, 3)
    f = r1.rank1_step(d, z, tau=1e-14)
    assert f.mk == 100
    assert abs(f.lam.sum() - (d.sum() + z @ z)) < 1e-13 * (abs(d).sum() + z @ z)
    s2 = (d ** 2).sum() + 2 * (d * z * z).sum() + (z @ z) ** 2
    assert abs((f.lam ** 2).sum() - s2) < 1e-12 * s2
    # last root bound lambda_m <= d_m + ||z||^2
    assert f.lam[-1] <= d[-1] + z @ z


def test_special_m1():
    f = r1.rank1_step(np.array([0.3]), np.array([0.7]), tau=1e-12)
    assert abs(f.lam[0] - (0.3 + 0.49)) <= 2 * np.finfo(float).eps
    assert abs(abs(f.dense()[0, 0]) - 1) < 1e-15


def test_special_m2_closed_form():
    d = np.array([0.1, 0.5])
    z = np.array([0.3, -0.4])
    M = np.diag(d) + np.outer(z, z)
    tr, det = np.trace(M), np.linalg.det(M)
    disc = np.sqrt(tr * tr / 4 - det)
    exact = np.array([tr / 2 - disc, tr / 2 + disc])
    f = r1.rank1_step(d, z, tau=1e-12)
    assert np.allclose(f.lam, exact, rtol=1e-15, atol=1e-16)


def test_special_unit_vector():
    m = 12
    d = np.linspace(0, 1, m)
    z = np.zeros(m)
    z[5] = 1.0
    f = r1.rank1_step(d, z, tau=1e-12)
    exp = d.copy()
    exp[5] += 1.0
    assert np.allclose(f.lam, np.sort(exp), atol=1e-15)
    assert f.mk == 1


def test_special_zero_vector_all_deflated():
    m = 10
    d = np.linspace(-1, 1, m)
    f = r1.rank1_step(d, np.zeros(m), tau=1e-12)
    assert f.mk == 0
    assert np.array_equal(f.lam, d)
    assert np.array_equal(f.dense(), np.eye(m))


def test_deflation_rules():
    # step 1: |z| < tau deflates; step 2: the Givens test of Remark 4.1 on neighbours
    d = np.array([0.0, 0.5, 0.5 + 1e-13, 0.9, 1.0])
    z = np.array([0.5, 0.6, 0.8, 1e-13, 0.7])
    dd, zz, kept, giv = r1.deflate(d, z, 1e-12)
    assert list(kept) == [True, False, True, False, True]
    assert len(giv[0]) == 1 and giv[0][0] == 1 and giv[1][0] == 2
    rho = np.hypot(0.6, 0.8)
    assert abs(zz[2] - rho) < 1e-15 and zz[1] == 0.0
    # the rotation diagonalises the 2x2 block up to the dropped entry
    c, s = giv[2][0], giv[3][0]
    G = np.array([[c, -s], [s, c]])
    M2 = np.diag(d[1:3]) + np.outer(z[1:3], z[1:3])
    T = G @ M2 @ G.T
    assert abs(T[0, 1]) < 1e-12
    assert abs(T[0, 0] - dd[1]) < 1e-15 and abs(T[1, 1] - (dd[2] + rho ** 2)) < 1e-14
    # pair just outside the threshold stays
    d2 = np.array([0.0, 1e-10])
    z2 = np.array([1.0, 1.0])
    assert r1.deflate(d2, z2, 1e-11)[2].all()         # |dd z z| = 1e-10 > 2e-11
    assert not r1.deflate(d2, z2, 1e-10)[2].all()     # 1e-10 < 2e-10


def test_newton_matches_exact_on_config_distribution():
    b = inputs.secular_batch(6, 32, 300, seed=5)
    for p in range(b.nprob):
        d, z = b.problem(p)
        f0 = r1.rank1_step(d, z, tau=1e-12, mode=0)
        f1 = r1.rank1_step(d, z, tau=1e-12, mode=1)
        assert f1.nbad == 0
        assert np.abs(f0.lam - f1.lam).max() <= 1e-12 * np.abs(f0.lam).max()
        same = f0.K == f1.K
        assert same.mean() > 0.99
        g0, g1 = f0.eta[same], f1.eta[same]
        assert np.all(np.abs(g0 - g1) <= 1e-9 * np.abs(g0) + 1e-300)
