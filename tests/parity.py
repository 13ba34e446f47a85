"""Shared comparison helpers for the GPU parity tests (CUDA path vs oracle).

Tolerances (derived from the arithmetic):
  * eigenvalues: |lam - lam_o| <= 1e-10 * max(|lam_o|, scale)  (spec bound);
  * gaps eta (same origin): the GPU stops at the test of eq. (4.12), the
    oracle bisects to adjacent doubles; |y - y*| <= 8 m eps (1+|psi|+|phi|)/g'
    gives a relative gap error of a few 1e-12 -> bound 1e-9 relative;
  * vhat, b: products/sums of m such gaps -> bound 1e-8 relative;
  * deflation decisions, rotations and the kept/deflated layout: bit-exact
    (both sides evaluate them with the same IEEE operations in the same order);
  * the merge permutation: bit-exact unless two new eigenvalues are within
    rounding of each other.
"""
import numpy as np

from oracle import rank1 as r1

LAM_RTOL = 1e-10
ETA_RTOL = 1e-9
VEC_RTOL = 1e-8


def gpu_problem(out, offs, p):
    """Slice problem p from host copies of the batched outputs."""
    a, b = int(offs[p]), int(offs[p + 1])
    m = b - a
    mk = int(out["mk"][p])
    ng = int(out["ngiv"][p])
    g = {k: out[k][a:b] for k in ("lam", "dk", "zk", "eta", "vhat", "bnorm", "org", "src", "perm")}
    g["m"], g["mk"], g["ng"] = m, mk, ng
    g["giv_ab"] = out["giv_ab"][2 * a:2 * a + 2 * ng].reshape(-1, 2)
    g["giv_cs"] = out["giv_cs"][2 * a:2 * a + 2 * ng].reshape(-1, 2)
    if out.get("sweeps") is not None:
        g["sweeps"] = out["sweeps"][a:b]
    return g


def near_tie_count(d, z, tau):
    """Deflation tests of the oracle's scan whose value is within 1e-8 of the threshold."""
    n = 0
    zz = np.where(np.abs(z) < tau, 0.0, z)
    n += int(np.sum(np.abs(np.abs(z) - tau) <= 1e-8 * tau))
    idx = np.nonzero(zz)[0]
    for a, b in zip(idx[:-1], idx[1:]):
        lhs = abs((d[a] - d[b]) * zz[a] * zz[b])
        rhs = (zz[a] ** 2 + zz[b] ** 2) * tau
        if rhs > 0 and abs(lhs - rhs) <= 1e-8 * rhs:
            n += 1
    return n


def compare_problem(g, d, z, tau, rho=1.0, mode=0):
    """Compare one GPU problem with the oracle.  Returns a dict of stats; raises AssertionError."""
    f = r1.rank1_step(d, z, tau, rho=rho, mode=mode)
    m = g["m"]
    assert m == f.m
    # deflation is evaluated with the same IEEE operations in the same order
    # on both sides: decisions, rotations and the slot layout are bit-exact
    assert g["mk"] == f.mk, (g["mk"], f.mk)
    assert np.array_equal(g["src"][:g["mk"]], f.kidx), "kept set differs"
    assert g["ng"] == len(f.giv[0])
    if g["ng"]:
        assert np.array_equal(g["giv_ab"][:, 0], f.giv[0]) and np.array_equal(g["giv_ab"][:, 1], f.giv[1])
        assert np.array_equal(g["giv_cs"][:, 0], f.giv[2]) and np.array_equal(g["giv_cs"][:, 1], f.giv[3])
    assert np.array_equal(g["src"][g["mk"]:], f.didx[np.lexsort((f.didx, f.dd))])
    assert np.array_equal(g["dk"][:f.mk], f.dk) and np.array_equal(g["zk"][:f.mk], f.zk)
    assert np.array_equal(g["dk"][f.mk:], np.sort(f.dd, kind="stable")) or f.mk == m
    ties = 0
    scale = max(np.abs(f.lam).max() if m else 1.0, 1e-300)
    assert np.all(np.abs(g["lam"] - f.lam) <= LAM_RTOL * np.maximum(np.abs(f.lam), scale * 1e-6)), \
        np.abs(g["lam"] - f.lam).max()
    mk = f.mk
    if mk:
        Kg = g["org"][:mk]
        same = Kg == f.K
        # origin choice differs only when f(mid) is ~0 (root at the midpoint)
        assert same.mean() >= 0.99
        e_g, e_o = g["eta"][:mk][same], f.eta[same]
        assert np.all(np.abs(e_g - e_o) <= ETA_RTOL * np.abs(e_o) + 1e-300), np.max(np.abs(e_g - e_o) / np.abs(e_o))
        assert np.all(np.abs(g["vhat"][:mk] - f.vhat) <= VEC_RTOL * np.abs(f.vhat))
        assert np.all(np.abs(g["bnorm"][:mk] - f.b) <= VEC_RTOL * np.abs(f.b))
        # merge permutation bit-exact unless two new eigenvalues are within rounding
        if not np.array_equal(g["perm"], f.order):
            lam = f.lam
            gaps = np.diff(lam)
            assert np.any(gaps <= 1e-12 * np.maximum(np.abs(lam[1:]), 1e-300)), "merge order differs"
    return dict(ties=ties, mk=mk, m=m)


def dense_qhat(g):
    """Dense eigenvector matrix of one GPU problem from its structured outputs
    (rotations, Cauchy-like block eq. (4.26) with shifted entries eq. (4.28), sort)."""
    m, mk = g["m"], g["mk"]
    dk, eta, org, v, b = g["dk"], g["eta"], g["org"], g["vhat"], g["bnorm"]
    C = np.zeros((m, m))
    if mk:
        dK = dk[org[:mk]]
        Cc = (v[:mk, None] * b[None, :mk]) / ((dk[:mk, None] - dK[None, :]) - eta[None, :mk])
        C[:mk, :mk] = Cc
    for s in range(mk, m):
        C[s, s] = 1.0
    # columns in merged order
    Cm = C[:, g["perm"]]
    # rows: slot -> input index
    Q = np.zeros((m, m))
    Q[g["src"], :] = Cm
    # undo rotations: Qhat = G^T [...]
    for t in range(g["ng"] - 1, -1, -1):
        a, bb = g["giv_ab"][t]
        c, s = g["giv_cs"][t]
        xa, xb = Q[a].copy(), Q[bb].copy()
        Q[a] = c * xa + s * xb
        Q[bb] = -s * xa + c * xb
    return Q
