"""Shared comparison helpers for the GPU parity tests (CUDA path vs oracle).

Tolerances (derived from the arithmetic):
  * eigenvalues: |lam - lam_o| <= 1e-10 * max(|lam_o|, 1e-6 scale)  (the target bound);
  * gaps eta (same origin): both sides stop when the test of eq. (4.12),
    |f| < c m eps (1 + |psi| + |phi|), holds (the oracle's bisection mode goes
    to adjacent doubles), so each gap lies within that tolerance over f' of
    the exact one: per root, |eta - eta_o| <= 4 c m eps (1+|psi|+|phi|)/f'
    + 8 eps |eta_o|, with psi, phi, f' evaluated by the oracle at its root.
    For m up to a few thousand this is ~1e-12 relative; at m = 131072 and
    weakly coupled roots (z_k^2 small against the gap) it reaches ~1e-6;
  * vhat, b: the oracle's formulas (eqs. (4.23), (4.27)) evaluated on the
    GPU's own origins and gaps, max(1e-11, 4 mk eps) relative (products and
    sums of about 2 mk shifted differences on equal inputs: rounding only,
    plus the FMM's far-field error);
  * deflation decisions, rotations and the kept/deflated layout: bit-exact
    (both sides evaluate them with the same IEEE operations in the same order);
  * the merge permutation: bit-exact unless two new eigenvalues lie within
    the eigenvalue tolerance of each other.
"""
import numpy as np

from oracle import rank1 as r1

LAM_RTOL = 1e-10
ETA_RTOL = 1e-9
EPS = 2.0 ** -52


def vec_rtol(mk):
    """Relative tolerance of zhat and b of a problem with mk kept poles: each
    is a product (eq. (4.23)) or a sum (eq. (4.27)) of about 2 mk rounded
    factors or terms of one sign, so at most about 4 mk eps relative; the far
    field's log form adds ~1e-14 per far box; floor 1e-11."""
    return max(1e-11, 4.0 * mk * EPS)


def lam_check(lam, ref, anorm, nsteps, tau=0.0, decisions_differ=False, max_exceptions=8):
    """Per-entry eigenvalue check of a whole HSS eigendecomposition.

    Every entry must satisfy |lam - ref| <= 1e-10 max(|ref|, 1e-6 ||A||) (the
    relative bound with its floor for tiny eigenvalues), except entries
    explained by one of two causes, which are counted and returned:
      * "rounding": |lam - ref| <= 8 nsteps eps ||A||, the absolute error that
        nsteps rank-one steps (tree levels x rank) leave on any eigenvalue,
        however small (both sides evaluate every step with absolute error of a
        few eps ||A||; the two modes of the oracle itself differ by this much);
      * "deflation": |lam - ref| <= 4 tau, allowed only when the two sides took
        some deflation decision of Remark 4.1 differently (decisions_differ):
        their inputs of a step differ by rounding, a test that sits within
        rounding of tau flips, and the dropped coupling moves nearby
        eigenvalues by O(tau).
    At most max_exceptions entries may use either exception."""
    lam = np.asarray(lam)
    ref = np.asarray(ref)
    err = np.abs(lam - ref)
    rel_ok = err <= LAM_RTOL * np.maximum(np.abs(ref), 1e-6 * anorm)
    floor = 8.0 * nsteps * EPS * anorm
    round_ok = ~rel_ok & (err <= floor)
    defl_ok = ~rel_ok & ~round_ok & (err <= 4.0 * tau) & bool(decisions_differ)
    bad = ~(rel_ok | round_ok | defl_ok)
    exc = np.nonzero(round_ok | defl_ok)[0]
    info = dict(n=len(lam), max_abs=float(err.max()) if len(err) else 0.0,
                n_rounding=int(round_ok.sum()), n_deflation=int(defl_ok.sum()), n_bad=int(bad.sum()),
                exceptions=[(int(i), float(ref[i]), float(err[i])) for i in exc[:20]],
                bad=[(int(i), float(ref[i]), float(err[i])) for i in np.nonzero(bad)[0][:20]])
    ok = info["n_bad"] == 0 and len(exc) <= max_exceptions
    return ok, info


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


def check_roots(f, K_g, eta_g, vhat_g, b_g, stop_c=8.0):
    """Kept part of a rank-one step: origins, gaps within the per-root bound of
    the stopping test, zhat and b against the oracle's formulas on the GPU's
    roots.  f: oracle factor; K_g, eta_g, vhat_g, b_g: GPU kept-slot arrays."""
    mk = f.mk
    st = {}
    if not mk:
        return st
    same = K_g == f.K
    # origin choice differs only when f(mid) is ~0 (root at the midpoint)
    assert same.mean() >= 0.99, same.mean()
    ks = np.arange(mk)
    _, ps, ph, df = r1.secular_eval(f.dk, f.zk, ks, f.K, f.eta)
    bound = 4.0 * stop_c * mk * EPS * (1.0 + np.abs(ps) + np.abs(ph)) / df + 8.0 * EPS * np.abs(f.eta)
    err = np.abs(eta_g - f.eta)
    assert np.all(err[same] <= bound[same]), np.max((err / bound)[same])
    vh = r1.lowner(f.dk, f.zk, K_g, eta_g)
    bb = r1.bnorm(f.dk, vh, K_g, eta_g)
    rv = np.abs(vhat_g - vh) / np.abs(vh)
    rb = np.abs(b_g - bb) / np.abs(bb)
    assert rv.max() <= vec_rtol(mk), (rv.max(), int(rv.argmax()), mk)
    assert rb.max() <= vec_rtol(mk), (rb.max(), int(rb.argmax()), mk)
    st.update(origin_same=float(same.mean()), eta_over_bound=float(np.max((err / bound)[same])),
              eta_rel=float(np.max(err[same] / np.maximum(np.abs(f.eta[same]), 1e-300))),
              vhat_rel=float(rv.max()), b_rel=float(rb.max()))
    return st


def check_lam(lam_g, f, perm_g=None):
    """New eigenvalues per entry; merge order equal up to near-ties."""
    m = f.m
    scale = max(np.abs(f.lam).max() if m else 1.0, 1e-300)
    tl = LAM_RTOL * np.maximum(np.abs(f.lam), scale * 1e-6)
    err = np.abs(lam_g - f.lam)
    assert np.all(err <= tl), (err / tl).max()
    if perm_g is not None and f.mk < m:
        # GPU slots mk.. hold the deflated entries sorted by (value, input
        # index); the oracle numbers them mk + their rank in input order
        mk = f.mk
        L = np.lexsort((f.didx, f.dd))
        perm_g = np.where(perm_g < mk, perm_g, mk + L[np.maximum(perm_g - mk, 0)])
    if perm_g is not None and not np.array_equal(perm_g, f.order):
        lam = f.lam
        for p in np.nonzero(perm_g != f.order)[0]:
            near = min(abs(lam[p] - lam[p - 1]) if p > 0 else np.inf,
                       abs(lam[p + 1] - lam[p]) if p + 1 < m else np.inf)
            assert near <= 2.0 * tl[p], ("merge order differs", p)
    return float((err / tl).max()) if m else 0.0


def check_deflation(g, f):
    """Kept set, rotations and the slot layout, bit for bit."""
    m, mk = g["m"], g["mk"]
    assert m == f.m
    assert mk == f.mk, (mk, f.mk)
    assert np.array_equal(g["src"][:mk], f.kidx), "kept set differs"
    assert g["ng"] == len(f.giv[0])
    if g["ng"]:
        assert np.array_equal(g["giv_ab"][:, 0], f.giv[0]) and np.array_equal(g["giv_ab"][:, 1], f.giv[1])
        assert np.array_equal(g["giv_cs"][:, 0], f.giv[2]) and np.array_equal(g["giv_cs"][:, 1], f.giv[3])
    assert np.array_equal(g["src"][mk:], f.didx[np.lexsort((f.didx, f.dd))])
    assert np.array_equal(g["dk"][:mk], f.dk)
    assert np.array_equal(g["dk"][mk:], np.sort(f.dd, kind="stable"))


def compare_problem(g, d, z, tau, rho=1.0, mode=0):
    """Compare one GPU problem with the oracle.  Returns a dict of stats; raises AssertionError."""
    f = r1.rank1_step(d, z, tau, rho=rho, mode=mode)
    check_deflation(g, f)
    if f.mk:
        assert np.array_equal(g["zk"][:f.mk], f.zk)
    st = dict(m=f.m, mk=f.mk)
    st.update(check_roots(f, g["org"][:f.mk], g["eta"][:f.mk], g["vhat"][:f.mk], g["bnorm"][:f.mk]))
    st["lam_over_tol"] = check_lam(g["lam"], f, g["perm"])
    return st


def eigfact_problem(F, level, step, q, o, m, nxt_din=None):
    """Node q (rows [o, o+m)) of stored step (level, step) of a GPU eigenfactor
    in the per-problem layout of gpu_problem (lam: the step's output in merged
    order, from the next step's input poles when given)."""
    g = {k: F.get(level, step, k)[o:o + m] for k in ("dk", "eta", "dorg", "vhat", "bnorm", "src", "pinv")}
    mk = int(F.get(level, step, "mk")[q])
    ng = int(F.get(level, step, "ngiv")[q])
    ab = F.get(level, step, "giv_ab")
    cs = F.get(level, step, "giv_cs")
    g["m"], g["mk"], g["ng"] = m, mk, ng
    g["giv_ab"] = ab[2 * o:2 * o + 2 * ng].reshape(-1, 2)
    g["giv_cs"] = cs[2 * o:2 * o + 2 * ng].reshape(-1, 2)
    # origin index of each kept root: its own pole or the next one
    k = np.arange(mk)
    g["org"] = np.where(g["dorg"][:mk] == g["dk"][:mk], k, k + 1).astype(np.int32)
    val = np.where(np.arange(m) < mk, g["dorg"] + g["eta"], g["dk"])
    lam = np.empty(m)
    lam[g["pinv"]] = val
    g["lam_slots"] = lam
    if nxt_din is not None:
        g["lam"] = nxt_din[o:o + m]
    return g


def compare_stored_step(g, d, z, tau, mode=1, n_exact=0, seed=0):
    """Compare one stored step of a GPU eigenfactor (eigfact_problem) with the
    oracle's rank-one step on the same inputs (d, z): deflation bit for bit,
    origins, gaps, zhat, b and the new eigenvalues per entry; with n_exact > 0,
    that many sampled roots (plus the first and last) are also checked against
    the oracle's bisection to adjacent doubles.  Returns a dict of stats."""
    f = r1.rank1_step(d, z, tau, mode=mode)
    check_deflation(g, f)
    mk = f.mk
    st = dict(m=g["m"], mk=mk, ngiv=g["ng"])
    st.update(check_roots(f, g["org"], g["eta"][:mk], g["vhat"][:mk], g["bnorm"][:mk]))
    if mk and n_exact:
        rng = np.random.default_rng(seed)
        ks = np.unique(np.concatenate([[0, mk - 1], rng.choice(mk, min(n_exact, mk), replace=False)]))
        K0, e0, _, _ = r1.secular_some(f.dk, f.zk, ks, mode=0)
        s0 = g["org"][ks] == K0
        _, ps, ph, df = r1.secular_eval(f.dk, f.zk, ks, K0, e0)
        b0 = 2.0 * 8.0 * mk * EPS * (1.0 + np.abs(ps) + np.abs(ph)) / df + 8.0 * EPS * np.abs(e0)
        e = np.abs(g["eta"][ks] - e0)
        assert s0.mean() >= 0.99 and np.all(e[s0] <= b0[s0]), (s0.mean(), np.max(e / b0))
        st.update(exact_sample=len(ks), exact_eta_over_bound=float(np.max((e / b0)[s0])))
    st["lam_over_tol"] = check_lam(g.get("lam", g["lam_slots"]), f)
    return st


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
