"""CPU ORACLE (test infrastructure): one rank-one update step
diag(d) + rho z z^T of the conquering stage, and its Cauchy-like factor.

Step order (Algorithm 3, inner loop; readings of the paper's silences are
listed in the module docstrings of ``rank1.c``):
  1. deflation, Remark 4.1 -> rotations G, kept set, deflated values;
  2. shifted secular roots (Algorithm 2; eqs. (4.13), (4.14), (4.17));
  3. Loewner zhat, eq. (4.23);  4. b, eq. (4.27);
  5. the new eigenvalues: kept roots and deflated values sorted by
     (value, input index) -> the next step's poles.
The factor is Qhat = G^T [C (+) I] Pi^T with C the Cauchy-like matrix of
eq. (4.26) on the kept set and Pi the sort of step 5.
"""
import ctypes
import dataclasses

import numpy as np

from ._build import lib

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def deflate(d, z, tau):
    """Remark 4.1.  Returns (dd, zz, kept(bool), giv list [(a, b, c, s)])."""
    d = np.ascontiguousarray(d, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    m = len(d)
    dd = np.empty(m)
    zz = np.empty(m)
    kept = np.empty(m, np.int32)
    ga = np.empty(max(m, 1), np.int32)
    gb = np.empty(max(m, 1), np.int32)
    gc = np.empty(max(m, 1))
    gs = np.empty(max(m, 1))
    ng = lib().orc_deflate(ctypes.c_int(m), _d(d), _d(z), ctypes.c_double(tau), _d(dd), _d(zz),
                           _i(kept), _i(ga), _i(gb), _d(gc), _d(gs))
    return dd, zz, kept.astype(bool), (ga[:ng].copy(), gb[:ng].copy(), gc[:ng].copy(), gs[:ng].copy())


def secular(dk, zk, mode=0, stop_c=8.0, max_iter=50):
    """Shifted roots of 1 + sum z_j^2/(d_j - x) (Algorithm 2).  Returns
    (K origin indices, eta gaps, sweeps per root, number not converged)."""
    dk = np.ascontiguousarray(dk, np.float64)
    zk = np.ascontiguousarray(zk, np.float64)
    m = len(dk)
    K = np.zeros(m, np.int32)
    eta = np.zeros(m)
    it = np.zeros(m, np.int32)
    if m == 0:
        return K, eta, it, 0
    bad = lib().orc_secular_all(ctypes.c_int(m), _d(dk), _d(zk), ctypes.c_int(mode),
                                ctypes.c_double(stop_c), ctypes.c_int(max_iter),
                                _i(K), _d(eta), _i(it))
    return K, eta, it, int(bad)


def secular_some(dk, zk, ks, mode=0, stop_c=8.0, max_iter=50):
    """Roots ks only of the kept problem (dk, zk); same per-root routine as
    ``secular``.  Returns (K, eta, sweeps, number not converged) for ks."""
    dk = np.ascontiguousarray(dk, np.float64)
    zk = np.ascontiguousarray(zk, np.float64)
    ks = np.ascontiguousarray(ks, np.int32)
    m, nk = len(dk), len(ks)
    assert nk == 0 or (ks.min() >= 0 and ks.max() < m)
    K = np.zeros(nk, np.int32)
    eta = np.zeros(nk)
    it = np.zeros(nk, np.int32)
    if nk == 0:
        return K, eta, it, 0
    bad = lib().orc_secular_some(ctypes.c_int(m), _d(dk), _d(zk), ctypes.c_int(nk), _i(ks), ctypes.c_int(mode),
                                 ctypes.c_double(stop_c), ctypes.c_int(max_iter), _i(K), _d(eta), _i(it))
    return K, eta, it, int(bad)


def secular_eval(dk, zk, ks, Ks, ys):
    """g_K(y) = 1 + psi + phi and f' at the given points (root ks[t], origin
    Ks[t], gap ys[t]) by direct sums.  Returns (f, psi, phi, df)."""
    dk = np.ascontiguousarray(dk, np.float64)
    zk = np.ascontiguousarray(zk, np.float64)
    ks = np.ascontiguousarray(ks, np.int32)
    Ks = np.ascontiguousarray(Ks, np.int32)
    ys = np.ascontiguousarray(ys, np.float64)
    m, nk = len(dk), len(ks)
    assert len(Ks) == nk and len(ys) == nk
    assert nk == 0 or (ks.min() >= 0 and ks.max() < m and Ks.min() >= 0 and Ks.max() < m)
    out = [np.zeros(nk) for _ in range(4)]
    if nk:
        lib().orc_secular_eval(ctypes.c_int(m), _d(dk), _d(zk), ctypes.c_int(nk), _i(ks), _i(Ks), _d(ys),
                               *[_d(a) for a in out])
    return tuple(out)


def lowner(dk, zk, K, eta):
    m = len(dk)
    v = np.empty(m)
    if m:
        lib().orc_lowner(ctypes.c_int(m), _d(np.ascontiguousarray(dk)), _d(np.ascontiguousarray(zk)),
                         _i(np.ascontiguousarray(K, np.int32)), _d(np.ascontiguousarray(eta)), _d(v))
    return v


def bnorm(dk, vhat, K, eta):
    m = len(dk)
    b = np.empty(m)
    if m:
        lib().orc_bnorm(ctypes.c_int(m), _d(np.ascontiguousarray(dk)), _d(np.ascontiguousarray(vhat)),
                        _i(np.ascontiguousarray(K, np.int32)), _d(np.ascontiguousarray(eta)), _d(b))
    return b


def cauchy_apply(dk, vhat, b, K, eta, X, trans):
    """Y = C^T X (trans=1) or C X (trans=0), C_ij = vhat_i b_j/((d_i - d_{K_j}) - eta_j)."""
    X = np.ascontiguousarray(X, np.float64)
    m, c = X.shape
    Y = np.empty_like(X)
    if m:
        lib().orc_cauchy_apply(ctypes.c_int(m), ctypes.c_int(c), _d(np.ascontiguousarray(dk)),
                               _d(np.ascontiguousarray(vhat)), _d(np.ascontiguousarray(b)),
                               _i(np.ascontiguousarray(K, np.int32)), _d(np.ascontiguousarray(eta)),
                               ctypes.c_int(int(trans)), _d(X), _d(Y))
    return Y


@dataclasses.dataclass
class Rank1Factor:
    m: int
    giv: tuple            # (a, b, c, s) arrays, scan order
    kidx: np.ndarray      # kept input indices (ascending)
    didx: np.ndarray      # deflated input indices (ascending)
    dk: np.ndarray        # kept poles (after rotations)
    zk: np.ndarray
    dd: np.ndarray        # deflated values, in didx order
    K: np.ndarray         # origin index into dk for each kept root
    eta: np.ndarray
    vhat: np.ndarray
    b: np.ndarray
    order: np.ndarray     # merged position -> source (< mk: kept root; else mk + deflated slot)
    lam: np.ndarray       # new eigenvalues, ascending
    sweeps: np.ndarray
    nbad: int

    @property
    def mk(self):
        return len(self.kidx)

    @property
    def lam_kept(self):
        return self.dk[self.K] + self.eta

    def _rot(self, X, forward):
        a, bb, c, s = self.giv
        rng = range(len(a)) if forward else range(len(a) - 1, -1, -1)
        for g in rng:
            xa = X[a[g]].copy()
            xb = X[bb[g]].copy()
            if forward:
                X[a[g]] = c[g] * xa - s[g] * xb
                X[bb[g]] = s[g] * xa + c[g] * xb
            else:
                X[a[g]] = c[g] * xa + s[g] * xb
                X[bb[g]] = -s[g] * xa + c[g] * xb
        return X

    def apply_T(self, X):
        """Qhat^T X (X: m x c)."""
        X = np.array(X, dtype=np.float64, copy=True).reshape(self.m, -1)
        X = self._rot(X, True)
        Yk = cauchy_apply(self.dk, self.vhat, self.b, self.K, self.eta, X[self.kidx], 1)
        allrows = np.vstack([Yk, X[self.didx]])
        return allrows[self.order]

    def apply(self, X):
        """Qhat X (X: m x c)."""
        X = np.asarray(X, dtype=np.float64).reshape(self.m, -1)
        T = np.empty_like(X)
        T[self.order] = X
        mk = self.mk
        out = np.empty_like(X)
        out[self.kidx] = cauchy_apply(self.dk, self.vhat, self.b, self.K, self.eta, T[:mk], 0)
        out[self.didx] = T[mk:]
        return self._rot(out, False)

    def dense(self):
        return self.apply(np.eye(self.m))


def rank1_step(d, z, tau, rho=1.0, mode=0, stop_c=8.0, max_iter=50) -> Rank1Factor:
    d = np.asarray(d, np.float64)
    z = np.asarray(z, np.float64) * np.sqrt(rho) if rho != 1.0 else np.asarray(z, np.float64)
    m = len(d)
    dd, zz, kept, giv = deflate(d, z, tau)
    kidx = np.nonzero(kept)[0].astype(np.int64)
    didx = np.nonzero(~kept)[0].astype(np.int64)
    dk, zk = dd[kidx].copy(), zz[kidx].copy()
    K, eta, sweeps, nbad = secular(dk, zk, mode, stop_c, max_iter)
    vhat = lowner(dk, zk, K, eta)
    b = bnorm(dk, vhat, K, eta)
    vals = np.concatenate([dk[K] + eta, dd[didx]])
    idxs = np.concatenate([kidx, didx])
    order = np.lexsort((idxs, vals))
    return Rank1Factor(m, giv, kidx, didx, dk, zk, dd[didx].copy(), K, eta, vhat, b, order,
                       vals[order], sweeps, nbad)
