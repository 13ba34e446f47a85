"""CPU ORACLE (test infrastructure): SuperDC dividing and conquering stages.

* ``divide``   -- Algorithm 1 with the balanced dividing of eqs. (3.11)/(3.12)
                  (or eq. (3.15) when colsize(B) > rowsize(B)), generator
                  updates by Lemma 2.1 (``updhss``), Z_i formed bottom-up.
* ``conquer``  -- Algorithm 3: dense leaf eigendecompositions (cyclic
                  Jacobi), Zhat_i = diag(Q_c1^T, Q_c2^T) Z_i through
                  ``superdcmv`` (eq. (2.8)), the sort P_i, then r rank-one
                  steps, each followed by the transpose of its factor applied
                  to the remaining columns.
* ``superdcmv``-- Algorithm 4: y = Q_i x or Q_i^T x from the stored factors,
                  with Q_p = diag(Q_c1, Q_c2) P_p^T Qhat_p^(1) ... Qhat_p^(r)
                  (eq. (4.32), Lemma 4.1).
"""
import dataclasses

import numpy as np

from . import rank1 as r1
from ._build import lib
import ctypes


def jacobi_eig(A):
    """Dense cyclic Jacobi on a symmetric matrix; (lam ascending, V)."""
    n = A.shape[0]
    a = np.ascontiguousarray(A, np.float64).copy()
    V = np.empty((n, n))
    lam = np.empty(n)
    dp = ctypes.POINTER(ctypes.c_double)
    lib().orc_jacobi(ctypes.c_int(n), a.ctypes.data_as(dp), V.ctypes.data_as(dp),
                     lam.ctypes.data_as(dp), ctypes.c_int(100))
    return lam, V


@dataclasses.dataclass
class Divided:
    Dhat: dict        # leaf -> updated diagonal block
    Bt: dict          # node -> updated B (left children)
    beta: dict        # non-leaf node -> ||B_c1||_2 used at that node
    Z: dict           # non-leaf node -> Z_i (m_i x r)
    swapped: dict     # non-leaf node -> True if eq. (3.15) was used


def divide(h, balanced=True) -> Divided:
    """Algorithm 1.  balanced=True: eqs. (3.11)/(3.12) (scale beta = ||Bt||_2);
    balanced=False: the original dividing of eqs. (2.4)/(2.5) (scale 1), kept
    for the ablation of Section 5's Table 6.  Divided.beta holds ||Bt||_2 in
    both cases."""
    t = h.tree
    Dh = {i: h.leaf_D(i).copy() for i in t.leaves}
    Bt = {i: h.B[i].copy() for i in range(t.nnodes)}
    R = h.R
    beta, swapped = {}, {}

    def updhss(i, H):
        # Lemma 2.1: generators of D_i - U_i H U_i^T
        if t.lchild[i] < 0:
            Ui = h.leaf_U(i)
            Dh[i] -= Ui @ H @ Ui.T
            return
        a, b = int(t.lchild[i]), int(t.rchild[i])
        Bt[a] = Bt[a] - R[a] @ H @ R[b].T
        updhss(a, R[a] @ H @ R[a].T)
        updhss(b, R[b] @ H @ R[b].T)

    # top-down (reverse postorder visits every parent before its children)
    for i in range(t.nnodes - 1, -1, -1):
        if t.lchild[i] < 0:
            continue
        c1, c2 = int(t.lchild[i]), int(t.rchild[i])
        B1 = Bt[c1]
        beta[i] = np.linalg.norm(B1, 2)
        bn = beta[i] if balanced else 1.0
        if B1.shape[1] <= B1.shape[0]:
            swapped[i] = False
            updhss(c1, (B1 @ B1.T) / bn)
            updhss(c2, bn * np.eye(B1.shape[0]))
        else:
            swapped[i] = True
            updhss(c1, bn * np.eye(B1.shape[0]))
            updhss(c2, (B1.T @ B1) / bn)

    # bottom-up Z_i and nested U_i
    Ubig = {}
    Z = {}
    for i in range(t.nnodes):
        if t.lchild[i] < 0:
            Ubig[i] = h.leaf_U(i).copy()
            continue
        c1, c2 = int(t.lchild[i]), int(t.rchild[i])
        B1, bn = Bt[c1], (beta[i] if balanced else 1.0)
        if not swapped[i]:
            Z[i] = np.vstack([Ubig[c1] @ B1 / np.sqrt(bn), np.sqrt(bn) * Ubig[c2]])
        else:
            Z[i] = np.vstack([np.sqrt(bn) * Ubig[c1], Ubig[c2] @ B1.T / np.sqrt(bn)])
        if i != t.root:
            Ubig[i] = np.vstack([Ubig[c1] @ R[c1], Ubig[c2] @ R[c2]])
    return Divided(Dh, Bt, beta, Z, swapped)


@dataclasses.dataclass
class EigFactor:
    tree: object
    lam: dict          # node -> local eigenvalues (ascending)
    Qleaf: dict        # leaf -> dense eigenvectors
    P: dict            # non-leaf -> merge order (new position -> old position)
    fac: dict          # non-leaf -> list of Rank1Factor

    @property
    def eigenvalues(self):
        return self.lam[self.tree.root]

    def stats(self):
        sweeps = []
        nbad = 0
        defl = 0
        for fl in self.fac.values():
            for f in fl:
                sweeps.append(f.sweeps)
                nbad += f.nbad
                defl += f.m - f.mk
        return (np.concatenate(sweeps) if sweeps else np.zeros(0)), nbad, defl


def superdcmv(F: EigFactor, i, X, transpose):
    """Algorithm 4 (recursive form): Q_i X or Q_i^T X, X of height m_i."""
    t = F.tree
    X = np.asarray(X, np.float64).reshape(int(t.leaf_size[i]), -1)
    if t.lchild[i] < 0:
        Q = F.Qleaf[i]
        return Q.T @ X if transpose else Q @ X
    c1, c2 = int(t.lchild[i]), int(t.rchild[i])
    m1 = int(t.leaf_size[c1])
    if transpose:
        Y = np.vstack([superdcmv(F, c1, X[:m1], 1), superdcmv(F, c2, X[m1:], 1)])
        Y = Y[F.P[i]]
        for f in F.fac[i]:
            Y = f.apply_T(Y)
        return Y
    Y = X
    for f in reversed(F.fac[i]):
        Y = f.apply(Y)
    Z = np.empty_like(Y)
    Z[F.P[i]] = Y
    return np.vstack([superdcmv(F, c1, Z[:m1], 0), superdcmv(F, c2, Z[m1:], 0)])


def conquer(h, dv: Divided, tau=1e-10, mode=0, stop_c=8.0, max_iter=50) -> EigFactor:
    t = h.tree
    F = EigFactor(t, {}, {}, {}, {})
    # leaf eigendecompositions are independent: run them on a thread pool
    # (the C routine releases the GIL)
    from concurrent.futures import ThreadPoolExecutor
    leaves = t.leaves
    with ThreadPoolExecutor() as ex:
        for i, (lam, V) in zip(leaves, ex.map(lambda k: jacobi_eig(dv.Dhat[k]), leaves)):
            F.lam[i] = lam
            F.Qleaf[i] = V
    for i in range(t.nnodes):              # postorder
        if t.lchild[i] < 0:
            continue
        c1, c2 = int(t.lchild[i]), int(t.rchild[i])
        m1 = int(t.leaf_size[c1])
        Z = dv.Z[i]
        Zh = np.vstack([superdcmv(F, c1, Z[:m1], 1), superdcmv(F, c2, Z[m1:], 1)])
        vals = np.concatenate([F.lam[c1], F.lam[c2]])
        order = np.argsort(vals, kind="stable")
        F.P[i] = order
        d = vals[order]
        Zh = Zh[order]
        facs = []
        for j in range(Zh.shape[1]):
            f = r1.rank1_step(d, Zh[:, j], tau, mode=mode, stop_c=stop_c, max_iter=max_iter)
            facs.append(f)
            if j + 1 < Zh.shape[1]:
                Zh[:, j + 1:] = f.apply_T(Zh[:, j + 1:])
            d = f.lam
        F.fac[i] = facs
        F.lam[i] = d
    return F


def superdc(h, tau=1e-10, mode=0, stop_c=8.0, max_iter=50) -> EigFactor:
    return conquer(h, divide(h), tau=tau, mode=mode, stop_c=stop_c, max_iter=max_iter)
