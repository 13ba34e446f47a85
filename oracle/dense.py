"""CPU ORACLE (test infrastructure): dense assembly of an HSS matrix from its
generators (eq. (2.1), nested bases U_p = [U_i R_i; U_j R_j]) and the accuracy
metrics of Section 5 (residual gamma, relative eigenvalue error delta, loss of
orthogonality theta), plus cheap invariants of the generators."""
import numpy as np


def dense_from_hss(h) -> np.ndarray:
    t = h.tree
    n = t.n
    A = np.zeros((n, n))
    Ubig = {}
    for i in range(t.nnodes):      # postorder: children before parents
        o, m = int(t.offset[i]), int(t.leaf_size[i])
        if t.lchild[i] < 0:
            A[o:o + m, o:o + m] = h.leaf_D(i)
            Ubig[i] = h.leaf_U(i).copy()
            continue
        a, b = int(t.lchild[i]), int(t.rchild[i])
        oa, ma = int(t.offset[a]), int(t.leaf_size[a])
        ob, mb = int(t.offset[b]), int(t.leaf_size[b])
        blk = Ubig[a] @ h.B[a] @ Ubig[b].T
        A[oa:oa + ma, ob:ob + mb] = blk
        A[ob:ob + mb, oa:oa + ma] = blk.T
        if i != t.root:
            Ubig[i] = np.vstack([Ubig[a] @ h.R[a], Ubig[b] @ h.R[b]])
    return A


def gamma(A, lam, Q):
    """max_k ||A q_k - lam_k q_k|| / (n ||A||_2)"""
    n = A.shape[0]
    res = A @ Q - Q * lam[None, :]
    return np.max(np.linalg.norm(res, axis=0)) / (n * np.linalg.norm(A, 2))


def theta(Q):
    """max_k ||Q^T q_k - e_k|| / n"""
    n = Q.shape[0]
    E = Q.T @ Q - np.eye(n)
    return np.max(np.linalg.norm(E, axis=0)) / n


def delta(lam, lam_star):
    n = len(lam)
    return np.sqrt(np.sum((lam_star - lam) ** 2)) / (n * np.sqrt(np.sum(lam_star ** 2)))


def trace_from_generators(h):
    return sum(np.trace(h.leaf_D(i)) for i in h.tree.leaves)


def fro2_from_generators(h):
    """||A||_F^2 = sum ||D_k||_F^2 + 2 sum_{left children} ||U_a B_a U_b^T||_F^2;
    with orthonormal nested bases this is sum ||D_k||_F^2 + 2 sum ||B_a||_F^2."""
    t = h.tree
    s = sum(np.sum(h.leaf_D(i) ** 2) for i in t.leaves)
    for i in range(t.nnodes):
        if t.lchild[i] >= 0:
            s += 2.0 * np.sum(h.B[int(t.lchild[i])] ** 2)
    return s
