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


def dense_from_hss_hermitian(h) -> np.ndarray:
    """Complex Hermitian HSS matrix from complex generators: A(i, j) =
    U_i B_i U_j^H for a left child i and its sibling j, the conjugate
    transpose below the diagonal, nested U_p = [U_i R_i; U_j R_j]."""
    t = h.tree
    n = t.n
    A = np.zeros((n, n), np.complex128)
    Ubig = {}
    for i in range(t.nnodes):
        o, m = int(t.offset[i]), int(t.leaf_size[i])
        if t.lchild[i] < 0:
            A[o:o + m, o:o + m] = h.leaf_D(i)
            Ubig[i] = h.leaf_U(i).copy()
            continue
        a, b = int(t.lchild[i]), int(t.rchild[i])
        oa, ma = int(t.offset[a]), int(t.leaf_size[a])
        ob, mb = int(t.offset[b]), int(t.leaf_size[b])
        blk = Ubig[a] @ h.B[a] @ Ubig[b].conj().T
        A[oa:oa + ma, ob:ob + mb] = blk
        A[ob:ob + mb, oa:oa + ma] = blk.conj().T
        if i != t.root:
            Ubig[i] = np.vstack([Ubig[a] @ h.R[a], Ubig[b] @ h.R[b]])
    return A


def kernel_matrix(x, kind="sqrt_dist", param=1.0):
    """Dense kernel matrix at points x: sqrt|x_i - x_j| (Section 5, Example 4)
    or exp(-|x_i - x_j| / param)."""
    d = np.abs(np.asarray(x)[:, None] - np.asarray(x)[None, :])
    return np.sqrt(d) if kind == "sqrt_dist" else np.exp(-d / param)


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


def hss_matvec(h, X):
    """A X from the generators (eq. (2.1)) in O(n r k): upward pass
    Ut_c = U_c^T X_c (nested through R), downward pass of the incoming
    coupling F_c, leaves D X + U F."""
    t = h.tree
    X = np.asarray(X, np.float64).reshape(t.n, -1)
    Ut, F = {}, {}
    for i in range(t.nnodes):                        # postorder: upward
        if t.lchild[i] < 0:
            o, m = int(t.offset[i]), int(t.leaf_size[i])
            Ut[i] = h.leaf_U(i).T @ X[o:o + m]
        elif i != t.root:
            a, b = int(t.lchild[i]), int(t.rchild[i])
            Ut[i] = h.R[a].T @ Ut[a] + h.R[b].T @ Ut[b]
    Y = np.zeros_like(X)
    F[t.root] = None
    for i in range(t.nnodes - 1, -1, -1):            # reverse postorder: downward
        if t.lchild[i] < 0:
            o, m = int(t.offset[i]), int(t.leaf_size[i])
            Y[o:o + m] = h.leaf_D(i) @ X[o:o + m]
            if F[i] is not None:
                Y[o:o + m] += h.leaf_U(i) @ F[i]
            continue
        a, b = int(t.lchild[i]), int(t.rchild[i])
        Fa = h.B[a] @ Ut[b]
        Fb = h.B[a].T @ Ut[a]
        if F[i] is not None:
            Fa = Fa + h.R[a] @ F[i]
            Fb = Fb + h.R[b] @ F[i]
        F[a], F[b] = Fa, Fb
    return Y
