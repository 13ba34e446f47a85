"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only draws random numbers and lays them out; it contains none
of the eigensolver's arithmetic (no dividing, no secular solve, no
eigenvector formulas).  Both sides receive the very same arrays from here.

HSS layout (the paper's Section 2, eq. (2.1)):
  * the tree is a postordered full binary tree; node ids 0..nnodes-1 in
    postorder, root = nnodes-1; ``lchild``/``rchild`` are -1 at leaves;
  * ``D``: leaf diagonal blocks, m_k x m_k column-major, concatenated over
    leaves in postorder (= left-to-right order);
  * ``U``: leaf bases, m_k x r column-major, concatenated the same way;
  * ``R``: r x r column-major per node (nnodes blocks; the root's and its
    children's entries are never used);
  * ``B``: r x r column-major per node (nnodes blocks; only entries of
    left children are used: B_i couples left child i with its sibling).

All random draws use numpy's PCG64 ``default_rng(seed)`` in a fixed order.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Tree:
    n: int
    nnodes: int
    lchild: np.ndarray      # int32 [nnodes]
    rchild: np.ndarray      # int32 [nnodes]
    parent: np.ndarray      # int32 [nnodes]
    leaf_size: np.ndarray   # int64 [nnodes] (size of the index range of every node)
    offset: np.ndarray      # int64 [nnodes] first row of each node's range
    level: np.ndarray       # int32 [nnodes] root = 0
    rank: int

    @property
    def root(self) -> int:
        return self.nnodes - 1

    def is_leaf(self, i: int) -> bool:
        return self.lchild[i] < 0

    @property
    def leaves(self):
        return [i for i in range(self.nnodes) if self.lchild[i] < 0]

    @property
    def lmax(self) -> int:
        return int(self.level.max())


@dataclasses.dataclass
class HSS:
    tree: Tree
    D: np.ndarray   # concatenated leaf blocks (column-major), float64
    U: np.ndarray   # concatenated leaf bases (column-major), float64
    R: np.ndarray   # [nnodes, r, r] (row-major numpy view of column-major data is avoided: we keep [node][i][j])
    B: np.ndarray   # [nnodes, r, r]
    d_off: np.ndarray  # int64 [nnodes] offset of each leaf's D block (-1 for non-leaves)
    u_off: np.ndarray  # int64 [nnodes] offset of each leaf's U block

    def leaf_D(self, i):
        m = int(self.tree.leaf_size[i])
        o = int(self.d_off[i])
        return self.D[o:o + m * m].reshape(m, m, order="F")

    def leaf_U(self, i):
        m = int(self.tree.leaf_size[i])
        r = self.tree.rank
        o = int(self.u_off[i])
        return self.U[o:o + m * r].reshape(m, r, order="F")

    def packed(self):
        """Flat float64 arrays in the C-ABI packing (column-major blocks)."""
        r = self.tree.rank
        Rp = np.ascontiguousarray(np.transpose(self.R, (0, 2, 1))).reshape(-1)
        Bp = np.ascontiguousarray(np.transpose(self.B, (0, 2, 1))).reshape(-1)
        out = (np.ascontiguousarray(self.D), np.ascontiguousarray(self.U), Rp, Bp)
        if np.iscomplexobj(self.D):     # (re, im) pairs
            out = tuple(np.ascontiguousarray(x, np.complex128).view(np.float64) for x in out)
        return out


def perfect_tree(n: int, leaf: int, rank: int) -> Tree:
    """Postordered perfect binary tree with leaves of size ``leaf`` (n = leaf * 2^lmax)."""
    nleaves = n // leaf
    assert nleaves * leaf == n and nleaves & (nleaves - 1) == 0, "n/leaf must be a power of two"
    lmax = nleaves.bit_length() - 1
    nnodes = 2 * nleaves - 1
    lchild = -np.ones(nnodes, np.int32)
    rchild = -np.ones(nnodes, np.int32)
    parent = -np.ones(nnodes, np.int32)
    size = np.zeros(nnodes, np.int64)
    off = np.zeros(nnodes, np.int64)
    level = np.zeros(nnodes, np.int32)
    counter = [0]
    leafpos = [0]

    def build(lev):
        if lev == lmax:
            i = counter[0]
            counter[0] += 1
            size[i] = leaf
            off[i] = leafpos[0] * leaf
            leafpos[0] += 1
            level[i] = lev
            return i
        a = build(lev + 1)
        b = build(lev + 1)
        i = counter[0]
        counter[0] += 1
        lchild[i], rchild[i] = a, b
        parent[a] = parent[b] = i
        size[i] = size[a] + size[b]
        off[i] = off[a]
        level[i] = lev
        return i

    build(0)
    return Tree(n, nnodes, lchild, rchild, parent, size, off, level, rank)


def perfect_tree_sizes(sizes, rank: int) -> Tree:
    """Postordered perfect binary tree whose leaves (left to right) have the
    given row counts (len(sizes) a power of two; sizes may differ)."""
    sizes = [int(x) for x in sizes]
    nleaves = len(sizes)
    assert nleaves >= 1 and nleaves & (nleaves - 1) == 0, "the number of leaves must be a power of two"
    lmax = nleaves.bit_length() - 1
    nnodes = 2 * nleaves - 1
    lchild = -np.ones(nnodes, np.int32)
    rchild = -np.ones(nnodes, np.int32)
    parent = -np.ones(nnodes, np.int32)
    size = np.zeros(nnodes, np.int64)
    off = np.zeros(nnodes, np.int64)
    level = np.zeros(nnodes, np.int32)
    counter = [0]
    leafpos = [0, 0]                      # leaf index, row offset

    def build(lev):
        if lev == lmax:
            i = counter[0]
            counter[0] += 1
            size[i] = sizes[leafpos[0]]
            off[i] = leafpos[1]
            leafpos[0] += 1
            leafpos[1] += size[i]
            level[i] = lev
            return i
        a = build(lev + 1)
        b = build(lev + 1)
        i = counter[0]
        counter[0] += 1
        lchild[i], rchild[i] = a, b
        parent[a] = parent[b] = i
        size[i] = size[a] + size[b]
        off[i] = off[a]
        level[i] = lev
        return i

    build(0)
    return Tree(int(sum(sizes)), nnodes, lchild, rchild, parent, size, off, level, rank)


def hss_random_sizes(sizes, rank: int, seed: int) -> HSS:
    """Random symmetric HSS matrix on a perfect tree with ragged leaf sizes:
    the recipe of ``hss_random`` (leaf D = (G + G^T)/2; leaf U the Q-factor of
    an m x r N(0,1) matrix when m >= r, else an m x r N(0,1) matrix scaled by
    1/sqrt(r); [R_c1; R_c2] the Q-factor of a 2r x r N(0,1) matrix; B = N(0,1)
    diag(2^-k)), same draw order."""
    tree = perfect_tree_sizes(sizes, rank)
    rng = np.random.default_rng(seed)
    D, U, R, B, d_off, u_off = _alloc(tree)
    h = HSS(tree, D, U, R, B, d_off, u_off)
    colscale = 2.0 ** (-np.arange(rank, dtype=np.float64))
    for i in range(tree.nnodes):
        m = int(tree.leaf_size[i])
        if tree.lchild[i] < 0:
            G = rng.standard_normal((m, m))
            h.leaf_D(i)[:, :] = 0.5 * (G + G.T)
            g = rng.standard_normal((m, rank))
            h.leaf_U(i)[:, :] = _qfactor(g) if m >= rank else g / np.sqrt(rank)
        else:
            c1, c2 = int(tree.lchild[i]), int(tree.rchild[i])
            if i != tree.root:
                q = _qfactor(rng.standard_normal((2 * rank, rank)))
                R[c1] = q[:rank]
                R[c2] = q[rank:]
            B[c1] = rng.standard_normal((rank, rank)) * colscale[None, :]
    return h


def _alloc(tree: Tree):
    r = tree.rank
    d_off = -np.ones(tree.nnodes, np.int64)
    u_off = -np.ones(tree.nnodes, np.int64)
    dpos = upos = 0
    for i in range(tree.nnodes):
        if tree.lchild[i] < 0:
            m = int(tree.leaf_size[i])
            d_off[i] = dpos
            u_off[i] = upos
            dpos += m * m
            upos += m * r
    D = np.zeros(dpos)
    U = np.zeros(upos)
    R = np.zeros((tree.nnodes, r, r))
    B = np.zeros((tree.nnodes, r, r))
    return D, U, R, B, d_off, u_off


def _qfactor(g):
    q, _ = np.linalg.qr(g)
    return q


def _expm(S):
    from scipy.linalg import expm
    return expm(S)


def hss_random(n: int, leaf: int, rank: int, seed: int, bscale: float = 1.0,
               clustered: bool = False, tilt: float = 1e-5) -> HSS:
    """Random symmetric HSS matrix as in the plain configurations.

    * leaf D = (G + G^T)/2, G ~ N(0,1);
    * with ``clustered``: leaf D = V diag(mu) V^T with V = [U_k, U_perp] exp(S):
      r eigenvalues N(0,1) on span(U_k); the other m - r eigenvalues are N(0,1)
      values repeated 4 times plus U[0, 1e-12] offsets; U_perp completes U_k
      to an orthonormal basis (QR of [U_k, N(0,1)]); S is skew-symmetric with
      N(0, tilt^2) entries (tilt = 1e-5), tilting the clustered eigenvectors
      slightly into span(U_k) so that they reach the rank-one updates;
    * leaf U = Q-factor of an m x r N(0,1) matrix;
    Draw order: nodes in postorder; leaf: D then U (clustered: U, then the
    completion, cluster values, offsets, span(U) values, S); non-leaf: R pair
    (non-root), then B.
    """
    tree = perfect_tree(n, leaf, rank)
    rng = np.random.default_rng(seed)
    D, U, R, B, d_off, u_off = _alloc(tree)
    h = HSS(tree, D, U, R, B, d_off, u_off)
    colscale = 2.0 ** (-np.arange(rank, dtype=np.float64))
    for i in range(tree.nnodes):
        m = int(tree.leaf_size[i])
        if tree.lchild[i] < 0:
            if clustered:
                Ul = _qfactor(rng.standard_normal((m, rank)))
                full = _qfactor(np.hstack([Ul, rng.standard_normal((m, m - rank))]))
                base = rng.standard_normal((m - rank + 3) // 4)
                mu = np.repeat(base, 4)[:m - rank] + rng.uniform(0.0, 1e-12, m - rank)
                muU = rng.standard_normal(rank)
                Sk = rng.standard_normal((m, m)) * tilt
                Sk = Sk - Sk.T
                V = np.hstack([Ul, full[:, rank:]]) @ _expm(Sk)
                Dl = (V * np.concatenate([muU, mu])) @ V.T
                Dl = 0.5 * (Dl + Dl.T)
                h.leaf_D(i)[:, :] = Dl
                h.leaf_U(i)[:, :] = Ul
            else:
                G = rng.standard_normal((m, m))
                h.leaf_D(i)[:, :] = 0.5 * (G + G.T)
                h.leaf_U(i)[:, :] = _qfactor(rng.standard_normal((m, rank)))
        else:
            c1, c2 = int(tree.lchild[i]), int(tree.rchild[i])
            if i != tree.root:
                q = _qfactor(rng.standard_normal((2 * rank, rank)))
                R[c1] = q[:rank]
                R[c2] = q[rank:]
            B[c1] = rng.standard_normal((rank, rank)) * colscale[None, :] * bscale
    return h


def hss_random_hermitian(n: int, leaf: int, rank: int, seed: int) -> HSS:
    """Random complex Hermitian HSS matrix, the complex analogue of
    ``hss_random``: leaf D = (G + G^H)/2 and B = G diag(2^-k) with
    G = N(0,1) + i N(0,1); leaf U and the stacked [R_c1; R_c2] are the
    Q-factors of complex Gaussian matrices (orthonormal columns).  Arrays are
    complex128 in the same layout as ``hss_random`` (``packed`` then yields the
    (re, im) pairs that superdc_build_hss_hermitian reads).  Draw order as
    ``hss_random``, each complex matrix drawn as its real part then its
    imaginary part."""
    tree = perfect_tree(n, leaf, rank)
    rng = np.random.default_rng(seed)
    D, U, R, B, d_off, u_off = _alloc(tree)
    D, U, R, B = (x.astype(np.complex128) for x in (D, U, R, B))
    h = HSS(tree, D, U, R, B, d_off, u_off)
    colscale = 2.0 ** (-np.arange(rank, dtype=np.float64))

    def cg(shape):
        re = rng.standard_normal(shape)
        return re + 1j * rng.standard_normal(shape)

    for i in range(tree.nnodes):
        m = int(tree.leaf_size[i])
        if tree.lchild[i] < 0:
            G = cg((m, m))
            h.leaf_D(i)[:, :] = 0.5 * (G + G.conj().T)
            h.leaf_U(i)[:, :] = _qfactor(cg((m, rank)))
        else:
            c1, c2 = int(tree.lchild[i]), int(tree.rchild[i])
            if i != tree.root:
                q = _qfactor(cg((2 * rank, rank)))
                R[c1] = q[:rank]
                R[c2] = q[rank:]
            B[c1] = cg((rank, rank)) * colscale[None, :]
    return h


def chebyshev_points(n: int) -> np.ndarray:
    """cos((2i - 1) pi / (2n)), i = 1..n: the points of the paper's Example 4
    (decreasing, so index order is position order)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.cos((2.0 * i - 1.0) * np.pi / (2.0 * n))


def real_layout(h: HSS, X: np.ndarray) -> np.ndarray:
    """Complex n x k block -> the 2n x k real block of a Hermitian HSS
    handle's layout: each leaf's rows as [Re rows; Im rows]."""
    X = np.asarray(X).reshape(h.tree.n, -1)
    out = np.empty((2 * h.tree.n, X.shape[1]))
    for i in h.tree.leaves:
        o, m = int(h.tree.offset[i]), int(h.tree.leaf_size[i])
        out[2 * o:2 * o + m] = X[o:o + m].real
        out[2 * o + m:2 * o + 2 * m] = X[o:o + m].imag
    return out


def complex_layout(h: HSS, Y: np.ndarray) -> np.ndarray:
    """Inverse of ``real_layout``."""
    Y = np.asarray(Y).reshape(2 * h.tree.n, -1)
    out = np.empty((h.tree.n, Y.shape[1]), np.complex128)
    for i in h.tree.leaves:
        o, m = int(h.tree.offset[i]), int(h.tree.leaf_size[i])
        out[o:o + m] = Y[2 * o:2 * o + m] + 1j * Y[2 * o + m:2 * o + 2 * m]
    return out


def hss_tridiag(n: int, leaf: int, diag: float = 3.0, off: float = -1.0) -> HSS:
    """Explicit rank-2 HSS form of the symmetric tridiagonal matrix of the
    paper's Example 1 (Section 5): leaf D = tridiag(off, diag, off),
    U_leaf = [e_first, e_last], R_c1 = [[1,0],[0,0]], R_c2 = [[0,0],[0,1]],
    B_c1 = [[0,0],[off,0]].  Eigenvalues: diag + 2*off*cos(k pi/(n+1))."""
    tree = perfect_tree(n, leaf, 2)
    D, U, R, B, d_off, u_off = _alloc(tree)
    h = HSS(tree, D, U, R, B, d_off, u_off)
    for i in range(tree.nnodes):
        m = int(tree.leaf_size[i])
        if tree.lchild[i] < 0:
            T = np.diag(np.full(m, diag)) + np.diag(np.full(m - 1, off), 1) + np.diag(np.full(m - 1, off), -1)
            h.leaf_D(i)[:, :] = T
            Ul = np.zeros((m, 2))
            Ul[0, 0] = 1.0
            Ul[m - 1, 1] = 1.0
            h.leaf_U(i)[:, :] = Ul
        else:
            c1, c2 = int(tree.lchild[i]), int(tree.rchild[i])
            R[c1] = np.array([[1.0, 0.0], [0.0, 0.0]])
            R[c2] = np.array([[0.0, 0.0], [0.0, 1.0]])
            B[c1] = np.array([[0.0, 0.0], [off, 0.0]])
    return h


# ---------------------------------------------------------------------------
# Batched independent rank-one problems diag(d) + rho z z^T
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class SecularBatch:
    offsets: np.ndarray   # int64 [nprob+1]
    d: np.ndarray         # float64 [sum m], ascending within each problem
    z: np.ndarray         # float64 [sum m]
    rho: float

    @property
    def nprob(self):
        return len(self.offsets) - 1

    def problem(self, p):
        a, b = int(self.offsets[p]), int(self.offsets[p + 1])
        return self.d[a:b], self.z[a:b]


def secular_batch(nprob: int, mlo: int, mhi: int, seed: int, cluster_frac: float = 0.1,
                  cluster_size: int = 8, cluster_width: float = 1e-10, rho: float = 1.0,
                  sizes=None) -> SecularBatch:
    """Independent rank-one problems: m ~ U{mlo..mhi}; d = sorted U[0,1]^m;
    then floor(cluster_frac*m/cluster_size) clusters: pick cluster_size
    consecutive sorted poles (random start) and replace them by c + U[0, width]
    (c = their first value), re-sort; z ~ N(0,1).  Draw order per problem:
    m (all problems first), then per problem d, cluster starts/offsets, z."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = rng.integers(mlo, mhi + 1, size=nprob)
    sizes = np.asarray(sizes, np.int64)
    offsets = np.zeros(nprob + 1, np.int64)
    offsets[1:] = np.cumsum(sizes)
    d = np.empty(int(offsets[-1]))
    z = np.empty(int(offsets[-1]))
    for p in range(nprob):
        m = int(sizes[p])
        dp = np.sort(rng.uniform(0.0, 1.0, m))
        ncl = int(cluster_frac * m) // cluster_size
        for _ in range(ncl):
            s = int(rng.integers(0, max(1, m - cluster_size + 1)))
            e = min(m, s + cluster_size)
            c = dp[s]
            dp[s:e] = c + rng.uniform(0.0, cluster_width, e - s)
            dp.sort()
        d[offsets[p]:offsets[p + 1]] = dp
        z[offsets[p]:offsets[p + 1]] = rng.standard_normal(m)
    return SecularBatch(offsets, d, z, rho)


def normal_block(n: int, ncols: int, seed: int) -> np.ndarray:
    """N(0,1) n x ncols block, column-major (Fortran order)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, ncols)))


# Workload recipes named by what they are.
def cfg_small_hss():
    """n=512, leaf 32 (4 levels), rank 4, seed 0."""
    return hss_random(512, 32, 4, seed=0)


def cfg_secular_4096(seed: int = 1):
    """4096 problems, m ~ U{32..2048}, 10% of poles in clusters of width 1e-10."""
    return secular_batch(4096, 32, 2048, seed=seed)


def cfg_clustered_16384():
    """n=16384, leaf 64, rank 8, clustered leaf spectra, seed 2."""
    return hss_random(16384, 64, 8, seed=2, clustered=True)


def cfg_backward_8192():
    """n=8192, leaf 64, rank 6, seed 3."""
    return hss_random(8192, 64, 6, seed=3)


def cfg_large_131072():
    """n=131072, leaf 128, rank 10, seed 4."""
    return hss_random(131072, 128, 10, seed=4)
