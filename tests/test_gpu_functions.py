"""Uses of the structured eigendecomposition: matrix functions f(A) X through
superdc_apply_function (Section 1's motivation: matrix function evaluations,
linear systems), and the complex Hermitian case through
superdc_build_hss_hermitian (Section 1: the real symmetric treatment extends
to Hermitian matrices), against dense FP64 references on the CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import inputs  # noqa: E402
from oracle import dense  # noqa: E402
from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def _fvals(lam, kind, sigma=0.0):
    if kind == "exp":
        return torch.exp(-lam)
    if kind == "inv":
        return 1.0 / (lam - sigma)
    if kind == "id":
        return lam.clone()
    return torch.ones_like(lam)


@pytest.mark.parametrize("kind", ["exp", "inv", "id", "one"])
def test_matrix_function_vs_dense(kind):
    """n = 512, leaf 32, rank 4: f(A) X for exp(-A), the shifted inverse
    (A - sigma I)^-1 with sigma halfway between two eigenvalues, A itself and
    the identity, against Q_d f(L_d) Q_d^T X from numpy's eigh of the dense A."""
    h = inputs.cfg_small_hss()
    A = dense.dense_from_hss(h)
    n = h.tree.n
    H = sdc.HSSMatrix(h)
    lam, F = H.eig()
    ln = lam.cpu().numpy()
    sigma = 0.5 * (ln[200] + ln[201])
    Xn = inputs.normal_block(n, 6, seed=8)
    Y = F.apply_function(_fvals(lam, kind, sigma), torch.from_numpy(Xn).to(DEV)).cpu().numpy()
    ld, Qd = np.linalg.eigh(A)
    fd = {"exp": np.exp(-ld), "inv": 1.0 / (ld - sigma), "id": ld, "one": np.ones(n)}[kind]
    Yref = Qd @ (fd[:, None] * (Qd.T @ Xn))
    rel = np.linalg.norm(Y - Yref) / np.linalg.norm(Yref)
    # the shifted inverse amplifies rounding by ||A|| / min|lambda - sigma|
    cond = np.abs(fd).max() / np.abs(fd).min() if kind == "inv" else 1.0
    print(kind, "relative error", rel)
    assert rel <= 1e-13 * max(1.0, cond) * 10, (kind, rel)
    if kind == "id":
        assert np.linalg.norm(Y - A @ Xn) / np.linalg.norm(A @ Xn) <= 1e-12
    if kind == "one":
        assert np.abs(Y - Xn).max() <= 1e-12 * np.abs(Xn).max()


def test_matrix_function_identity_is_matvec_16384():
    """Clustered n = 16384: Q diag(lambda) Q^T X equals the HSS matrix-vector
    product A X from the generators (no dense matrix), measured like the
    probe residual, ||Y - A X|| / (||A|| ||X||) <= 1e-12 sqrt(n): about 2e5
    deflations with tau = 1e-10 perturb A by O(tau) here (Remark 4.1)."""
    h = inputs.cfg_clustered_16384()
    H = sdc.HSSMatrix(h)
    lam, F = H.eig()
    Xn = inputs.normal_block(h.tree.n, 8, seed=9)
    Y = F.apply_function(lam, torch.from_numpy(Xn).to(DEV)).cpu().numpy()
    ref = dense.hss_matvec(h, Xn)
    an = max(float(lam.abs().max()), 1.0)
    rel = np.linalg.norm(Y - ref) / (an * np.linalg.norm(Xn))
    print("f = lambda at n = 16384: relative error", rel)
    assert rel <= 1e-12 * np.sqrt(h.tree.n)


@pytest.mark.parametrize("n,leaf,rank", [(256, 32, 3), (2048, 64, 4)])
def test_hermitian_eigenvalues_vectors_and_functions(n, leaf, rank):
    """Complex Hermitian HSS matrices: every eigenvalue twice in the real form,
    each copy against numpy's eigvalsh of the dense complex matrix per entry;
    the complex eigenvectors read from every other column of the real Q give
    the paper's residual and orthogonality metrics (gamma, theta) <= 1e-12;
    exp(-A) x for complex x against the dense reference."""
    h = inputs.hss_random_hermitian(n, leaf, rank, seed=11)
    A = dense.dense_from_hss_hermitian(h)
    ld = np.linalg.eigvalsh(A)
    an = np.abs(ld).max()
    H = sdc.HSSMatrix(h, hermitian=True)
    lam, F = H.eig()
    lr = lam.cpu().numpy()
    assert len(lr) == 2 * n
    nsteps = F.lmax * F.rank
    for half in (lr[0::2], lr[1::2]):
        ok, info = P.lam_check(half, ld, an, nsteps)
        print("hermitian n=%d eigenvalues" % n, info)
        assert ok, info
    # eigenvectors: column 2k of the real Q, read in the complex layout
    k = min(n, 256)
    sel = torch.zeros((2 * n, k), dtype=torch.float64, device=DEV)
    cols = np.arange(0, 2 * k, 2) if n <= 256 else np.linspace(0, 2 * n - 2, k).astype(int) // 2 * 2
    sel[torch.from_numpy(cols).to(DEV), torch.arange(k, device=DEV)] = 1.0
    Qr = F.apply_Q(sel).cpu().numpy()
    Xc = inputs.complex_layout(h, Qr)
    lk = lr[cols]
    res = np.linalg.norm(A @ Xc - Xc * lk[None, :], axis=0).max() / (n * np.linalg.norm(A, 2))
    orth = np.linalg.norm(Xc.conj().T @ Xc - np.eye(k), axis=0).max() / n
    print("hermitian gamma", res, "theta", orth)
    assert res <= 1e-12 and orth <= 1e-12
    # exp(-A) x for complex x, in the real layout
    rng = np.random.default_rng(12)
    x = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    xr = torch.from_numpy(inputs.real_layout(h, x)).to(DEV)
    y = inputs.complex_layout(h, F.apply_function(torch.exp(-lam), xr).cpu().numpy())
    Ld, Qd = np.linalg.eigh(A)
    yref = Qd @ (np.exp(-Ld)[:, None] * (Qd.conj().T @ x))
    rel = np.linalg.norm(y - yref) / np.linalg.norm(yref)
    print("hermitian exp(-A) x relative error", rel)
    assert rel <= 1e-15 * 2 * n          # a few eps per row of the real form
