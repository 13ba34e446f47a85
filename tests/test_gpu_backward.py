"""Adjoint of the batched rank-one step (superdc_secular_batched_backward):
against the dense eigen-adjoint of diag(d) + z z^T built from the oracle's
dense eigenvectors, against central finite differences of the GPU forward,
and through the torch.autograd.Function wrapper."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import inputs  # noqa: E402
from oracle import rank1 as r1  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def separated_batch(seed, sizes):
    rng = np.random.default_rng(seed)
    ds, zs = [], []
    for m in sizes:
        ds.append(np.sort(rng.uniform(0, 1, m)))
        zs.append(rng.standard_normal(m))
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    return inputs.SecularBatch(offs, np.concatenate(ds), np.concatenate(zs), 1.0)


def dense_adjoint(d, z, tau, lam_bar, X, Ybar):
    """Eigen-adjoint of M = diag(d) + z z^T with the oracle's eigenvectors
    (merged order, sign(zhat) convention): Mbar = Q (diag(lam_bar) +
    sym(F o (Y Ybar^T))) Q^T, F_kl = 1/(lambda_l - lambda_k)."""
    f = r1.rank1_step(d, z, tau)
    Q, lam = f.dense(), f.lam
    Y = Q.T @ X
    F = lam[None, :] - lam[:, None]
    np.fill_diagonal(F, 1.0)
    F = 1.0 / F
    np.fill_diagonal(F, 0.0)
    A = F * (Y @ Ybar.T)
    E = np.diag(lam_bar) + 0.5 * (A + A.T)
    Mb = Q @ E @ Q.T
    return np.diag(Mb).copy(), 2.0 * Mb @ z, Q @ Ybar, Y


def gpu_fwd_bwd(b, tau, lam_bar, X, Ybar):
    offs = torch.from_numpy(b.offsets).to(DEV)
    out = sdc.secular_batched(offs, torch.from_numpy(b.d).to(DEV), torch.from_numpy(b.z).to(DEV), 1.0,
                              sdc.default_opts(tau=tau))
    Xt = torch.from_numpy(X).to(DEV)
    Y = sdc.apply_rank1(offs, out, Xt, trans=True)
    db, zb, Xb = sdc.secular_batched_backward(offs, out, 1.0, torch.from_numpy(lam_bar).to(DEV), Xt,
                                              torch.from_numpy(Ybar).to(DEV))
    return out, Y.cpu().numpy(), db.cpu().numpy(), zb.cpu().numpy(), Xb.cpu().numpy()


def test_against_dense_eigen_adjoint():
    b = separated_batch(1, [5, 37, 130, 200])
    rng = np.random.default_rng(2)
    total = int(b.offsets[-1])
    lam_bar = rng.standard_normal(total)
    X = rng.standard_normal((total, 3))
    Ybar = rng.standard_normal((total, 3))
    out, Y, db, zb, Xb = gpu_fwd_bwd(b, 1e-14, lam_bar, X, Ybar)
    for p in range(b.nprob):
        a, e = int(b.offsets[p]), int(b.offsets[p + 1])
        d, z = b.problem(p)
        rd, rz, rX, rY = dense_adjoint(d, z, 1e-14, lam_bar[a:e], X[a:e], Ybar[a:e])
        assert np.allclose(Y[a:e], rY, rtol=0, atol=1e-11 * np.abs(rY).max())
        assert np.allclose(Xb[a:e], rX, rtol=0, atol=1e-11 * np.abs(rX).max())
        scale_d, scale_z = np.abs(rd).max(), np.abs(rz).max()
        assert np.abs(db[a:e] - rd).max() <= 1e-9 * scale_d, (p, np.abs(db[a:e] - rd).max(), scale_d)
        assert np.abs(zb[a:e] - rz).max() <= 1e-9 * scale_z, (p, np.abs(zb[a:e] - rz).max(), scale_z)


def _loss(b, d, z, w, X, Ybar, tau):
    offs = torch.from_numpy(b.offsets).to(DEV)
    out = sdc.secular_batched(offs, torch.from_numpy(d).to(DEV), torch.from_numpy(z).to(DEV), 1.0,
                              sdc.default_opts(tau=tau))
    Y = sdc.apply_rank1(offs, out, torch.from_numpy(X).to(DEV), trans=True).cpu().numpy()
    return float(w @ out["lam"].cpu().numpy() + np.sum(Ybar * Y))


@pytest.mark.parametrize("with_zdefl", [False, True])
def test_central_finite_differences(with_zdefl):
    b = separated_batch(3, [64, 150, 300])
    tau = 1e-12
    z = b.z.copy()
    small = np.zeros_like(z, dtype=bool)
    if with_zdefl:
        small[[3, 70, 100, 400]] = True
        z[small] = 1e-14                     # |z| < tau: deflated, zero derivative by construction
    b = inputs.SecularBatch(b.offsets, b.d, z, 1.0)
    rng = np.random.default_rng(4)
    total = int(b.offsets[-1])
    w = rng.standard_normal(total)
    X = rng.standard_normal((total, 2))
    Ybar = rng.standard_normal((total, 2))
    out, Y, db, zb, Xb = gpu_fwd_bwd(b, tau, w, X, Ybar)
    h = 1e-6
    for trial in range(5):
        dd = rng.standard_normal(total) * 1e-3     # keeps the poles sorted (spacing >> h * 1e-3)
        dz = rng.standard_normal(total)
        dz[small] = 0.0
        lp = _loss(b, b.d + h * dd, b.z + h * dz, w, X, Ybar, tau)
        lm = _loss(b, b.d - h * dd, b.z - h * dz, w, X, Ybar, tau)
        fd = (lp - lm) / (2 * h)
        an = float(db @ dd + zb @ dz)
        assert abs(fd - an) <= 1e-6 * max(abs(an), abs(fd)), (trial, fd, an)


def test_autograd_function():
    b = separated_batch(5, [40, 90])
    rng = np.random.default_rng(6)
    total = int(b.offsets[-1])
    offs = torch.from_numpy(b.offsets).to(DEV)
    d = torch.from_numpy(b.d).to(DEV).requires_grad_(True)
    z = torch.from_numpy(b.z).to(DEV).requires_grad_(True)
    X = torch.from_numpy(rng.standard_normal((total, 2))).to(DEV).requires_grad_(True)
    w = torch.from_numpy(rng.standard_normal(total)).to(DEV)
    G = torch.from_numpy(rng.standard_normal((total, 2))).to(DEV)
    lam, Y = sdc.SecularEig.apply(offs, d, z, X, 1.0, 1e-14)
    loss = (w * lam).sum() + (G * Y).sum()
    loss.backward()
    out, Yn, db, zb, Xb = gpu_fwd_bwd(b, 1e-14, w.cpu().numpy(), X.detach().cpu().numpy(), G.cpu().numpy())
    assert np.allclose(d.grad.cpu().numpy(), db, rtol=1e-12, atol=1e-14 * np.abs(db).max())
    assert np.allclose(z.grad.cpu().numpy(), zb, rtol=1e-12, atol=1e-14 * np.abs(zb).max())
    assert np.allclose(X.grad.cpu().numpy(), Xb, rtol=1e-12, atol=1e-14 * np.abs(Xb).max())
