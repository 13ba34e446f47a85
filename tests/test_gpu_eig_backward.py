"""Reverse mode of the HSS eigendecomposition (superdc_eig_backward through
the HSSEig autograd Function): against torch.linalg.eigh autograd of the
assembled dense matrix, and against central finite differences on the
n = 8192 workload (leaf 64, rank 6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def packed_tensors(h, device, grad=False):
    return [torch.from_numpy(x).to(device).requires_grad_(grad) for x in h.packed()]


def dense_torch(tree, D, U, R, B):
    """Dense A from packed generators (column-major blocks), differentiable."""
    n, r = int(tree.n), int(tree.rank)
    A = torch.zeros((n, n), dtype=torch.float64, device=D.device)
    Ub, dpos, upos = {}, 0, 0
    for i in range(tree.nnodes):
        o, m = int(tree.offset[i]), int(tree.leaf_size[i])
        if tree.lchild[i] < 0:
            A[o:o + m, o:o + m] = D[dpos:dpos + m * m].view(m, m).t()
            Ub[i] = U[upos:upos + m * r].view(r, m).t()
            dpos += m * m
            upos += m * r
            continue
        a, b = int(tree.lchild[i]), int(tree.rchild[i])
        oa, ma = int(tree.offset[a]), int(tree.leaf_size[a])
        ob, mb = int(tree.offset[b]), int(tree.leaf_size[b])
        Ba = B[a * r * r:(a + 1) * r * r].view(r, r).t()
        blk = Ub[a] @ Ba @ Ub[b].t()
        A[oa:oa + ma, ob:ob + mb] = blk
        A[ob:ob + mb, oa:oa + ma] = blk.t()
        if i != tree.nnodes - 1:
            Ra = R[a * r * r:(a + 1) * r * r].view(r, r).t()
            Rb = R[b * r * r:(b + 1) * r * r].view(r, r).t()
            Ub[i] = torch.cat([Ub[a] @ Ra, Ub[b] @ Rb], 0)
    return 0.5 * (A + A.t())


@pytest.mark.parametrize("clustered", [False, True])
def test_against_dense_eigh_autograd(clustered):
    """Well-separated spectrum: eigenvalue and eigenvector loss.  Clustered
    spectrum (eigenvalues repeated to 1e-12): individual eigenpairs are not
    differentiable there, so the loss is the trace sum(lambda), whose gradient
    is the identity on the leaf blocks and zero elsewhere."""
    h = inputs.hss_random(256, 32, 3, seed=41, clustered=clustered)
    n, k = h.tree.n, 2
    rng = np.random.default_rng(42)
    w = torch.from_numpy(rng.standard_normal(n)).to(DEV)
    G = torch.from_numpy(rng.standard_normal((n, k))).to(DEV)
    if clustered:
        w = torch.ones(n, dtype=torch.float64, device=DEV)
        G = torch.zeros((n, k), dtype=torch.float64, device=DEV)
    Vn = rng.standard_normal((n, k))
    # GPU path
    D, U, R, B = packed_tensors(h, DEV, grad=True)
    V = torch.from_numpy(Vn).to(DEV).requires_grad_(True)
    lam, Y = sdc.HSSEig.apply(h.tree, D, U, R, B, V, None)
    ((w * lam).sum() + (G * Y).sum()).backward()
    # dense reference (CPU, torch autograd of eigh), signs aligned with the GPU's Q
    Qg = sdc.HSSMatrix(h).eig(sdc.default_opts())[1].apply_Q(torch.eye(n, dtype=torch.float64, device=DEV))
    Dc, Uc, Rc, Bc = packed_tensors(h, "cpu", grad=True)
    Vc = torch.from_numpy(Vn).requires_grad_(True)
    lc, Qc = torch.linalg.eigh(dense_torch(h.tree, Dc, Uc, Rc, Bc))
    sgn = torch.sign((Qg.cpu() * Qc.detach()).sum(0))
    Yc = (Qc * sgn).t() @ Vc
    ((w.cpu() * lc).sum() + (G.cpu() * Yc).sum()).backward()
    assert torch.allclose(lam.cpu(), lc.detach(), atol=1e-10 * lc.abs().max().item())
    for name, gg, gc in (("D", D.grad, Dc.grad), ("U", U.grad, Uc.grad), ("R", R.grad, Rc.grad),
                         ("B", B.grad, Bc.grad), ("V", V.grad, Vc.grad)):
        gg, gc = gg.cpu(), gc
        scale = max(gc.abs().max().item(), 1.0 if clustered else 0.0)
        err = (gg - gc).abs().max().item()
        # clustered: the eigenvector couplings of pairs just above the degeneracy
        # cutoff cancel only to eps/gap ~ 1e-16/1e-10 relative on this spectrum
        tol = 1e-5 if clustered else 1e-8
        assert err <= tol * scale, (name, err, scale)


def test_finite_differences_8192():
    """Central differences, step 1e-6, along 20 seeded unit-norm directions in
    generator space (symmetric in the leaf blocks), for
    L = sum w_i lambda_i + sum u_i (q_i^T v)^2 (w, u, v ~ N(0,1)).

    Tolerance: 1e-6 relative (the O(h^2) truncation is far below it) plus the
    central difference's rounding term eps_L / h, with eps_L taken as
    1e-13 * (sum |w_i| max|lambda| + sum |u_i| (q_i^T v)^2), a forward error of
    the loss about ten times the eigensolver's backward error n * eps * ||A||."""
    h = inputs.cfg_backward_8192()
    n = h.tree.n
    rng = np.random.default_rng(3)
    w = torch.from_numpy(rng.standard_normal(n)).to(DEV)
    u = torch.from_numpy(rng.standard_normal(n)).to(DEV)
    v = torch.from_numpy(rng.standard_normal((n, 1))).to(DEV)
    opts = sdc.default_opts(tau=1e-10, stop_c=0.25)      # roots to adjacent doubles: smooth FD

    def loss(gens, grad=False):
        ts = [g.clone().requires_grad_(grad) for g in gens]
        lam, Y = sdc.HSSEig.apply(h.tree, *ts, v, opts)
        L = (w * lam).sum() + (u * Y[:, 0] ** 2).sum()
        if grad:
            L.backward()
            scale = (w.abs().sum() * lam.abs().max() + (u.abs() * Y[:, 0] ** 2).sum()).item()
            return L.item(), [t.grad for t in ts], scale
        return L.item()

    base = packed_tensors(h, DEV)
    L0, grads, lscale = loss(base, grad=True)
    drng = np.random.default_rng(103)
    hstep = 1e-6
    t = h.tree
    for trial in range(20):
        dirs = []
        for g in base:
            dirs.append(torch.from_numpy(drng.standard_normal(g.numel())).to(DEV))
        # symmetric perturbations of the leaf blocks
        dD = dirs[0].cpu().numpy()
        pos = 0
        for i in t.leaves:
            m = int(t.leaf_size[i])
            blk = dD[pos:pos + m * m].reshape(m, m)
            dD[pos:pos + m * m] = (0.5 * (blk + blk.T)).reshape(-1)
            pos += m * m
        dirs[0] = torch.from_numpy(dD).to(DEV)
        nrm = float(torch.sqrt(sum((d * d).sum() for d in dirs)))
        dirs = [d / nrm for d in dirs]
        Lp = loss([g + hstep * d for g, d in zip(base, dirs)])
        Lm = loss([g - hstep * d for g, d in zip(base, dirs)])
        fd = (Lp - Lm) / (2 * hstep)
        an = sum(float((g * d).sum()) for g, d in zip(grads, dirs))
        tol = 1e-6 * max(abs(an), abs(fd)) + 1e-13 * lscale / hstep
        assert abs(fd - an) <= tol, (trial, fd, an, tol)


def test_literal_projection_loss_has_zero_gradient():
    """||Q^T v||^2 = ||v||^2 for orthogonal Q: its gradient in the generators vanishes."""
    h = inputs.hss_random(1024, 64, 4, seed=44)
    n = h.tree.n
    v = torch.from_numpy(np.random.default_rng(45).standard_normal((n, 1))).to(DEV)
    D, U, R, B = packed_tensors(h, DEV, grad=True)
    lam, Y = sdc.HSSEig.apply(h.tree, D, U, R, B, v, None)
    (Y ** 2).sum().backward()
    ref = float((v ** 2).sum())
    for g in (D.grad, U.grad, R.grad, B.grad):
        assert g.abs().max().item() <= 1e-9 * ref
