"""Reverse mode of the HSS eigendecomposition (superdc_eig_backward through
the HSSEig autograd Function): against torch.linalg.eigh autograd of the
assembled dense matrix (n = 256 and the n = 8192 workload, leaf 64, rank 6),
and against central finite differences on the n = 8192 workload."""
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


class _Backward8192:
    """The n = 8192 workload (leaf 64, rank 6) and its loss
    L = sum w_i lambda_i + sum u_i (q_i^T v)^2 (w, u, v ~ N(0,1), seed 3),
    with the analytic gradient from superdc_eig_backward; FD directions are
    seeded unit vectors in generator space (symmetric in the leaf blocks)."""

    def __init__(self):
        self.h = inputs.cfg_backward_8192()
        n = self.h.tree.n
        rng = np.random.default_rng(3)
        self.w = torch.from_numpy(rng.standard_normal(n)).to(DEV)
        self.u = torch.from_numpy(rng.standard_normal(n)).to(DEV)
        self.v = torch.from_numpy(rng.standard_normal((n, 1))).to(DEV)
        self.opts = sdc.default_opts(tau=1e-10, stop_c=0.25)      # roots to adjacent doubles: smooth FD
        self.base = packed_tensors(self.h, DEV)
        self.L0, self.grads = self.loss(self.base, grad=True)
        self.drng = np.random.default_rng(103)

    def loss(self, gens, grad=False):
        ts = [g.clone().requires_grad_(grad) for g in gens]
        lam, Y = sdc.HSSEig.apply(self.h.tree, *ts, self.v, self.opts)
        L = (self.w * lam).sum() + (self.u * Y[:, 0] ** 2).sum()
        if grad:
            L.backward()
            return L.item(), [t.grad for t in ts]
        return L.item()

    def direction(self):
        dirs = [torch.from_numpy(self.drng.standard_normal(g.numel())).to(DEV) for g in self.base]
        dD = dirs[0].cpu().numpy()
        pos = 0
        for i in self.h.tree.leaves:
            m = int(self.h.tree.leaf_size[i])
            blk = dD[pos:pos + m * m].reshape(m, m)
            dD[pos:pos + m * m] = (0.5 * (blk + blk.T)).reshape(-1)
            pos += m * m
        dirs[0] = torch.from_numpy(dD).to(DEV)
        nrm = float(torch.sqrt(sum((d * d).sum() for d in dirs)))
        return [d / nrm for d in dirs]

    def central(self, dirs, hstep):
        Lp = self.loss([g + hstep * d for g, d in zip(self.base, dirs)])
        Lm = self.loss([g - hstep * d for g, d in zip(self.base, dirs)])
        return (Lp - Lm) / (2 * hstep)

    def analytic(self, dirs):
        return sum(float((g * d).sum()) for g, d in zip(self.grads, dirs))


@pytest.fixture(scope="module")
def bw8192():
    return _Backward8192()


def ridders(central, h0=1e-3, c=2.0, kmax=9):
    """Derivative by central differences extrapolated over a falling step
    (Ridders' method, 1982): a Neville tableau of the central differences at
    h0, h0/c, h0/c^2, ..., each column cancelling the next even power of h;
    the entry whose two neighbours agree best is returned with that
    disagreement as its error estimate.  Stops once the diagonal's error has
    grown to twice the best one (rounding has taken over)."""
    prev = [central(h0)]
    best, err = prev[0], float("inf")
    h = h0
    for k in range(1, kmax):
        h /= c
        row = [central(h)]
        fac = c * c
        for j in range(1, k + 1):
            row.append(row[j - 1] + (row[j - 1] - prev[j - 1]) / (fac - 1.0))
            fac *= c * c
            e = max(abs(row[j] - row[j - 1]), abs(row[j] - prev[j - 1]))
            if e <= err:
                best, err = row[j], e
        if abs(row[k] - prev[k - 1]) >= 2.0 * err:
            break
        prev = row
    return best, err


def test_finite_differences_8192(bw8192):
    """20 directions: the directional derivative from central differences,
    extrapolated by Ridders' method over steps 1e-3, 5e-4, ... (each
    direction takes the step range where neither truncation, which grows near
    a close pair of eigenvalues, nor rounding of the loss, ~eps_L / h,
    dominates), against the analytic one: 1e-6 relative with no further
    allowance.  A plain step of 1e-6 is rounding-limited at a few 1e-6
    (test_fd_step_sweep_shows_rounding_floor)."""
    worst = 0.0
    for trial in range(20):
        dirs = bw8192.direction()
        fd, est = ridders(lambda hs: bw8192.central(dirs, hs))
        an = bw8192.analytic(dirs)
        rel = abs(fd - an) / abs(an)
        worst = max(worst, rel)
        assert rel <= 1e-6, (trial, fd, an, rel, est)
    print("Ridders-extrapolated central differences: worst relative error", worst)


def test_fd_step_sweep_shows_rounding_floor(bw8192):
    """Plain central differences over h = 1e-3 .. 1e-7 on 3 directions: the
    error falls like h^2 from 1e-3 to 1e-4 (truncation) and grows again from
    1e-5 to 1e-7 (rounding of the loss, ~eps_L / h), so the ~1e-6 relative
    error of the step 1e-6 is the rounding floor of the loss evaluation, not a
    gradient error (measured at step 1e-6: up to 5.8e-6 relative)."""
    for trial in range(3):
        dirs = bw8192.direction()
        an = bw8192.analytic(dirs)
        err = {hs: abs(bw8192.central(dirs, hs) - an) / abs(an) for hs in (1e-3, 1e-4, 1e-5, 1e-6, 1e-7)}
        print("step sweep", trial, {k: "%.2e" % v for k, v in err.items()})
        assert err[1e-3] >= 30.0 * err[1e-4], err        # h^2 truncation
        assert err[1e-7] >= 3.0 * err[1e-5], err         # 1/h rounding
        assert err[1e-6] <= 1e-5, err


def test_dense_gradient_8192(bw8192):
    """The gradients with respect to every generator against FP64
    torch.linalg.eigh autograd of the assembled dense matrix (n = 8192, on the
    host cores), for the same loss (sign-invariant in the eigenvectors)."""
    h = bw8192.h
    Dc, Uc, Rc, Bc = packed_tensors(h, "cpu", grad=True)
    lc, Qc = torch.linalg.eigh(dense_torch(h.tree, Dc, Uc, Rc, Bc))
    Yc = Qc.t() @ bw8192.v.cpu()
    L = (bw8192.w.cpu() * lc).sum() + (bw8192.u.cpu() * Yc[:, 0] ** 2).sum()
    L.backward()
    assert abs(L.item() - bw8192.L0) <= 1e-10 * abs(L.item())
    for name, gg, gc in zip("DURB", bw8192.grads, (Dc.grad, Uc.grad, Rc.grad, Bc.grad)):
        gg = gg.cpu()
        rel = (gg - gc).abs().max().item() / gc.abs().max().item()
        print("dense gradient", name, "max relative error", rel)
        assert rel <= 1e-8, (name, rel)


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
