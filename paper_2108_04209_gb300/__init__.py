"""SuperDC conquering stage on GB300 (sm_103a CUDA, FP64).

Public Python API over the C ABI of ``include/superdc.h``.  PyTorch provides
device memory and streams only; every step of the method runs in the CUDA
library ``_lib/libsuperdc.so``.
"""
import ctypes

import torch

from . import _lib as L
from ._lib import SuperDCError, default_opts  # noqa: F401

__all__ = ["secular_batched", "secular_batched_host", "default_opts", "SuperDCError", "check_status"]


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def check_status(status_tensor, where=""):
    """Raise if the device status word has error bits (synchronises)."""
    s = int(status_tensor.item())
    if s & L.DEV_NONFINITE:
        raise SuperDCError(4, where)
    if s & L.DEV_NOCONV:
        raise SuperDCError(5, where)
    if s & L.DEV_INDEX:
        raise SuperDCError(2, where + " (index guard)")


def alloc_rank1_out(nprob, total, device, sweeps=True):
    f64 = dict(dtype=torch.float64, device=device)
    i32 = dict(dtype=torch.int32, device=device)
    n = max(total, 1)
    out = dict(lam=torch.empty(n, **f64), dk=torch.empty(n, **f64), zk=torch.empty(n, **f64),
               eta=torch.empty(n, **f64), vhat=torch.empty(n, **f64), bnorm=torch.empty(n, **f64),
               org=torch.empty(n, **i32), src=torch.empty(n, **i32), perm=torch.empty(n, **i32),
               giv_ab=torch.empty(2 * n, **i32), giv_cs=torch.empty(2 * n, **f64),
               mk=torch.empty(max(nprob, 1), **i32), ngiv=torch.empty(max(nprob, 1), **i32),
               sweeps=torch.empty(n, **i32) if sweeps else None,
               status=torch.zeros(1, **i32), fmm=torch.zeros(max(nprob, 1), **i32))
    return out


def secular_batched(offsets, d, z, rho=1.0, opts=None, out=None, check=True):
    """Batched rank-one steps diag(d_p) + rho z_p z_p^T (device tensors).

    offsets: int64 [nprob+1] on the GPU; d, z: float64 [total] on the GPU.
    Returns a dict of device tensors (layout of superdc_rank1_out in
    include/superdc.h).  With ``check`` the device status is read and errors
    raise (this synchronises the stream)."""
    assert d.is_cuda and z.is_cuda and offsets.is_cuda, "device tensors required"
    assert d.dtype == torch.float64 and z.dtype == torch.float64 and offsets.dtype == torch.int64
    nprob = offsets.numel() - 1
    total = d.numel()
    if opts is None:
        opts = default_opts(tau=1e-12)
    if out is None:
        out = alloc_rank1_out(nprob, total, d.device)
    else:
        out["status"].zero_()
    ro = L.Rank1Out(**{k: (_ptr(v).value or None) for k, v in out.items()})
    code = L.lib().superdc_secular_batched(nprob, _ptr(offsets), total, _ptr(d), _ptr(z), float(rho),
                                           ctypes.byref(opts), ctypes.byref(ro), _stream())
    L.check(code, "superdc_secular_batched")
    if check:
        check_status(out["status"], "superdc_secular_batched")
    return out


def secular_batched_host(offsets, d, z, rho=1.0, opts=None, fields=("lam", "eta", "org", "vhat", "bnorm"),
                         out=None):
    """End-to-end variant through the host-buffer entry point
    superdc_secular_batched_host: CPU tensors in (pinned for asynchronous
    copies), CPU tensors out.  ``fields`` selects the outputs copied back;
    ``out`` (optional) is a dict of preallocated CPU tensors to reuse."""
    assert not d.is_cuda and not z.is_cuda and not offsets.is_cuda, "host tensors required"
    assert d.dtype == torch.float64 and z.dtype == torch.float64 and offsets.dtype == torch.int64
    nprob = offsets.numel() - 1
    total = d.numel()
    if opts is None:
        opts = default_opts(tau=1e-12)
    if out is None:
        pin = torch.cuda.is_available()
        out = {}
        for k in fields:
            dt = torch.int32 if k in ("org", "src", "perm", "giv_ab", "mk", "ngiv", "sweeps", "fmm") else torch.float64
            n = {"giv_ab": 2 * total, "giv_cs": 2 * total, "mk": nprob, "ngiv": nprob, "fmm": nprob}.get(k, total)
            out[k] = torch.empty(max(n, 1), dtype=dt, pin_memory=pin)
        out["status"] = torch.zeros(1, dtype=torch.int32, pin_memory=pin)
    ro = L.Rank1Out(**{k: (_ptr(out[k]).value if k in out else None) for k, _ in L.Rank1Out._fields_})
    code = L.lib().superdc_secular_batched_host(nprob, _ptr(offsets), total, _ptr(d), _ptr(z), float(rho),
                                                ctypes.byref(opts), ctypes.byref(ro), _stream())
    L.check(code, "superdc_secular_batched_host")
    return {k: v for k, v in out.items() if k != "status"}


# ---------------------------------------------------------------------------
# HSS eigendecomposition
# ---------------------------------------------------------------------------
class HSSMatrix:
    """Library-owned device copy of a symmetric HSS matrix (superdc_build_hss).

    ``h`` is an ``inputs.HSS`` (tree + generators); the generators are copied
    to the GPU and then into the library handle."""

    def __init__(self, h, device=None, tensors=None, hermitian=False):
        """``hermitian``: ``h`` holds complex Hermitian generators; the handle
        is the real form of order 2n (superdc_build_hss_hermitian)."""
        import numpy as np
        dev = torch.device(device or "cuda")
        t = h.tree if hasattr(h, "tree") else h
        self.hermitian = bool(hermitian)
        self.n, self.rank = int(t.n) * (2 if hermitian else 1), int(t.rank) * (2 if hermitian else 1)
        self.tree = t
        self._lch = np.ascontiguousarray(t.lchild, np.int32)
        self._rch = np.ascontiguousarray(t.rchild, np.int32)
        self._sz = np.ascontiguousarray(t.leaf_size, np.int64)
        tree = L.Tree(int(t.n), int(t.nnodes), self._lch.ctypes.data, self._rch.ctypes.data,
                      self._sz.ctypes.data, int(t.rank))
        if tensors is not None:
            D, U, R, B = (x.detach().contiguous() for x in tensors)
        else:
            D, U, R, B = (torch.from_numpy(x).to(dev) for x in h.packed())
        self.sizes = (D.numel(), U.numel(), R.numel(), B.numel())
        self._h = ctypes.c_void_p()
        build = L.lib().superdc_build_hss_hermitian if hermitian else L.lib().superdc_build_hss
        code = build(ctypes.byref(tree), _ptr(D), _ptr(U), _ptr(R), _ptr(B), _stream(), ctypes.byref(self._h))
        L.check(code, "superdc_build_hss_hermitian" if hermitian else "superdc_build_hss")

    def eig(self, opts=None):
        """Eigendecomposition; returns (lambda [n] device tensor ascending, EigFactor)."""
        if opts is None:
            opts = default_opts()
        lam = torch.empty(self.n, dtype=torch.float64, device="cuda")
        f = ctypes.c_void_p()
        code = L.lib().superdc_eig(self._h, ctypes.byref(opts), _stream(), _ptr(lam), ctypes.byref(f))
        fac = EigFactor(f, self) if f.value else None
        L.check(code, "superdc_eig")
        return lam, fac

    @classmethod
    def from_entries(cls, n, leaf, rank, kind="sqrt_dist", A=None, x=None, param=0.0, nsamp=None, seed=0):
        """HSS approximation by off-diagonal compression (superdc_build_hss_compress)
        of the symmetric matrix with entries sqrt|x_i - x_j| ("sqrt_dist"),
        exp(-|x_i - x_j| / param) ("exp_dist") at the points x (float64 CUDA
        tensor), or the dense matrix A ("dense", float64 CUDA n x n).  The
        Gaussian sample (n x nsamp, nsamp = rank + 10 by default) is drawn by
        inputs.gaussian_block(seed).  The estimate sigma_{r+1}/sigma_1 of the
        dropped part is in .err_est."""
        import numpy as np
        from . import inputs
        kinds = {"dense": 0, "sqrt_dist": 1, "exp_dist": 2}
        s = int(nsamp or min(64, rank + 10))
        Om = torch.from_numpy(inputs.normal_block(n, s, seed=seed)).cuda()
        ent = L.MatrixEntries(kinds[kind], _ptr(A).value if A is not None else None,
                              int(A.stride(1)) if A is not None else 0,
                              _ptr(x).value if x is not None else None, float(param))
        hp = ctypes.c_void_p()
        est = ctypes.c_double()
        code = L.lib().superdc_build_hss_compress(int(n), int(leaf), int(rank), ctypes.byref(ent), _ptr(Om), s,
                                                  _stream(), ctypes.byref(hp), ctypes.byref(est))
        L.check(code, "superdc_build_hss_compress")
        self = cls.__new__(cls)
        t = inputs.perfect_tree(int(n), int(leaf), int(rank))
        self.hermitian = False
        self.n, self.rank, self.tree = int(n), int(rank), t
        self._lch = np.ascontiguousarray(t.lchild, np.int32)
        self._rch = np.ascontiguousarray(t.rchild, np.int32)
        self._sz = np.ascontiguousarray(t.leaf_size, np.int64)
        self.sizes = (int(n) * int(leaf), int(n) * int(rank), t.nnodes * rank * rank, t.nnodes * rank * rank)
        self._h = hp
        self.err_est = est.value
        return self

    def generators(self):
        """The handle's generators as an inputs.HSS (host arrays; superdc_hss_get)."""
        import numpy as np
        from . import inputs
        t = self.tree
        D, U, R, B, d_off, u_off = inputs._alloc(t)
        r = t.rank
        for name, arr in (("D", D), ("U", U)):
            L.check(L.lib().superdc_hss_get(self._h, name.encode(), arr.ctypes.data), "superdc_hss_get")
        for name, arr in (("R", R), ("B", B)):
            flat = np.empty(t.nnodes * r * r)
            L.check(L.lib().superdc_hss_get(self._h, name.encode(), flat.ctypes.data), "superdc_hss_get")
            arr[:] = np.transpose(flat.reshape(t.nnodes, r, r), (0, 2, 1))
        return inputs.HSS(t, D, U, R, B, d_off, u_off)

    def eig_plan(self, opts=None):
        """superdc_eig_plan: a factor handle with every buffer allocated; run it
        with EigFactor.run (which can be captured into a CUDA graph)."""
        if opts is None:
            opts = default_opts()
        f = ctypes.c_void_p()
        L.check(L.lib().superdc_eig_plan(self._h, ctypes.byref(opts), ctypes.byref(f)), "superdc_eig_plan")
        return EigFactor(f, self)

    def __del__(self):
        try:
            if self._h and self._h.value:
                L.lib().superdc_hss_free(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass


class EigFactor:
    """Structured Q of an HSS eigendecomposition (superdc_eigfact)."""

    def __init__(self, handle, owner):
        self._f = handle
        self._owner = owner   # keeps the HSS handle alive
        lm, r, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        L.check(L.lib().superdc_eigfact_shape(self._f, ctypes.byref(lm), ctypes.byref(r), ctypes.byref(n)))
        self.lmax, self.rank, self.n = lm.value, r.value, n.value

    def apply_Q(self, X, trans=False):
        """Y = Q X (trans False) or Q^T X; X: float64 CUDA tensor n or n x k."""
        vec = X.dim() == 1
        Xc = X.reshape(self.n, -1)
        Xf = Xc.t().contiguous().t() if not Xc.t().is_contiguous() else Xc    # column-major view
        k = Xf.shape[1]
        Y = torch.empty((k, self.n), dtype=torch.float64, device=X.device).t()
        ldx = Xf.stride(1) if k > 1 else self.n
        code = L.lib().superdc_apply_Q(self._f, 1 if trans else 0, k, _ptr(Xf), ldx, _ptr(Y),
                                       self.n, _stream())
        L.check(code, "superdc_apply_Q")
        return Y.reshape(-1) if vec else Y

    def run(self, lam):
        """superdc_eig_run on the current stream into lam (float64 CUDA, n):
        enqueue only, no synchronisation; errors via sync_status()."""
        assert lam.is_cuda and lam.dtype == torch.float64 and lam.numel() == self.n
        L.check(L.lib().superdc_eig_run(self._f, _stream(), _ptr(lam)), "superdc_eig_run")
        return lam

    def sync_status(self):
        """Raise if the handle's device status word holds an error (synchronises)."""
        L.check(L.lib().superdc_sync_status(self._f), "superdc_sync_status")

    def apply_function(self, fvals, X):
        """f(A) X = Q diag(fvals) Q^T X (superdc_apply_function); fvals: float64
        CUDA tensor of f(lambda_i) for the ascending eigenvalues; X: n or n x k."""
        vec = X.dim() == 1
        Xc = X.reshape(self.n, -1)
        Xf = Xc.t().contiguous().t() if not Xc.t().is_contiguous() else Xc
        k = Xf.shape[1]
        fv = fvals.contiguous()
        assert fv.numel() == self.n and fv.dtype == torch.float64 and fv.is_cuda
        Y = torch.empty((k, self.n), dtype=torch.float64, device=X.device).t()
        ldx = Xf.stride(1) if k > 1 else self.n
        code = L.lib().superdc_apply_function(self._f, _ptr(fv), k, _ptr(Xf), ldx, _ptr(Y), self.n, _stream())
        L.check(code, "superdc_apply_function")
        return Y.reshape(-1) if vec else Y

    def set_fmm_min_m(self, fmm_min_m):
        """FMM threshold of later apply_Q calls (opts.fmm_min_m meaning)."""
        L.check(L.lib().superdc_eigfact_set_fmm_min_m(self._f, int(fmm_min_m)), "superdc_eigfact_set_fmm_min_m")

    def stats(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        L.check(L.lib().superdc_eigfact_stats(self._f, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"deflated": a.value, "sweeps": b.value, "max_sweeps": c.value}

    def get(self, level, step, field):
        import numpy as np
        n = self.n
        nn = 2 ** level
        spec = {"dk": (n, np.float64), "eta": (n, np.float64), "dorg": (n, np.float64), "vhat": (n, np.float64),
                "bnorm": (n, np.float64), "din": (n, np.float64), "zin": (n, np.float64), "src": (n, np.int32), "pinv": (n, np.int32), "sweeps": (n, np.int32), "P": (n, np.int32),
                "giv_cs": (2 * n, np.float64), "giv_ab": (2 * n, np.int32), "mk": (nn, np.int32),
                "ngiv": (nn, np.int32), "fmm": (nn, np.int32)}
        cnt, dt = spec[field]
        out = np.empty(cnt, dt)
        L.check(L.lib().superdc_eigfact_get(self._f, level, step, field.encode(), out.ctypes.data),
                "superdc_eigfact_get")
        return out

    def __del__(self):
        try:
            if self._f and self._f.value:
                L.lib().superdc_eigfact_free(self._f)
                self._f = ctypes.c_void_p()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Adjoint of the batched rank-one step and its autograd wrapper
# ---------------------------------------------------------------------------
def secular_batched_backward(offsets, out, rho, lam_bar=None, X=None, Ybar=None):
    """Reverse mode of ``secular_batched`` (superdc_secular_batched_backward).

    ``out`` is the dict returned by the forward call.  Returns (d_bar, z_bar,
    X_bar); X_bar is None when no columns are given."""
    total = out["lam"].numel() if offsets.numel() > 1 else 0
    total = int(offsets[-1].item()) if total else 0
    nprob = offsets.numel() - 1
    dev = out["lam"].device
    d_bar = torch.empty(max(total, 1), dtype=torch.float64, device=dev)
    z_bar = torch.empty(max(total, 1), dtype=torch.float64, device=dev)
    ncols = 0
    Xf = Yf = Xb = None
    if X is not None:
        ncols = X.shape[1]
        Xf = X.t().contiguous().t()
        Yf = Ybar.t().contiguous().t()
        Xb = torch.empty((ncols, total), dtype=torch.float64, device=dev).t()
    ro = L.Rank1Out(**{k: (_ptr(v).value or None) for k, v in out.items()})
    code = L.lib().superdc_secular_batched_backward(
        nprob, _ptr(offsets), total, float(rho), ctypes.byref(ro), _ptr(lam_bar), ncols,
        _ptr(Xf), total, _ptr(Yf), total, _ptr(d_bar), _ptr(z_bar), _ptr(Xb), total, _stream())
    L.check(code, "superdc_secular_batched_backward")
    return d_bar[:total], z_bar[:total], Xb


class SecularEig(torch.autograd.Function):
    """(d, z, X) -> (lambda, Y = Qhat^T X) for a batch of rank-one problems,
    differentiable in d, z and X.  offsets (int64, device) and rho are
    constants.  The backward runs superdc_secular_batched_backward."""

    @staticmethod
    def forward(ctx, offsets, d, z, X, rho=1.0, tau=1e-12):
        out = secular_batched(offsets, d.detach(), z.detach(), rho, default_opts(tau=tau))
        Y = None
        if X is not None and X.numel():
            Y = _apply_rank1_T(offsets, out, X.detach())
        ctx.save_for_backward(offsets, X if X is not None else torch.empty(0, device=d.device))
        ctx.out, ctx.rho = out, rho
        lam = out["lam"][:d.numel()].clone()
        return (lam, Y) if Y is not None else (lam, torch.empty(0, device=d.device, dtype=torch.float64))

    @staticmethod
    def backward(ctx, lam_bar, Y_bar):
        offsets, X = ctx.saved_tensors
        has_x = X.numel() > 0
        d_bar, z_bar, X_bar = secular_batched_backward(
            offsets, ctx.out, ctx.rho, lam_bar.contiguous(),
            X if has_x else None, Y_bar if has_x else None)
        return None, d_bar, z_bar, (X_bar if has_x else None), None, None


def _apply_rank1_T(offsets, out, X):
    return apply_rank1(offsets, out, X, trans=True)


def apply_rank1(offsets, out, X, trans=True, opts=None):
    """Qhat^T X (trans) or Qhat X for the factors of a secular_batched result
    (opts: only fmm_min_m is used; None = defaults)."""
    total = int(offsets[-1].item())
    ncols = X.shape[1]
    Xf = X.t().contiguous().t()
    Y = torch.empty((ncols, total), dtype=torch.float64, device=X.device).t()
    ro = L.Rank1Out(**{k: (_ptr(v).value or None) for k, v in out.items()})
    code = L.lib().superdc_rank1_apply(offsets.numel() - 1, _ptr(offsets), total, ctypes.byref(ro),
                                       1 if trans else 0, ncols, _ptr(Xf), total, _ptr(Y), total,
                                       ctypes.byref(opts) if opts is not None else None, _stream())
    L.check(code, "superdc_rank1_apply")
    return Y


class HSSEig(torch.autograd.Function):
    """(D, U, R, B, V) -> (lambda, Y = Q^T V) for a symmetric HSS matrix given
    by its packed generators (layout of superdc_build_hss; ``tree`` is an
    ``inputs.Tree``).  Differentiable in D (symmetric perturbations), U, R, B
    and V; the backward runs superdc_eig_backward on the forward's tape."""

    @staticmethod
    def forward(ctx, tree, D, U, R, B, V, opts=None):
        H = HSSMatrix(tree, tensors=(D, U, R, B))
        o = opts if opts is not None else default_opts()
        o.tape = 1
        lam, F = H.eig(o)
        Vc = V.detach().reshape(H.n, -1)
        Y = F.apply_Q(Vc, trans=True)
        ctx.H, ctx.F = H, F
        ctx.save_for_backward(Vc)
        return lam, Y

    @staticmethod
    def backward(ctx, lam_bar, Y_bar):
        (V,) = ctx.saved_tensors
        H, F = ctx.H, ctx.F
        n, k = V.shape
        dev = V.device
        gD, gU, gR, gB = (torch.empty(sz, dtype=torch.float64, device=dev) for sz in H.sizes)
        gV = torch.empty((k, n), dtype=torch.float64, device=dev).t()
        Vf = V.t().contiguous().t()
        Yb = (Y_bar if Y_bar is not None else torch.zeros_like(V)).t().contiguous().t()
        lb = lam_bar.contiguous() if lam_bar is not None else None
        code = L.lib().superdc_eig_backward(H._h, F._f, _ptr(lb), k, _ptr(Vf), n, _ptr(Yb), n, _ptr(gD), _ptr(gU),
                                            _ptr(gR), _ptr(gB), _ptr(gV), n, _stream())
        L.check(code, "superdc_eig_backward")
        return None, gD, gU, gR, gB, gV.reshape(V.shape), None
