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
               status=torch.zeros(1, **i32))
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


def secular_batched_host(offsets, d, z, rho=1.0, opts=None, fields=("lam", "eta", "org", "vhat", "bnorm")):
    """End-to-end variant: host (CPU) tensors in, host tensors out.  Copies the
    inputs to the device, runs the batched step, copies ``fields`` back."""
    dev = torch.device("cuda")
    offs = offsets.to(dev, non_blocking=True)
    dd = d.to(dev, non_blocking=True)
    zz = z.to(dev, non_blocking=True)
    out = secular_batched(offs, dd, zz, rho, opts, check=False)
    res = {k: out[k].to("cpu", non_blocking=True) for k in fields}
    st = out["status"].to("cpu", non_blocking=True)
    torch.cuda.current_stream().synchronize()
    check_status(st, "superdc_secular_batched")
    return res
