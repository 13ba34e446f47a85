"""The allocation-free entry point superdc_secular_batched_noalloc, for
callers that cannot allocate device memory while they run (graph replay,
latency-bound paths, fixed memory budgets).  Called twice in a row through the
C ABI; each call must match superdc_secular_batched on the same inputs.  Kept
in a file that is collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import _lib as L, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _call_noalloc(b, opts, out):
    fn = L.lib().superdc_secular_batched_noalloc
    fn.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_double, ctypes.POINTER(L.Opts), ctypes.POINTER(L.Rank1Out), ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    dev = torch.device("cuda")
    offs = torch.from_numpy(b.offsets).to(dev)
    d = torch.from_numpy(b.d).to(dev)
    z = torch.from_numpy(b.z).to(dev)
    out["status"].zero_()
    ro = L.Rank1Out(**{k: (v.data_ptr() if v is not None else None) for k, v in out.items()})
    code = fn(b.nprob, offs.data_ptr(), int(b.offsets[-1]), d.data_ptr(), z.data_ptr(), 1.0,
              ctypes.byref(opts), ctypes.byref(ro), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return code, offs, d, z


def test_noalloc_matches_allocating_entry_point_twice():
    opts = sdc.default_opts(tau=1e-12)
    batches = [inputs.secular_batch(96, 32, 2048, seed=21),           # whole-problem units
               inputs.secular_batch(3, 20000, 30000, seed=22)]        # large problems: split mode
    for b in batches:
        total = int(b.offsets[-1])
        assert total <= 262144
        dev = torch.device("cuda")
        ref = sdc.secular_batched(torch.from_numpy(b.offsets).to(dev), torch.from_numpy(b.d).to(dev),
                                  torch.from_numpy(b.z).to(dev), 1.0, opts)
        ref = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
        for call in range(2):
            out = sdc.alloc_rank1_out(b.nprob, total, dev)
            code, *_ = _call_noalloc(b, opts, out)
            assert code == 0, L.STATUS.get(code)
            got = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
            assert got["status"][0] == 0
            for k in ("mk", "ngiv", "src", "perm", "org"):
                assert np.array_equal(got[k][:len(ref[k])], ref[k]), (call, k)
            for k in ("lam", "eta", "vhat", "bnorm", "dk"):
                r, g = ref[k], got[k]
                assert np.all(np.abs(g - r) <= 1e-10 * np.abs(r) + 1e-300), (call, k, np.abs(g - r).max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    b = inputs.secular_batch(2, 140000, 140000, seed=23)      # 280000 entries > 262144
    out = sdc.alloc_rank1_out(b.nprob, int(b.offsets[-1]), torch.device("cuda"))
    code, *_ = _call_noalloc(b, sdc.default_opts(tau=1e-12), out)
    assert code == 1     # SUPERDC_ERR_ARG
