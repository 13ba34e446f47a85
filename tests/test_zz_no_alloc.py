"""The allocation-free entry point superdc_secular_batched_noalloc, for
callers that cannot allocate device memory while they run (device memory
reserved up front by another framework, latency-bound paths on which an
allocation may block, plug-ins with a fixed memory footprint).  Called twice
in a row through the C ABI; each call must match superdc_secular_batched on
the same inputs, and the results are checked against the oracle as well.
Kept in a file that is collected last."""
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


@pytest.mark.parametrize("case", ["whole_problems", "pole_split"])
def test_noalloc_matches_allocating_entry_point_twice(case):
    """Two calls in a row against the allocating entry point (direct evaluator:
    fmm_min_m < 0 there, as the allocation-free path has no FMM) and against
    the oracle.  sched = 1 runs the whole-problem units, which the automatic
    choice does not pick below the size limit; sched = 2 the pole split."""
    from tests import parity as P
    if case == "whole_problems":
        b, sched = inputs.secular_batch(96, 32, 2048, seed=21), 1
    else:
        b, sched = inputs.secular_batch(3, 20000, 30000, seed=22), 2
    opts = sdc.default_opts(tau=1e-12, sched=sched)
    total = int(b.offsets[-1])
    assert total <= 262144
    dev = torch.device("cuda")
    ref = sdc.secular_batched(torch.from_numpy(b.offsets).to(dev), torch.from_numpy(b.d).to(dev),
                              torch.from_numpy(b.z).to(dev), 1.0, sdc.default_opts(tau=1e-12, sched=sched,
                                                                                   fmm_min_m=-1))
    ref = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
    for call in range(2):
        out = sdc.alloc_rank1_out(b.nprob, total, dev)
        out["fmm"].fill_(7)
        code, *_ = _call_noalloc(b, opts, out)
        assert code == 0, L.STATUS.get(code)
        got = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
        assert got["status"][0] == 0
        assert np.all(got["fmm"][:b.nprob] == 0)
        for k in ("mk", "ngiv", "src", "perm", "org"):
            assert np.array_equal(got[k][:len(ref[k])], ref[k]), (call, k)
        for k in ("lam", "eta", "vhat", "bnorm", "dk"):
            r, g = ref[k], got[k]
            assert np.all(np.abs(g - r) <= 1e-10 * np.abs(r) + 1e-300), (call, k, np.abs(g - r).max())
    # the same results against the oracle, problem by problem
    for p in range(b.nprob):
        d, z = b.problem(p)
        P.compare_problem(P.gpu_problem(got, b.offsets, p), d, z, 1e-12, mode=1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    b = inputs.secular_batch(2, 140000, 140000, seed=23)      # 280000 entries > 262144
    out = sdc.alloc_rank1_out(b.nprob, int(b.offsets[-1]), torch.device("cuda"))
    code, *_ = _call_noalloc(b, sdc.default_opts(tau=1e-12), out)
    assert code == 1     # SUPERDC_ERR_ARG
