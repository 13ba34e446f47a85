"""Failure paths of the C ABI, reached by host-side injection only: non-finite
inputs (the kernels' own checks latch SUPERDC_DEV_NONFINITE), an iteration
cap that cannot be met (SUPERDC_DEV_NOCONV), sizes beyond what a call accepts
(SUPERDC_ERR_ARG, nothing enqueued) and device allocations refused through the
library's allocation-limit test hook (SUPERDC_ERR_OOM).  No case faults, traps
or hangs the GPU; after every failure the library stays usable."""
import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import _lib as L, inputs  # noqa: E402
from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu

ERR_ARG, ERR_OOM, ERR_NONFINITE, ERR_NOCONV = 1, 3, 4, 5


def _batch(seed=0, sizes=(100, 700, 60)):
    rng = np.random.default_rng(seed)
    ds = [np.sort(rng.uniform(0, 1, m)) for m in sizes]
    zs = [rng.standard_normal(m) for m in sizes]
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    return inputs.SecularBatch(offs, np.concatenate(ds), np.concatenate(zs), 1.0)


def _dev(b):
    dev = torch.device("cuda")
    return (torch.from_numpy(b.offsets).to(dev), torch.from_numpy(b.d).to(dev), torch.from_numpy(b.z).to(dev))


@pytest.fixture
def no_alloc_limit():
    yield
    L.lib().superdc_debug_alloc_limit(0)


@pytest.mark.parametrize("where", ["z_direct", "z_fmm", "d_direct"])
def test_nonfinite_input_batched(where):
    """A NaN in z of a direct-path problem or of an FMM-path problem (700 kept
    poles), or in d of a direct-path problem: the status word carries
    NONFINITE and the call raises it; the untouched problem is still right."""
    b = _batch()
    if where == "z_direct":
        b.z[10] = np.nan
    elif where == "z_fmm":
        b.z[100 + 333] = np.nan
    else:
        b.d[50] = np.nan
    offs, d, z = _dev(b)
    with pytest.raises(sdc.SuperDCError) as ei:
        sdc.secular_batched(offs, d, z, 1.0, sdc.default_opts(tau=1e-12))
    assert ei.value.code == ERR_NONFINITE
    # check=False: the outputs of the clean problem (the last) are intact
    out = sdc.secular_batched(offs, d, z, 1.0, sdc.default_opts(tau=1e-12), check=False)
    assert int(out["status"].item()) & L.DEV_NONFINITE
    host = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    dd, zz = b.problem(2)
    P.compare_problem(P.gpu_problem(host, b.offsets, 2), dd, zz, 1e-12, mode=1)


def test_nonfinite_input_host_entry_point():
    b = _batch()
    b.z[5] = np.inf
    with pytest.raises(sdc.SuperDCError) as ei:
        sdc.secular_batched_host(torch.from_numpy(b.offsets), torch.from_numpy(b.d), torch.from_numpy(b.z), 1.0,
                                 sdc.default_opts(tau=1e-12))
    assert ei.value.code == ERR_NONFINITE


def test_nonfinite_leaf_block_eig():
    """A NaN on the diagonal of one leaf block of an HSS matrix (the blocks
    are read as symmetric, one triangle): superdc_eig returns
    SUPERDC_ERR_NONFINITE (direct evaluator, as the FMM needs finite poles to
    build its boxes meaningfully)."""
    h = inputs.cfg_small_hss()
    m = int(h.tree.leaf_size[h.tree.leaves[0]])
    h.D[int(h.d_off[h.tree.leaves[0]]) + 5 * m + 5] = np.nan
    H = sdc.HSSMatrix(h)
    with pytest.raises(sdc.SuperDCError) as ei:
        H.eig(sdc.default_opts(fmm_min_m=-1))
    assert ei.value.code == ERR_NONFINITE


def test_nonfinite_leaf_block_divide_and_conquer_leaves():
    """The same with leaves of 128 rows (the leaf divide-and-conquer path): a
    NaN on a diagonal entry bounds every loop (QL chases hit their iteration
    cap, the merge steps' deflation latches NONFINITE) and the call returns
    SUPERDC_ERR_NONFINITE; the library is still usable afterwards."""
    h = inputs.hss_random(512, 128, 4, seed=2)
    m = int(h.tree.leaf_size[h.tree.leaves[1]])
    h.D[int(h.d_off[h.tree.leaves[1]]) + 40 * m + 40] = np.nan
    H = sdc.HSSMatrix(h)
    with pytest.raises(sdc.SuperDCError) as ei:
        H.eig(sdc.default_opts(fmm_min_m=-1))
    assert ei.value.code == ERR_NONFINITE
    lam, F = sdc.HSSMatrix(inputs.hss_random(512, 128, 4, seed=2)).eig()
    assert torch.isfinite(lam).all()


def test_zero_matrix_divide_and_conquer_leaves():
    """All generators zero (leaves of 128): every coupling is zero, every
    rank-one update deflates; eigenvalues 0 and Q orthogonal."""
    h = inputs.hss_random(256, 128, 3, seed=1)
    h.D[:] = 0.0
    h.U[:] = 0.0
    h.B[:] = 0.0
    lam, F = sdc.HSSMatrix(h).eig()
    assert float(lam.abs().max()) == 0.0
    Q = F.apply_Q(torch.eye(256, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.abs(Q.T @ Q - np.eye(256)).max() <= 1e-14


def test_iteration_cap_reports_noconv_promptly():
    """max_iter = 1: roots stop after one step past the midpoint sweep; the
    status carries NOCONV and the call takes no longer than a normal one."""
    b = inputs.cfg_secular_4096()
    offs, d, z = _dev(b)
    ok = sdc.default_opts(tau=1e-12)
    sdc.secular_batched(offs, d, z, 1.0, ok)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sdc.secular_batched(offs, d, z, 1.0, ok)
    t_ok = time.perf_counter() - t0
    t0 = time.perf_counter()
    with pytest.raises(sdc.SuperDCError) as ei:
        sdc.secular_batched(offs, d, z, 1.0, sdc.default_opts(tau=1e-12, max_iter=1))
    t_cap = time.perf_counter() - t0
    assert ei.value.code == ERR_NOCONV
    assert t_cap <= 2.0 * t_ok + 0.05, (t_cap, t_ok)
    H = sdc.HSSMatrix(inputs.cfg_small_hss())
    with pytest.raises(sdc.SuperDCError) as ei:
        H.eig(sdc.default_opts(max_iter=1))
    assert ei.value.code == ERR_NOCONV
    lam, F = H.eig()                       # the library is still usable
    assert F is not None and torch.isfinite(lam).all()


def test_argument_errors_enqueue_nothing():
    lib = L.lib()
    b = _batch()
    offs, d, z = _dev(b)
    out = sdc.alloc_rank1_out(b.nprob, int(b.offsets[-1]), torch.device("cuda"))
    ro = L.Rank1Out(**{k: (v.data_ptr() if v is not None else None) for k, v in out.items()})
    st = torch.cuda.current_stream().cuda_stream
    fn = lib.superdc_secular_batched
    good = sdc.default_opts(tau=1e-12)
    # a total beyond the int32 row indices the kernels use
    assert fn(b.nprob, offs.data_ptr(), 2 ** 31, d.data_ptr(), z.data_ptr(), 1.0, ctypes.byref(good),
              ctypes.byref(ro), st) == ERR_ARG
    for bad in (dict(tau=-1.0), dict(max_iter=0), dict(sched=3), dict(stop_c=0.0)):
        o = sdc.default_opts(**dict(dict(tau=1e-12), **bad))
        assert fn(b.nprob, offs.data_ptr(), int(b.offsets[-1]), d.data_ptr(), z.data_ptr(), 1.0, ctypes.byref(o),
                  ctypes.byref(ro), st) == ERR_ARG, bad
    assert fn(b.nprob, offs.data_ptr(), int(b.offsets[-1]), d.data_ptr(), z.data_ptr(), -1.0, ctypes.byref(good),
              ctypes.byref(ro), st) == ERR_ARG
    assert lib.superdc_debug_alloc_limit(-5) == ERR_ARG


def test_refused_allocations_return_oom_and_recover(no_alloc_limit):
    """Every device allocation above 64 KiB refused: the batched step,
    superdc_eig and superdc_apply_Q return SUPERDC_ERR_OOM (and free what they
    took); without the limit the same calls succeed and agree with a run that
    never saw the limit."""
    lib = L.lib()
    b = inputs.secular_batch(64, 32, 2048, seed=9)
    offs, d, z = _dev(b)
    opts = sdc.default_opts(tau=1e-12)
    ref = sdc.secular_batched(offs, d, z, 1.0, opts)["lam"].clone()
    h = inputs.hss_random(2048, 64, 4, seed=5)
    H = sdc.HSSMatrix(h)
    lam_ref, F = H.eig()
    X = torch.from_numpy(inputs.normal_block(2048, 8, seed=1)).cuda()
    y_ref = F.apply_Q(X, trans=True).clone()
    torch.cuda.synchronize()
    assert lib.superdc_debug_alloc_limit(64 * 1024) == 0
    for call in (lambda: sdc.secular_batched(offs, d, z, 1.0, opts),
                 lambda: H.eig(),
                 lambda: F.apply_Q(X, trans=True)):
        with pytest.raises(sdc.SuperDCError) as ei:
            call()
        assert ei.value.code == ERR_OOM
    torch.cuda.synchronize()
    assert lib.superdc_debug_alloc_limit(0) == 0
    assert torch.equal(sdc.secular_batched(offs, d, z, 1.0, opts)["lam"], ref)
    lam2, F2 = H.eig()
    assert torch.equal(lam2, lam_ref)
    assert torch.equal(F2.apply_Q(X, trans=True), y_ref)
