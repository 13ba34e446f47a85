"""The level-batched eigendecomposition as one CUDA graph: superdc_eig_plan
allocates every buffer, superdc_eig_run only enqueues device work (kernels,
device copies, stream-ordered scratch), so the whole launch sequence of all
tree levels is captured once and replayed.  Replays must reproduce the
uncaptured factorisation bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2108_04209_gb300 as sdc  # noqa: E402
from paper_2108_04209_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.mark.parametrize("n,leaf,rank,clustered", [(2048, 64, 5, True), (16384, 128, 6, False)])
def test_eig_run_replayed_from_a_cuda_graph(n, leaf, rank, clustered):
    h = inputs.hss_random(n, leaf, rank, seed=31, clustered=clustered)
    H = sdc.HSSMatrix(h)
    lam_ref, Fref = H.eig()
    F = H.eig_plan()
    lam = torch.empty(n, dtype=torch.float64, device=DEV)
    F.run(lam)                       # first run outside the capture
    torch.cuda.synchronize()
    F.sync_status()
    assert torch.equal(lam, lam_ref)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.run(lam)
    X = torch.from_numpy(inputs.normal_block(n, 3, seed=2)).to(DEV)
    y_ref = Fref.apply_Q(X, trans=True)
    for _ in range(2):
        lam.zero_()
        g.replay()
        torch.cuda.synchronize()
        F.sync_status()
        assert torch.equal(lam, lam_ref)
        assert torch.equal(F.apply_Q(X, trans=True), y_ref)
    st = F.stats()
    assert st["sweeps"] > 0
