"""Run one named workload through the public API (for profilers such as ncu).

    python -m paper_2108_04209_gb300.profile_case secular <nprob> [fmm_min_m] [sched]
        two batched secular calls on the 4096-problem distribution
        (m ~ U{32..2048}, seed 1) restricted to <nprob> problems, with the
        FMM threshold fmm_min_m (default: the library's) and the secular
        schedule sched (0 automatic, 1 whole problems, 2 pole split);
    python -m paper_2108_04209_gb300.profile_case eig <n> <leaf> <rank>
        superdc_eig twice on a random HSS matrix (seed 4);
    python -m paper_2108_04209_gb300.profile_case applyq <n> <leaf> <rank> <ncols>
        superdc_eig once, then Q^T times an n x ncols N(0,1) block twice;
    python -m paper_2108_04209_gb300.profile_case clustered
        superdc_eig once on the clustered n=16384 matrix (leaf 64, rank 8, seed 2);
    python -m paper_2108_04209_gb300.profile_case secular_m <m> <nprob>
        two batched secular calls on <nprob> problems of size m (seed 5).
"""
import sys

import torch

import paper_2108_04209_gb300 as sdc
from paper_2108_04209_gb300 import inputs


def main(argv):
    what = argv[1]
    dev = torch.device("cuda")
    if what == "secular":
        n = int(argv[2]) if len(argv) > 2 else 4096
        fm = int(argv[3]) if len(argv) > 3 else 0
        sc = int(argv[4]) if len(argv) > 4 else 0
        b = inputs.secular_batch(n, 32, 2048, seed=1)
        o, d, z = (torch.from_numpy(x).to(dev) for x in (b.offsets, b.d, b.z))
        for _ in range(2):
            sdc.secular_batched(o, d, z, 1.0, sdc.default_opts(tau=1e-12, fmm_min_m=fm, sched=sc))
        torch.cuda.synchronize()
        print("ok", int(b.offsets[-1]))
    elif what in ("eig", "applyq"):
        n, leaf, r = int(argv[2]), int(argv[3]), int(argv[4])
        H = sdc.HSSMatrix(inputs.hss_random(n, leaf, r, seed=4))
        lam, F = H.eig(sdc.default_opts(tau=1e-10))
        if what == "eig":
            lam, F = H.eig(sdc.default_opts(tau=1e-10))
        else:
            X = torch.from_numpy(inputs.normal_block(n, int(argv[5]), seed=104)).to(dev)
            for _ in range(2):
                F.apply_Q(X, trans=True)
        torch.cuda.synchronize()
        print("ok", n)
    elif what == "secular_m":
        m, nprob = int(argv[2]), int(argv[3])
        b = inputs.secular_batch(nprob, m, m, seed=5)
        o, d, z = (torch.from_numpy(x).to(dev) for x in (b.offsets, b.d, b.z))
        for _ in range(2):
            sdc.secular_batched(o, d, z, 1.0, sdc.default_opts(tau=1e-12))
        torch.cuda.synchronize()
        print("ok", int(b.offsets[-1]))
    elif what == "clustered":
        H = sdc.HSSMatrix(inputs.cfg_clustered_16384())
        lam, F = H.eig(sdc.default_opts(tau=1e-10))
        torch.cuda.synchronize()
        print("ok", 16384)
    else:
        raise SystemExit(__doc__)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
