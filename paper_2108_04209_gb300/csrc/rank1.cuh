// Internal interface of the batched rank-one step (see rank1.cu).
#pragma once
#include "common.cuh"

// Device output arrays of one batched rank-one step (layout as documented
// for superdc_rank1_out in superdc.h), plus library scratch.
struct R1Out {
    double *lam, *dk, *zk, *eta, *vhat, *bnorm;
    int32_t *org, *src, *perm, *giv_ab;
    double *giv_cs;
    int32_t *mk, *ngiv, *sweeps, *status;
    double *dorg;   // d_{K} of every kept root (scratch or stored), total entries
    int32_t *pinv;  // merged position of every slot (inverse of perm), total entries
    double *wsum;   // sum of kept z^2 per problem (scratch), nprob entries
    double *lamk;   // d_K + eta of every kept root, slot order (scratch), total entries
    int32_t *fmm_used = nullptr;   // per problem: 1 if it took the FMM path (may be NULL)
    int32_t unshifted = 0;         // ablation: roots as plain positions (origin 0, no local shifting)
};

struct FmmPlan;

struct R1Args {
    int64_t nprob, total;   // problems; extent of the row-indexed arrays (rows are absolute)
    int64_t rows = -1;      // rows covered by the problems (scheduling), -1 = total
    const int64_t *off;     // device, nprob+1
    const double *d, *z;    // device inputs
    double sqrt_rho, tau, stop_c;
    int max_iter, tile_roots;
    int sched = 0;          // 0 automatic, 1 whole problems per CTA (root pools per warp), 2 pole split
    int fmm_min_m = 0;      // kept size from which a problem takes the FMM path (0: direct only)
    int64_t max_m = -1;     // upper bound on the problem sizes (-1: unknown)
    // keep (may be NULL): receives the step's FMM plan instead of freeing it,
    // with workspaces keep_width columns wide, for a Cauchy-like application
    // of the same factor (cauchy_apply_T with that plan); the caller frees it
    FmmPlan *keep = nullptr;
    int keep_width = 0;
    R1Out o;
};

superdc_status r1_run(const R1Args &a, cudaStream_t st);

// One-time per-device set-up of the batched step's kernels (attributes);
// r1_run does it on first use, callers that capture work into a graph call it
// before the capture.
cudaError_t r1_prepare();
