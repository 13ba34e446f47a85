// Application of one batched rank-one factor Qhat = G^T [C (+) I] Pi^T
// (Cauchy-like block C_ij = vhat_i b_j / ((d_i - d_{K_j}) - eta_j), eqs. (4.26)
// and (4.28); rotations G of the deflation; sort Pi of the new eigenvalues) to
// a block of columns.  Used inside the conquering stage (Algorithm 3: the
// transpose applied to the remaining columns) and by superdc_apply_Q
// (Algorithm 4).
#pragma once
#include "common.cuh"

struct FactorView {
    int64_t nprob;
    const int64_t *off;                 // device, nprob+1 (problem row ranges)
    const int32_t *mk, *ngiv;           // device, nprob
    const double *dk, *eta, *dorg, *vhat, *bnorm;   // device, per slot
    const int32_t *src, *perm, *pinv, *giv_ab;      // device
    const double *giv_cs;
    int32_t fmm_min_m = 0;   // kept size from which a problem takes the FMM path (0: direct only)
    int64_t max_m = -1;      // upper bound on the problem sizes (-1: unknown)
#ifdef SUPERDC_CHECK
    int32_t *status = nullptr;   // device status word of the index guards (checked build)
#endif
};

struct FmmPlan;

// Y = Qhat^T X.  X (rows in the step's input order) is overwritten by the
// rotations; Y rows in merged order.  Column-major with leading dims ldx/ldy;
// row r of problem p lives at off[p] + r.  ncols columns.  plan (may be NULL):
// the FMM plan the rank-one step of this factor kept (R1Args::keep), used
// instead of a new one when its boxes and widths fit.
superdc_status cauchy_apply_T(const FactorView &f, int64_t total, double *X, int64_t ldx,
                              double *Y, int64_t ldy, int ncols, cudaStream_t st, const FmmPlan *plan = nullptr);

// Y = Qhat X.  X rows in merged order (read only); Y rows in input order.
superdc_status cauchy_apply_N(const FactorView &f, int64_t total, const double *X, int64_t ldx,
                              double *Y, int64_t ldy, int ncols, cudaStream_t st);

// Adjoint of one batched rank-one step (backward.cu): d_bar, z_bar (input
// order), X_bar = Qhat Ybar, from lam_bar (merged order, may be NULL) and the
// cotangent Ybar of Qhat^T X.
superdc_status r1_backward_fv(const FactorView &f, int64_t total, const double *lam_bar, int ncols,
                              const double *X, int64_t ldx, const double *Ybar, int64_t ldy, double *d_bar,
                              double *z_bar, double *X_bar, int64_t ldxb, double sqrt_rho, cudaStream_t st);
