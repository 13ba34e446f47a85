// Triangular FMM with local shifting for the large problems of a batched
// rank-one step (Sections 4.1.2, 4.2.2 and 4.3): the secular sweeps (the lower
// and upper triangular sums psi, phi and their derivatives, eq. (4.10)), the
// Loewner zhat in logarithmic form (eq. (4.25)), the normalisation b
// (eq. (4.27)) and the Cauchy-like applications of eq. (4.29).
//
// Problems whose kept size is at least min_m take this path; the direct
// evaluators skip them (each direct kernel reads the plan's fslot array).
#pragma once
#include <vector>
#include "common.cuh"
#include "rank1.cuh"
#include "cauchy.cuh"

constexpr int FMM_P = 22;      // Chebyshev nodes (expansion order) per box
constexpr int FMM_NPOOL = 24;  // near-list pool entries per box (average; lists have any length)

// State of a secular root handed from the per-box sweep kernel to the tail
// pass (the box's last few unconverged roots).
struct FmmTail {
    int64_t p;                             // problem
    int32_t k, K, phase, nsw;              // root index, origin, iteration state
    double dK, y, lo, hi;
};

// Device view of a plan: which problems of the batch use the FMM and their
// box trees (index-based binary tree over the kept poles, near lists from the
// geometric admissibility test).
struct FmmDev {
    int64_t nprob;
    const int64_t *box_base, *leaf_base;   // nprob+1: boxes / leaf boxes per problem (prefix)
    int32_t *fslot;                        // nprob: >= 0 FMM problem, -1 direct
    const int32_t *fprob, *nfmm;           // FMM problem -> batch problem; count
    const double *blo, *bhi;               // per box: interval [lo, hi] of its points
    const int32_t *nnear, *near;           // per box: near-list length (< 0: every source direct); list pool
    const int64_t *nstart;                 // per box: start of its near list in the pool
    double *W, *coef;                      // workspace: node weights, leaf coefficients
    double *F;                             // workspace: far field at every box's nodes
    double *lastp;                         // workspace: per leaf box (ncol wide), its sources' share of
                                           // the sums for the last eigenvalue (outside the tree)
    FmmTail *tail;                         // roots left to the tail pass (capacity: every kept root)
    unsigned int *ntail;                   // their count, then the tail pass's next unclaimed entry
    double *kmat;                          // per box, its first kslots interaction pairs: the P x P
    int kslots;                            // matrix 1/(s_q2 - t_q) of nodes (M2L kernel, shared by
                                           // the far fields built on one plan)
    const int64_t *lev_off;                // per level: prefix of the FMM problems' box counts
    const int64_t *top_off;                // the same per level counted from each problem's top box
    int32_t *upcnt;                        // per box: children whose moments are done in the current
                                           // upward pass (the last one computes the box; reset by it)
    unsigned long long *upq;               // upward pass: next unclaimed leaf box, CTAs past the end
    int64_t *split;                        // leaf boxes with long near lists (any order) and their
    int32_t *nsplit;                       // count, filled by the tree build
    int64_t cap_f;                         // capacity of the FMM problem list
    int ncol, nfield;                      // workspace widths
    unsigned long long *flops;             // algorithmic FP64 work of the far fields and of the
                                           // zhat / b / Cauchy-like consumers (profiling only; NULL
                                           // otherwise): FMA 2, other operations 1
};

struct FmmPlan {
    FmmDev dv{};
    int64_t cap_boxes = 0, cap_leaves = 0, cap_f = 0;
    int lmax = 0;                          // upper bound on tree levels
    int nb0max = 0;                        // upper bound on leaf boxes per problem
    int box = 0;                           // indices per leaf box (32 or 64) of this plan
    bool on = false;                       // some problem may take the FMM path
    std::vector<void *> bufs;
};

// Decide per problem (kept size mk >= min_m) and build the box trees from the
// kept poles dk.  max_m: an upper bound on the problem sizes (-1 unknown).
// ncol / nfield: widths of the moment and coefficient workspaces.
// used (may be NULL): per problem 1 if it takes the FMM path, else 0.
// box: indices per leaf box, 32 or 64 (smaller boxes halve the near field,
// larger ones halve the number of box pairs whose expansions are translated).
// kslots: M2L kernel matrices kept per box for the later far fields of the
// same plan (0: none).
superdc_status fmm_plan(FmmPlan &pl, int64_t nprob, const int64_t *off, int64_t total, int64_t max_m,
                        const int32_t *mk, const double *dk, int min_m, int ncol, int nfield, int32_t *used,
                        int box, int kslots, cudaStream_t st);
void fmm_free(FmmPlan &pl, cudaStream_t st);

// Roots of the FMM problems (same outputs as the direct secular kernel).
superdc_status fmm_secular(const FmmPlan &pl, const int64_t *off, const R1Out &o, double stop_c, int max_iter,
                           cudaStream_t st);
// zhat (eq. (4.23) via eq. (4.25)) and b (eq. (4.27)) of the FMM problems.
superdc_status fmm_lowner(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st);
superdc_status fmm_bnorm(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st);
// Columns [col0, col0 + nc) of Y = Qhat^T X (trans) or Y = Qhat X for the FMM
// problems (layouts as cauchy_apply_T / cauchy_apply_N; X already rotated for trans).
superdc_status fmm_cauchy(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y,
                          int64_t ldy, int col0, int nc, bool trans, cudaStream_t st);

// Library default of the FMM threshold (kept problem size), and the
// threshold an option value selects (> 0 itself, 0 the default, < 0 off).
int fmm_default_min_m();
inline int fmm_resolve(int32_t opt) { return opt > 0 ? opt : (opt == 0 ? fmm_default_min_m() : 0); }
