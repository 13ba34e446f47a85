// Internal layout of the library handles (shared by the forward and the adjoint).
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "cauchy.cuh"
#include "rank1.cuh"

struct superdc_hss {
    int64_t n = 0;
    int nnodes = 0, r = 0, lmax = 0, nleaves = 0, mmax = 0;
    std::vector<int> lch, rch, level;
    std::vector<int64_t> size, off;
    std::vector<std::vector<int>> lev_nodes;       // nodes of each level, left to right
    std::vector<int> leaves;                       // left to right
    // device
    double *D = nullptr, *U = nullptr, *R = nullptr, *B = nullptr;
    int32_t *d_lch = nullptr, *d_rch = nullptr;
    int64_t *d_size = nullptr;
    int64_t *d_leaf_off = nullptr, *d_leaf_m = nullptr, *d_leaf_doff = nullptr, *d_leaf_uoff = nullptr;
    int32_t *d_leaf_id = nullptr;
    std::vector<int64_t *> d_lev_off;              // per level: node row offsets (nodes+1)
    std::vector<int32_t *> d_lev_nodes;            // per level: node ids
};

struct StepF {   // stored factor of one rank-one step of one level
    double *dk, *eta, *dorg, *vhat, *bnorm, *giv_cs;
    double *din, *zin;   // the step's input poles d and column z (before deflation)
    int32_t *src, *pinv, *giv_ab, *mk, *ngiv, *sweeps;
    int32_t *fmm;   // per node: 1 if the step took the FMM path
};

// Forward intermediates kept for superdc_eig_backward (opts.tape = 1).
struct Tape {
    bool on = false;
    std::vector<double *> lam_prev;             // [level] children's eigenvalues (n), input of the level build
    std::vector<double *> Wprev;                // [level] children's W = Q_c^T U_c (n x r)
    std::vector<std::vector<double *>> WKb;     // [level][step] columns step..ctot-1 before the step (n x (ctot-step))
    double *H = nullptr, *Bt = nullptr, *Bts = nullptr, *beta = nullptr, *sqb = nullptr, *u1 = nullptr, *v1 = nullptr;
};

// Work buffers of superdc_eig_run, allocated by superdc_eig_plan.
struct EigWork {
    double *H = nullptr, *Bts = nullptr, *sqb = nullptr, *lamA = nullptr, *lamB = nullptr, *Wp = nullptr;
    double *WK = nullptr, *WK2 = nullptr, *zk = nullptr, *wsum = nullptr, *dq = nullptr, *eq = nullptr;
    double *bnrm = nullptr;                // per node: ||Bt||_2 of its left child (dividing stage)
    double *rho_d = nullptr;               // max over leaves of ||Dhat_k||_2
    int32_t *org = nullptr, *perm = nullptr, *nsw = nullptr;
    double2 *rot = nullptr;
    int2 *hdr = nullptr;
    bool leaf_batched = false;
    size_t smem1 = 0, smem2 = 0, smem3 = 0, smem4 = 0, smem5 = 0;
    int ql_lpw = 32;                       // leaves per warp of the batched QL chase
    int64_t cap = 0, caps = 0;
    // leaves of 128 rows: divide and conquer on the tridiagonal form
    // (blocks of 32 by implicit QL, two levels of batched rank-one merges)
    bool leaf_dc = false;
    int64_t *dc_boff = nullptr, *dc_bm = nullptr, *dc_bq = nullptr;   // per 32-row block
    int64_t *dc_off[2] = {nullptr, nullptr};  // merge levels (64, 128 rows): problem offsets
    double *dc_scale = nullptr;            // per leaf: power of two >= ||T||_inf
    double *dc_beta = nullptr;             // per row: the coupling torn at that row (block starts)
    double *dc_QB = nullptr;               // 32 x 32 block eigenvectors (row-major)
    double *dc_Ya = nullptr, *dc_Yb = nullptr, *dc_X = nullptr;   // n x 128, column-major
    double *dc_Qh = nullptr;               // Householder factors of the leaves (row-major)
    double *dc_lam = nullptr, *dc_din = nullptr, *dc_zin = nullptr;
    R1Out dc_o{};                          // outputs of the merge steps
};

struct superdc_eigfact {
    const superdc_hss *h = nullptr;
    Tape tape;
    int64_t n = 0;
    int r = 0, lmax = 0;
    std::vector<char *> slabs;             // device allocations owned by the handle
    double *Qleaf = nullptr;               // concatenated leaf eigenvector blocks (column-major)
    int64_t *d_qoff = nullptr;             // offset of each leaf's block
    std::vector<int32_t *> P;              // per non-leaf level: merge order (node-local old position)
    std::vector<std::vector<StepF>> F;     // [level][step]
    int32_t *status = nullptr;             // device status word
    int fmm_min_m = 0;                     // resolved FMM threshold of the factorisation (0: direct)
    cudaStream_t last_stream = nullptr;
    superdc_opts opts{};                   // options of the plan
    EigWork work;                          // buffers of the run
    bool ran = false;                      // superdc_eig_run has been enqueued at least once
};


// the stored factor of rank-one step j of level l, as a batched view
FactorView factor_view(const superdc_eigfact *f, int l, int j);
// dense leaf blocks: Y = Q_leaf^T X (trans) or Q_leaf X, all leaves
superdc_status leaves_apply(const superdc_eigfact *f, int trans, int ncols, const double *X, int64_t ldx, double *Y,
                            int64_t ldy, cudaStream_t st);

// Leaves above 128 rows refined into exact rank-r subtrees (compress.cu); new
// device arrays returned in D2.. (cudaFree by the caller).
superdc_status refine_leaves(const superdc_tree *tree, const double *D, const double *U, const double *R,
                             const double *B, cudaStream_t st, std::vector<int32_t> &lch2,
                             std::vector<int32_t> &rch2, std::vector<int64_t> &lsize2, double **D2, double **U2,
                             double **R2, double **B2);
