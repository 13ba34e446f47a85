/*
 * superdc.h -- C ABI of the GB300 (sm_103a) SuperDC conquering-stage library.
 *
 * Method: Ou & Xia, "SuperDC: superfast divide-and-conquer eigenvalue
 * decomposition with improved stability for rank-structured matrices"
 * (arXiv 2108.04209).  Symmetric HSS matrix A (Section 2, eq. (2.1)) ->
 * A = Q Lambda Q^T with Q kept in structured form (Lemma 4.1, eq. (4.34)).
 *
 * Conventions for every entry point
 *   - numeric data are FP64; matrices are column-major;
 *   - pointers are DEVICE pointers unless the comment says HOST;
 *   - work is enqueued on the given CUDA stream and is stream-ordered; the
 *     caller keeps inputs alive and outputs allocated until the stream has
 *     reached the work (e.g. cudaStreamSynchronize);
 *   - argument errors are returned synchronously and enqueue nothing;
 *   - errors found by the GPU (non-finite values, a root that misses the
 *     stopping test within max_iter, an index guard) are latched in a device
 *     status word and reported by superdc_sync_status / the status output;
 *     the library never traps, asserts or aborts, and every device loop is
 *     bounded;
 *   - no C++ exception crosses this interface.
 */
#ifndef SUPERDC_H
#define SUPERDC_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SUPERDC_OK = 0,
    SUPERDC_ERR_ARG = 1,        /* invalid argument (sizes, null pointers, options) */
    SUPERDC_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    SUPERDC_ERR_OOM = 3,        /* device allocation failed */
    SUPERDC_ERR_NONFINITE = 4,  /* NaN/Inf met in the inputs or intermediate values */
    SUPERDC_ERR_NOCONV = 5,     /* a secular root missed the stopping test eq. (4.12) in max_iter sweeps */
    SUPERDC_ERR_STATE = 6       /* handle used in the wrong state */
} superdc_status;

/* Device status word bits (written by kernels, OR-ed). */
#define SUPERDC_DEV_NONFINITE 1
#define SUPERDC_DEV_NOCONV    2
#define SUPERDC_DEV_INDEX     4   /* checked build only (-DSUPERDC_CHECK, libsuperdc_check.so): an index
                                   read from device data (a near-list box, a kept count) was out of
                                   range; the access used 0 instead; reported as SUPERDC_ERR_CUDA */

typedef struct {
    double  tau;          /* deflation tolerance of Remark 4.1 (absolute; strict '<' tests) */
    double  stop_c;       /* constant c of the stopping test eq. (4.12): |f| < c m (1+|psi|+|phi|) eps */
    int32_t max_iter;     /* iteration cap of the secular solver (the paper is silent; default 50) */
    int32_t tile_roots;   /* secular schedule: roots per work unit (32..4096, multiple of 32);
                             other values: chosen from the batch size */
    int32_t batching;     /* superdc_eig: 1 = a whole tree level per launch (default); 0 = one
                             launch sequence per node (the unbatched baseline) */
    int32_t sched;        /* secular schedule: 0 automatic, 1 whole problems per CTA with per-warp
                             root pools, 2 CTA warps split the poles of one 32-root group */
    int32_t tape;         /* superdc_eig: 1 = keep the forward intermediates that
                             superdc_eig_backward needs (O(r^2 n log n) doubles) */
    int32_t fmm_min_m;    /* rank-one problems whose kept size is at least this use the triangular
                             FMM with local shifting (Sections 4.1.2, 4.2.2, 4.3) for the secular
                             sweeps, zhat, b and the Cauchy-like applications; smaller ones the
                             direct tiled evaluator.  0 = the library default (the crossover
                             measured on GB300), < 0 = direct evaluator only */
    int32_t shifted;      /* 1 (default): every secular root is solved and stored relative to its
                             nearest pole (the local shifting of Section 4.2, eqs. (4.13)-(4.21));
                             0: ablation, the roots are solved and stored as plain positions, so
                             every difference d_j - lambda is formed from rounded values (the
                             unshifted variant Section 5 compares against) */
    int32_t balanced;     /* 1 (default): the balanced dividing of eqs. (3.11)/(3.12); 0: ablation,
                             the original dividing of eqs. (2.4)/(2.5) (no scaling by ||B||_2),
                             whose generator norms can grow exponentially (Proposition 3.1;
                             not with opts.tape = 1) */
} superdc_opts;

/* Fills *opts with the defaults: tau = 1e-10, stop_c = 8, max_iter = 50,
 * tile_roots = 0 (automatic), batching = 1, sched = 0, tape = 0, fmm_min_m = 0 (default crossover),
 * shifted = 1, balanced = 1. */
superdc_status superdc_opts_default(superdc_opts *opts);

/* Test hook (no counterpart in the paper): from now on every device
 * allocation the library makes that is larger than max_bytes fails as if the
 * device were out of memory, so the SUPERDC_ERR_OOM paths can be exercised
 * without exhausting a GPU; 0 removes the limit.  Process-wide; not meant
 * for production use.  Negative values: SUPERDC_ERR_ARG. */
superdc_status superdc_debug_alloc_limit(int64_t max_bytes);

/* Human-readable name of a status code (static string). */
const char *superdc_status_string(superdc_status s);

/* ------------------------------------------------------------------------
 * Batched independent rank-one problems  diag(d_p) + rho z_p z_p^T.
 *
 * One call performs, for every problem p, the rank-one step of Algorithm 3:
 * deflation (Remark 4.1), the shifted secular roots (Algorithm 2, shifted
 * equation eqs. (4.13)/(4.14), gap update eq. (4.17), the triangular
 * psi/phi split of eqs. (4.7)-(4.10), stopping test eq. (4.12)), Loewner's
 * zhat (eq. (4.23)), the normalisation b (eq. (4.27)), and the sorted new
 * eigenvalues.  The eigenvector matrix of
 * problem p is  Qhat = G^T [C (+) I] Pi^T  with G the recorded rotations,
 * C_ij = vhat_i b_j / ((d_i - d_{K_j}) - eta_j) on the kept set
 * (eqs. (4.26), (4.28)), identity on the deflated set, and Pi the sort.
 *
 * Inputs (device): offsets[nprob+1] (int64, offsets[0] = 0, ascending),
 * d[total] ascending inside every problem, z[total]; total = offsets[nprob]
 * (also passed by value, HOST-known).  rho > 0.
 *
 * Outputs: caller-allocated device arrays in superdc_rank1_out, each of
 * length `total` (problem p owns entries [offsets[p], offsets[p+1])) unless
 * noted.  Inside problem p with m entries and mk kept:
 *   slots 0..mk-1   = kept entries in ascending order, slots mk..m-1 =
 *   deflated entries sorted by (value, input index);
 *   dk[slot]     pole (after rotations) / deflated value;
 *   zk[slot]     z after rotations (0 for deflated slots);
 *   src[slot]    input index (0-based inside the problem) of the slot;
 *   org[slot]    origin K (kept slot index) of the root, -1 for deflated;
 *   eta[slot]    gap lambda - d_K (0 for deflated);
 *   vhat[slot], bnorm[slot]  Loewner zhat and b (0 / 1 for deflated);
 *   lam[pos]     new eigenvalues ascending, perm[pos] = slot it came from
 *                (ties broken by input index);
 *   giv_ab[2*(off+g)+{0,1}], giv_cs[2*(off+g)+{0,1}]: rotation g (scan
 *                order) between input indices a, b with cosine c, sine s:
 *                [x_a; x_b] <- [c x_a - s x_b; s x_a + c x_b];
 *   mk[p], ngiv[p] (int32, length nprob);
 *   sweeps[slot] (may be NULL) secular sweeps used per root;
 *   status (int32, length 1): SUPERDC_DEV_* bits, OR-ed (caller zeroes it);
 *   fmm[p] (may be NULL; int32, length nprob): 1 if problem p took the
 *                triangular FMM path (opts.fmm_min_m), else 0.
 * Scratch is taken from the stream-ordered allocator and released on the
 * same stream.
 * -------------------------------------------------------------------- */
typedef struct {
    double  *lam;
    double  *dk;
    double  *zk;
    double  *eta;
    double  *vhat;
    double  *bnorm;
    int32_t *org;
    int32_t *src;
    int32_t *perm;
    int32_t *giv_ab;
    double  *giv_cs;
    int32_t *mk;
    int32_t *ngiv;
    int32_t *sweeps;
    int32_t *status;
    int32_t *fmm;
} superdc_rank1_out;

superdc_status superdc_secular_batched(int64_t nprob, const int64_t *offsets, int64_t total,
                                       const double *d, const double *z, double rho,
                                       const superdc_opts *opts, superdc_rank1_out *out,
                                       cudaStream_t stream);

/* superdc_secular_batched with HOST buffers, for callers whose data live in
 * host memory: offsets[nprob+1], d[total], z[total] are HOST arrays (pinned
 * memory makes the copies asynchronous; pageable memory works too), every
 * non-NULL field of *out is a HOST array of the length given above, and
 * out->status (HOST, required) receives the device status word.  The call
 * copies the inputs to a stream-ordered device slab, runs the batched step,
 * copies the requested outputs back, releases the slab and synchronises the
 * stream; it returns SUPERDC_ERR_NONFINITE / SUPERDC_ERR_NOCONV when the
 * status word says so.  A batch of 2^20 entries or more (and at least 16
 * problems) runs as four chunks of problems on two library-owned streams
 * that wait for the work already queued on `stream`, so that one chunk's
 * copies overlap another chunk's kernels; every chunk uses the schedule of
 * the whole batch and absolute rows, so the results are bit-identical to one
 * superdc_secular_batched call over the batch.  Argument errors as
 * superdc_secular_batched, plus offsets[0] != 0, offsets[nprob] != total or
 * decreasing offsets.
 *
 * Device scratch of every entry point comes from a stream-ordered memory
 * pool of the library on each device, which keeps up to 16 GiB of freed
 * scratch across synchronisations (so a call after a synchronising one does
 * not map its scratch again); that memory stays reserved by the process. */
superdc_status superdc_secular_batched_host(int64_t nprob, const int64_t *offsets, int64_t total,
                                            const double *d, const double *z, double rho,
                                            const superdc_opts *opts, superdc_rank1_out *out,
                                            cudaStream_t stream);

/* Y = Qhat^T X (trans = 1) or Y = Qhat X (trans = 0) for every problem of a
 * superdc_secular_batched result `fwd` (the structured eigenvector matrices of
 * eq. (4.26) with the rotations and the sort), applied to caller columns:
 * X, Y total x ncols column-major (ld ldx, ldy >= total), problem p owning rows
 * [offsets[p], offsets[p+1]).  X is read only; X and Y must not overlap.
 * opts (may be NULL: defaults): only fmm_min_m is used (problems whose kept
 * size reaches it use the triangular FMM for the Cauchy-like sums). */
superdc_status superdc_rank1_apply(int64_t nprob, const int64_t *offsets, int64_t total,
                                   const superdc_rank1_out *fwd, int32_t trans, int64_t ncols,
                                   const double *X, int64_t ldx, double *Y, int64_t ldy,
                                   const superdc_opts *opts, cudaStream_t stream);

/* Adjoint of superdc_secular_batched (reverse mode through the secular roots
 * by the implicit-function theorem; the row-12 building block).
 * fwd: the forward outputs of the same call (unchanged since); rho, offsets,
 * total as in the forward.  Cotangents (DEVICE, may be NULL / ncols = 0):
 *   lam_bar[total] of the new eigenvalues (merged order, as fwd->lam);
 *   Ybar (total x ncols, column-major, ld ldy) of Y = Qhat^T X for the caller
 *   columns X (total x ncols, ld ldx, input order).
 * Outputs: d_bar[total], z_bar[total] (input order), X_bar = Qhat Ybar
 * (total x ncols, ld ldxb; written only when ncols > 0).
 * Kept block: eigen-adjoint of diag(d_k) + z_k z_k^T through the Cauchy-like
 * factor (eq. (4.26)), reading zhat and b from fwd (the structured factor
 * keeps them for its applications, so they are not formed again) with every
 * difference in shifted form (eq. (4.28)); deflation rotations are
 * treated as fixed linear maps (their dependence on z is of order tau). */
superdc_status superdc_secular_batched_backward(int64_t nprob, const int64_t *offsets, int64_t total,
                                                double rho, const superdc_rank1_out *fwd,
                                                const double *lam_bar, int64_t ncols, const double *X,
                                                int64_t ldx, const double *Ybar, int64_t ldy,
                                                double *d_bar, double *z_bar, double *X_bar, int64_t ldxb,
                                                cudaStream_t stream);

/* ------------------------------------------------------------------------
 * superdc_secular_batched_noalloc: the batched rank-one step of
 * superdc_secular_batched for callers that cannot allocate device memory
 * while they run: a host whose device memory was reserved up front by
 * another framework or pool it does not own, a latency-bound path on which
 * cudaMalloc may block or synchronise the device, or a plug-in that must not
 * change the process's memory footprint after it has been loaded.  The paper
 * has no counterpart; this is an interface variant only.  Same arguments and
 * output layout as superdc_secular_batched, but the call makes no device
 * allocation: its scratch is a static device array of about 11 MB that every
 * GPU which loads the library holds until the process exits.
 *   - evaluator: the direct tiled evaluator only (the triangular FMM needs
 *     scratch proportional to its tree); opts.fmm_min_m is ignored and
 *     out->fmm (if given) is set to 0.  opts.sched and opts.tile_roots select
 *     the schedule as in superdc_secular_batched; for a problem below the
 *     FMM threshold the results are those of superdc_secular_batched;
 *   - limits: nprob <= SDC_NOALLOC_MAX_PROB and total <= SDC_NOALLOC_MAX_TOTAL,
 *     else SUPERDC_ERR_ARG (nothing enqueued);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it, and
 *     sets a kernel attribute once per device; make that first call before
 *     any stream capture;
 *   - all calls on a device share the array and it keeps the last call's
 *     contents (each call writes every word it reads, so nothing needs
 *     clearing in between): calls whose work overlaps on the GPU (other
 *     streams, other host threads) race and must be serialised.
 * -------------------------------------------------------------------- */
#define SDC_NOALLOC_MAX_TOTAL 262144
#define SDC_NOALLOC_MAX_PROB 16384
superdc_status superdc_secular_batched_noalloc(int64_t nprob, const int64_t *offsets, int64_t total,
                                               const double *d, const double *z, double rho,
                                               const superdc_opts *opts, superdc_rank1_out *out,
                                               cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Symmetric HSS matrix (Section 2, eq. (2.1)) and its eigendecomposition.
 *
 * Tree (HOST arrays): a postordered full binary tree with nnodes nodes, the
 * root is node nnodes-1; lchild/rchild are -1 at leaves; every leaf lies at
 * the same depth (perfect tree); leaf_size[i] = rows of leaf i (ignored for
 * non-leaves), 1 <= leaf_size <= 128, or all leaves of one size M <= 4096
 * that is 2^k times a size of at most 128 (see below); rank = r, the common HSS rank
 * (1 <= r <= 32): every U_i is m_i x r, every R_i and B_i is r x r.
 *
 * Generators (DEVICE, FP64, column-major blocks, caller-owned, read only):
 *   D : leaf diagonal blocks m_i x m_i concatenated over the leaves in
 *       postorder (= left-to-right);
 *   U : leaf bases m_i x r concatenated the same way;
 *   R : nnodes blocks r x r (node i at R + i r^2); the entries of the root
 *       and of its two children are not used;
 *   B : nnodes blocks r x r; B_i of a left child i couples it with its
 *       sibling: A(i, j) = U_i B_i U_j^T (nested U_p = [U_i R_i; U_j R_j]).
 * superdc_build_hss copies them into a library-owned handle (stream-ordered);
 * the caller may free its arrays once the stream has passed the call.
 * Leaves of more than 128 rows (the paper's examples use 2048) are refined:
 * each leaf block becomes a subtree with leaves of M / 2^k <= 128 rows whose
 * top basis is the leaf's U, by the compression of superdc_build_hss_compress
 * applied to the block with U as exact extra columns.  The refinement must be
 * exact at rank r (relative projection residual <= 1e-12 at every node, as
 * for banded or tridiagonal leaf blocks, Section 5's Examples 1-2), else
 * SUPERDC_ERR_ARG; the handle then describes the refined tree (superdc_eig's
 * levels count the refined levels).
 * -------------------------------------------------------------------- */
typedef struct superdc_hss superdc_hss;
typedef struct superdc_eigfact superdc_eigfact;

typedef struct {
    int64_t n;
    int32_t nnodes;
    const int32_t *lchild;
    const int32_t *rchild;
    const int64_t *leaf_size;
    int32_t rank;
} superdc_tree;

superdc_status superdc_build_hss(const superdc_tree *tree, const double *D, const double *U,
                                 const double *R, const double *B, cudaStream_t stream,
                                 superdc_hss **out);
void superdc_hss_free(superdc_hss *h);

/* Copy one generator array of a handle to HOST memory `dst` (inspection;
 * synchronous): "D", "U" (leaf blocks, the packing of superdc_build_hss),
 * "R", "B" (nnodes blocks of r x r). */
superdc_status superdc_hss_get(const superdc_hss *h, const char *field, void *dst);

/* Complex Hermitian HSS matrix (the extension the paper notes in Section 1:
 * its real symmetric treatment carries over to the Hermitian case).  Same
 * tree and packing as superdc_build_hss, but every generator entry is
 * complex, stored as an (re, im) pair of doubles (column-major blocks of
 * pairs): D_i Hermitian, A(i, j) = U_i B_i U_j^H for a left child i and its
 * sibling j, nested U_p = [U_i R_i; U_j R_j].  The handle holds the real form
 * of A: every complex block M becomes [[Re M, -Im M], [Im M, Re M]] and the
 * rows of every leaf are ordered [Re rows; Im rows], which keeps the tree and
 * gives a real symmetric HSS matrix of order 2n, leaves 2m_i, rank 2r (so
 * 2 m_i <= 128 and 2r <= 32).  Its eigenvalues are those of A, each twice
 * (superdc_eig returns 2n values, pairs equal up to rounding); for a real
 * function f, superdc_apply_function applies f(A) to complex columns in the
 * same real layout ([Re x_leaf; Im x_leaf] per leaf), and column 2k of the
 * real Q read as x = (first half of each leaf's rows) + i (second half) is
 * a unit eigenvector of A for the k-th eigenvalue when that eigenvalue is
 * simple. */
superdc_status superdc_build_hss_hermitian(const superdc_tree *tree, const double *D, const double *U,
                                           const double *R, const double *B, cudaStream_t stream,
                                           superdc_hss **out);

/* HSS approximation of a symmetric matrix given by its entries, by
 * compression of the off-diagonal block rows (Section 5, Example 4: the HSS
 * form of a kernel matrix built by off-diagonal compression; the paper uses
 * an existing routine of that kind, this one is randomized range finding on
 * one sample of the whole matrix, with nested bases):
 *   entries: kind 0 = dense matrix A (DEVICE, n x n column-major, ld lda >= n,
 *            symmetric, both triangles read), kind 1 = sqrt(|x_i - x_j|),
 *            kind 2 = exp(-|x_i - x_j| / param), at points x (DEVICE, n);
 *   tree: perfect, leaves of `leaf` rows (n = leaf * 2^L, L >= 1, leaf <= 128),
 *   one rank `rank` at every node (rank <= leaf, rank <= 32);
 *   Omega: DEVICE n x nsamp column-major N(0,1) sample drawn by the caller
 *   (rank <= nsamp <= 64; nsamp = rank + 10 is the usual oversampling).
 * For a leaf i, U_i spans the leading rank left singular vectors of the
 * sampled block row Y(I_i) - A(I_i, I_i) Omega(I_i); up the tree the children's
 * projected samples, corrected for the sibling block, give [R_c1; R_c2]; every
 * B_c1 = U_c1^T A(I_c1, I_c2) U_c2 is an exact block product; D_i = A(I_i, I_i).
 * *err_est (HOST, may be NULL) receives the largest relative residual
 * ||M - U U^T M||_F / ||M||_F over the nodes' samples M, the relative size of
 * what the rank-`rank` bases leave out.
 * The result is a handle as from superdc_build_hss; synchronous; work buffers
 * from the stream-ordered allocator. */
typedef struct {
    int32_t kind;
    const double *A;
    int64_t lda;
    const double *x;
    double param;
} superdc_matrix_entries;

superdc_status superdc_build_hss_compress(int64_t n, int32_t leaf, int32_t rank,
                                          const superdc_matrix_entries *entries, const double *Omega,
                                          int32_t nsamp, cudaStream_t stream, superdc_hss **out, double *err_est);

/* Eigendecomposition A = Q diag(lambda) Q^T (Algorithms 1-3):
 *   dividing stage (Algorithm 1, balanced eqs. (3.11)/(3.12), generator
 *   updates of Lemma 2.1); leaf eigendecompositions (Householder
 *   tridiagonalisation, then implicit QL with Wilkinson's shift, or for
 *   leaves all of 128 rows a divide and conquer on the tridiagonal form:
 *   blocks of 32 by QL, two levels of batched rank-one merges); conquering
 *   stage bottom-up over the tree levels: merge sort P_p
 *   (eq. (4.31)), Zhat_p = diag(Q_c1^T, Q_c2^T) Z_p (eq. (2.8)), r rank-one
 *   steps per node, each step applied to the remaining columns.
 * lambda: DEVICE, n entries, ascending (caller-allocated).
 * *fact receives a library-owned handle holding Q in structured form
 * (Lemma 4.1, eq. (4.34)): dense leaf blocks, the permutations and, for every
 * node and step, the factor vectors of eq. (4.30) plus the deflation
 * rotations.  Device-detected errors are latched in the handle; the call
 * synchronises the stream once at the end and returns them (it is
 * superdc_eig_plan + superdc_eig_run + that synchronisation). */
superdc_status superdc_eig(const superdc_hss *h, const superdc_opts *opts, cudaStream_t stream,
                           double *lambda, superdc_eigfact **fact);

/* superdc_eig in two parts, for callers that record the work once into a CUDA
 * graph and replay it (the level-batched launch sequence as one graph):
 *   superdc_eig_plan allocates the handle with every buffer the
 *   factorisation needs and sets the kernels' attributes (synchronous, no
 *   work enqueued);
 *   superdc_eig_run enqueues the whole factorisation on the stream: no host
 *   synchronisation, no host memory read, only device work and the
 *   stream-ordered (cudaMallocAsync) scratch of its steps, so the call can be
 *   captured; each replay recomputes the factor in place and writes lambda
 *   (DEVICE, n).  Device-detected errors are latched in the handle's status
 *   word (cleared at the start of every run) and read by superdc_sync_status.
 * The handle's options are those given to the plan. */
superdc_status superdc_eig_plan(const superdc_hss *h, const superdc_opts *opts, superdc_eigfact **fact);
superdc_status superdc_eig_run(superdc_eigfact *fact, cudaStream_t stream, double *lambda);
void superdc_eigfact_free(superdc_eigfact *f);

/* Y = Q X (trans = 0) or Y = Q^T X (trans = 1), Algorithm 4 applied at the
 * root.  X, Y: DEVICE, n x ncols column-major with leading dimensions
 * ldx, ldy >= n; X and Y must not overlap.  Work buffers come from the
 * stream-ordered allocator. */
superdc_status superdc_apply_Q(const superdc_eigfact *f, int32_t trans, int64_t ncols,
                               const double *X, int64_t ldx, double *Y, int64_t ldy,
                               cudaStream_t stream);

/* Reverse mode of superdc_eig (Algorithms 1-3 differentiated; no counterpart
 * in the paper): gradients of a loss L(lambda, Y = Q^T V) with respect to the
 * generators and V, given the cotangents lambda_bar (n, may be NULL) and Ybar
 * (n x k, ld ldy; k = 0 for eigenvalue-only losses).  The factor must come
 * from superdc_eig with opts.tape = 1 on the same handle (else
 * SUPERDC_ERR_STATE).  Each rank-one step is reversed through its secular
 * roots (the adjoint of superdc_secular_batched_backward); the level build,
 * the leaf eigendecompositions and the dividing stage (H, B~, beta = ||B~||_2)
 * are reversed exactly.  Outputs (DEVICE, caller-allocated, packing of
 * superdc_build_hss): gD (gradient for symmetric perturbations of the leaf
 * blocks), gU, gR, gB (zero where a generator is not used), gV (n x k, ld
 * ldgv).  Deflation rotations are treated as fixed (their dependence is of
 * the order of tau); degenerate eigenvalues make eigenvector losses
 * non-differentiable. */
superdc_status superdc_eig_backward(const superdc_hss *h, const superdc_eigfact *f,
                                    const double *lambda_bar, int64_t k, const double *V, int64_t ldv,
                                    const double *Ybar, int64_t ldy, double *gD, double *gU, double *gR,
                                    double *gB, double *gV, int64_t ldgv, cudaStream_t stream);

/* Matrix function of A applied to a block (the use of the structured
 * eigendecomposition the paper's introduction motivates, Section 1):
 * Y = Q diag(fvals) Q^T X, i.e. f(A) X when fvals[i] = f(lambda_i) for the
 * eigenvalues in the ascending order superdc_eig returned them.  fvals: DEVICE,
 * n entries (any real function values: exp(-t lambda), 1/(lambda - sigma),
 * a spectral window, ...).  X, Y: DEVICE, n x ncols column-major, ld >= n,
 * not overlapping.  Two Algorithm 4 sweeps (Q^T, then Q) and a row scaling;
 * work buffers from the stream-ordered allocator. */
superdc_status superdc_apply_function(const superdc_eigfact *f, const double *fvals, int64_t ncols,
                                      const double *X, int64_t ldx, double *Y, int64_t ldy,
                                      cudaStream_t stream);

/* FMM threshold of later superdc_apply_Q calls on this factor (same meaning
 * as superdc_opts.fmm_min_m; superdc_eig sets it from its options).  The
 * factor itself does not depend on it. */
superdc_status superdc_eigfact_set_fmm_min_m(superdc_eigfact *f, int32_t fmm_min_m);

/* Latched device status of a handle (synchronises the handle's last work):
 * SUPERDC_OK, SUPERDC_ERR_NONFINITE or SUPERDC_ERR_NOCONV. */
superdc_status superdc_sync_status(const superdc_eigfact *f);

/* Statistics of the last superdc_eig on this handle (HOST outputs, any may be
 * NULL): total deflated entries over all steps, total secular sweeps, and the
 * largest number of sweeps used by a root. */
superdc_status superdc_eigfact_stats(const superdc_eigfact *f, int64_t *deflated, int64_t *sweeps,
                                     int32_t *max_sweeps);

/* Copy one stored array of the structured Q to HOST memory `dst` (test and
 * inspection access).  level: 0 (root) .. lmax-1; step: 0 .. r-1.  Fields of
 * length n (one entry per row of the level; node i owns its row range):
 *   "dk", "eta", "dorg", "vhat", "bnorm"  (double), "src", "pinv" (int32),
 *   "din", "zin" (double: the step's input poles, ascending inside each
 *   node, and its input column z, both before deflation), "sweeps" (int32:
 *   secular sweeps of each kept root, the midpoint sweep included),
 *   "P" (int32, the merge order of eq. (4.31); step ignored),
 *   "giv_cs" (double, 2n), "giv_ab" (int32, 2n);
 * per node of the level: "mk", "ngiv", "fmm" (int32; fmm = 1 where the
 * node's step took the triangular FMM path).  Synchronous. */
superdc_status superdc_eigfact_get(const superdc_eigfact *f, int32_t level, int32_t step,
                                   const char *field, void *dst);
/* Generator norms after the dividing stage of the last run on this handle
 * (HOST outputs, any may be NULL; synchronous): rho_bt = max over non-leaf
 * nodes p of ||Bt_c1||_2 (the updated B of p's left child, eq. (3.8)),
 * rho_dt = max over leaves of ||Dhat_k||_2 (the updated leaf blocks, from
 * their eigenvalues) -- the quantities of Section 5's Table 6. */
superdc_status superdc_eigfact_norms(const superdc_eigfact *f, double *rho_bt, double *rho_dt);

/* Tree depth lmax (levels of non-leaf nodes are 0 .. lmax-1), rank r, order n. */
superdc_status superdc_eigfact_shape(const superdc_eigfact *f, int32_t *lmax, int32_t *r, int64_t *n);

/* ------------------------------------------------------------------------
 * Kernel timing (instrumentation; no counterpart in the paper).
 * superdc_profile_enable(1) makes every later call record CUDA events on its
 * stream around each kernel; superdc_profile_read synchronises on those
 * events and returns, for kernel `name` (e.g. "secular"), the number of
 * launches and their summed device time in milliseconds since the last
 * superdc_profile_reset.  Returns SUPERDC_ERR_ARG for an unknown name.
 * Not thread-safe; meant for benchmarks.
 * -------------------------------------------------------------------- */
superdc_status superdc_profile_enable(int32_t on);
superdc_status superdc_profile_reset(void);
superdc_status superdc_profile_read(const char *name, int64_t *launches, double *ms);
/* Work counters recorded while profiling (synchronous read; zeroed by
 * superdc_profile_reset): "fmm_secular_terms" = pole terms summed directly by
 * the FMM secular kernel (near fields), "fmm_secular_last_terms" = terms of
 * the last roots (summed over every pole), both over all sweeps. */
superdc_status superdc_profile_counter(const char *name, int64_t *value);

#ifdef __cplusplus
}
#endif
#endif /* SUPERDC_H */
