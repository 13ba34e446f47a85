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
#define SUPERDC_DEV_INDEX     4

typedef struct {
    double  tau;          /* deflation tolerance of Remark 4.1 (absolute; strict '<' tests) */
    double  stop_c;       /* constant c of the stopping test eq. (4.12): |f| < c m (1+|psi|+|phi|) eps */
    int32_t max_iter;     /* iteration cap of the secular solver (the paper is silent; default 50) */
    int32_t tile_roots;   /* roots per CTA of the direct evaluator (32..512, multiple of 32) */
    int32_t batching;     /* 1: whole tree level per launch (default); 0: one launch per node */
    int32_t reserved;
} superdc_opts;

/* Fills *opts with the defaults: tau = 1e-10, stop_c = 8, max_iter = 50,
 * tile_roots = 128, batching = 1. */
superdc_status superdc_opts_default(superdc_opts *opts);

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
 *   status (int32, length 1): SUPERDC_DEV_* bits, OR-ed (caller zeroes it).
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
} superdc_rank1_out;

superdc_status superdc_secular_batched(int64_t nprob, const int64_t *offsets, int64_t total,
                                       const double *d, const double *z, double rho,
                                       const superdc_opts *opts, superdc_rank1_out *out,
                                       cudaStream_t stream);

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

#ifdef __cplusplus
}
#endif
#endif /* SUPERDC_H */
