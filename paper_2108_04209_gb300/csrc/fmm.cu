// Entry points of the triangular FMM: each plan records its leaf-box size and
// the calls go to the build of fmm_impl.cuh for that size (fmm32.cu, fmm64.cu).
#include "fmm.cuh"

namespace fmm_b32 {
superdc_status plan(FmmPlan &pl, int64_t nprob, const int64_t *off, int64_t total, int64_t max_m,
                    const int32_t *mk, const double *dk, int min_m, int ncol, int nfield, int32_t *used,
                    int kslots, cudaStream_t st);
void free_plan(FmmPlan &pl, cudaStream_t st);
superdc_status secular(const FmmPlan &pl, const int64_t *off, const R1Out &o, double stop_c, int max_iter,
                       cudaStream_t st);
superdc_status lowner(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st);
superdc_status bnorm(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st);
superdc_status cauchy(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y,
                      int64_t ldy, int col0, int nc, bool trans, cudaStream_t st);
}
namespace fmm_b64 {
superdc_status plan(FmmPlan &pl, int64_t nprob, const int64_t *off, int64_t total, int64_t max_m,
                    const int32_t *mk, const double *dk, int min_m, int ncol, int nfield, int32_t *used,
                    int kslots, cudaStream_t st);
void free_plan(FmmPlan &pl, cudaStream_t st);
superdc_status secular(const FmmPlan &pl, const int64_t *off, const R1Out &o, double stop_c, int max_iter,
                       cudaStream_t st);
superdc_status lowner(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st);
superdc_status bnorm(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st);
superdc_status cauchy(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y,
                      int64_t ldy, int col0, int nc, bool trans, cudaStream_t st);
}

// measured on GB300 (python -m paper_2108_04209_gb300.crossover: batches of
// equal-size rank-one problems, whole step direct vs FMM): at m = 256 few
// problems keep enough poles for the tree and the direct path is 10 % faster;
// at m = 512 the FMM step is 1.4x faster (4096 problems), at 1024 2.6x, at
// 2048 7x; in the n = 131072 eigendecomposition (256 problems of 512 on that
// level) the threshold 512 beats 1024 and 256.  The autotuner refines it per
// batch.
int fmm_default_min_m() { return 512; }

superdc_status fmm_plan(FmmPlan &pl, int64_t nprob, const int64_t *off, int64_t total, int64_t max_m,
                        const int32_t *mk, const double *dk, int min_m, int ncol, int nfield, int32_t *used,
                        int box, int kslots, cudaStream_t st)
{
    if (box == 64)
        return fmm_b64::plan(pl, nprob, off, total, max_m, mk, dk, min_m, ncol, nfield, used, kslots, st);
    if (box == 32)
        return fmm_b32::plan(pl, nprob, off, total, max_m, mk, dk, min_m, ncol, nfield, used, kslots, st);
    return SUPERDC_ERR_ARG;
}

void fmm_free(FmmPlan &pl, cudaStream_t st)
{
    if (pl.box == 64) fmm_b64::free_plan(pl, st);
    else fmm_b32::free_plan(pl, st);
}

superdc_status fmm_secular(const FmmPlan &pl, const int64_t *off, const R1Out &o, double stop_c, int max_iter,
                           cudaStream_t st)
{
    return pl.box == 64 ? fmm_b64::secular(pl, off, o, stop_c, max_iter, st)
                        : fmm_b32::secular(pl, off, o, stop_c, max_iter, st);
}

superdc_status fmm_lowner(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st)
{
    return pl.box == 64 ? fmm_b64::lowner(pl, off, o, st) : fmm_b32::lowner(pl, off, o, st);
}

superdc_status fmm_bnorm(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st)
{
    return pl.box == 64 ? fmm_b64::bnorm(pl, off, o, st) : fmm_b32::bnorm(pl, off, o, st);
}

superdc_status fmm_cauchy(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y,
                          int64_t ldy, int col0, int nc, bool trans, cudaStream_t st)
{
    return pl.box == 64 ? fmm_b64::cauchy(pl, f, X, ldx, Y, ldy, col0, nc, trans, st)
                        : fmm_b32::cauchy(pl, f, X, ldx, Y, ldy, col0, nc, trans, st);
}
