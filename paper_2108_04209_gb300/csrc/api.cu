// extern "C" entry points of libsuperdc (declared in include/superdc.h).
#include <cuda_runtime.h>
#include "common.cuh"
#include "rank1.cuh"
#include "fmm.cuh"

int sdc_num_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

extern "C" {

superdc_status superdc_opts_default(superdc_opts *opts)
{
    if (!opts) return SUPERDC_ERR_ARG;
    opts->tau = 1e-10;
    opts->stop_c = 8.0;
    opts->max_iter = 50;
    opts->tile_roots = 0;
    opts->batching = 1;
    opts->sched = 0;
    opts->tape = 0;
    opts->fmm_min_m = 0;
    return SUPERDC_OK;
}

const char *superdc_status_string(superdc_status s)
{
    switch (s) {
    case SUPERDC_OK: return "SUPERDC_OK";
    case SUPERDC_ERR_ARG: return "SUPERDC_ERR_ARG: invalid argument";
    case SUPERDC_ERR_CUDA: return "SUPERDC_ERR_CUDA: CUDA runtime error";
    case SUPERDC_ERR_OOM: return "SUPERDC_ERR_OOM: device allocation failed";
    case SUPERDC_ERR_NONFINITE: return "SUPERDC_ERR_NONFINITE: NaN or Inf encountered";
    case SUPERDC_ERR_NOCONV: return "SUPERDC_ERR_NOCONV: secular iteration did not converge";
    case SUPERDC_ERR_STATE: return "SUPERDC_ERR_STATE: handle in wrong state";
    }
    return "unknown superdc_status";
}

static bool opts_ok(const superdc_opts *op)
{
    return op && op->tau >= 0.0 && op->stop_c > 0.0 && op->max_iter >= 1 && op->max_iter <= 10000 &&
           op->sched >= 0 && op->sched <= 2;
}

superdc_status superdc_secular_batched(int64_t nprob, const int64_t *offsets, int64_t total,
                                       const double *d, const double *z, double rho,
                                       const superdc_opts *opts, superdc_rank1_out *out,
                                       cudaStream_t stream)
{
    superdc_opts def;
    if (!opts) { superdc_opts_default(&def); opts = &def; }
    if (nprob < 0 || total < 0 || !(rho > 0.0) || !opts_ok(opts) || !out) return SUPERDC_ERR_ARG;
    if (nprob == 0) return SUPERDC_OK;
    if (!offsets || !d || !z || total > INT32_MAX) return SUPERDC_ERR_ARG;
    if (!out->lam || !out->dk || !out->zk || !out->eta || !out->vhat || !out->bnorm || !out->org ||
        !out->src || !out->perm || !out->giv_ab || !out->giv_cs || !out->mk || !out->ngiv ||
        !out->status)
        return SUPERDC_ERR_ARG;
    R1Args a;
    a.nprob = nprob;
    a.total = total;
    a.off = offsets;
    a.d = d;
    a.z = z;
    a.sqrt_rho = sqrt(rho);
    a.tau = opts->tau;
    a.stop_c = opts->stop_c;
    a.max_iter = opts->max_iter;
    a.tile_roots = opts->tile_roots;
    a.sched = opts->sched;
    a.fmm_min_m = fmm_resolve(opts->fmm_min_m);
    a.o.lam = out->lam; a.o.dk = out->dk; a.o.zk = out->zk; a.o.eta = out->eta;
    a.o.vhat = out->vhat; a.o.bnorm = out->bnorm; a.o.org = out->org; a.o.src = out->src;
    a.o.perm = out->perm; a.o.giv_ab = out->giv_ab; a.o.giv_cs = out->giv_cs; a.o.mk = out->mk;
    a.o.ngiv = out->ngiv; a.o.sweeps = out->sweeps; a.o.status = out->status; a.o.fmm_used = out->fmm;
    SDC_CHECK(sdc_alloc(&a.o.dorg, total, stream));
    SDC_CHECK(sdc_alloc(&a.o.wsum, nprob, stream));
    SDC_CHECK(sdc_alloc(&a.o.pinv, total, stream));
    superdc_status st = r1_run(a, stream);
    cudaFreeAsync(a.o.dorg, stream);
    cudaFreeAsync(a.o.wsum, stream);
    cudaFreeAsync(a.o.pinv, stream);
    return st;
}

}  // extern "C"
