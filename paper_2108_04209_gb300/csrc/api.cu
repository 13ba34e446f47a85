// extern "C" entry points of libsuperdc (declared in include/superdc.h).
#include <algorithm>
#include <atomic>
#include <cuda_runtime.h>
#include "common.cuh"
#include "rank1.cuh"
#include "fmm.cuh"

namespace {
std::atomic<int64_t> g_alloc_limit{0};
}

bool sdc_alloc_denied(size_t bytes)
{
    const int64_t lim = g_alloc_limit.load(std::memory_order_relaxed);
    return lim > 0 && (int64_t)bytes > lim;
}

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

superdc_status superdc_debug_alloc_limit(int64_t max_bytes)
{
    if (max_bytes < 0) return SUPERDC_ERR_ARG;
    g_alloc_limit.store(max_bytes, std::memory_order_relaxed);
    return SUPERDC_OK;
}

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
    opts->shifted = 1;
    opts->balanced = 1;
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
           op->sched >= 0 && op->sched <= 2 && (op->shifted == 0 || op->shifted == 1) &&
           (op->balanced == 0 || op->balanced == 1);
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
    a.o.unshifted = opts->shifted ? 0 : 1;
    SdcScratch sc(stream);
    SDC_CHECK(sc.get(&a.o.dorg, total));
    SDC_CHECK(sc.get(&a.o.wsum, nprob));
    SDC_CHECK(sc.get(&a.o.pinv, total));
    return r1_run(a, stream);
}

superdc_status superdc_secular_batched_host(int64_t nprob, const int64_t *offsets, int64_t total,
                                            const double *d, const double *z, double rho,
                                            const superdc_opts *opts, superdc_rank1_out *out,
                                            cudaStream_t stream)
{
    superdc_opts def;
    if (!opts) { superdc_opts_default(&def); opts = &def; }
    if (nprob < 0 || total < 0 || !(rho > 0.0) || !opts_ok(opts) || !out || !out->status) return SUPERDC_ERR_ARG;
    if (nprob == 0) { *out->status = 0; return SUPERDC_OK; }
    if (!offsets || !d || !z || total > INT32_MAX) return SUPERDC_ERR_ARG;
    if (offsets[0] != 0 || offsets[nprob] != total) return SUPERDC_ERR_ARG;
    const size_t T = (size_t)std::max<int64_t>(total, 1), NP = (size_t)nprob;
    // one device slab: inputs, every output, status (8-byte fields first)
    const size_t n8 = (NP + 1) + 3 * T + 6 * T + 2 * T, n4 = 3 * T + 2 * T + 2 * NP + T + 1 + NP;
    char *slab = nullptr;
    SDC_CHECK(sdc_alloc(&slab, n8 * 8 + n4 * 4, stream));
    int64_t *doff = (int64_t *)slab;
    double *dd = (double *)(doff + NP + 1), *dz = dd + T;
    superdc_rank1_out o;
    o.lam = dz + T; o.dk = o.lam + T; o.zk = o.dk + T; o.eta = o.zk + T; o.vhat = o.eta + T; o.bnorm = o.vhat + T;
    o.giv_cs = o.bnorm + T;
    int32_t *ip = (int32_t *)(o.giv_cs + 2 * T);
    o.org = ip; o.src = o.org + T; o.perm = o.src + T; o.giv_ab = o.perm + T; o.mk = o.giv_ab + 2 * T;
    o.ngiv = o.mk + NP; o.sweeps = o.ngiv + NP; o.status = o.sweeps + T; o.fmm = o.status + 1;
    cudaError_t e = cudaMemcpyAsync(doff, offsets, (NP + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, d, (size_t)total * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dz, z, (size_t)total * sizeof(double), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(o.status, 0, sizeof(int32_t), stream);
    superdc_status st = (e == cudaSuccess)
        ? superdc_secular_batched(nprob, doff, total, dd, dz, rho, opts, &o, stream) : SUPERDC_ERR_CUDA;
    // results back to the caller's host arrays (NULL fields are skipped)
    struct Cp { void *h; const void *dv; size_t bytes; };
    const Cp cps[] = {
        {out->lam, o.lam, T * 8}, {out->dk, o.dk, T * 8}, {out->zk, o.zk, T * 8}, {out->eta, o.eta, T * 8},
        {out->vhat, o.vhat, T * 8}, {out->bnorm, o.bnorm, T * 8}, {out->giv_cs, o.giv_cs, 2 * T * 8},
        {out->org, o.org, T * 4}, {out->src, o.src, T * 4}, {out->perm, o.perm, T * 4},
        {out->giv_ab, o.giv_ab, 2 * T * 4}, {out->mk, o.mk, NP * 4}, {out->ngiv, o.ngiv, NP * 4},
        {out->sweeps, o.sweeps, T * 4}, {out->fmm, o.fmm, NP * 4}, {out->status, o.status, 4}};
    if (st == SUPERDC_OK)
        for (const Cp &c : cps)
            if (c.h && e == cudaSuccess) e = cudaMemcpyAsync(c.h, c.dv, c.bytes, cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(slab, stream);
    cudaError_t es = cudaStreamSynchronize(stream);
    if (st != SUPERDC_OK) return st;
    if (e != cudaSuccess || es != cudaSuccess) return SUPERDC_ERR_CUDA;
    const int32_t w = *out->status;
    if (w & SUPERDC_DEV_NONFINITE) return SUPERDC_ERR_NONFINITE;
    if (w & SUPERDC_DEV_NOCONV) return SUPERDC_ERR_NOCONV;
    if (w & SUPERDC_DEV_INDEX) return SUPERDC_ERR_CUDA;
    return SUPERDC_OK;
}

}  // extern "C"
