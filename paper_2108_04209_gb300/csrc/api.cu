// extern "C" entry points of libsuperdc (declared in include/superdc.h).
#include <algorithm>
#include <atomic>
#include <cuda_runtime.h>
#include <mutex>
#include <vector>
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

// the batched step's arguments from the public options (device arrays)
static R1Args r1args(int64_t nprob, const int64_t *offsets, int64_t total, const double *d, const double *z,
                     double rho, const superdc_opts *opts)
{
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
    a.o.unshifted = opts->shifted ? 0 : 1;
    return a;
}

// two non-blocking streams of the library on the current device (created on
// first use), for the host-buffer entry point's copy/compute pipeline
static cudaError_t sdc_side_streams(cudaStream_t *s2)
{
    static std::mutex mu;
    static cudaStream_t ss[64][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    for (int k = 0; k < 2; k++)
        if (!ss[dev][k] && (e = cudaStreamCreateWithFlags(&ss[dev][k], cudaStreamNonBlocking)) != cudaSuccess) return e;
    s2[0] = ss[dev][0];
    s2[1] = ss[dev][1];
    return cudaSuccess;
}

cudaMemPool_t sdc_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool tried[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        cudaMemPoolProps pp = {};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.handleTypes = cudaMemHandleTypeNone;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &pp) == cudaSuccess) {
            unsigned long long keep = SDC_POOL_KEEP;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            // no dependencies inserted between streams to reuse a block (the
            // host entry's two streams would otherwise be serialised)
            int no = 0;
            cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
            pools[dev] = pool;
        } else {
            cudaGetLastError();
        }
    }
    return pools[dev];
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
    R1Args a = r1args(nprob, offsets, total, d, z, rho, opts);
    a.o.lam = out->lam; a.o.dk = out->dk; a.o.zk = out->zk; a.o.eta = out->eta;
    a.o.vhat = out->vhat; a.o.bnorm = out->bnorm; a.o.org = out->org; a.o.src = out->src;
    a.o.perm = out->perm; a.o.giv_ab = out->giv_ab; a.o.giv_cs = out->giv_cs; a.o.mk = out->mk;
    a.o.ngiv = out->ngiv; a.o.sweeps = out->sweeps; a.o.status = out->status; a.o.fmm_used = out->fmm;
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
    for (int64_t p = 0; p < nprob; p++)
        if (offsets[p + 1] < offsets[p]) return SUPERDC_ERR_ARG;
    const size_t T = (size_t)std::max<int64_t>(total, 1), NP = (size_t)nprob;
    // one device slab: offsets, inputs, every output, the step's per-row and
    // per-problem scratch, status (8-byte fields first)
    const size_t n8 = (NP + 1) + 2 * T + 6 * T + 2 * T + T + NP;
    const size_t n4 = 3 * T + 2 * T + 2 * NP + T + 1 + NP + T;
    char *slab = nullptr;
    SDC_CHECK(sdc_alloc(&slab, n8 * 8 + n4 * 4, stream));
    int64_t *doff = (int64_t *)slab;
    double *dd = (double *)(doff + NP + 1), *dz = dd + T;
    superdc_rank1_out o;
    o.lam = dz + T; o.dk = o.lam + T; o.zk = o.dk + T; o.eta = o.zk + T; o.vhat = o.eta + T; o.bnorm = o.vhat + T;
    o.giv_cs = o.bnorm + T;
    double *dorg = o.giv_cs + 2 * T, *wsum = dorg + T;
    int32_t *ip = (int32_t *)(wsum + NP);
    o.org = ip; o.src = o.org + T; o.perm = o.src + T; o.giv_ab = o.perm + T; o.mk = o.giv_ab + 2 * T;
    o.ngiv = o.mk + NP; o.sweeps = o.ngiv + NP; o.status = o.sweeps + T; o.fmm = o.status + 1;
    int32_t *pinv = o.fmm + NP;
    // chunks of about equal root counts at problem boundaries, on two streams:
    // one chunk's copies overlap another's kernels.  Rows stay absolute and the
    // schedule is that of the whole batch, so every problem's arithmetic (and
    // result) is the same as in one call over the batch.
    const int nch = (total >= (1 << 20) && nprob >= 16) ? 4 : 1;
    std::vector<int64_t> cut(nch + 1, nprob);
    cut[0] = 0;
    for (int c = 1; c < nch; c++)
        cut[c] = std::lower_bound(offsets, offsets + nprob + 1, (total * c) / nch) - offsets;
    cudaStream_t side[2] = {stream, stream};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaMemcpyAsync(doff, offsets, (NP + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(o.status, 0, sizeof(int32_t), stream);
    if (e == cudaSuccess && nch > 1) {
        e = sdc_side_streams(side);
        for (int k = 0; k < 3 && e == cudaSuccess; k++) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], stream);
        for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaStreamWaitEvent(side[k], ev[0], 0);
    }
    superdc_status st = (e == cudaSuccess) ? SUPERDC_OK : SUPERDC_ERR_CUDA;
    for (int c = 0; c < nch && st == SUPERDC_OK; c++) {
        const int64_t p0 = cut[c], p1 = cut[c + 1];
        if (p1 <= p0) continue;
        cudaStream_t sc = side[c & 1];
        const int64_t o0 = offsets[p0], o1 = offsets[p1];
        const size_t nr = (size_t)(o1 - o0), npc = (size_t)(p1 - p0);
        e = cudaMemcpyAsync(dd + o0, d + o0, nr * sizeof(double), cudaMemcpyHostToDevice, sc);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dz + o0, z + o0, nr * sizeof(double), cudaMemcpyHostToDevice, sc);
        if (e != cudaSuccess) { st = SUPERDC_ERR_CUDA; break; }
        R1Args a = r1args(p1 - p0, doff + p0, total, dd, dz, rho, opts);
        a.rows = total;
        a.o.lam = o.lam; a.o.dk = o.dk; a.o.zk = o.zk; a.o.eta = o.eta; a.o.vhat = o.vhat; a.o.bnorm = o.bnorm;
        a.o.org = o.org; a.o.src = o.src; a.o.perm = o.perm; a.o.giv_ab = o.giv_ab; a.o.giv_cs = o.giv_cs;
        a.o.mk = o.mk + p0; a.o.ngiv = o.ngiv + p0; a.o.sweeps = o.sweeps; a.o.status = o.status;
        a.o.fmm_used = o.fmm + p0; a.o.dorg = dorg; a.o.wsum = wsum + p0; a.o.pinv = pinv;
        st = r1_run(a, sc);
        if (st != SUPERDC_OK) break;
        // this chunk's results to the caller's host arrays (NULL fields are skipped)
        struct Cp { void *h; const void *dv; size_t bytes; };
        const Cp cps[] = {
            {out->lam, o.lam, 8}, {out->dk, o.dk, 8}, {out->zk, o.zk, 8}, {out->eta, o.eta, 8},
            {out->vhat, o.vhat, 8}, {out->bnorm, o.bnorm, 8}, {out->giv_cs, o.giv_cs, 16},
            {out->org, o.org, 4}, {out->src, o.src, 4}, {out->perm, o.perm, 4},
            {out->giv_ab, o.giv_ab, 8}, {out->sweeps, o.sweeps, 4}};
        for (const Cp &cp : cps)
            if (cp.h && e == cudaSuccess)
                e = cudaMemcpyAsync((char *)cp.h + o0 * cp.bytes, (const char *)cp.dv + o0 * cp.bytes, nr * cp.bytes,
                                    cudaMemcpyDeviceToHost, sc);
        const Cp pps[] = {{out->mk, o.mk, 4}, {out->ngiv, o.ngiv, 4}, {out->fmm, o.fmm, 4}};
        for (const Cp &cp : pps)
            if (cp.h && e == cudaSuccess)
                e = cudaMemcpyAsync((char *)cp.h + p0 * cp.bytes, (const char *)cp.dv + p0 * cp.bytes, npc * cp.bytes,
                                    cudaMemcpyDeviceToHost, sc);
        if (e != cudaSuccess) st = SUPERDC_ERR_CUDA;
    }
    // join the side streams before the status is read and the slab freed
    if (nch > 1 && ev[1] && ev[2]) {
        for (int k = 0; k < 2; k++)
            if (cudaEventRecord(ev[1 + k], side[k]) == cudaSuccess) cudaStreamWaitEvent(stream, ev[1 + k], 0);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->status, o.status, 4, cudaMemcpyDeviceToHost, stream);
    cudaFreeAsync(slab, stream);
    cudaError_t es = cudaStreamSynchronize(stream);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (st != SUPERDC_OK) return st;
    if (e != cudaSuccess || es != cudaSuccess) return SUPERDC_ERR_CUDA;
    const int32_t w = *out->status;
    if (w & SUPERDC_DEV_NONFINITE) return SUPERDC_ERR_NONFINITE;
    if (w & SUPERDC_DEV_NOCONV) return SUPERDC_ERR_NOCONV;
    if (w & SUPERDC_DEV_INDEX) return SUPERDC_ERR_CUDA;
    return SUPERDC_OK;
}

}  // extern "C"
