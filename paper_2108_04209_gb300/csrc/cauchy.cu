// Cauchy-like factor application kernels (direct tiled evaluator).
//
// Transpose (conquering stage, Algorithm 3; superdcmv with transpose,
// Algorithm 4):   y_j = b_j sum_i vhat_i x_i / ((d_i - d_{K_j}) - eta_j)
// Forward (superdcmv without transpose):
//                 y_i = vhat_i sum_j b_j x_j / ((d_i - d_{K_j}) - eta_j)
// Every entry uses the shifted difference of eq. (4.28).  One reciprocal per
// (i, j) pair is shared by all columns of the block; the column sums run as
// FP64 FMAs in registers, the operands of the other side are staged in shared
// memory in chunks of TI rows.
#include "common.cuh"
#include <algorithm>
#include "cauchy.cuh"
#include "fmm.cuh"
#include "prof.cuh"

namespace {

__device__ __forceinline__ float mufu_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// full-accuracy FP64 reciprocal: MUFU seed on the mantissa, exponent by
// integer arithmetic, two Newton-Raphson steps (see rank1.cu)
__device__ __forceinline__ double rcp2(double t)
{
    const int hi = __double2hiint(t);
    const unsigned lo = (unsigned)__double2loint(t);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int e = (hi >> 20) & 0x7FF;
    const unsigned mb = (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
    const float rm = mufu_rcp(__uint_as_float(0x3F800000u | mb));
    const unsigned rb = __float_as_uint(rm);
    const int E = (int)(rb >> 23) - 127 - (e - 1023) + 1023;
    const unsigned rmant = rb & 0x7FFFFFu;
    double r = __hiloint2double((int)(sign | ((unsigned)E << 20) | (rmant >> 3)), (int)(rmant << 29));
    double q = fma(-t, r, 1.0);
    r = fma(r, q, r);
    q = fma(-t, r, 1.0);
    return fma(r, q, r);
}

constexpr int TJ = 128;   // outputs per CTA (one per thread)
constexpr int TI = 128;   // staged rows per chunk

__global__ void k_tiles_c(int64_t nprob, const int32_t *__restrict__ mk, int tr, int64_t *__restrict__ tile_off)
{
    __shared__ int64_t part[1024];
    const int T = blockDim.x;
    int64_t per = (nprob + T - 1) / T;
    int64_t beg = threadIdx.x * per, end = min(nprob, beg + per);
    int64_t s = 0;
    for (int64_t p = beg; p < end; p++) s += (mk[p] + tr - 1) / tr;
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int i = 0; i < T; i++) { int64_t v = part[i]; part[i] = acc; acc += v; }
        tile_off[nprob] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t p = beg; p < end; p++) { tile_off[p] = acc; acc += (mk[p] + tr - 1) / tr; }
}

// rotations of the deflation, in scan order (forward) or reversed with the
// transposed rotation (inverse).  The rotation list is a sequence of chains
// (rotation k + 1 continues rotation k when its first index is the second
// index of k); different chains touch disjoint entries, so one thread per
// (chain, column) applies its chain in order (reversed for the inverse).
__global__ void k_givens(FactorView f, int64_t total, double *X, int64_t ldx, int ncols, int inverse)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total * ncols;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % total;
        const int col = (int)(t / total);
        if (x < f.off[0] || x >= f.off[f.nprob]) continue;
        const int64_t p = sdc_upper_index(f.off, f.nprob, x);
        const int64_t b0 = f.off[p];
        const int g = (int)(x - b0);
        const int ng = f.ngiv[p];
        if (g >= ng) continue;
        const int32_t *ab = f.giv_ab + 2 * b0;
        const double *cs = f.giv_cs + 2 * b0;
        double *xv = X + b0 + (int64_t)col * ldx;
        if (!inverse) {
            if (g > 0 && ab[2 * g] == ab[2 * (g - 1) + 1]) continue;      // not a chain start
            for (int k = g; k < ng; k++) {
                if (k > g && ab[2 * k] != ab[2 * (k - 1) + 1]) break;
                const int a = ab[2 * k], b = ab[2 * k + 1];
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double xa = xv[a], xb = xv[b];
                xv[a] = c * xa - s * xb;
                xv[b] = s * xa + c * xb;
            }
        } else {
            if (g + 1 < ng && ab[2 * (g + 1)] == ab[2 * g + 1]) continue;  // not a chain end
            for (int k = g; k >= 0; k--) {
                if (k < g && ab[2 * (k + 1)] != ab[2 * k + 1]) break;
                const int a = ab[2 * k], b = ab[2 * k + 1];
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double xa = xv[a], xb = xv[b];
                xv[a] = c * xa + s * xb;
                xv[b] = -s * xa + c * xb;
            }
        }
    }
}

// y_j = b_j sum_i vhat_i x_{src_i} / ((d_i - d_{K_j}) - eta_j), written at
// merged position pinv[j]; columns [col0, col0 + NC) (fewer at the tail)
template <int NC>
__global__ void __launch_bounds__(TJ)
k_cauchy_T(FactorView f, const int64_t *__restrict__ tile_off, const double *__restrict__ X, int64_t ldx,
           double *__restrict__ Y, int64_t ldy, int col0, int ncols, const int32_t *__restrict__ fslot)
{
    __shared__ double sd[TI];
    __shared__ double sx[NC][TI];
    const int64_t ntiles = tile_off[f.nprob];
    const int nc = min(NC, ncols - col0);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, f.nprob, tile);
        if (fslot && fslot[p] >= 0) continue;   // FMM problem (uniform per CTA)
        const int64_t b0 = f.off[p];
        const int m = f.mk[p];
        const int j = (int)(tile - tile_off[p]) * TJ + threadIdx.x;
        const bool act = j < m;
        const double dK = act ? f.dorg[b0 + j] : 0.0;
        const double e = act ? f.eta[b0 + j] : 1.0;
        double acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) acc[q] = 0.0;
        for (int i0 = 0; i0 < m; i0 += TI) {
            const int cn = min(TI, m - i0);
            __syncthreads();
            for (int ii = threadIdx.x; ii < cn; ii += TJ) {
                const int64_t row = b0 + SDC_IDX(f.src[b0 + i0 + ii], f.off[p + 1] - b0, f.status);
                const double v = f.vhat[b0 + i0 + ii];
                sd[ii] = f.dk[b0 + i0 + ii];
#pragma unroll
                for (int q = 0; q < NC; q++)
                    sx[q][ii] = (q < nc) ? v * X[row + (int64_t)(col0 + q) * ldx] : 0.0;
            }
            __syncthreads();
            if (act) {
                for (int ii = 0; ii < cn; ii++) {
                    const double r = rcp2((sd[ii] - dK) - e);
#pragma unroll
                    for (int q = 0; q < NC; q++) acc[q] = fma(sx[q][ii], r, acc[q]);
                }
            }
        }
        if (act) {
            const double bj = f.bnorm[b0 + j];
            const int64_t row = b0 + SDC_IDX(f.pinv[b0 + j], f.off[p + 1] - b0, f.status);
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) Y[row + (int64_t)(col0 + q) * ldy] = bj * acc[q];
        }
    }
}

// y_{src_i} = vhat_i sum_j b_j x_{pinv_j} / ((d_i - d_{K_j}) - eta_j)
template <int NC>
__global__ void __launch_bounds__(TJ)
k_cauchy_N(FactorView f, const int64_t *__restrict__ tile_off, const double *__restrict__ X, int64_t ldx,
           double *__restrict__ Y, int64_t ldy, int col0, int ncols, const int32_t *__restrict__ fslot)
{
    __shared__ double sk[TI], se[TI];
    __shared__ double sx[NC][TI];
    const int64_t ntiles = tile_off[f.nprob];
    const int nc = min(NC, ncols - col0);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, f.nprob, tile);
        if (fslot && fslot[p] >= 0) continue;   // FMM problem (uniform per CTA)
        const int64_t b0 = f.off[p];
        const int m = f.mk[p];
        const int i = (int)(tile - tile_off[p]) * TJ + threadIdx.x;
        const bool act = i < m;
        const double di = act ? f.dk[b0 + i] : 0.0;
        double acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) acc[q] = 0.0;
        for (int j0 = 0; j0 < m; j0 += TI) {
            const int cn = min(TI, m - j0);
            __syncthreads();
            for (int jj = threadIdx.x; jj < cn; jj += TJ) {
                const int64_t row = b0 + SDC_IDX(f.pinv[b0 + j0 + jj], f.off[p + 1] - b0, f.status);
                const double bj = f.bnorm[b0 + j0 + jj];
                sk[jj] = f.dorg[b0 + j0 + jj];
                se[jj] = f.eta[b0 + j0 + jj];
#pragma unroll
                for (int q = 0; q < NC; q++)
                    sx[q][jj] = (q < nc) ? bj * X[row + (int64_t)(col0 + q) * ldx] : 0.0;
            }
            __syncthreads();
            if (act) {
                for (int jj = 0; jj < cn; jj++) {
                    const double r = rcp2((di - sk[jj]) - se[jj]);
#pragma unroll
                    for (int q = 0; q < NC; q++) acc[q] = fma(sx[q][jj], r, acc[q]);
                }
            }
        }
        if (act) {
            const double v = f.vhat[b0 + i];
            const int64_t row = b0 + SDC_IDX(f.src[b0 + i], f.off[p + 1] - b0, f.status);
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) Y[row + (int64_t)(col0 + q) * ldy] = v * acc[q];
        }
    }
}

// deflated slots: identity part of the factor
__global__ void k_defl_copy(FactorView f, int64_t total, const double *__restrict__ X, int64_t ldx,
                            double *__restrict__ Y, int64_t ldy, int ncols, int trans)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total * ncols;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slotg = x % total;
        const int col = (int)(x / total);
        if (slotg < f.off[0] || slotg >= f.off[f.nprob]) continue;
        const int64_t p = sdc_upper_index(f.off, f.nprob, slotg);
        const int64_t b0 = f.off[p];
        const int s = (int)(slotg - b0);
        if (s < f.mk[p]) continue;
        const int64_t ps = SDC_IDX(f.pinv[slotg], f.off[p + 1] - b0, f.status);
        const int64_t sr = SDC_IDX(f.src[slotg], f.off[p + 1] - b0, f.status);
        if (trans) Y[b0 + ps + (int64_t)col * ldy] = X[b0 + sr + (int64_t)col * ldx];
        else       Y[b0 + sr + (int64_t)col * ldy] = X[b0 + ps + (int64_t)col * ldx];
    }
}

template <template <int> class K>
struct Dummy {};

// the inner loops run all NC columns: even widths up to 20 (the ranks of
// typical HSS generators) waste at most one FMA per term
int pick_nc(int c)
{
    if (c <= 20) return std::max(2, (c + 1) & ~1);
    if (c <= 24) return 24;
    return 32;
}

template <int NC>
void launch_T(const FactorView &f, const int64_t *tile_off, const double *X, int64_t ldx, double *Y, int64_t ldy,
              int col0, int ncols, unsigned grid, const int32_t *fslot, cudaStream_t st)
{
    k_cauchy_T<NC><<<grid, TJ, 0, st>>>(f, tile_off, X, ldx, Y, ldy, col0, ncols, fslot);
}

template <int NC>
void launch_N(const FactorView &f, const int64_t *tile_off, const double *X, int64_t ldx, double *Y, int64_t ldy,
              int col0, int ncols, unsigned grid, const int32_t *fslot, cudaStream_t st)
{
    k_cauchy_N<NC><<<grid, TJ, 0, st>>>(f, tile_off, X, ldx, Y, ldy, col0, ncols, fslot);
}

typedef void (*LaunchFn)(const FactorView &, const int64_t *, const double *, int64_t, double *, int64_t, int, int,
                         unsigned, const int32_t *, cudaStream_t);

LaunchFn pick(bool trans, int nc)
{
    switch (nc) {
#define SDC_NC(W) case W: return trans ? launch_T<W> : launch_N<W>;
    SDC_NC(2) SDC_NC(4) SDC_NC(6) SDC_NC(8) SDC_NC(10) SDC_NC(12) SDC_NC(14) SDC_NC(16) SDC_NC(18) SDC_NC(20)
    SDC_NC(24)
#undef SDC_NC
    default: return trans ? launch_T<32> : launch_N<32>;
    }
}

superdc_status run(const FactorView &f, int64_t total, double *Xmut, const double *X, int64_t ldx, double *Y,
                   int64_t ldy, int ncols, bool trans, cudaStream_t st, const FmmPlan *shared)
{
    if (ncols <= 0 || total <= 0) return SUPERDC_OK;
    const int nsm = sdc_num_sms();
    int64_t *tile_off = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&tile_off, f.nprob + 1));
    k_tiles_c<<<1, 1024, 0, st>>>(f.nprob, f.mk, TJ, tile_off);
    const int gthreads = 128;
    if (trans)
        PROF_LAUNCH("givens", st, k_givens<<<(unsigned)(nsm * 8), gthreads, 0, st>>>(f, total, Xmut, ldx, ncols, 0));
    // problems whose kept size reaches the threshold: triangular FMM
    FmmPlan fp;
    const int w = std::min(32, ncols);
    const int box = (w <= 24) ? 32 : 64;
    // the plan of this factor's rank-one step serves when its boxes and widths fit
    const bool use_shared = shared && shared->on && shared->box == box && shared->dv.ncol >= w &&
                            shared->dv.nfield >= w;
    if (!use_shared) {
        // boxes of 32 halve the near field; with many columns the translations
        // (P^2 per column and box pair) dominate and boxes of 64 halve those
        superdc_status fs = fmm_plan(fp, f.nprob, f.off, total, f.max_m, f.mk, f.dk, f.fmm_min_m, w, w, nullptr,
                                     box, 0, st);
        if (fs != SUPERDC_OK) { fmm_free(fp, st); return fs; }
    }
    const FmmPlan &pl = use_shared ? *shared : fp;
    const int32_t *fslot = pl.on ? pl.dv.fslot : nullptr;
    superdc_status fs = SUPERDC_OK;
    const unsigned grid = (unsigned)(nsm * 4);
    for (int c0 = 0; c0 < ncols; c0 += 32) {
        const int c = min(32, ncols - c0);
        LaunchFn fn = pick(trans, pick_nc(c));
        PROF_LAUNCH("cauchy", st, fn(f, tile_off, X, ldx, Y, ldy, c0, ncols, grid, fslot, st));
        if (fs == SUPERDC_OK) fs = fmm_cauchy(pl, f, X, ldx, Y, ldy, c0, c, trans, st);
    }
    PROF_LAUNCH("deflcopy", st, k_defl_copy<<<(unsigned)(nsm * 8), 256, 0, st>>>(f, total, X, ldx, Y, ldy, ncols,
                                                                                  trans ? 1 : 0));
    if (!trans)
        PROF_LAUNCH("givens", st, k_givens<<<(unsigned)(nsm * 8), gthreads, 0, st>>>(f, total, Y, ldy, ncols, 1));
    const cudaError_t le = cudaGetLastError();
    fmm_free(fp, st);
    if (le != cudaSuccess) return SUPERDC_ERR_CUDA;
    return fs;
}

}  // namespace

superdc_status cauchy_apply_T(const FactorView &f, int64_t total, double *X, int64_t ldx, double *Y, int64_t ldy,
                              int ncols, cudaStream_t st, const FmmPlan *plan)
{
    return run(f, total, X, X, ldx, Y, ldy, ncols, true, st, plan);
}

superdc_status cauchy_apply_N(const FactorView &f, int64_t total, const double *X, int64_t ldx, double *Y,
                              int64_t ldy, int ncols, cudaStream_t st)
{
    return run(f, total, nullptr, X, ldx, Y, ldy, ncols, false, st, nullptr);
}
