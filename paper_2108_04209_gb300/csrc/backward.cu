// Adjoint of the batched rank-one step (reverse mode through the secular roots).
//
// Forward, per problem: M = diag(d) + rho z z^T  ->  new eigenvalues lambda
// (sorted) and, for caller columns X, Y = Qhat^T X with
// Qhat = G^T [C (+) I] Pi^T (rotations G, Cauchy-like block C of eq. (4.26)
// on the kept set, identity on the deflated set, sort Pi).
// Given cotangents lambda_bar (merged order) and Ybar, this computes
// d_bar, z_bar (input order) and X_bar = Qhat Ybar.
//
// Kept block (implicit-function theorem on the secular equation, i.e. the
// eigen-adjoint of M_k = diag(d_k) + z_k z_k^T = C Lambda C^T):
//   Mbar = C E C^T,  E = diag(lambda_bar) + sym(F o (Y Ybar^T)),
//   F_kl = 1/(lambda_l - lambda_k) (k != l);  d_bar = diag(Mbar), z_bar = 2 Mbar z.
// With C^T z = -b (Loewner's zhat makes sum_i zhat_i^2/(d_i - lambda_k) = -1),
//   u_k = -lambda_bar_k b_k - 1/2 sum_c (y_kc P_kc - ybar_kc R_kc),
//   P_kc = sum_{l!=k} b_l ybar_lc/(lambda_l - lambda_k), R_kc = sum_{l!=k} b_l y_lc/(lambda_l - lambda_k),
//   z_bar_i = 2 (C u)_i = 2 vhat_i sum_k b_k u_k / (d_i - lambda_k),
// and, by partial fractions 1/((d-l_k)(d-l_l)) = [1/(d-l_k) - 1/(d-l_l)]/(l_k - l_l),
//   d_bar_i = vhat_i^2 sum_k [h_k/(d_i - lambda_k)^2 + g_k/(d_i - lambda_k)],
//   h_k = b_k^2 lambda_bar_k,  g_k = sum_c (beta_kc Delta_kc - alpha_kc Gamma_kc),
//   alpha_kc = b_k y_kc, beta_kc = b_k ybar_kc,
//   Gamma_kc = sum_{l!=k} beta_lc/(lambda_k - lambda_l)^2, Delta_kc = sum_{l!=k} alpha_lc/(lambda_k - lambda_l)^2.
// Every difference is taken in shifted form: d_i - lambda_k = (d_i - d_{K_k}) - eta_k
// (eq. (4.28)) and lambda_k - lambda_l = (d_{K_k} - d_{K_l}) + (eta_k - eta_l).
// Deflation: the rotations are treated as fixed linear maps (their dependence
// on z is of the order of tau); deflated eigenvalues are the rotated poles.
// Eigenvalue pairs with |lambda_k - lambda_l| <= 1e-10 max(|lambda_k|, |lambda_l|)
// are treated as one eigenspace (no coupling term): eigenvector losses are not
// differentiable there, and losses invariant within the eigenspace are exact.
#include <algorithm>
#include <cuda_runtime.h>
#include "common.cuh"
#include "cauchy.cuh"
#include "fmm.cuh"
#include "prof.cuh"

namespace {

constexpr int BW_C = 8;      // columns per pass of the lambda-lambda kernel
constexpr int TB = 128;

__device__ __forceinline__ double rcp_full(double t) { return 1.0 / t; }

// pinv from perm, d_K from org (inputs are the public forward outputs)
__global__ void k_prep(int64_t nprob, const int64_t *__restrict__ off, int64_t total, const int32_t *__restrict__ mk,
                       const int32_t *__restrict__ perm, const int32_t *__restrict__ org, const double *__restrict__ dk,
                       int32_t *__restrict__ pinv, double *__restrict__ dorg)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = sdc_upper_index(off, nprob, x);
        const int64_t b0 = off[p];
        const int pos = (int)(x - b0);
        pinv[b0 + perm[x]] = pos;
        const int s = (int)(x - b0);
        dorg[x] = (s < mk[p]) ? dk[b0 + org[x]] : dk[x];
    }
}

// per kept root k: u_k and g_k (lambda-lambda sums), columns [c0, c0+nc)
__global__ void __launch_bounds__(TB)
k_bw_lamlam(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off,
            const int32_t *__restrict__ mk, const double *__restrict__ dorg, const double *__restrict__ eta,
            const double *__restrict__ bnorm, const int32_t *__restrict__ pinv,
            const double *__restrict__ Y, int64_t ld, const double *__restrict__ Ybar, int64_t ldb, int c0, int nc,
            double *__restrict__ u, double *__restrict__ g)
{
    __shared__ double sK[TB], sE[TB], sA[BW_C][TB], sB[BW_C][TB];
    const int64_t ntiles = tile_off[nprob];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        const int64_t b0 = off[p];
        const int m = mk[p];
        const int k = (int)(tile - tile_off[p]) * TB + threadIdx.x;
        const bool act = k < m;
        const double dKk = act ? dorg[b0 + k] : 0.0, ek = act ? eta[b0 + k] : 0.0;
        double P[BW_C], R[BW_C], Ga[BW_C], De[BW_C];
#pragma unroll
        for (int c = 0; c < BW_C; c++) { P[c] = R[c] = Ga[c] = De[c] = 0.0; }
        for (int l0 = 0; l0 < m; l0 += TB) {
            const int cn = min(TB, m - l0);
            __syncthreads();
            for (int ll = threadIdx.x; ll < cn; ll += TB) {
                const int64_t s = b0 + l0 + ll;
                const double bl = bnorm[s];
                const int64_t row = b0 + pinv[s];
                sK[ll] = dorg[s];
                sE[ll] = eta[s];
#pragma unroll
                for (int c = 0; c < BW_C; c++) {
                    sA[c][ll] = (c < nc) ? bl * Y[row + ld * (c0 + c)] : 0.0;
                    sB[c][ll] = (c < nc) ? bl * Ybar[row + ldb * (c0 + c)] : 0.0;
                }
            }
            __syncthreads();
            if (act) {
                for (int ll = 0; ll < cn; ll++) {
                    if (l0 + ll == k) continue;
                    const double dl = (dKk - sK[ll]) + (ek - sE[ll]);     // lambda_k - lambda_l
                    // numerically degenerate pairs form one eigenspace: no coupling
                    if (fabs(dl) <= 1e-10 * fmax(fabs(dKk + ek), fabs(sK[ll] + sE[ll]))) continue;
                    const double r = rcp_full(dl);
                    const double r2 = r * r;
#pragma unroll
                    for (int c = 0; c < BW_C; c++) {
                        P[c] = fma(-sB[c][ll], r, P[c]);     // sum beta_l/(lambda_l - lambda_k)
                        R[c] = fma(-sA[c][ll], r, R[c]);
                        Ga[c] = fma(sB[c][ll], r2, Ga[c]);
                        De[c] = fma(sA[c][ll], r2, De[c]);
                    }
                }
            }
        }
        if (act) {
            const double bk = bnorm[b0 + k];
            const int64_t row = b0 + pinv[b0 + k];
            double uu = 0.0, gg = 0.0;
#pragma unroll
            for (int c = 0; c < BW_C; c++) {
                if (c >= nc) break;
                const double y = Y[row + ld * (c0 + c)], yb = Ybar[row + ldb * (c0 + c)];
                uu += -0.5 * (y * P[c] - yb * R[c]);
                gg += (bk * yb) * De[c] - (bk * y) * Ga[c];
            }
            u[b0 + k] += uu;
            g[b0 + k] += gg;
        }
    }
}

// d_bar_i, z_bar_i of the kept rows
__global__ void __launch_bounds__(TB)
k_bw_dz(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off,
        const int32_t *__restrict__ mk, const double *__restrict__ dk, const double *__restrict__ dorg,
        const double *__restrict__ eta, const double *__restrict__ vhat, const double *__restrict__ bnorm,
        const int32_t *__restrict__ pinv, const double *__restrict__ lam_bar, const double *__restrict__ u,
        const double *__restrict__ g, double *__restrict__ dbar_s, double *__restrict__ zbar_s)
{
    __shared__ double sK[TB], sE[TB], sH[TB], sG[TB], sU[TB];
    const int64_t ntiles = tile_off[nprob];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        const int64_t b0 = off[p];
        const int m = mk[p];
        const int i = (int)(tile - tile_off[p]) * TB + threadIdx.x;
        const bool act = i < m;
        const double di = act ? dk[b0 + i] : 0.0;
        double a1 = 0.0, a2 = 0.0;
        for (int k0 = 0; k0 < m; k0 += TB) {
            const int cn = min(TB, m - k0);
            __syncthreads();
            for (int kk = threadIdx.x; kk < cn; kk += TB) {
                const int64_t s = b0 + k0 + kk;
                const double bk = bnorm[s];
                const double lb = lam_bar ? lam_bar[b0 + pinv[s]] : 0.0;
                sK[kk] = dorg[s];
                sE[kk] = eta[s];
                sH[kk] = bk * bk * lb;
                sG[kk] = g[s];
                sU[kk] = bk * (u[s] - lb * bk);
            }
            __syncthreads();
            if (act) {
                for (int kk = 0; kk < cn; kk++) {
                    const double r = rcp_full((di - sK[kk]) - sE[kk]);
                    a1 = fma(fma(sH[kk], r, sG[kk]), r, a1);
                    a2 = fma(sU[kk], r, a2);
                }
            }
        }
        if (act) {
            const double v = vhat[b0 + i];
            dbar_s[b0 + i] = v * v * a1;
            zbar_s[b0 + i] = 2.0 * v * a2;
        }
    }
}

// scatter to input order, deflated eigenvalues, reverse rotations, rho scaling
__global__ void k_bw_deflate(int64_t nprob, const int64_t *__restrict__ off, const int32_t *__restrict__ mk,
                             const int32_t *__restrict__ ngiv, const int32_t *__restrict__ src,
                             const int32_t *__restrict__ pinv, const int32_t *__restrict__ giv_ab,
                             const double *__restrict__ giv_cs, const double *__restrict__ lam_bar,
                             const double *__restrict__ dbar_s, const double *__restrict__ zbar_s,
                             double sqrt_rho, double *__restrict__ dbar, double *__restrict__ zbar)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    const int64_t b0 = off[p];
    const int m = (int)(off[p + 1] - b0), k = mk[p];
    for (int s = 0; s < m; s++) {
        const int64_t in = b0 + src[b0 + s];
        if (s < k) {
            dbar[in] = dbar_s[b0 + s];
            zbar[in] = zbar_s[b0 + s];
        } else {
            dbar[in] = lam_bar ? lam_bar[b0 + pinv[b0 + s]] : 0.0;
            zbar[in] = 0.0;
        }
    }
    for (int t = ngiv[p] - 1; t >= 0; t--) {
        const int a = giv_ab[2 * (b0 + t)], bb = giv_ab[2 * (b0 + t) + 1];
        const double c = giv_cs[2 * (b0 + t)], s = giv_cs[2 * (b0 + t) + 1];
        const double da = dbar[b0 + a], db = dbar[b0 + bb];
        dbar[b0 + a] = c * c * da + s * s * db;
        dbar[b0 + bb] = s * s * da + c * c * db;
        const double za = zbar[b0 + a], zb = zbar[b0 + bb];
        zbar[b0 + a] = c * za + s * zb;
        zbar[b0 + bb] = -s * za + c * zb;
    }
    for (int i = 0; i < m; i++) zbar[b0 + i] *= sqrt_rho;
}

__global__ void k_tiles_b(int64_t nprob, const int32_t *__restrict__ mk, int tr, int64_t *__restrict__ tile_off)
{
    __shared__ int64_t part[1024];
    const int T = blockDim.x;
    int64_t per = (nprob + T - 1) / T;
    int64_t beg = threadIdx.x * per, end = min(nprob, beg + per);
    int64_t s = 0;
    for (int64_t q = beg; q < end; q++) s += (mk[q] + tr - 1) / tr;
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int i = 0; i < T; i++) { int64_t v = part[i]; part[i] = acc; acc += v; }
        tile_off[nprob] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t q = beg; q < end; q++) { tile_off[q] = acc; acc += (mk[q] + tr - 1) / tr; }
}

}  // namespace

// Adjoint of one batched rank-one step given its factor view (pinv and d_K
// available).  X: the columns the step transformed (input order, read only),
// Ybar: cotangent of Qhat^T X (merged order); lam_bar may be NULL.
superdc_status r1_backward_fv(const FactorView &f, int64_t total, const double *lam_bar, int ncols,
                              const double *X, int64_t ldx, const double *Ybar, int64_t ldy, double *d_bar,
                              double *z_bar, double *X_bar, int64_t ldxb, double sqrt_rho, cudaStream_t st)
{
    const int nsm = sdc_num_sms();
    double *u = nullptr, *g = nullptr, *dbs = nullptr, *zbs = nullptr, *Y = nullptr, *Xw = nullptr;
    int64_t *tile_off = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&u, total));
    SDC_CHECK(sc.get(&g, total));
    SDC_CHECK(sc.get(&dbs, total));
    SDC_CHECK(sc.get(&zbs, total));
    SDC_CHECK(sc.get(&tile_off, f.nprob + 1));
    SDC_CHECK(cudaMemsetAsync(u, 0, total * sizeof(double), st));
    SDC_CHECK(cudaMemsetAsync(g, 0, total * sizeof(double), st));
    k_tiles_b<<<1, 1024, 0, st>>>(f.nprob, f.mk, TB, tile_off);
    superdc_status s = SUPERDC_OK;
    if (ncols > 0) {
        // Y = Qhat^T X is recomputed (the rotations act on a copy of X)
        SDC_CHECK(sc.get(&Y, (size_t)total * ncols));
        SDC_CHECK(sc.get(&Xw, (size_t)total * ncols));
        SDC_CHECK(cudaMemcpy2DAsync(Xw, total * sizeof(double), X, ldx * sizeof(double), total * sizeof(double),
                                    ncols, cudaMemcpyDeviceToDevice, st));
        s = cauchy_apply_T(f, total, Xw, total, Y, total, ncols, st);
        if (s == SUPERDC_OK) s = cauchy_apply_N(f, total, Ybar, ldy, X_bar, ldxb, ncols, st);
        for (int c0 = 0; c0 < ncols && s == SUPERDC_OK; c0 += BW_C) {
            PROF_LAUNCH("bw_lamlam", st, k_bw_lamlam<<<(unsigned)(nsm * 4), TB, 0, st>>>(
                f.nprob, f.off, tile_off, f.mk, f.dorg, f.eta, f.bnorm, f.pinv, Y, total, Ybar, ldy, c0,
                std::min(BW_C, ncols - c0), u, g));
        }
    }
    PROF_LAUNCH("bw_dz", st, k_bw_dz<<<(unsigned)(nsm * 4), TB, 0, st>>>(
        f.nprob, f.off, tile_off, f.mk, f.dk, f.dorg, f.eta, f.vhat, f.bnorm, f.pinv, lam_bar, u, g, dbs, zbs));
    k_bw_deflate<<<(unsigned)((f.nprob + 127) / 128), 128, 0, st>>>(f.nprob, f.off, f.mk, f.ngiv, f.src, f.pinv,
                                                                    f.giv_ab, f.giv_cs, lam_bar, dbs, zbs, sqrt_rho,
                                                                    d_bar, z_bar);
    cudaError_t e = cudaGetLastError();
    if (s != SUPERDC_OK) return s;
    return e == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}

extern "C" superdc_status superdc_secular_batched_backward(
    int64_t nprob, const int64_t *offsets, int64_t total, double rho, const superdc_rank1_out *fwd,
    const double *lam_bar, int64_t ncols, const double *X, int64_t ldx, const double *Ybar, int64_t ldy,
    double *d_bar, double *z_bar, double *X_bar, int64_t ldxb, cudaStream_t st)
{
    if (nprob < 0 || total < 0 || !(rho > 0.0) || !fwd || ncols < 0 || ncols > 4096) return SUPERDC_ERR_ARG;
    if (nprob == 0 || total == 0) return SUPERDC_OK;
    if (!offsets || !d_bar || !z_bar || !fwd->dk || !fwd->eta || !fwd->vhat || !fwd->bnorm || !fwd->org ||
        !fwd->src || !fwd->perm || !fwd->giv_ab || !fwd->giv_cs || !fwd->mk || !fwd->ngiv)
        return SUPERDC_ERR_ARG;
    if (ncols > 0 && (!X || !Ybar || !X_bar || ldx < total || ldy < total || ldxb < total)) return SUPERDC_ERR_ARG;
    const int nsm = sdc_num_sms();
    int32_t *pinv = nullptr;
    double *dorg = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&pinv, total));
    SDC_CHECK(sc.get(&dorg, total));
    k_prep<<<(unsigned)(nsm * 8), 256, 0, st>>>(nprob, offsets, total, fwd->mk, fwd->perm, fwd->org, fwd->dk, pinv,
                                                 dorg);
    FactorView f;
    f.nprob = nprob; f.off = offsets; f.mk = fwd->mk; f.ngiv = fwd->ngiv; f.dk = fwd->dk; f.eta = fwd->eta;
    f.dorg = dorg; f.vhat = fwd->vhat; f.bnorm = fwd->bnorm; f.src = fwd->src; f.perm = fwd->perm; f.pinv = pinv;
    f.giv_ab = fwd->giv_ab; f.giv_cs = fwd->giv_cs;
#ifdef SUPERDC_CHECK
    f.status = fwd->status;
#endif
    return r1_backward_fv(f, total, lam_bar, (int)ncols, X, ldx, Ybar, ldy, d_bar, z_bar, X_bar, ldxb, sqrt(rho), st);
}

extern "C" superdc_status superdc_rank1_apply(int64_t nprob, const int64_t *offsets, int64_t total,
                                              const superdc_rank1_out *fwd, int32_t trans, int64_t ncols,
                                              const double *X, int64_t ldx, double *Y, int64_t ldy,
                                              const superdc_opts *opts, cudaStream_t st)
{
    superdc_opts def;
    if (!opts) { superdc_opts_default(&def); opts = &def; }
    if (nprob < 0 || total < 0 || !fwd || ncols < 0 || (trans != 0 && trans != 1)) return SUPERDC_ERR_ARG;
    if (nprob == 0 || total == 0 || ncols == 0) return SUPERDC_OK;
    if (!offsets || !X || !Y || ldx < total || ldy < total || !fwd->dk || !fwd->eta || !fwd->vhat ||
        !fwd->bnorm || !fwd->org || !fwd->src || !fwd->perm || !fwd->giv_ab || !fwd->giv_cs || !fwd->mk ||
        !fwd->ngiv)
        return SUPERDC_ERR_ARG;
    const int nsm = sdc_num_sms();
    int32_t *pinv = nullptr;
    double *dorg = nullptr, *Xw = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&pinv, total));
    SDC_CHECK(sc.get(&dorg, total));
    k_prep<<<(unsigned)(nsm * 8), 256, 0, st>>>(nprob, offsets, total, fwd->mk, fwd->perm, fwd->org, fwd->dk, pinv,
                                                 dorg);
    FactorView f;
    f.nprob = nprob; f.off = offsets; f.mk = fwd->mk; f.ngiv = fwd->ngiv; f.dk = fwd->dk; f.eta = fwd->eta;
    f.dorg = dorg; f.vhat = fwd->vhat; f.bnorm = fwd->bnorm; f.src = fwd->src; f.perm = fwd->perm; f.pinv = pinv;
    f.giv_ab = fwd->giv_ab; f.giv_cs = fwd->giv_cs;
#ifdef SUPERDC_CHECK
    f.status = fwd->status;
#endif
    f.fmm_min_m = fmm_resolve(opts->fmm_min_m);
    superdc_status s;
    if (trans) {
        SDC_CHECK(sc.get(&Xw, (size_t)total * ncols));
        SDC_CHECK(cudaMemcpy2DAsync(Xw, total * sizeof(double), X, ldx * sizeof(double), total * sizeof(double),
                                    ncols, cudaMemcpyDeviceToDevice, st));
        s = cauchy_apply_T(f, total, Xw, total, Y, ldy, (int)ncols, st);
    } else {
        s = cauchy_apply_N(f, total, X, ldx, Y, ldy, (int)ncols, st);
    }
    cudaError_t e = cudaGetLastError();
    if (s != SUPERDC_OK) return s;
    return e == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}
