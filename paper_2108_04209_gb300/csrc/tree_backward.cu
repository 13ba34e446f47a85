// superdc_eig_backward: reverse mode of the whole eigendecomposition
// (Algorithms 1-3) for a loss L(lambda, Y = Q^T V).
//
// The forward keeps a tape (opts.tape = 1): the children's eigenvalues and
// W = Q_c^T U_c at every level, the work columns before every rank-one step,
// and the dividing-stage matrices (H, B~, beta = ||B~||_2, its top singular
// pair).  The reverse walks the tree from the root to the leaves:
//   * every rank-one step of a level: the batched adjoint through the secular
//     roots (r1_backward_fv), with the step's remaining work columns and the
//     V columns as the transformed block;
//   * the level build (merge P_p, Zhat_p = [W_c1 B~/sqrt(beta); sqrt(beta) W_c2],
//     X_p = [W_c1 R_c1; W_c2 R_c2]) reversed: cotangents of the children's
//     eigenvalues and W, of B~/sqrt(beta), sqrt(beta) and R;
//   * the leaves: the dense eigen-adjoint of Dhat = Q diag(lambda) Q^T with
//     W = Q^T U and Q^T V, then Dhat = D - U H U^T;
//   * the dividing stage bottom-up: H_c1 = R_c1 H R_c1^T + B~B~^T/beta,
//     H_c2 = R_c2 H R_c2^T + beta I, B~ = B_c1 - R_c1 H R_c2^T, d beta = u1^T dB~ v1.
#include <mutex>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "handles.cuh"
#include "cauchy.cuh"
#include "prof.cuh"

namespace {

__global__ void k_perm_rows(int64_t n, int nl, const int64_t *__restrict__ loff, const int32_t *__restrict__ P,
                            const double *__restrict__ X, int64_t ldx, double *__restrict__ Y, int64_t ldy,
                            int ncols, int scatter)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ncols;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % n;
        const int col = (int)(t / n);
        const int64_t q = sdc_upper_index(loff, (int64_t)nl, x);
        const int64_t src = loff[q] + P[x];
        if (scatter) Y[src + ldy * col] = X[x + ldx * col];
        else         Y[x + ldy * col] = X[src + ldx * col];
    }
}

// level build reversed, per merged row y of node p: cotangents of the
// children's eigenvalue and W rows
__global__ void k_build_bw_rows(int64_t n, int r, int nl, const int64_t *__restrict__ loff,
                                const int32_t *__restrict__ lnodes, int root, const int32_t *__restrict__ lch,
                                const int32_t *__restrict__ rch, const int64_t *__restrict__ size,
                                const double *__restrict__ R, const double *__restrict__ Bts,
                                const double *__restrict__ sqb, const int32_t *__restrict__ P,
                                const double *__restrict__ lamb, const double *__restrict__ WKbar,
                                double *__restrict__ lamb_child, double *__restrict__ Wbar_child)
{
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < n; y += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = sdc_upper_index(loff, (int64_t)nl, y);
        const int64_t o = loff[q];
        const int node = lnodes[q];
        const int c1 = lch[node], c2 = rch[node];
        const int m1 = (int)size[c1];
        const int i = P[y];
        const int64_t x = o + i;
        lamb_child[x] = lamb[y];
        const bool top = i < m1;
        const int rr = r * r;
        const double *Rc = R + (int64_t)(top ? c1 : c2) * rr;
        const double *Bs = Bts + (int64_t)node * rr;
        const double sb = sqb[node];
        for (int a = 0; a < r; a++) {
            double w = 0.0;
            for (int col = 0; col < r; col++) {
                if (top) w += WKbar[y + n * col] * Bs[a + r * col];
                if (node != root) w += WKbar[y + n * (r + col)] * Rc[a + r * col];
            }
            if (!top) w += sb * WKbar[y + n * a];
            Wbar_child[x + n * a] = w;
        }
    }
}

// per node p: Btsbar_p = sum_top W_c1^T Zbar, sqbbar_p = sum_bottom <W_c2, Zbar>,
// gR[c1] += sum_top W_c1^T Xbar, gR[c2] += sum_bottom W_c2^T Xbar
__global__ void k_build_bw_red(int64_t n, int r, const int64_t *__restrict__ loff,
                               const int32_t *__restrict__ lnodes, int root, const int32_t *__restrict__ lch,
                               const int32_t *__restrict__ rch, const int64_t *__restrict__ size,
                               const int32_t *__restrict__ P, const double *__restrict__ Wp,
                               const double *__restrict__ WKbar, double *__restrict__ Btsbar,
                               double *__restrict__ sqbbar, double *__restrict__ gR)
{
    const int q = blockIdx.x;
    const int64_t o = loff[q];
    const int m = (int)(loff[q + 1] - o);
    const int node = lnodes[q];
    const int c1 = lch[node], c2 = rch[node];
    const int m1 = (int)size[c1];
    const int rr = r * r;
    const int nent = 3 * rr + 1;
    for (int e = threadIdx.x; e < nent; e += blockDim.x) {
        const int kind = (e < rr) ? 0 : (e < 2 * rr) ? 1 : (e < 3 * rr) ? 2 : 3;
        const int ee = e - kind * rr;
        const int a = ee % r, col = ee / r;
        if (kind >= 1 && kind <= 2 && node == root) continue;
        double s = 0.0;
        for (int yy = 0; yy < m; yy++) {
            const int64_t y = o + yy;
            const int i = P[y];
            const bool top = i < m1;
            const int64_t x = o + i;
            if (kind == 0 && top) s += Wp[x + n * a] * WKbar[y + n * col];
            else if (kind == 1 && top) s += Wp[x + n * a] * WKbar[y + n * (r + col)];
            else if (kind == 2 && !top) s += Wp[x + n * a] * WKbar[y + n * (r + col)];
            else if (kind == 3 && !top)
                for (int b = 0; b < r; b++) s += Wp[x + n * b] * WKbar[y + n * b];
        }
        if (kind == 0) Btsbar[(int64_t)node * rr + ee] = s;
        else if (kind == 1) gR[(int64_t)c1 * rr + ee] += s;
        else if (kind == 2) gR[(int64_t)c2 * rr + ee] += s;
        else sqbbar[node] = s;
    }
}

// leaf eigen-adjoint, one CTA per leaf; scratch: three m x m blocks per leaf
__global__ void k_leaf_bw(int64_t n, int r, int k, const int64_t *__restrict__ leaf_off,
                          const int64_t *__restrict__ leaf_m, const int64_t *__restrict__ leaf_doff,
                          const int64_t *__restrict__ leaf_uoff, const int32_t *__restrict__ leaf_id,
                          const int64_t *__restrict__ qoff, const double *__restrict__ Qleaf,
                          const double *__restrict__ U, const double *__restrict__ H,
                          const double *__restrict__ lam, const double *__restrict__ lamb,
                          const double *__restrict__ Wbar, const double *__restrict__ V, int64_t ldv,
                          const double *__restrict__ Vbar, double *__restrict__ scratch,
                          double *__restrict__ gD, double *__restrict__ gU, double *__restrict__ gV, int64_t ldgv,
                          double *__restrict__ Hbar)
{
    const int L = blockIdx.x;
    const int m = (int)leaf_m[L];
    const int64_t o = leaf_off[L];
    const double *Q = Qleaf + qoff[L];
    const double *Ul = U + leaf_uoff[L];
    const double *Hl = H + (int64_t)leaf_id[L] * r * r;
    double *S1 = scratch + 3 * qoff[L], *S2 = S1 + (int64_t)m * m, *S3 = S2 + (int64_t)m * m;
    const int T = blockDim.x;
    // S1 = Qbar = U Wbar^T + V Vbar^T
    for (int e = threadIdx.x; e < m * m; e += T) {
        const int i = e % m, j = e / m;
        double s = 0.0;
        for (int a = 0; a < r; a++) s += Ul[i + (int64_t)m * a] * Wbar[o + j + n * a];
        for (int c = 0; c < k; c++) s += V[o + i + ldv * c] * Vbar[o + j + n * c];
        S1[e] = s;
    }
    __syncthreads();
    // S2 = Q^T Qbar
    for (int e = threadIdx.x; e < m * m; e += T) {
        const int i = e % m, j = e / m;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += Q[l + (int64_t)m * i] * S1[l + (int64_t)m * j];
        S2[e] = s;
    }
    __syncthreads();
    // S3 = E = diag(lamb) + sym(F o S2), F_ij = 1/(lambda_j - lambda_i)
    for (int e = threadIdx.x; e < m * m; e += T) {
        const int i = e % m, j = e / m;
        double v;
        if (i == j) v = lamb[o + i];
        else {
            // numerically degenerate pairs form one eigenspace: no coupling
            const double dl = lam[o + j] - lam[o + i];
            const double sc = fmax(fabs(lam[o + i]), fabs(lam[o + j]));
            v = (fabs(dl) > 1e-10 * sc) ? 0.5 * (S2[i + (int64_t)m * j] - S2[j + (int64_t)m * i]) / dl : 0.0;
        }
        S3[e] = v;
    }
    __syncthreads();
    // S1 = Q E
    for (int e = threadIdx.x; e < m * m; e += T) {
        const int i = e % m, j = e / m;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += Q[i + (int64_t)m * l] * S3[l + (int64_t)m * j];
        S1[e] = s;
    }
    __syncthreads();
    // S2 = Dhat_bar = (Q E) Q^T  -> gD
    double *gDl = gD + leaf_doff[L];
    for (int e = threadIdx.x; e < m * m; e += T) {
        const int i = e % m, j = e / m;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += S1[i + (int64_t)m * l] * Q[j + (int64_t)m * l];
        S2[e] = s;
        gDl[e] = s;
    }
    __syncthreads();
    // S3 (m x r) = Dbar U; gU = Q Wbar - 2 (Dbar U) H; gV = Q Vbar
    for (int e = threadIdx.x; e < m * r; e += T) {
        const int i = e % m, a = e / m;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += S2[i + (int64_t)m * l] * Ul[l + (int64_t)m * a];
        S3[e] = s;
    }
    __syncthreads();
    double *gUl = gU + leaf_uoff[L];
    for (int e = threadIdx.x; e < m * r; e += T) {
        const int i = e % m, a = e / m;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += Q[i + (int64_t)m * l] * Wbar[o + l + n * a];
        double t = 0.0;
        for (int b = 0; b < r; b++) t += S3[i + (int64_t)m * b] * Hl[b + r * a];
        gUl[e] = s - 2.0 * t;
    }
    for (int e = threadIdx.x; e < m * k; e += T) {
        const int i = e % m, c = e / m;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += Q[i + (int64_t)m * l] * Vbar[o + l + n * c];
        gV[o + i + ldgv * c] = s;
    }
    // Hbar_leaf = -U^T Dbar U
    for (int e = threadIdx.x; e < r * r; e += T) {
        const int a = e % r, b = e / r;
        double s = 0.0;
        for (int l = 0; l < m; l++) s += Ul[l + (int64_t)m * a] * S3[l + (int64_t)m * b];
        Hbar[(int64_t)leaf_id[L] * r * r + e] = -s;
    }
}

// dividing stage reversed for the non-leaf nodes of one level (bottom-up)
__global__ void k_divide_bw(const int32_t *__restrict__ nodes, int root, int r, const int32_t *__restrict__ lch,
                            const int32_t *__restrict__ rch, const double *__restrict__ R,
                            const double *__restrict__ H, const double *__restrict__ Bt,
                            const double *__restrict__ beta, const double *__restrict__ u1,
                            const double *__restrict__ v1, const double *__restrict__ Btsbar,
                            const double *__restrict__ sqbbar, double *__restrict__ Hbar,
                            double *__restrict__ gR, double *__restrict__ gB)
{
    extern __shared__ double sm[];
    const int rr = r * r;
    double *A1 = sm, *A2 = sm + rr, *Hx = sm + 2 * rr, *R1 = sm + 3 * rr, *R2 = sm + 4 * rr, *Bb = sm + 5 * rr,
           *Bs = sm + 6 * rr, *T1 = sm + 7 * rr, *T2 = sm + 8 * rr;
    __shared__ double s_bb;
    const int x = nodes[blockIdx.x];
    const int c1 = lch[x], c2 = rch[x];
    const bool isroot = (x == root);
    const double bet = beta[x];
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int a = e % r, b = e / r;
        // symmetric parts of the children's H cotangents
        A1[e] = Hbar[(int64_t)c1 * rr + e] + Hbar[(int64_t)c1 * rr + b + r * a];
        A2[e] = Hbar[(int64_t)c2 * rr + e] + Hbar[(int64_t)c2 * rr + b + r * a];
        Hx[e] = isroot ? 0.0 : H[(int64_t)x * rr + e];
        R1[e] = isroot ? 0.0 : R[(int64_t)c1 * rr + e];
        R2[e] = isroot ? 0.0 : R[(int64_t)c2 * rr + e];
        Bb[e] = Bt[(int64_t)x * rr + e];
        Bs[e] = Btsbar[(int64_t)x * rr + e];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // beta_bar = -<H1bar, B B^T>/beta^2 + tr(H2bar) - 1/2 <Btsbar, B> beta^-3/2 + sqbbar/(2 sqrt(beta))
        double bb = 0.0;
        if (bet > 0) {
            double hbb = 0.0, tr2 = 0.0, sb = 0.0;
            for (int a = 0; a < r; a++) {
                tr2 += Hbar[(int64_t)c2 * rr + a + r * a];
                for (int b = 0; b < r; b++) {
                    double bbt = 0.0;
                    for (int c = 0; c < r; c++) bbt += Bb[a + r * c] * Bb[b + r * c];
                    hbb += Hbar[(int64_t)c1 * rr + a + r * b] * bbt;
                    sb += Bs[a + r * b] * Bb[a + r * b];
                }
            }
            bb = -hbb / (bet * bet) + tr2 - 0.5 * sb / (bet * sqrt(bet)) + sqbbar[x] / (2.0 * sqrt(bet));
        }
        s_bb = bb;
    }
    __syncthreads();
    const double bbar = s_bb;
    // Btbar = (H1bar + H1bar^T) B / beta + Btsbar / sqrt(beta) + beta_bar u1 v1^T  -> T1
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int a = e % r, b = e / r;
        double s = 0.0;
        if (bet > 0) {
            for (int c = 0; c < r; c++) s += A1[a + r * c] * Bb[c + r * b];
            s = s / bet + Bs[e] / sqrt(bet) + bbar * u1[(int64_t)x * r + a] * v1[(int64_t)x * r + b];
        }
        T1[e] = s;
        gB[(int64_t)c1 * rr + e] = s;
    }
    __syncthreads();
    if (isroot) return;
    // gR[c1] += A1 R1 Hx - Btbar R2 Hx ; gR[c2] += A2 R2 Hx - Btbar^T R1 Hx ;
    // Hbar[x] = R1^T H1bar R1 + R2^T H2bar R2 - R1^T Btbar R2   (H symmetric)
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {       // T2 = R1 Hx, Bs <- R2 Hx
        const int a = e % r, b = e / r;
        double s1 = 0.0, s2 = 0.0;
        for (int c = 0; c < r; c++) { s1 += R1[a + r * c] * Hx[c + r * b]; s2 += R2[a + r * c] * Hx[c + r * b]; }
        T2[e] = s1;
        Bs[e] = s2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int a = e % r, b = e / r;
        double g1 = 0.0, g2 = 0.0, hb = 0.0;
        for (int c = 0; c < r; c++) {
            g1 += A1[a + r * c] * T2[c + r * b] - T1[a + r * c] * Bs[c + r * b];
            g2 += A2[a + r * c] * Bs[c + r * b] - T1[c + r * a] * T2[c + r * b];
        }
        for (int c = 0; c < r; c++)
            for (int d = 0; d < r; d++) {
                hb += R1[c + r * a] * Hbar[(int64_t)c1 * rr + c + r * d] * R1[d + r * b];
                hb += R2[c + r * a] * Hbar[(int64_t)c2 * rr + c + r * d] * R2[d + r * b];
                hb -= R1[c + r * a] * T1[c + r * d] * R2[d + r * b];
            }
        gR[(int64_t)c1 * rr + e] += g1;
        gR[(int64_t)c2 * rr + e] += g2;
        Hbar[(int64_t)x * rr + e] = hb;
    }
}

}  // namespace

namespace {
// dynamic shared memory of k_divide_bw above the 48 KiB default (9 r^2
// doubles: 72 KiB at the largest rank), once per device
cudaError_t divide_bw_attr()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        e = cudaFuncSetAttribute(k_divide_bw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(9 * 32 * 32 * sizeof(double)));
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}
}  // namespace

extern "C" superdc_status superdc_eig_backward(const superdc_hss *h, const superdc_eigfact *f,
                                               const double *lam_bar, int64_t k, const double *V, int64_t ldv,
                                               const double *Ybar, int64_t ldy, double *gD, double *gU,
                                               double *gR, double *gB, double *gV, int64_t ldgv, cudaStream_t st)
{
    if (!h || !f || f->h != h || !gD || !gU || !gR || !gB || k < 0 || k > 1024) return SUPERDC_ERR_ARG;
    if (!f->tape.on) return SUPERDC_ERR_STATE;
    const int64_t n = f->n;
    if (k > 0 && (!V || !Ybar || !gV || ldv < n || ldy < n || ldgv < n)) return SUPERDC_ERR_ARG;
    const int r = f->r, lmax = f->lmax, rr = r * r, nn = h->nnodes;
    const int kc = (int)k;
    const int nsm = sdc_num_sms();
    const unsigned g = (unsigned)(nsm * 8);
    const Tape &T = f->tape;
    if (divide_bw_attr() != cudaSuccess) return SUPERDC_ERR_CUDA;
    std::vector<void *> tmp;
    auto alloc = [&](auto **p, size_t cnt) -> cudaError_t {
        cudaError_t e = sdc_alloc(p, cnt, st);
        if (e == cudaSuccess) tmp.push_back((void *)*p);
        return e;
    };
    auto release = [&]() { for (auto p : tmp) cudaFreeAsync(p, st); tmp.clear(); };
#define BW_CHECK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { release(); \
        return e_ == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA; } } while (0)
    // ---- V tape: values of the V columns before every factor (apply_Q with snapshots)
    std::vector<std::vector<double *>> Vb(lmax, std::vector<double *>(r, nullptr));
    double *B0 = nullptr, *B1 = nullptr;
    int64_t dsz = 0, usz = 0;
    for (int L : h->leaves) { dsz += h->size[L] * h->size[L]; usz += h->size[L] * r; }
    if (kc > 0) {
        BW_CHECK(alloc(&B0, (size_t)n * kc));
        BW_CHECK(alloc(&B1, (size_t)n * kc));
        for (int l = 0; l < lmax; l++)
            for (int j = 0; j < r; j++) BW_CHECK(alloc(&Vb[l][j], (size_t)n * kc));
    }
    double *lamb = nullptr, *dbar = nullptr, *zbar = nullptr, *WKbar = nullptr, *Xs = nullptr, *Ys = nullptr,
           *Xb = nullptr, *Wbar = nullptr, *Vbar = nullptr, *Vbar2 = nullptr, *lamb2 = nullptr, *Btsbar = nullptr,
           *sqbbar = nullptr, *Hbar = nullptr, *scr = nullptr;
    BW_CHECK(alloc(&lamb, n));
    BW_CHECK(alloc(&lamb2, n));
    BW_CHECK(alloc(&dbar, n));
    BW_CHECK(alloc(&zbar, n));
    BW_CHECK(alloc(&WKbar, (size_t)n * 2 * r));
    BW_CHECK(alloc(&Wbar, (size_t)n * r));
    const int cmax = 2 * r + kc;
    BW_CHECK(alloc(&Xs, (size_t)n * cmax));
    BW_CHECK(alloc(&Ys, (size_t)n * cmax));
    BW_CHECK(alloc(&Xb, (size_t)n * cmax));
    BW_CHECK(alloc(&Vbar, (size_t)n * (kc > 0 ? kc : 1)));
    BW_CHECK(alloc(&Vbar2, (size_t)n * (kc > 0 ? kc : 1)));
    BW_CHECK(alloc(&Btsbar, (size_t)nn * rr));
    BW_CHECK(alloc(&sqbbar, nn));
    BW_CHECK(alloc(&Hbar, (size_t)nn * rr));
    BW_CHECK(alloc(&scr, (size_t)3 * dsz));
    BW_CHECK(cudaMemsetAsync(gR, 0, (size_t)nn * rr * sizeof(double), st));
    BW_CHECK(cudaMemsetAsync(gB, 0, (size_t)nn * rr * sizeof(double), st));
    BW_CHECK(cudaMemsetAsync(Btsbar, 0, (size_t)nn * rr * sizeof(double), st));
    BW_CHECK(cudaMemsetAsync(sqbbar, 0, nn * sizeof(double), st));
    BW_CHECK(cudaMemsetAsync(Hbar, 0, (size_t)nn * rr * sizeof(double), st));
    BW_CHECK(cudaMemsetAsync(WKbar, 0, (size_t)n * 2 * r * sizeof(double), st));
    if (lam_bar) BW_CHECK(cudaMemcpyAsync(lamb, lam_bar, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else BW_CHECK(cudaMemsetAsync(lamb, 0, n * sizeof(double), st));
    superdc_status s = SUPERDC_OK;
    if (kc > 0) {
        // forward of the V columns with snapshots
        s = leaves_apply(f, 1, kc, V, ldv, B0, n, st);
        for (int l = lmax - 1; l >= 0 && s == SUPERDC_OK; l--) {
            const int nl = (int)h->lev_nodes[l].size();
            k_perm_rows<<<g, 256, 0, st>>>(n, nl, h->d_lev_off[l], f->P[l], B0, n, B1, n, kc, 0);
            std::swap(B0, B1);
            for (int j = 0; j < r && s == SUPERDC_OK; j++) {
                BW_CHECK(cudaMemcpyAsync(Vb[l][j], B0, (size_t)n * kc * sizeof(double), cudaMemcpyDeviceToDevice, st));
                s = cauchy_apply_T(factor_view(f, l, j), n, B0, n, B1, n, kc, st);
                std::swap(B0, B1);
            }
        }
        BW_CHECK(cudaMemcpy2DAsync(Vbar, n * sizeof(double), Ybar, ldy * sizeof(double), n * sizeof(double), kc,
                                   cudaMemcpyDeviceToDevice, st));
    }
    // ---- reverse over the levels, root first
    for (int l = 0; l < lmax && s == SUPERDC_OK; l++) {
        const int nl = (int)h->lev_nodes[l].size();
        const int ctot = (l == 0) ? r : 2 * r;
        for (int j = r - 1; j >= 0 && s == SUPERDC_OK; j--) {
            const int c = ctot - j - 1;
            const int cw = c + kc;
            // transformed block: remaining work columns (before the step) and the V columns
            if (c > 0)
                BW_CHECK(cudaMemcpyAsync(Xs, T.WKb[l][j] + n, (size_t)n * c * sizeof(double), cudaMemcpyDeviceToDevice,
                                         st));
            if (kc > 0)
                BW_CHECK(cudaMemcpyAsync(Xs + (size_t)n * c, Vb[l][j], (size_t)n * kc * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
            if (c > 0)
                BW_CHECK(cudaMemcpyAsync(Ys, WKbar + (size_t)n * (j + 1), (size_t)n * c * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
            if (kc > 0)
                BW_CHECK(cudaMemcpyAsync(Ys + (size_t)n * c, Vbar, (size_t)n * kc * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
            s = r1_backward_fv(factor_view(f, l, j), n, lamb, cw, Xs, n, Ys, n, dbar, zbar, Xb, n, 1.0, st);
            if (s != SUPERDC_OK) break;
            BW_CHECK(cudaMemcpyAsync(lamb, dbar, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            BW_CHECK(cudaMemcpyAsync(WKbar + (size_t)n * j, zbar, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            if (c > 0)
                BW_CHECK(cudaMemcpyAsync(WKbar + (size_t)n * (j + 1), Xb, (size_t)n * c * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
            if (kc > 0)
                BW_CHECK(cudaMemcpyAsync(Vbar, Xb + (size_t)n * c, (size_t)n * kc * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
        }
        if (s != SUPERDC_OK) break;
        // level build reversed
        PROF_LAUNCH("build_bw", st, k_build_bw_rows<<<g, 256, 0, st>>>(
            n, r, nl, h->d_lev_off[l], h->d_lev_nodes[l], nn - 1, h->d_lch, h->d_rch, h->d_size, h->R, T.Bts, T.sqb,
            f->P[l], lamb, WKbar, lamb2, Wbar));
        k_build_bw_red<<<(unsigned)nl, 128, 0, st>>>(n, r, h->d_lev_off[l], h->d_lev_nodes[l], nn - 1, h->d_lch,
                                                     h->d_rch, h->d_size, f->P[l], T.Wprev[l], WKbar, Btsbar, sqbbar,
                                                     gR);
        if (kc > 0) {
            k_perm_rows<<<g, 256, 0, st>>>(n, nl, h->d_lev_off[l], f->P[l], Vbar, n, Vbar2, n, kc, 1);
            std::swap(Vbar, Vbar2);
        }
        std::swap(lamb, lamb2);
        BW_CHECK(cudaMemsetAsync(WKbar, 0, (size_t)n * r * sizeof(double), st));
        BW_CHECK(cudaMemcpyAsync(WKbar + (size_t)n * r, Wbar, (size_t)n * r * sizeof(double), cudaMemcpyDeviceToDevice,
                                 st));
    }
    if (s != SUPERDC_OK) { release(); return s; }
    // ---- leaves
    PROF_LAUNCH("leaf_bw", st, k_leaf_bw<<<(unsigned)h->nleaves, 256, 0, st>>>(
        n, r, kc, h->d_leaf_off, h->d_leaf_m, h->d_leaf_doff, h->d_leaf_uoff, h->d_leaf_id, f->d_qoff, f->Qleaf, h->U,
        T.H, T.lam_prev[lmax - 1], lamb, WKbar + (size_t)n * r, V, ldv, Vbar, scr, gD, gU, gV, ldgv, Hbar));
    // ---- dividing stage, bottom-up
    for (int l = lmax - 1; l >= 0; l--) {
        std::vector<int> nodes;
        for (int i : h->lev_nodes[l]) if (h->lch[i] >= 0) nodes.push_back(i);
        if (nodes.empty()) continue;
        PROF_LAUNCH("divide_bw", st, k_divide_bw<<<(unsigned)nodes.size(), 128, 9 * rr * sizeof(double), st>>>(
            h->d_lev_nodes[l], nn - 1, r, h->d_lch, h->d_rch, h->R, T.H, T.Bt, T.beta, T.u1, T.v1, Btsbar, sqbbar,
            Hbar, gR, gB));
    }
    cudaError_t e = cudaGetLastError();
    release();
#undef BW_CHECK
    return e == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}
