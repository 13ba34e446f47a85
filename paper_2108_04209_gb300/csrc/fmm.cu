// Triangular FMM with local shifting on sm_103a (Sections 4.1.2, 4.2.2, 4.3).
//
// Geometry.  The kept poles d_0 < ... < d_{m-1} of a problem and the targets
// (roots x_k in (d_k, d_{k+1}), eigenvalues lambda_j, or the poles themselves)
// interlace (eq. (4.4)), so one index-based binary tree serves both: a leaf
// box holds FMM_B consecutive indices (d_k and x_k of the same k always share
// a box, the paper's first design point) and every box carries the interval
// [d_{i0}, d_{i1}] of its points (the last box ends at d_{m-1}).  The index
// split adapts the boxes to clustered spectra (second design point); whether
// two boxes interact through expansions is decided geometrically: boxes S, T
// of one level are admissible when their gap is at least FMM_KAPPA times the
// larger width.  Near lists are built top-down (children of the parent's near
// list that are not admissible).  A box whose list would exceed FMM_NCAP (a
// box straddling a wide gap of the spectrum is close to everything) is marked
// "all near", and so is its subtree: the targets of such leaves are summed
// directly over every source, the other leaves keep the expansions.  Only the last eigenvalue
// lambda_{m-1} lies outside the tree (to the right of d_{m-1}): as a target it
// is summed directly, as a source it is added directly to every target.
//
// Expansions.  Chebyshev interpolation with FMM_P first-kind nodes per box:
// source moments M_n = sum_j w_j T_n(u_j) of the leaf boxes, translated
// exactly to the parents (T_n(alpha u + beta) expands in T_0..T_n), node
// weights W_q = sum_j w_j L_q(u_j) from the moments; every leaf box receives
// the kernel sums of all boxes admissible to it or to one of its ancestors
// (while the ancestor's parent was not) at its own Chebyshev nodes, converted
// to Chebyshev coefficients and evaluated at the targets by Clenshaw.  Work is
// O(m P^2 log m / FMM_B) for the far field plus O(m FMM_B) for the near field.
//
// Triangularity.  A far box lies entirely to the left or right of the target
// box in index order, so its sums go to the lower (psi, C_L w, S_L w) or the
// upper (phi, C_U w, S_U w) part; inside the near field the split is by index
// as in the direct evaluator (eq. (4.10)).
//
// Local shifting.  Near-field terms use the shifted differences of eqs.
// (4.14)/(4.28) exactly as the direct kernels; far-field terms use the plain
// positions x = d_K + y and lambda_j = d_{K_j} + eta_j (eq. (4.21)), which is
// accurate there because far points are separated by at least a box width.
//
// Because the poles and weights of a secular equation do not change during
// the iteration and every root stays inside its bracket, the far-field
// expansions on the leaf boxes' (fixed) intervals are computed once per
// problem; each sweep costs a near-field pass plus one Clenshaw evaluation.
#include <algorithm>
#include "common.cuh"
#include "fmm.cuh"
#include "secular.cuh"
#include "prof.cuh"

namespace {

constexpr int P = FMM_P;
constexpr int B = FMM_B;
constexpr double FMM_KAPPA = 1.0;
constexpr int WMAX = 32;          // widest moment / coefficient block (columns)

// ---------------------------------------------------------------------------
// tree shape of a problem with m kept indices: nb0 = ceil(m / B) leaf boxes,
// level l has ceil(nb0 / 2^l) boxes, the top level one box; boxes of a problem
// are stored level by level from the leaves up.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int lev_nb(int nb0, int l) { return ((nb0 - 1) >> l) + 1; }

__host__ __device__ __forceinline__ int lev_count(int nb0)
{
    int L = 1;
    while (lev_nb(nb0, L - 1) > 1) L++;
    return L;
}

__host__ __device__ __forceinline__ int lev_base(int nb0, int l)
{
    int s = 0;
    for (int i = 0; i < l; i++) s += lev_nb(nb0, i);
    return s;
}

__device__ __forceinline__ bool fmm_cand(int m, int min_m) { return min_m > 0 && m >= min_m && m >= 4 * B; }

__device__ __forceinline__ void box_range(int m, int l, int b, int &i0, int &i1)
{
    const int64_t span = (int64_t)B << l;
    const int64_t a = (int64_t)b * span;
    i0 = (int)a;
    i1 = (int)std::min<int64_t>((int64_t)m, a + span);
}

__device__ __forceinline__ void box_ch(double lo, double hi, double &c, double &h)
{
    c = 0.5 * (lo + hi);
    h = 0.5 * (hi - lo);
    if (!(h > 0.0)) h = fmax(fabs(c) * 1e-15, 1e-300);
}

__device__ __forceinline__ bool adm(double loS, double hiS, double loT, double hiT)
{
    double gap;
    if (hiS <= loT) gap = loT - hiS;
    else if (hiT <= loS) gap = loS - hiT;
    else return false;
    return gap > 0.0 && gap >= FMM_KAPPA * fmax(hiS - loS, hiT - loT);
}

// near list of a leaf box: nn >= 0 entries, or (nn < 0) every leaf box
__device__ __forceinline__ int near_len(int nn, int nb0) { return nn < 0 ? nb0 : nn; }
__device__ __forceinline__ int near_box(const int32_t *__restrict__ near, int64_t g, int nn, int i)
{
    return nn < 0 ? i : near[g * FMM_NCAP + i];
}

// Chebyshev nodes x_q = cos((2q+1) pi / 2P) and T_n(x_q) (Tx[q * P + n])
__device__ void cheb_tables(double *xq, double *Tx)
{
    for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
        const int q = t / P, n = t % P;
        Tx[t] = cospi((double)(n * (2 * q + 1)) / (2.0 * P));
    }
    for (int q = threadIdx.x; q < P; q += blockDim.x) xq[q] = cospi((double)(2 * q + 1) / (2.0 * P));
}

// Clenshaw evaluation of sum_n a_n T_n(u)
__device__ __forceinline__ double clenshaw(const double *__restrict__ a, double u)
{
    const double u2 = u + u;
    double b1 = 0.0, b2 = 0.0;
#pragma unroll 4
    for (int n = P - 1; n >= 1; n--) {
        const double b0 = fma(u2, b1, a[n] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(u, b1, a[0] - b2);
}

// ---------------------------------------------------------------------------
// Plan: which problems take the FMM path, and the prefix of their boxes.
// ---------------------------------------------------------------------------
__global__ void k_fmm_plan(int64_t nprob, const int32_t *__restrict__ mk, int min_m, int64_t cap_boxes,
                           int64_t cap_leaves, int64_t cap_f, int64_t *__restrict__ box_base,
                           int64_t *__restrict__ leaf_base, int32_t *__restrict__ fslot,
                           int32_t *__restrict__ fprob, int32_t *__restrict__ nfmm)
{
    __shared__ int64_t sb[1024], sl[1024];
    __shared__ int sf[1024];
    __shared__ int ok;
    const int T = blockDim.x;
    const int64_t per = (nprob + T - 1) / T;
    const int64_t beg = std::min<int64_t>(nprob, (int64_t)threadIdx.x * per);
    const int64_t end = std::min<int64_t>(nprob, beg + per);
    int64_t nbx = 0, nlf = 0;
    int nf = 0;
    for (int64_t p = beg; p < end; p++) {
        const int m = mk[p];
        if (!fmm_cand(m, min_m)) continue;
        const int nb0 = (m + B - 1) / B;
        nbx += lev_base(nb0, lev_count(nb0));
        nlf += nb0;
        nf++;
    }
    sb[threadIdx.x] = nbx;
    sl[threadIdx.x] = nlf;
    sf[threadIdx.x] = nf;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t ab = 0, al = 0;
        int af = 0;
        for (int i = 0; i < T; i++) {
            int64_t vb = sb[i], vl = sl[i];
            int vf = sf[i];
            sb[i] = ab; sl[i] = al; sf[i] = af;
            ab += vb; al += vl; af += vf;
        }
        ok = (ab <= cap_boxes && al <= cap_leaves && af <= cap_f) ? 1 : 0;
        box_base[nprob] = ok ? ab : 0;
        leaf_base[nprob] = ok ? al : 0;
        *nfmm = ok ? af : 0;
    }
    __syncthreads();
    int64_t ab = ok ? sb[threadIdx.x] : 0, al = ok ? sl[threadIdx.x] : 0;
    int af = ok ? sf[threadIdx.x] : 0;
    for (int64_t p = beg; p < end; p++) {
        box_base[p] = ab;
        leaf_base[p] = al;
        const int m = mk[p];
        if (ok && fmm_cand(m, min_m)) {
            const int nb0 = (m + B - 1) / B;
            fslot[p] = af;
            fprob[af] = (int32_t)p;
            ab += lev_base(nb0, lev_count(nb0));
            al += nb0;
            af++;
        } else {
            fslot[p] = -1;
        }
    }
}

// Box intervals and near lists, one CTA per problem, top level first.
__global__ void __launch_bounds__(256)
k_fmm_tree(int64_t nprob, const int64_t *__restrict__ off, const int32_t *__restrict__ mk,
           const double *__restrict__ dk, const int64_t *__restrict__ box_base, int32_t *__restrict__ fslot,
           double *__restrict__ blo, double *__restrict__ bhi, int32_t *__restrict__ nnear,
           int32_t *__restrict__ near, int32_t *__restrict__ used)
{
    for (int64_t p = blockIdx.x; p < nprob; p += gridDim.x) {
        if (fslot[p] < 0) continue;
        const int m = mk[p];
        const double *d = dk + off[p];
        const int64_t g0 = box_base[p];
        const int nb0 = (m + B - 1) / B;
        const int L = lev_count(nb0);
        for (int l = L - 1; l >= 0; l--) {
            const int nb = lev_nb(nb0, l);
            const int64_t gb = g0 + lev_base(nb0, l);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int i0, i1;
                box_range(m, l, b, i0, i1);
                blo[gb + b] = d[i0];
                bhi[gb + b] = (i1 < m) ? d[i1] : d[m - 1];
            }
            __syncthreads();
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int cnt = 0;
                if (l == L - 1) {
                    near[(gb + b) * FMM_NCAP] = b;
                    cnt = 1;
                } else {
                    const int64_t gp = g0 + lev_base(nb0, l + 1) + (b >> 1);
                    const int npn = nnear[gp];
                    if (npn < 0) {
                        cnt = -1;                                  // parent: all near
                    } else {
                        const double loT = blo[gb + b], hiT = bhi[gb + b];
                        for (int i = 0; i < npn && cnt >= 0; i++) {
                            const int s = near[gp * FMM_NCAP + i];
                            for (int S = 2 * s; S <= 2 * s + 1 && S < nb; S++) {
                                if (S != b && adm(blo[gb + S], bhi[gb + S], loT, hiT)) continue;
                                if (cnt == FMM_NCAP) { cnt = -1; break; }   // overflow: all near
                                near[(gb + b) * FMM_NCAP + cnt] = S;
                                cnt++;
                            }
                        }
                    }
                }
                nnear[gb + b] = cnt;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && used) used[p] = 1;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sources of the five sums
// ---------------------------------------------------------------------------
enum { M_SEC = 0, M_BN = 1, M_LOW = 2, M_CT = 3, M_CN = 4 };

struct SrcArgs {
    const int64_t *off;
    const int32_t *mk;
    const double *dk, *zk, *vhat, *bnorm, *dorg, *eta;
    const int32_t *src, *pinv;
    const double *X;
    int64_t ldx;
    int col0, nc;
};

// leaf moments and node weights
//   M_SEC: w_j = z_j^2 at d_j            M_BN: w_i = vhat_i^2 at d_i
//   M_LOW: +1 at lambda_j, -1 at d_j (j < m-1; Chebyshev differences of the pair)
//   M_CT:  vhat_i x_{src_i} at d_i       M_CN: b_j x_{pinv_j} at lambda_j (j < m-1)
template <int MODE>
__global__ void __launch_bounds__(B) k_fmm_leafmom(FmmDev pl, SrcArgs a)
{
    __shared__ double Tt[B][P + 1];
    __shared__ double Wt[B][WMAX + 1];
    __shared__ double Ms[P][WMAX + 1];
    __shared__ double Tx[P * P], xq[P];
    cheb_tables(xq, Tx);
    const int nw = (MODE == M_CT || MODE == M_CN) ? a.nc : 1;
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = blockIdx.x; gl < nleaf; gl += gridDim.x) {
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = a.off[p];
        const int m = a.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        double c, h;
        box_ch(pl.blo[g], pl.bhi[g], c, h);
        const int j = Tb * B + tid;
        const int jend = (MODE == M_LOW || MODE == M_CN) ? m - 1 : m;
        const bool act = j < jend;
        __syncthreads();
        if (MODE == M_LOW) {
            // D_n = T_n(b) - T_n(a) with b = a + delta, by the recurrence
            // D_{n+1} = 2 delta T_n(b) + 2 a D_n - D_{n-1} (no cancellation)
            double av = 0.0, dl = 0.0;
            if (act) {
                av = (a.dk[b0 + j] - c) / h;
                dl = ((a.dorg[b0 + j] - a.dk[b0 + j]) + a.eta[b0 + j]) / h;
            }
            const double bv = av + dl;
            double tb0 = 1.0, tb1 = bv, D0 = 0.0, D1 = dl;
            Tt[tid][0] = 0.0;
            Tt[tid][1] = D1;
            for (int n = 1; n < P - 1; n++) {
                const double D2 = 2.0 * dl * tb1 + 2.0 * av * D1 - D0;
                const double tb2 = 2.0 * bv * tb1 - tb0;
                Tt[tid][n + 1] = D2;
                D0 = D1; D1 = D2; tb0 = tb1; tb1 = tb2;
            }
            Wt[tid][0] = act ? 1.0 : 0.0;
        } else {
            double u = 0.0;
            if (act) {
                const double s = (MODE == M_CN) ? a.dorg[b0 + j] + a.eta[b0 + j] : a.dk[b0 + j];
                u = (s - c) / h;
            }
            double t0 = 1.0, t1 = u;
            Tt[tid][0] = 1.0;
            Tt[tid][1] = u;
            for (int n = 2; n < P; n++) {
                const double t2 = 2.0 * u * t1 - t0;
                Tt[tid][n] = t2;
                t0 = t1; t1 = t2;
            }
            if (MODE == M_SEC) {
                const double z = act ? a.zk[b0 + j] : 0.0;
                Wt[tid][0] = z * z;
            } else if (MODE == M_BN) {
                const double v = act ? a.vhat[b0 + j] : 0.0;
                Wt[tid][0] = v * v;
            } else if (MODE == M_CT) {
                const double v = act ? a.vhat[b0 + j] : 0.0;
                const int64_t row = act ? b0 + a.src[b0 + j] : 0;
                for (int q = 0; q < nw; q++) Wt[tid][q] = act ? v * a.X[row + (int64_t)(a.col0 + q) * a.ldx] : 0.0;
            } else {
                const double bj = act ? a.bnorm[b0 + j] : 0.0;
                const int64_t row = act ? b0 + a.pinv[b0 + j] : 0;
                for (int q = 0; q < nw; q++) Wt[tid][q] = act ? bj * a.X[row + (int64_t)(a.col0 + q) * a.ldx] : 0.0;
            }
        }
        __syncthreads();
        for (int t = tid; t < P * nw; t += B) {
            const int n = t / nw, q = t % nw;
            double s = 0.0;
            for (int jj = 0; jj < B; jj++) s = fma(Tt[jj][n], Wt[jj][q], s);
            Ms[n][q] = s;
            pl.M[(g * P + n) * pl.ncol + q] = s;
        }
        __syncthreads();
        for (int t = tid; t < P * nw; t += B) {
            const int qn = t / nw, q = t % nw;
            double s = Ms[0][q];
            for (int n = 1; n < P; n++) s = fma(2.0 * Tx[qn * P + n], Ms[n][q], s);
            pl.W[(g * P + qn) * pl.ncol + q] = s / P;
        }
    }
}

// moments of the boxes of level l from their children (exact translation)
__global__ void __launch_bounds__(128) k_fmm_m2m(FmmDev pl, const int32_t *__restrict__ mk, int l, int nw)
{
    __shared__ double A[P][P + 1];
    __shared__ double Mc[P][WMAX + 1];
    __shared__ double Ms[P][WMAX + 1];
    __shared__ double Tx[P * P], xq[P];
    cheb_tables(xq, Tx);
    const int tid = threadIdx.x;
    const int64_t nbox = pl.box_base[pl.nprob];
    for (int64_t g = blockIdx.x; g < nbox; g += gridDim.x) {
        const int64_t p = sdc_upper_index(pl.box_base, pl.nprob, g);
        if (pl.fslot[p] < 0) continue;
        const int m = mk[p];
        const int nb0 = (m + B - 1) / B;
        if (l >= lev_count(nb0)) continue;
        const int64_t local = g - pl.box_base[p];
        const int lb = lev_base(nb0, l), nbl = lev_nb(nb0, l);
        if (local < lb || local >= lb + nbl) continue;
        const int b = (int)(local - lb);
        double cP, hP;
        box_ch(pl.blo[g], pl.bhi[g], cP, hP);
        __syncthreads();
        for (int t = tid; t < P * nw; t += blockDim.x) Ms[t / nw][t % nw] = 0.0;
        const int nbc = lev_nb(nb0, l - 1);
        const int64_t gcb = pl.box_base[p] + lev_base(nb0, l - 1);
        for (int ci = 0; ci < 2; ci++) {
            const int cb = 2 * b + ci;
            if (cb >= nbc) break;
            const int64_t gc = gcb + cb;
            double cc, hc;
            box_ch(pl.blo[gc], pl.bhi[gc], cc, hc);
            const double al = hc / hP, be = (cc - cP) / hP;
            __syncthreads();
            for (int t = tid; t < P * nw; t += blockDim.x)
                Mc[t / nw][t % nw] = pl.M[(gc * P + t / nw) * pl.ncol + t % nw];
            if (tid < P) {
                A[0][tid] = (tid == 0) ? 1.0 : 0.0;
                A[1][tid] = (tid == 0) ? be : ((tid == 1) ? al : 0.0);
            }
            __syncthreads();
            // T_{n+1}(v) = 2 v T_n(v) - T_{n-1}(v), v = al u + be, in coefficient space
            for (int n = 1; n < P - 1; n++) {
                if (tid < P) {
                    const int k = tid;
                    double U;
                    if (k == 0) U = 0.5 * A[n][1];
                    else if (k == 1) U = A[n][0] + 0.5 * A[n][2];
                    else U = 0.5 * (A[n][k - 1] + ((k + 1 < P) ? A[n][k + 1] : 0.0));
                    A[n + 1][k] = 2.0 * (al * U + be * A[n][k]) - A[n - 1][k];
                }
                __syncthreads();
            }
            for (int t = tid; t < P * nw; t += blockDim.x) {
                const int n = t / nw, q = t % nw;
                double s = 0.0;
                for (int k = 0; k <= n; k++) s = fma(A[n][k], Mc[k][q], s);
                Ms[n][q] += s;
            }
        }
        __syncthreads();
        for (int t = tid; t < P * nw; t += blockDim.x) pl.M[(g * P + t / nw) * pl.ncol + t % nw] = Ms[t / nw][t % nw];
        for (int t = tid; t < P * nw; t += blockDim.x) {
            const int qn = t / nw, q = t % nw;
            double s = Ms[0][q];
            for (int n = 1; n < P; n++) s = fma(2.0 * Tx[qn * P + n], Ms[n][q], s);
            pl.W[(g * P + qn) * pl.ncol + q] = s / P;
        }
    }
}

// far-field sums at the Chebyshev nodes of every leaf box, converted to
// Chebyshev coefficients.  Kernels (s source, t target):
//   K_SEC: 1/(s-t) and 1/(s-t)^2 into four fields (psi, phi, psi', phi' by side)
//   K_1: 1/(s-t)   K_2: 1/(s-t)^2   K_1N: 1/(t-s)   K_LOG: log|s-t|
enum { K_SEC = 0, K_1 = 1, K_2 = 2, K_1N = 3, K_LOG = 4 };

template <int KER>
__global__ void __launch_bounds__(128) k_fmm_m2l(FmmDev pl, const int32_t *__restrict__ mk, int nw)
{
    constexpr int NT = 128;
    constexpr int RMAX = (P * WMAX + NT - 1) / NT;
    __shared__ double Tx[P * P], xq[P], tq[P];
    __shared__ double Ws[P][WMAX + 1];
    __shared__ double K1[P][P + 1];
    __shared__ double K2[(KER == K_SEC) ? P : 1][P + 1];
    __shared__ double Fs[P][WMAX + 1];
    cheb_tables(xq, Tx);
    const int nf = (KER == K_SEC) ? 4 : nw;
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = blockIdx.x; gl < nleaf; gl += gridDim.x) {
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int m = mk[p];
        const int nb0 = (m + B - 1) / B;
        const int L = lev_count(nb0);
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t gp0 = pl.box_base[p];
        double cT, hT;
        box_ch(pl.blo[gp0 + Tb], pl.bhi[gp0 + Tb], cT, hT);
        __syncthreads();
        if (tid < P) tq[tid] = cT + hT * xq[tid];
        double acc[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; r++) acc[r] = 0.0;
        // an all-near leaf sums every source directly: no far field
        const int Lf = (pl.nnear[gp0 + Tb] < 0) ? 1 : L;
        for (int l = 0; l < Lf - 1; l++) {
            const int Ab = Tb >> l;
            const int64_t gbl = gp0 + lev_base(nb0, l);
            const int64_t gPA = gp0 + lev_base(nb0, l + 1) + (Ab >> 1);
            const double loA = pl.blo[gbl + Ab], hiA = pl.bhi[gbl + Ab];
            const int nbl = lev_nb(nb0, l);
            const int npn = pl.nnear[gPA];
            for (int i = 0; i < npn; i++) {
                const int s = pl.near[gPA * FMM_NCAP + i];
                for (int S = 2 * s; S <= 2 * s + 1 && S < nbl; S++) {
                    if (S == Ab) continue;
                    const int64_t gS = gbl + S;
                    const double loS = pl.blo[gS], hiS = pl.bhi[gS];
                    if (!adm(loS, hiS, loA, hiA)) continue;
                    const bool left = S < Ab;
                    double cS, hS;
                    box_ch(loS, hiS, cS, hS);
                    __syncthreads();
                    for (int t = tid; t < P * nw; t += NT) Ws[t / nw][t % nw] = pl.W[(gS * P + t / nw) * pl.ncol + t % nw];
                    for (int t = tid; t < P * P; t += NT) {
                        const int q = t / P, q2 = t % P;
                        const double diff = (cS + hS * xq[q2]) - tq[q];
                        if (KER == K_LOG) {
                            K1[q][q2] = log(fabs(diff));
                        } else {
                            const double r = 1.0 / diff;
                            if (KER == K_SEC) { K1[q][q2] = r; K2[q][q2] = r * r; }
                            else if (KER == K_1) K1[q][q2] = r;
                            else if (KER == K_1N) K1[q][q2] = -r;
                            else K1[q][q2] = r * r;
                        }
                    }
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < RMAX; r++) {
                        const int t = tid + r * NT;
                        if (t >= P * nf) break;
                        const int q = t / nf, f = t % nf;
                        if (KER == K_SEC) {
                            if ((f & 1) != (left ? 0 : 1)) continue;
                            const double(*Km)[P + 1] = (f < 2) ? K1 : K2;
                            double s2 = 0.0;
                            for (int q2 = 0; q2 < P; q2++) s2 = fma(Km[q][q2], Ws[q2][0], s2);
                            acc[r] += s2;
                        } else {
                            double s2 = 0.0;
                            for (int q2 = 0; q2 < P; q2++) s2 = fma(K1[q][q2], Ws[q2][f], s2);
                            acc[r] += s2;
                        }
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RMAX; r++) {
            const int t = tid + r * NT;
            if (t < P * nf) Fs[t / nf][t % nf] = acc[r];
        }
        __syncthreads();
        for (int t = tid; t < P * nf; t += NT) {
            const int n = t / nf, f = t % nf;
            double s = 0.0;
            for (int q = 0; q < P; q++) s = fma(Fs[q][f], Tx[q * P + n], s);
            pl.coef[(gl * pl.nfield + f) * P + n] = s * ((n == 0) ? 1.0 : 2.0) / P;
        }
    }
}

// ---------------------------------------------------------------------------
// Secular roots of the FMM problems.  Units: first one per problem for its
// last root (outside the tree; every pole direct, the warp splits the poles),
// then one per 32 roots of a leaf box.  One root per lane; each sweep sums
// the near boxes with shifted differences (staged per warp) and evaluates the
// four far-field expansions at x = d_K + y.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64)
k_secular_fmm(FmmDev pl, const int64_t *__restrict__ off, R1Out o, double stop_c, int max_iter)
{
    __shared__ double sd[2][B], sw[2][B];
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nf = *pl.nfmm;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    const int64_t nunits = nf + nleaf * (B / 32);
    for (int64_t u = (int64_t)blockIdx.x * 2 + warp; u < nunits; u += (int64_t)gridDim.x * 2) {
        if (u < nf) {
            const int64_t p = pl.fprob[u];
            if (pl.fslot[p] < 0) continue;
            const int64_t b0 = off[p];
            const int m = o.mk[p];
            const double *dk = o.dk + b0, *zk = o.zk + b0;
            const double W = o.wsum[p];
            const double tol = stop_c * (double)m * SDC_EPS;
            Root R;
            R.init(dk, zk, m - 1, m, W);
            bool fin = false;
            while (!fin) {
                const bool p0 = (R.phase == 0);
                double ps = 0.0, dps = 0.0;
                for (int j = lane; j < m; j += 32) {
                    const double t = shifted_t(dk[j], R.dK, R.y);
                    const double r = rcp_nr1(t);
                    const double z = zk[j];
                    const double a = (z * z) * r;
                    ps += a;
                    if (!p0) dps = fma(a, r, dps);
                }
                for (int sh = 16; sh > 0; sh >>= 1) {
                    ps += __shfl_down_sync(FULL, ps, sh);
                    dps += __shfl_down_sync(FULL, dps, sh);
                }
                Acc A;
                A.psi = __shfl_sync(FULL, ps, 0);
                A.dpsi = __shfl_sync(FULL, dps, 0);
                A.phi = 0.0;
                A.dphi = 0.0;
                fin = R.update(A, tol, max_iter, lane == 0 ? o.status : nullptr);
            }
            if (lane == 0) {
                const int k = m - 1;
                o.org[b0 + k] = R.K;
                o.eta[b0 + k] = R.y;
                o.dorg[b0 + k] = R.dK;
                o.lamk[b0 + k] = R.dK + R.y;
                if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
            }
            continue;
        }
        const int64_t lu = u - nf;
        const int64_t gl = lu / (B / 32);
        const int half = (int)(lu % (B / 32));
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int k0 = Tb * B + half * 32;
        const int kend = min(k0 + 32, m - 1);
        if (k0 >= kend) continue;
        const double *dk = o.dk + b0, *zk = o.zk + b0;
        const double W = o.wsum[p];
        const double tol = stop_c * (double)m * SDC_EPS;
        const int64_t g = pl.box_base[p] + Tb;
        double cT, hT;
        box_ch(pl.blo[g], pl.bhi[g], cT, hT);
        const double ihT = 1.0 / hT;
        const double *cf = pl.coef + gl * pl.nfield * P;
        const int nnr = pl.nnear[g];
        const int nn = near_len(nnr, (m + B - 1) / B);
        int k = k0 + lane;
        bool act = k < kend;
        Root R;
        R.dK = 0.0; R.y = 1.0; R.phase = 1;
        if (act) R.init(dk, zk, k, m, W);
        while (__any_sync(FULL, act)) {
            const int kwlo = __reduce_min_sync(FULL, act ? k : 0x7fffffff);
            const int kwhi = __reduce_max_sync(FULL, act ? k : -1);
            const int kk = act ? k : kwlo;
            const bool p0 = __all_sync(FULL, !act || R.phase == 0);
            Acc A = {0.0, 0.0, 0.0, 0.0};
            if (act) {
                // far field at the plain position x = d_K + y (local shifting)
                const double uu = ((R.dK + R.y) - cT) * ihT;
                const double u2 = uu + uu;
                double a1 = 0, a2 = 0, b1 = 0, b2 = 0, c1 = 0, c2 = 0, e1 = 0, e2 = 0;
                for (int n = P - 1; n >= 1; n--) {
                    double t;
                    t = fma(u2, a1, cf[n] - a2);         a2 = a1; a1 = t;
                    t = fma(u2, b1, cf[P + n] - b2);     b2 = b1; b1 = t;
                    t = fma(u2, c1, cf[2 * P + n] - c2); c2 = c1; c1 = t;
                    t = fma(u2, e1, cf[3 * P + n] - e2); e2 = e1; e1 = t;
                }
                A.psi = fma(uu, a1, cf[0] - a2);
                A.phi = fma(uu, b1, cf[P] - b2);
                A.dpsi = fma(uu, c1, cf[2 * P] - c2);
                A.dphi = fma(uu, e1, cf[3 * P] - e2);
            }
            for (int i = 0; i < nn; i++) {
                const int S = near_box(pl.near, g, nnr, i);
                const int j0 = S * B;
                const int cnt = min(B, m - j0);
                __syncwarp();
                for (int jj = lane; jj < cnt; jj += 32) {
                    sd[warp][jj] = dk[j0 + jj];
                    const double z = zk[j0 + jj];
                    sw[warp][jj] = z * z;
                }
                __syncwarp();
                if (p0) sweep<false>(sd[warp], sw[warp], 0, cnt, j0, kk, kwlo, kwhi, R.dK, R.y, A);
                else    sweep<true>(sd[warp], sw[warp], 0, cnt, j0, kk, kwlo, kwhi, R.dK, R.y, A);
            }
            if (act && R.update(A, tol, max_iter, o.status)) {
                o.org[b0 + k] = R.K;
                o.eta[b0 + k] = R.y;
                o.dorg[b0 + k] = R.dK;
                o.lamk[b0 + k] = R.dK + R.y;
                if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                act = false;
            }
        }
    }
}

// running product with exponent renormalisation every 8 factors
struct Prod {
    double pn = 1.0, pd = 1.0;
    int ex = 0, cnt = 0;
    __device__ __forceinline__ void mul(double num, double den)
    {
        pn *= num;
        pd *= den;
        if ((++cnt & 7) == 0) {
            const int hn = __double2hiint(pn), hd = __double2hiint(pd);
            const int en = (hn >> 20) & 0x7FF, ed = (hd >> 20) & 0x7FF;
            if (en != 0 && ed != 0 && en != 0x7FF && ed != 0x7FF) {
                ex += en - ed;
                pn = __hiloint2double((hn & 0x800FFFFF) | (1022 << 20), __double2loint(pn));
                pd = __hiloint2double((hd & 0x800FFFFF) | (1022 << 20), __double2loint(pd));
            }
        }
    }
};

// zhat of the FMM problems, eq. (4.23) as
//   vhat_i^2 = (lambda_i - d_i) prod_{j != i} (lambda_j - d_i) / (d_j - d_i):
// near boxes and the pair j = m-1 as products of shifted differences, the far
// boxes through the logarithmic form eq. (4.25) (dipole charges +1 at
// lambda_j, -1 at d_j).  One CTA of B threads per leaf box, one target each.
__global__ void __launch_bounds__(B) k_lowner_fmm(FmmDev pl, const int64_t *__restrict__ off, R1Out o)
{
    __shared__ double sd[B], so[B], se[B];
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = blockIdx.x; gl < nleaf; gl += gridDim.x) {
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        const double *dk = o.dk + b0, *dorg = o.dorg + b0, *eta = o.eta + b0;
        const int i = Tb * B + tid;
        const bool act = i < m;
        const double di = act ? dk[i] : 0.0;
        Prod pr;
        if (act) {
            const double num = (dorg[m - 1] - di) + eta[m - 1];
            const double den = (i == m - 1) ? 1.0 : dk[m - 1] - di;
            pr.mul(num, den);
        }
        const int nnr = pl.nnear[g];
        const int nn = near_len(nnr, (m + B - 1) / B);
        for (int s = 0; s < nn; s++) {
            const int S = near_box(pl.near, g, nnr, s);
            const int j0 = S * B;
            const int cnt = min(B, (m - 1) - j0);
            __syncthreads();
            if (tid < cnt) { sd[tid] = dk[j0 + tid]; so[tid] = dorg[j0 + tid]; se[tid] = eta[j0 + tid]; }
            __syncthreads();
            if (act) {
                for (int jj = 0; jj < cnt; jj++) {
                    const double num = (so[jj] - di) + se[jj];
                    const double den = (j0 + jj == i) ? 1.0 : sd[jj] - di;
                    pr.mul(num, den);
                }
            }
        }
        if (act) {
            double cT, hT;
            box_ch(pl.blo[g], pl.bhi[g], cT, hT);
            const double Lf = clenshaw(pl.coef + gl * pl.nfield * P, (di - cT) / hT);
            double prod = pr.pn / pr.pd;
            int ex = pr.ex;
            if (ex & 1) { prod *= 2.0; ex -= 1; }
            double v = ldexp(sqrt(prod), ex / 2) * exp(0.5 * Lf);
            if (!isfinite(v)) sdc_latch(o.status, SUPERDC_DEV_NONFINITE);
            o.vhat[b0 + i] = (o.zk[b0 + i] < 0.0) ? -v : v;
        }
    }
}

// b of the FMM problems, eq. (4.27): near boxes with the shifted entries of
// eq. (4.28), far boxes by expansion at lambda_j = d_{K_j} + eta_j; the last
// target j = m-1 (outside the tree) summed directly by a whole CTA.
__global__ void __launch_bounds__(B) k_bnorm_fmm(FmmDev pl, const int64_t *__restrict__ off, R1Out o)
{
    __shared__ double sd[B], sv[B];
    __shared__ double red[B];
    const int tid = threadIdx.x;
    const int nf = *pl.nfmm;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t u = blockIdx.x; u < nf + nleaf; u += gridDim.x) {
        if (u < nf) {
            const int64_t p = pl.fprob[u];
            if (pl.fslot[p] < 0) continue;
            const int64_t b0 = off[p];
            const int m = o.mk[p];
            const double dK = o.dorg[b0 + m - 1], e = o.eta[b0 + m - 1];
            double s = 0.0;
            for (int i = tid; i < m; i += B) {
                const double r = rcp_nr2((o.dk[b0 + i] - dK) - e);
                const double vr = o.vhat[b0 + i] * r;
                s = fma(vr, vr, s);
            }
            __syncthreads();
            red[tid] = s;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < B; q++) t += red[q];
                o.bnorm[b0 + m - 1] = 1.0 / sqrt(t);
            }
            continue;
        }
        const int64_t gl = u - nf;
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        const int j = Tb * B + tid;
        const bool act = j < m - 1;
        const double dK = act ? o.dorg[b0 + j] : 0.0, e = act ? o.eta[b0 + j] : 0.0;
        double s = 0.0;
        if (act) {
            double cT, hT;
            box_ch(pl.blo[g], pl.bhi[g], cT, hT);
            s = clenshaw(pl.coef + gl * pl.nfield * P, ((dK + e) - cT) / hT);
        }
        const int nnr = pl.nnear[g];
        const int nn = near_len(nnr, (m + B - 1) / B);
        for (int q = 0; q < nn; q++) {
            const int S = near_box(pl.near, g, nnr, q);
            const int i0 = S * B;
            const int cnt = min(B, m - i0);
            __syncthreads();
            if (tid < cnt) { sd[tid] = o.dk[b0 + i0 + tid]; sv[tid] = o.vhat[b0 + i0 + tid]; }
            __syncthreads();
            if (act) {
                for (int ii = 0; ii < cnt; ii++) {
                    const double r = rcp_nr2((sd[ii] - dK) - e);
                    const double vr = sv[ii] * r;
                    s = fma(vr, vr, s);
                }
            }
        }
        if (act) o.bnorm[b0 + j] = 1.0 / sqrt(s);
    }
}

// Y = Qhat^T X (columns [col0, col0+nc)) for the FMM problems:
//   y_{pinv_j} = b_j sum_i vhat_i x_{src_i} / ((d_i - d_{K_j}) - eta_j)
template <int NC>
__global__ void __launch_bounds__(B)
k_cauchyT_fmm(FmmDev pl, FactorView f, const double *__restrict__ X, int64_t ldx, double *__restrict__ Y,
              int64_t ldy, int col0, int nc)
{
    __shared__ double sd[B];
    __shared__ double sx[NC][B + 1];
    const int tid = threadIdx.x;
    const int nf = *pl.nfmm;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t u = blockIdx.x; u < nf + nleaf; u += gridDim.x) {
        double acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) acc[q] = 0.0;
        if (u < nf) {
            const int64_t p = pl.fprob[u];
            if (pl.fslot[p] < 0) continue;
            const int64_t b0 = f.off[p];
            const int m = f.mk[p];
            const int j = m - 1;
            const double dK = f.dorg[b0 + j], e = f.eta[b0 + j];
            for (int i = tid; i < m; i += B) {
                const double r = rcp_nr2((f.dk[b0 + i] - dK) - e);
                const double v = f.vhat[b0 + i] * r;
                const int64_t row = b0 + f.src[b0 + i];
#pragma unroll
                for (int q = 0; q < NC; q++)
                    if (q < nc) acc[q] = fma(v, X[row + (int64_t)(col0 + q) * ldx], acc[q]);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NC; q++) sx[q][tid] = acc[q];
            __syncthreads();
            if (tid < nc) {
                double t = 0.0;
                for (int i = 0; i < B; i++) t += sx[tid][i];
                Y[b0 + f.pinv[b0 + j] + (int64_t)(col0 + tid) * ldy] = f.bnorm[b0 + j] * t;
            }
            continue;
        }
        const int64_t gl = u - nf;
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = f.off[p];
        const int m = f.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        const int j = Tb * B + tid;
        const bool act = j < m - 1;
        const double dK = act ? f.dorg[b0 + j] : 0.0, e = act ? f.eta[b0 + j] : 1.0;
        if (act) {
            double cT, hT;
            box_ch(pl.blo[g], pl.bhi[g], cT, hT);
            const double uu = ((dK + e) - cT) / hT;
            const double *cf = pl.coef + gl * pl.nfield * P;
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) acc[q] = clenshaw(cf + q * P, uu);
        }
        const int nnr = pl.nnear[g];
        const int nn = near_len(nnr, (m + B - 1) / B);
        for (int s = 0; s < nn; s++) {
            const int S = near_box(pl.near, g, nnr, s);
            const int i0 = S * B;
            const int cnt = min(B, m - i0);
            __syncthreads();
            if (tid < cnt) {
                const int i = i0 + tid;
                sd[tid] = f.dk[b0 + i];
                const double v = f.vhat[b0 + i];
                const int64_t row = b0 + f.src[b0 + i];
#pragma unroll
                for (int q = 0; q < NC; q++) sx[q][tid] = (q < nc) ? v * X[row + (int64_t)(col0 + q) * ldx] : 0.0;
            }
            __syncthreads();
            if (act) {
                for (int ii = 0; ii < cnt; ii++) {
                    const double r = rcp_nr2((sd[ii] - dK) - e);
#pragma unroll
                    for (int q = 0; q < NC; q++) acc[q] = fma(sx[q][ii], r, acc[q]);
                }
            }
        }
        if (act) {
            const double bj = f.bnorm[b0 + j];
            const int64_t row = b0 + f.pinv[b0 + j];
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) Y[row + (int64_t)(col0 + q) * ldy] = bj * acc[q];
        }
    }
}

// Y = Qhat X (columns [col0, col0+nc)) for the FMM problems:
//   y_{src_i} = vhat_i sum_j b_j x_{pinv_j} / ((d_i - d_{K_j}) - eta_j)
template <int NC>
__global__ void __launch_bounds__(B)
k_cauchyN_fmm(FmmDev pl, FactorView f, const double *__restrict__ X, int64_t ldx, double *__restrict__ Y,
              int64_t ldy, int col0, int nc)
{
    __shared__ double sk[B], se[B];
    __shared__ double sx[NC][B + 1];
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = blockIdx.x; gl < nleaf; gl += gridDim.x) {
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = f.off[p];
        const int m = f.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        const int i = Tb * B + tid;
        const bool act = i < m;
        const double di = act ? f.dk[b0 + i] : 0.0;
        double acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) acc[q] = 0.0;
        if (act) {
            double cT, hT;
            box_ch(pl.blo[g], pl.bhi[g], cT, hT);
            const double uu = (di - cT) / hT;
            const double *cf = pl.coef + gl * pl.nfield * P;
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) acc[q] = clenshaw(cf + q * P, uu);
            // the last eigenvalue (outside the tree) as a source
            const int jl = m - 1;
            const double r = rcp_nr2((di - f.dorg[b0 + jl]) - f.eta[b0 + jl]);
            const double bl = f.bnorm[b0 + jl] * r;
            const int64_t row = b0 + f.pinv[b0 + jl];
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) acc[q] = fma(bl, X[row + (int64_t)(col0 + q) * ldx], acc[q]);
        }
        const int nnr = pl.nnear[g];
        const int nn = near_len(nnr, (m + B - 1) / B);
        for (int s = 0; s < nn; s++) {
            const int S = near_box(pl.near, g, nnr, s);
            const int j0 = S * B;
            const int cnt = min(B, (m - 1) - j0);
            __syncthreads();
            if (tid < cnt) {
                const int j = j0 + tid;
                sk[tid] = f.dorg[b0 + j];
                se[tid] = f.eta[b0 + j];
                const double bj = f.bnorm[b0 + j];
                const int64_t row = b0 + f.pinv[b0 + j];
#pragma unroll
                for (int q = 0; q < NC; q++) sx[q][tid] = (q < nc) ? bj * X[row + (int64_t)(col0 + q) * ldx] : 0.0;
            }
            __syncthreads();
            if (act) {
                for (int jj = 0; jj < cnt; jj++) {
                    const double r = rcp_nr2((di - sk[jj]) - se[jj]);
#pragma unroll
                    for (int q = 0; q < NC; q++) acc[q] = fma(sx[q][jj], r, acc[q]);
                }
            }
        }
        if (act) {
            const double v = f.vhat[b0 + i];
            const int64_t row = b0 + f.src[b0 + i];
#pragma unroll
            for (int q = 0; q < NC; q++)
                if (q < nc) Y[row + (int64_t)(col0 + q) * ldy] = v * acc[q];
        }
    }
}

unsigned fmm_grid() { return (unsigned)(sdc_num_sms() * 8); }

SrcArgs src_from_r1(const int64_t *off, const R1Out &o)
{
    SrcArgs a{};
    a.off = off; a.mk = o.mk; a.dk = o.dk; a.zk = o.zk; a.vhat = o.vhat; a.bnorm = o.bnorm;
    a.dorg = o.dorg; a.eta = o.eta; a.src = o.src; a.pinv = o.pinv;
    return a;
}

template <int MODE, int KER>
superdc_status far_field(const FmmPlan &pl, const SrcArgs &a, int nw, cudaStream_t st)
{
    const unsigned g = fmm_grid();
    PROF_LAUNCH("fmm_mom", st, k_fmm_leafmom<MODE><<<g, B, 0, st>>>(pl.dv, a));
    for (int l = 1; l < pl.lmax; l++)
        PROF_LAUNCH("fmm_m2m", st, k_fmm_m2m<<<g, 128, 0, st>>>(pl.dv, a.mk, l, nw));
    PROF_LAUNCH("fmm_m2l", st, k_fmm_m2l<KER><<<g, 128, 0, st>>>(pl.dv, a.mk, nw));
    return SUPERDC_OK;
}

template <int NC>
void launch_ct(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y, int64_t ldy, int col0,
               int nc, cudaStream_t st)
{
    k_cauchyT_fmm<NC><<<fmm_grid(), B, 0, st>>>(pl.dv, f, X, ldx, Y, ldy, col0, nc);
}

template <int NC>
void launch_cn(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y, int64_t ldy, int col0,
               int nc, cudaStream_t st)
{
    k_cauchyN_fmm<NC><<<fmm_grid(), B, 0, st>>>(pl.dv, f, X, ldx, Y, ldy, col0, nc);
}

}  // namespace

int fmm_default_min_m() { return 4096; }

superdc_status fmm_plan(FmmPlan &pl, int64_t nprob, const int64_t *off, int64_t total, int64_t max_m,
                        const int32_t *mk, const double *dk, int min_m, int ncol, int nfield, int32_t *used,
                        cudaStream_t st)
{
    pl = FmmPlan();
    if (nprob <= 0) return SUPERDC_OK;
    if (used) SDC_CHECK(cudaMemsetAsync(used, 0, (size_t)nprob * sizeof(int32_t), st));
    if (min_m <= 0) return SUPERDC_OK;
    const int64_t mm = (max_m >= 0) ? std::min(max_m, total) : total;
    const int eff = std::max(min_m, 4 * B);
    if (mm < eff) return SUPERDC_OK;
    const int64_t nf_cap = std::min<int64_t>(nprob, total / eff + 1);
    pl.cap_f = nf_cap;
    pl.cap_leaves = total / B + nf_cap + 1;
    pl.cap_boxes = 2 * pl.cap_leaves + nf_cap * 40;
    const int nb0max = (int)((mm + B - 1) / B);
    pl.lmax = lev_count(nb0max);
    ncol = std::max(1, std::min(ncol, WMAX));
    nfield = std::max(1, std::min(nfield, WMAX));
    FmmDev &d = pl.dv;
    d.nprob = nprob;
    d.ncol = ncol;
    d.nfield = nfield;
    auto al = [&](auto **ptr, size_t cnt) -> cudaError_t {
        cudaError_t e = sdc_alloc(ptr, cnt, st);
        if (e == cudaSuccess) pl.bufs.push_back((void *)*ptr);
        return e;
    };
    int64_t *box_base, *leaf_base;
    int32_t *fslot, *fprob, *nfmm, *nnear, *near;
    double *blo, *bhi;
    SDC_CHECK(al(&box_base, nprob + 1));
    SDC_CHECK(al(&leaf_base, nprob + 1));
    SDC_CHECK(al(&fslot, nprob));
    SDC_CHECK(al(&fprob, nf_cap));
    SDC_CHECK(al(&nfmm, 1));
    SDC_CHECK(al(&blo, pl.cap_boxes));
    SDC_CHECK(al(&bhi, pl.cap_boxes));
    SDC_CHECK(al(&nnear, pl.cap_boxes));
    SDC_CHECK(al(&near, pl.cap_boxes * FMM_NCAP));
    SDC_CHECK(al(&d.M, (size_t)pl.cap_boxes * P * ncol));
    SDC_CHECK(al(&d.W, (size_t)pl.cap_boxes * P * ncol));
    SDC_CHECK(al(&d.coef, (size_t)pl.cap_leaves * nfield * P));
    d.box_base = box_base; d.leaf_base = leaf_base; d.fslot = fslot; d.fprob = fprob; d.nfmm = nfmm;
    d.blo = blo; d.bhi = bhi; d.nnear = nnear; d.near = near;
    PROF_LAUNCH("fmm_plan", st, k_fmm_plan<<<1, 1024, 0, st>>>(nprob, mk, min_m, pl.cap_boxes, pl.cap_leaves,
                                                               pl.cap_f, box_base, leaf_base, fslot, fprob, nfmm));
    const unsigned gt = (unsigned)std::min<int64_t>(nprob, (int64_t)sdc_num_sms() * 4);
    PROF_LAUNCH("fmm_tree", st, k_fmm_tree<<<gt, 256, 0, st>>>(nprob, off, mk, dk, box_base, fslot, blo, bhi,
                                                               nnear, near, used));
    SDC_CHECK(cudaGetLastError());
    pl.on = true;
    return SUPERDC_OK;
}

void fmm_free(FmmPlan &pl, cudaStream_t st)
{
    for (void *p : pl.bufs) cudaFreeAsync(p, st);
    pl.bufs.clear();
    pl.on = false;
}

superdc_status fmm_secular(const FmmPlan &pl, const int64_t *off, const R1Out &o, double stop_c, int max_iter,
                           cudaStream_t st)
{
    if (!pl.on) return SUPERDC_OK;
    far_field<M_SEC, K_SEC>(pl, src_from_r1(off, o), 1, st);
    PROF_LAUNCH("fmm_secular", st, k_secular_fmm<<<fmm_grid(), 64, 0, st>>>(pl.dv, off, o, stop_c, max_iter));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

superdc_status fmm_lowner(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st)
{
    if (!pl.on) return SUPERDC_OK;
    far_field<M_LOW, K_LOG>(pl, src_from_r1(off, o), 1, st);
    PROF_LAUNCH("fmm_lowner", st, k_lowner_fmm<<<fmm_grid(), B, 0, st>>>(pl.dv, off, o));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

superdc_status fmm_bnorm(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st)
{
    if (!pl.on) return SUPERDC_OK;
    far_field<M_BN, K_2>(pl, src_from_r1(off, o), 1, st);
    PROF_LAUNCH("fmm_bnorm", st, k_bnorm_fmm<<<fmm_grid(), B, 0, st>>>(pl.dv, off, o));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

superdc_status fmm_cauchy(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y,
                          int64_t ldy, int col0, int nc, bool trans, cudaStream_t st)
{
    if (!pl.on || nc <= 0) return SUPERDC_OK;
    if (nc > WMAX || nc > pl.dv.ncol || nc > pl.dv.nfield) return SUPERDC_ERR_ARG;
    SrcArgs a{};
    a.off = f.off; a.mk = f.mk; a.dk = f.dk; a.vhat = f.vhat; a.bnorm = f.bnorm; a.dorg = f.dorg; a.eta = f.eta;
    a.src = f.src; a.pinv = f.pinv; a.X = X; a.ldx = ldx; a.col0 = col0; a.nc = nc;
    if (trans) far_field<M_CT, K_1>(pl, a, nc, st);
    else far_field<M_CN, K_1N>(pl, a, nc, st);
    typedef void (*Fn)(const FmmPlan &, const FactorView &, const double *, int64_t, double *, int64_t, int, int,
                       cudaStream_t);
    Fn fn;
    if (nc <= 4) fn = trans ? launch_ct<4> : launch_cn<4>;
    else if (nc <= 8) fn = trans ? launch_ct<8> : launch_cn<8>;
    else if (nc <= 16) fn = trans ? launch_ct<16> : launch_cn<16>;
    else if (nc <= 24) fn = trans ? launch_ct<24> : launch_cn<24>;
    else fn = trans ? launch_ct<32> : launch_cn<32>;
    PROF_LAUNCH("fmm_cauchy", st, fn(pl, f, X, ldx, Y, ldy, col0, nc, st));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}
