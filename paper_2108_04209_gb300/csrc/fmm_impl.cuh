// Triangular FMM with local shifting on sm_103a (Sections 4.1.2, 4.2.2, 4.3).
//
// Geometry.  The kept poles d_0 < ... < d_{m-1} of a problem and the targets
// (roots x_k in (d_k, d_{k+1}), eigenvalues lambda_j, or the poles themselves)
// interlace (eq. (4.4)), so one index-based binary tree serves both: a leaf
// box holds B consecutive indices (32 or 64; this file is compiled once per
// box size, fmm32.cu and fmm64.cu), so d_k and x_k of the same k always share
// a box (the paper's first design point), and every box carries the interval
// [d_{i0}, d_{i1}] of its points (the last box ends at d_{m-1}).  The index
// split adapts the boxes to clustered spectra (second design point); whether
// two boxes interact through expansions is decided geometrically: boxes S, T
// of one level are admissible when their gap is at least FMM_KAPPA times the
// larger width.  Near lists are built top-down (children of the parent's near
// list that are not admissible) and have any length (a wide box, e.g. in a
// tail of the spectrum, is close to many boxes; its narrow children are not).
// Only when the list pool is exhausted is a box marked "all near", with its
// subtree: the targets of such leaves are summed directly over every source.
// Only the last eigenvalue lambda_{m-1} lies outside the tree (to the right of
// d_{m-1}): as a target its sums run over the tree (node weights of the boxes
// far from it, direct sums over the leaf boxes next to it) or are spread over
// the leaf boxes; as a source it is added directly to every target.
//
// Expansions.  Chebyshev interpolation with FMM_P first-kind nodes per box:
// source moments M_n = sum_j w_j T_n(u_j) of the leaf boxes, node weights
// W_q = sum_j w_j L_q(u_j) from the moments, parents' moments exactly from
// the children's weights (T_n(alpha u + beta) has degree n < P; upward
// pass); every box
// receives the kernel sums of its interaction list (children of its parent's
// near list that are admissible to it) at its own Chebyshev nodes (M2L), the
// parents' fields are interpolated down the tree (L2L), and on the leaves the
// field becomes Chebyshev coefficients evaluated at the targets by Clenshaw.
// Work is O(m P^2 / B) for the far field plus O(m B) for the near field.
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
#include <mutex>
#include "common.cuh"
#include "fmm.cuh"
#include "secular.cuh"
#include "prof.cuh"

#if !defined(FMM_BOX) || !defined(FMM_NS)
#error "define FMM_BOX (indices per leaf box) and FMM_NS (namespace) before including fmm_impl.cuh"
#endif

namespace FMM_NS {
namespace {

constexpr int P = FMM_P;
constexpr int B = FMM_BOX;
// admissibility: gap >= 0.75 x the larger width.  The nearest source then lies
// at least 2.5 half-widths from either box's centre (Bernstein ellipse
// rho >= 2.5 + sqrt(5.25) = 4.79): at 22 nodes the interpolated 1/(s-t) stays at
// the rounding floor (~1e-14 relative) and 1/(s-t)^2 within ~1e-13 over box-width
// ratios 1e-3..1e3, while index-based boxes of random spectra drop from ~4.3
// to ~3.2-3.4 near boxes per leaf (with 1.0 the box between two neighbours must
// be at least as wide as both, which a random width sequence meets a third of
// the time)
constexpr double FMM_KAPPA = 0.75;
constexpr int SPLIT_NEAR = 512 / B;   // leaf boxes with this many near boxes (512 poles) or more: CTA-split sweeps
constexpr int TAIL_X = 12;        // k_secular_fmm hands a box's last roots to the tail pass below this many busy lanes
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
__device__ __forceinline__ int near_box(const FmmDev &pl, int64_t g, int nn, int i)
{
    return nn < 0 ? i : pl.near[pl.nstart[g] + i];
}
// a near box of a consumer kernel: in the checked build the list entry is
// tested against the problem's leaf box count nb0 (latched into word)
__device__ __forceinline__ int near_box_chk(const FmmDev &pl, int64_t g, int nn, int i, int nb0, int32_t *word)
{
    return SDC_IDX(near_box(pl, g, nn, i), nb0, word);
}

// Chebyshev nodes x_q = cos((2q+1) pi / 2P) and T_n(x_q) (Tx[q * P + n], by
// the three-term recurrence, one row per thread); the caller synchronises
// before the first use.  sc scales the entries n >= 1 (2: the weights of the
// moments -> node weights sums, exact, saving a multiply per term)
__device__ __forceinline__ void cheb_tables(double *xq, double *Tx, double sc = 1.0)
{
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        const double x = cospi((double)(2 * q + 1) / (2.0 * P));
        xq[q] = x;
        double t0 = 1.0, t1 = x;
        Tx[q * P] = 1.0;
        Tx[q * P + 1] = sc * x;
        for (int n = 2; n < P; n++) {
            const double t2 = 2.0 * x * t1 - t0;
            Tx[q * P + n] = sc * t2;
            t0 = t1; t1 = t2;
        }
    }
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

// algorithmic work counter (profiling): one add per box by thread 0
__device__ __forceinline__ void fl_add(const FmmDev &pl, int64_t v)
{
    if (pl.flops && threadIdx.x == 0 && v > 0) atomicAdd(pl.flops, (unsigned long long)v);
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

// Box intervals and near lists, one CTA per problem, top level first.  Near
// lists have any length; they are stored back to back in the problem's share
// of the pool (FMM_NPOOL entries per box on average).  A box whose list no
// longer fits, and its subtree, is marked "all near" (nnear = -1).
__device__ __forceinline__ int near_count(const double *__restrict__ blo, const double *__restrict__ bhi,
                                          const int32_t *__restrict__ near, int64_t gb, int nb, int b,
                                          int64_t pst, int npn)
{
    const double loT = blo[gb + b], hiT = bhi[gb + b];
    int cnt = 0;
    for (int i = 0; i < npn; i++) {
        const int s = near[pst + i];
        for (int S = 2 * s; S <= 2 * s + 1 && S < nb; S++)
            if (S == b || !adm(blo[gb + S], bhi[gb + S], loT, hiT)) cnt++;
    }
    return cnt;
}

// exclusive scan of one value per thread of the CTA (warp shuffles, then the
// warp totals); sh holds one entry per warp
__device__ __forceinline__ int64_t cta_exscan(int64_t v, int64_t *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; w++) before += sh[w];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(1024)
k_fmm_tree(int64_t nprob, const int64_t *__restrict__ off, const int32_t *__restrict__ mk,
           const double *__restrict__ dk, const int64_t *__restrict__ box_base, int32_t *__restrict__ fslot,
           double *__restrict__ blo, double *__restrict__ bhi, int32_t *__restrict__ nnear,
           int64_t *__restrict__ nstart, int32_t *__restrict__ near, int32_t *__restrict__ used,
           const int64_t *__restrict__ leaf_base, int64_t *__restrict__ split, int32_t *__restrict__ nsplit)
{
    __shared__ int64_t wsum[32];
    __shared__ int64_t s_pos;
    const int T = blockDim.x;
    for (int64_t p = blockIdx.x; p < nprob; p += gridDim.x) {
        if (fslot[p] < 0) continue;
        const int m = mk[p];
        const double *d = dk + off[p];
        const int64_t g0 = box_base[p];
        const int64_t pool_end = box_base[p + 1] * FMM_NPOOL;
        const int nb0 = (m + B - 1) / B;
        const int L = lev_count(nb0);
        if (threadIdx.x == 0) s_pos = g0 * FMM_NPOOL;
        __syncthreads();
        for (int l = L - 1; l >= 0; l--) {
            const int nb = lev_nb(nb0, l);
            const int64_t gb = g0 + lev_base(nb0, l);
            const int64_t gp0 = (l < L - 1) ? g0 + lev_base(nb0, l + 1) : 0;
            for (int b = threadIdx.x; b < nb; b += T) {
                int i0, i1;
                box_range(m, l, b, i0, i1);
                blo[gb + b] = d[i0];
                bhi[gb + b] = (i1 < m) ? d[i1] : d[m - 1];
            }
            __syncthreads();
            // each thread a contiguous range of boxes: count, block prefix, fill
            const int per = (nb + T - 1) / T;
            const int bb = min(nb, (int)threadIdx.x * per), be = min(nb, bb + per);
            int64_t sum = 0;
            for (int b = bb; b < be; b++) {
                if (l == L - 1) { sum += 1; continue; }
                const int64_t gp = gp0 + (b >> 1);
                const int npn = nnear[gp];
                if (npn >= 0) sum += near_count(blo, bhi, near, gb, nb, b, nstart[gp], npn);
            }
            int64_t pos = s_pos + cta_exscan(sum, wsum);
            for (int b = bb; b < be; b++) {
                int cnt;
                if (l == L - 1) {
                    cnt = 1;
                    if (pos + 1 <= pool_end) near[pos] = b; else cnt = -1;
                    nstart[gb + b] = pos;
                    pos += 1;
                } else {
                    const int64_t gp = gp0 + (b >> 1);
                    const int npn = nnear[gp];
                    if (npn < 0) {
                        cnt = -1;                                           // parent all near
                        nstart[gb + b] = pos;
                    } else {
                        const int64_t pst = nstart[gp];
                        const int c = near_count(blo, bhi, near, gb, nb, b, pst, npn);
                        nstart[gb + b] = pos;
                        if (pos + c <= pool_end) {
                            const double loT = blo[gb + b], hiT = bhi[gb + b];
                            int w = 0;
                            for (int i = 0; i < npn; i++) {
                                const int s2 = near[pst + i];
                                for (int S = 2 * s2; S <= 2 * s2 + 1 && S < nb; S++)
                                    if (S == b || !adm(blo[gb + S], bhi[gb + S], loT, hiT)) near[pos + w++] = S;
                            }
                            cnt = c;
                        } else {
                            cnt = -1;                                       // pool exhausted: all near
                        }
                        pos += c;
                    }
                }
                nnear[gb + b] = cnt;
                // leaf boxes with long near lists, for k_secular_fmm_split (in
                // any order: each box's sweeps are independent of the others)
                if (l == 0 && (cnt < 0 || cnt >= SPLIT_NEAR)) split[atomicAdd(nsplit, 1)] = leaf_base[p] + b;
            }
            __syncthreads();
            if (threadIdx.x == T - 1) s_pos = pos;
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

// leaf moments and node weights of leaf box gl (box g, index Tb within its
// problem p); one thread per source (threads B.. only join the sums)
//   M_SEC: w_j = z_j^2 at d_j            M_BN: w_i = vhat_i^2 at d_i
//   M_LOW: +1 at lambda_j, -1 at d_j (j < m-1; Chebyshev differences of the pair)
//   M_CT:  vhat_i x_{src_i} at d_i       M_CN: b_j x_{pinv_j} at lambda_j (j < m-1)
constexpr int UP_ROWS = (B > 2 * P) ? B : 2 * P;   // rows of the staging arrays (sources, or 2 children x P)

template <int MODE, int WW>
__device__ __forceinline__ void leaf_moments(const FmmDev &pl, const SrcArgs &a, int64_t p, int64_t gl, int64_t g,
                                             int Tb, int nw, double (*Tt)[P + 1], double (*Wt)[WW + 1],
                                             double (*Ms)[WW + 1], const double *Tx)
{
    const int tid = threadIdx.x;
    const int64_t b0 = a.off[p];
    const int m = a.mk[p];
    double c, h;
    box_ch(pl.blo[g], pl.bhi[g], c, h);
    const int j = Tb * B + tid;
    const int jend = (MODE == M_LOW || MODE == M_CN) ? m - 1 : m;
    const bool act = tid < B && j < jend;
    __syncthreads();
    if (tid < B) {
        if (MODE == M_LOW) {
            // D_n = T_n(b) - T_n(a) with b = a + delta, by the recurrence
            // D_{n+1} = 2 delta T_n(b) + 2 a D_n - D_{n-1} (no cancellation)
            double av = 0.0, dl = 0.0;
            if (act) {
                const double ih = 1.0 / h;
                av = (a.dk[b0 + j] - c) * ih;
                dl = ((a.dorg[b0 + j] - a.dk[b0 + j]) + a.eta[b0 + j]) * ih;
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
    }
    __syncthreads();
    for (int t = tid; t < P * nw; t += blockDim.x) {
        const int n = t / nw, q = t % nw;
        double s = 0.0;
        for (int jj = 0; jj < B; jj++) s = fma(Tt[jj][n], Wt[jj][q], s);
        Ms[n][q] = s;
    }
    __syncthreads();
    for (int t = tid; t < P * nw; t += blockDim.x) {
        const int qn = t / nw, q = t % nw;
        double s = Ms[0][q];
        for (int n = 1; n < P; n++) s = fma(Tx[qn * P + n], Ms[n][q], s);     // Tx holds 2 T_n
        pl.W[(g * P + qn) * pl.ncol + q] = s * (1.0 / P);
    }
    // Chebyshev recurrence per source, moments, moments -> node weights
    const int64_t cnt = max(0, min(B, jend - Tb * B));
    fl_add(pl, cnt * ((MODE == M_LOW) ? 4 : 2) * (P - 2) + 2 * cnt * P * nw + 2 * P * P * nw);
}

// Boxes of level l of the FMM problems, enumerated as (FMM problem f, box b)
// with b below the widest level-l box count nbl_max (host bound); returns
// false for slots without a box.
// Box u of level l over all FMM problems (per-level prefix lev_off[l][f]).
__device__ __forceinline__ bool level_box(const FmmDev &pl, const int32_t *__restrict__ mk, int l, int64_t u,
                                          int64_t &p, int &nb0, int &b, int64_t &g)
{
    const int nf = *pl.nfmm;
    const int64_t *lo = pl.lev_off + (int64_t)l * (pl.cap_f + 1);
    const int64_t f = sdc_upper_index(lo, (int64_t)nf, u);
    b = (int)(u - lo[f]);
    p = pl.fprob[f];
    if (pl.fslot[p] < 0) return false;
    nb0 = (mk[p] + B - 1) / B;
    if (l >= lev_count(nb0) || b >= lev_nb(nb0, l)) return false;
    g = pl.box_base[p] + lev_base(nb0, l) + b;
    return true;
}

// per-level prefix of the box counts of the FMM problems (one CTA per level):
// lev_off by absolute level (leaves 0), top_off by level counted from each
// problem's top box (top 0)
__device__ __forceinline__ int levoff_count(int nb0, int l, bool top)
{
    const int L = lev_count(nb0);
    if (l >= L) return 0;
    return lev_nb(nb0, top ? L - 1 - l : l);
}

__global__ void k_fmm_levoff(const int32_t *__restrict__ mk, const int32_t *__restrict__ fprob,
                             const int32_t *__restrict__ nfmm, int64_t cap_f, int64_t *__restrict__ lev_off,
                             int64_t *__restrict__ top_off)
{
    __shared__ int64_t part[1024];
    const int l = blockIdx.x;
    const int nf = *nfmm;
    const int T = blockDim.x;
    const int per = (nf + T - 1) / T;
    const int beg = min(nf, (int)threadIdx.x * per), end = min(nf, beg + per);
    for (int pass = 0; pass < 2; pass++) {
        const bool top = pass == 1;
        int64_t *out = (top ? top_off : lev_off) + (int64_t)l * (cap_f + 1);
        int64_t sum = 0;
        for (int f = beg; f < end; f++) sum += levoff_count((mk[fprob[f]] + B - 1) / B, l, top);
        __syncthreads();
        part[threadIdx.x] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t acc = 0;
            for (int i = 0; i < T; i++) { const int64_t v = part[i]; part[i] = acc; acc += v; }
            out[nf] = acc;
        }
        __syncthreads();
        int64_t acc = part[threadIdx.x];
        for (int f = beg; f < end; f++) {
            out[f] = acc;
            acc += levoff_count((mk[fprob[f]] + B - 1) / B, l, top);
        }
    }
}

// moments of box g (level l >= 1, index b) from its children's node weights:
// M_n(parent) = sum_children sum_q W_q(child) T_n(alpha x_q + beta), exact
// because T_n(alpha u + beta) has degree n < P and the children's weights
// reproduce every moment of degree < P.  The children's weights are read
// through L2 (ld.global.cg): the sibling's were written by another CTA of the
// same launch, which published them before its arrival count.
template <int WW>
__device__ __forceinline__ void m2m_box(const FmmDev &pl, int64_t p, int nb0, int l, int b, int64_t g, int nw,
                                        double (*Tv)[P + 1], double (*Wc)[WW + 1], double (*Ms)[WW + 1],
                                        const double *Tx, const double *xq)
{
    const int tid = threadIdx.x;
    double cP = 0.0, ihP = 1.0;
    if (tid < 2 * P) {                 // the threads that build Tv (uniform FP64 work costs every warp)
        double hP;
        box_ch(pl.blo[g], pl.bhi[g], cP, hP);
        ihP = rcp_nr2(hP);
    }
    const int nbc = lev_nb(nb0, l - 1);
    const int64_t gcb = pl.box_base[p] + lev_base(nb0, l - 1);
    const int nch = (2 * b + 1 < nbc) ? 2 : 1;
    __syncthreads();
    for (int t = tid; t < 2 * P; t += blockDim.x) {
        const int ci = t / P, q = t % P;
        if (ci >= nch) continue;
        const int64_t gc = gcb + 2 * b + ci;
        double cc, hc;
        box_ch(pl.blo[gc], pl.bhi[gc], cc, hc);
        const double v = fma(hc * ihP, xq[q], (cc - cP) * ihP);    // as scale and shift (see l2l_box)
        double t0 = 1.0, t1 = v;
        Tv[t][0] = 1.0;
        Tv[t][1] = v;
        for (int n = 2; n < P; n++) {
            const double t2 = 2.0 * v * t1 - t0;
            Tv[t][n] = t2;
            t0 = t1; t1 = t2;
        }
    }
    for (int t = tid; t < 2 * P * nw; t += blockDim.x) {
        const int ci = t / (P * nw), r = t % (P * nw);
        if (ci >= nch) continue;
        const int64_t gc = gcb + 2 * b + ci;
        Wc[ci * P + r / nw][r % nw] = __ldcg(&pl.W[(gc * P + r / nw) * pl.ncol + r % nw]);
    }
    __syncthreads();
    for (int t = tid; t < P * nw; t += blockDim.x) {
        const int n = t / nw, q = t % nw;
        double s = 0.0;
        for (int ci = 0; ci < nch; ci++)
            for (int k = 0; k < P; k++) s = fma(Tv[ci * P + k][n], Wc[ci * P + k][q], s);
        Ms[n][q] = s;
    }
    __syncthreads();
    for (int t = tid; t < P * nw; t += blockDim.x) {
        const int qn = t / nw, q = t % nw;
        double s = Ms[0][q];
        for (int n = 1; n < P; n++) s = fma(Tx[qn * P + n], Ms[n][q], s);     // Tx holds 2 T_n
        pl.W[(g * P + qn) * pl.ncol + q] = s * (1.0 / P);
    }
    // children's node positions, the children's weights into moments, moments -> weights
    fl_add(pl, (int64_t)nch * 2 * P * (P - 2) + (int64_t)nch * 2 * P * P * nw + 2 * P * P * nw);
}

// The whole upward pass in one launch: the leaf boxes' moments and node
// weights (grid-stride over the leaf boxes of the FMM problems), then each
// box climbs towards its problem's top box.  A box that has finished its
// weights counts itself into its parent's arrival counter (after a device-
// scope fence); the child that arrives last computes the parent and climbs
// on, the other stops.  No CTA ever waits for another, so any grid size and
// any scheduling order are safe, and every box is computed exactly once, by
// the same arithmetic as a level-by-level pass.  The counter is reset by the
// child that consumes it, ready for the next far field built on the plan.
// Threads and staged columns of the upward pass: the one-column far fields
// (secular, b, Loewner) take 64 threads (one per source of a box of 64, and
// the 2P children's nodes of a box), the Cauchy-like ones 128 and WMAX columns.
template <int MODE> constexpr bool up_wide() { return MODE == M_CT || MODE == M_CN; }
template <int MODE> constexpr int up_threads() { return up_wide<MODE>() ? 128 : 64; }
template <int MODE> constexpr int up_cols() { return up_wide<MODE>() ? WMAX : 1; }

template <int MODE>
__global__ void __launch_bounds__(up_threads<MODE>()) k_fmm_up(FmmDev pl, SrcArgs a)
{
    constexpr int WW = up_cols<MODE>();
    __shared__ double Tt[UP_ROWS][P + 1];
    __shared__ double Wt[UP_ROWS][WW + 1];
    __shared__ double Ms[P][WW + 1];
    __shared__ double Tx[P * P], xq[P];
    __shared__ int last;
    __shared__ int64_t next;
    cheb_tables(xq, Tx, 2.0);          // 2 T_n(x_q), n >= 1: the moments -> weights sums
    const int nw = (MODE == M_CT || MODE == M_CN) ? a.nc : 1;
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (;;) {
        // leaf boxes are claimed one at a time: a CTA that climbs takes fewer
        // (a fixed stride would pile the climbs onto the CTAs that start late)
        __syncthreads();
        if (tid == 0) {
            next = (int64_t)atomicAdd(&pl.upq[0], 1ull);
            if (next >= nleaf && atomicAdd(&pl.upq[1], 1ull) == gridDim.x - 1) {
                pl.upq[0] = 0;                 // every CTA has run past the end: reset for the next launch
                pl.upq[1] = 0;
            }
        }
        __syncthreads();
        const int64_t gl = next;
        if (gl >= nleaf) break;
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        leaf_moments<MODE, WW>(pl, a, p, gl, g, Tb, nw, Tt, Wt, Ms, Tx);
        const int nb0 = (a.mk[p] + B - 1) / B;
        const int L = lev_count(nb0);
        int l = 0, b = Tb;
        while (l + 1 < L) {
            const int bp = b >> 1;
            const int nch = (2 * bp + 1 < lev_nb(nb0, l)) ? 2 : 1;
            const int64_t gp = pl.box_base[p] + lev_base(nb0, l + 1) + bp;
            __threadfence();               // this box's weights, visible before the count
            __syncthreads();
            if (tid == 0) {
                const int old = atomicAdd(&pl.upcnt[gp], 1);
                last = (old == nch - 1);
                if (last) pl.upcnt[gp] = 0;
            }
            __syncthreads();
            if (!last) break;
            __threadfence();
            m2m_box<WW>(pl, p, nb0, l + 1, bp, gp, nw, Tt, Wt, Ms, Tx, xq);
            l++;
            b = bp;
        }
    }
}

// Multipole-to-local: for every box T below the top, the kernel sums of the
// boxes of its interaction list (children of its parent's near list that are
// admissible to T) at T's Chebyshev nodes.  "All near" boxes and the top box
// get no far field.  Kernels (s source, t target):
//   K_SEC: 1/(s-t) and 1/(s-t)^2 into four fields (psi, phi, psi', phi' by side)
//   K_1: 1/(s-t)   K_2: 1/(s-t)^2   K_1N: 1/(t-s)
//   K_LOG: log|s-t|, as its t-derivative 1/(t-s) at the nodes plus the sum
//     itself at the box centre; the derivative's Chebyshev series is
//     integrated exactly, so a box pair costs P logs instead of P^2
enum { K_SEC = 0, K_1 = 1, K_2 = 2, K_1N = 3, K_LOG = 4 };

template <int KER>
// kmode: 0 evaluate the kernel matrices, 1 evaluate and keep the first
// kslots of every box (kmat), 2 read those back (the same enumeration of
// pairs: the plan's tree and near lists do not change between far fields)
__global__ void __launch_bounds__(128) k_fmm_m2l(FmmDev pl, const int32_t *__restrict__ mk, int nw, int kmode)
{
    constexpr int NT = 128;
    constexpr int RMAX = (P * WMAX + NT - 1) / NT;
    __shared__ double xq[P], tq[P], sq[P];
    __shared__ double Tx[P * P];
    __shared__ double Ws[P][WMAX + 1];
    __shared__ double K1[P][P + 1];
    __shared__ double K2[(KER == K_SEC) ? P : 1][P + 1];
    __shared__ double Fp[P], An[P + 2], Bk[P + 1], hk[P + 1], s_f0;
    __shared__ int s_list[32], s_nlist;
    cheb_tables(xq, Tx);
    if (KER == K_LOG && threadIdx.x >= 1 && threadIdx.x <= P) hk[threadIdx.x] = 0.5 / threadIdx.x;   // 1 / (2k)
    const int nf = (KER == K_SEC) ? 4 : nw;
    const int tid = threadIdx.x;
    const int64_t nbox = pl.box_base[pl.nprob];
    for (int64_t g = blockIdx.x; g < nbox; g += gridDim.x) {
        const int64_t p = sdc_upper_index(pl.box_base, pl.nprob, g);
        if (pl.fslot[p] < 0) continue;
        const int m = mk[p];
        const int nb0 = (m + B - 1) / B;
        const int L = lev_count(nb0);
        int local = (int)(g - pl.box_base[p]), l = 0;
        while (local >= lev_nb(nb0, l)) { local -= lev_nb(nb0, l); l++; }
        const int Tb = local;
        double acc[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; r++) acc[r] = 0.0;
        int npair = 0;            // interaction pairs of the box (work counter)
        double f0 = 0.0;          // K_LOG: the far field at the box centre (thread 0)
        double accL = 0.0, accR = 0.0;   // K_SEC: thread t < 2P, node t % P, kernel 1/(s-t)^(1 + t/P),
                                         // sums of the boxes to the left / right
        if (l < L - 1 && pl.nnear[g] >= 0) {
            // FP64 instructions cost a warp slot of the FP64 pipe even when every
            // lane computes the same value, so the box geometry and the
            // admissibility tests run once, in warp 0 (lane-parallel over the
            // candidates), not in every warp
            double cT = 0.0, hT = 1.0;
            if (tid < 32) box_ch(pl.blo[g], pl.bhi[g], cT, hT);
            __syncthreads();
            if (tid < P) tq[tid] = cT + hT * xq[tid];
            const int64_t gbl = pl.box_base[p] + lev_base(nb0, l);
            const int64_t gPT = pl.box_base[p] + lev_base(nb0, l + 1) + (Tb >> 1);
            const int nbl = lev_nb(nb0, l);
            const int npn = pl.nnear[gPT];
            const int64_t pst = pl.nstart[gPT];
            int js = 0;                                   // index of the pair in T's interaction list
            for (int c0 = 0; c0 < 2 * npn; c0 += 32) {
                // candidates c0 .. c0+31: children of the parent's near boxes, in list order
                if (tid < 32) {
                    const int c = c0 + tid;
                    int S = -1;
                    bool ok = false;
                    if (c < 2 * npn) {
                        S = 2 * pl.near[pst + (c >> 1)] + (c & 1);
                        ok = S < nbl && S != Tb && adm(pl.blo[gbl + S], pl.bhi[gbl + S], pl.blo[g], pl.bhi[g]);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    if (ok) s_list[__popc(bal & ((1u << tid) - 1u))] = S;
                    if (tid == 0) s_nlist = __popc(bal);
                }
                __syncthreads();
                const int nlist = s_nlist;
                npair += nlist;
                for (int ii = 0; ii < nlist; ii++) {
                    const int S = s_list[ii];
                    const bool left = S < Tb;
                    const int64_t gS = gbl + S;
                    if (ii > 0) __syncthreads();
                    for (int t = tid; t < P * nw; t += NT) Ws[t / nw][t % nw] = pl.W[(gS * P + t / nw) * pl.ncol + t % nw];
                    if (tid < P) {
                        double cS, hS;
                        box_ch(pl.blo[gS], pl.bhi[gS], cS, hS);
                        sq[tid] = cS + hS * xq[tid];
                    }
                    __syncthreads();
                    const bool kept = js < pl.kslots;
                    double *km = kept ? pl.kmat + ((g * pl.kslots + js) * P) * P : nullptr;
                    js++;
                    for (int t = tid; t < P * P; t += NT) {
                        const int q = t / P, q2 = t % P;
                        double r;                                // 1/(s - t)
                        if (kmode == 2 && kept) {
                            r = km[t];
                        } else {
                            r = rcp_nr2(sq[q2] - tq[q]);
                            if (kmode == 1 && kept) km[t] = r;
                        }
                        if (KER == K_LOG) K1[q][q2] = -r;        // d/dt log|s - t| = 1/(t - s)
                        else if (KER == K_SEC) { K1[q][q2] = r; K2[q][q2] = r * r; }
                        else if (KER == K_1) K1[q][q2] = r;
                        else if (KER == K_1N) K1[q][q2] = -r;
                        else K1[q][q2] = r * r;
                    }
                    __syncthreads();
                    if (KER == K_LOG && tid < 32) {
                        // the log sum itself only at the box centre
                        double v = (tid < P) ? Ws[tid][0] * log(fabs(sq[tid] - cT)) : 0.0;
                        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_down_sync(0xffffffffu, v, sh);
                        if (tid == 0) f0 += v;
                    }
                    if (KER == K_SEC) {
                        // a pair feeds two of the four fields (its side): threads
                        // own (node, kernel) and keep one sum per side, so no lane idles
                        if (tid < 2 * P) {
                            const int q = tid % P;
                            const double(*Km)[P + 1] = (tid < P) ? K1 : K2;
                            double s2 = 0.0;
                            for (int q2 = 0; q2 < P; q2++) s2 = fma(Km[q][q2], Ws[q2][0], s2);
                            if (left) accL += s2; else accR += s2;
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < RMAX; r++) {
                            const int t = tid + r * NT;
                            if (t >= P * nf) break;
                            const int q = t / nf, f = t % nf;
                            double s2 = 0.0;
                            for (int q2 = 0; q2 < P; q2++) s2 = fma(K1[q][q2], Ws[q2][f], s2);
                            acc[r] += s2;
                        }
                    }
                }
                __syncthreads();        // s_list, Ws and the kernel blocks are reused
            }
            if (KER == K_LOG) {
                // F' at the nodes (thread q holds it) -> Chebyshev coefficients,
                // integrated exactly in coefficient space; F = F(centre) +
                // h (G(x_q) - G(0)) with G the antiderivative in u
                if (tid < P) Fp[tid] = acc[0];
                if (tid == 0) s_f0 = f0;
                __syncthreads();
                if (tid < P) {
                    double a = 0.0;
                    for (int q = 0; q < P; q++) a = fma(Fp[q], Tx[q * P + tid], a);
                    An[tid] = a * ((tid == 0) ? (1.0 / P) : (2.0 / P));
                }
                if (tid == 0) { An[P] = 0.0; An[P + 1] = 0.0; }
                __syncthreads();
                // antiderivative coefficients b_k, k = 1..P, once (thread k)
                if (tid >= 1 && tid <= P) {
                    const int k = tid;
                    Bk[k] = (k == 1) ? 0.5 * (2.0 * An[0] - An[2]) : (An[k - 1] - An[k + 1]) * hk[k];
                }
                __syncthreads();
                if (tid < P) {
                    // the degree-P term vanishes at the first-kind nodes but not at 0
                    double gq = 0.0, g0 = 0.0;
                    for (int k = 1; k < P; k++) gq = fma(Bk[k], Tx[tid * P + k], gq);
                    for (int k = 2; k <= P; k += 2) g0 += (k & 2) ? -Bk[k] : Bk[k];      // T_k(0) = (-1)^(k/2)
                    acc[0] = s_f0 + hT * (gq - g0);
                }
            }
        }
        {
            // per pair: the kernel matrix (difference and reciprocal, squared
            // for 1/(s-t)^2) unless read back, and its products with the
            // fields; K_LOG adds the centre's log sum and the integration
            const bool evald = !(kmode == 2 && pl.kslots > 0);
            const int64_t kev = evald ? ((KER == K_SEC || KER == K_2) ? 3 : 2) * P * P : 0;
            const int64_t mv = (KER == K_SEC) ? 4 * P * P : 2 * P * P * nf;
            const int64_t lg = (KER == K_LOG) ? 3 * P : 0;
            fl_add(pl, npair * (kev + mv + lg) + ((KER == K_LOG && npair) ? 4 * P * P : 0));
        }
        if (KER == K_SEC) {
            // fields: 0 psi (left, 1/(s-t)), 1 phi (right), 2 psi', 3 phi'
            if (tid < 2 * P) {
                const int q = tid % P, f = (tid < P) ? 0 : 2;
                pl.F[(g * P + q) * pl.nfield + f] = accL;
                pl.F[(g * P + q) * pl.nfield + f + 1] = accR;
            }
        } else {
#pragma unroll
            for (int r = 0; r < RMAX; r++) {
                const int t = tid + r * NT;
                if (t < P * nf) pl.F[(g * P + t / nf) * pl.nfield + t % nf] = acc[r];
            }
        }
    }
}

// Local-to-local for box g (level l, index b, below its problem's top box):
// add the parent's far field, interpolated at the box's Chebyshev nodes
// (Chebyshev coefficients of the parent's node values, evaluated at
// alpha x_q + beta).  On the leaf level the field is converted to Chebyshev
// coefficients for the targets.  Computed by a group of G threads (a warp, or
// the whole CTA), tid in [0, G); WF the staged width.
template <int G>
__device__ __forceinline__ void grp_sync()
{
    if (G == 32) __syncwarp();
    else __syncthreads();
}

template <int G, int WF>
__device__ __forceinline__ void l2l_box(const FmmDev &pl, int64_t p, int nb0, int l, int b, int64_t g, int nf, int tid,
                                        double (*Fs)[WF + 1], double (*Ac)[WF + 1], double (*Tv)[P + 1],
                                        const double *Tx, const double *xq)
{
    const bool alln = pl.nnear[g] < 0;
    const int64_t gP = pl.box_base[p] + lev_base(nb0, l + 1) + (b >> 1);
    grp_sync<G>();
    if (!alln) {
        // parent's node values
        for (int t = tid; t < P * nf; t += G) Fs[t / nf][t % nf] = pl.F[(gP * P + t / nf) * pl.nfield + t % nf];
        if (tid < P) {
            double cP, hP, cT, hT;
            box_ch(pl.blo[gP], pl.bhi[gP], cP, hP);
            box_ch(pl.blo[g], pl.bhi[g], cT, hT);
            // the node in the parent's variable as alpha x_q + beta: forming the
            // node's position c + h x_q first would round it to the spacing of
            // c, which on a box of one point (h = |c| 1e-15) moves the nodes by
            // several percent of h; a chain of such boxes then re-evaluates the
            // field's rounding noise off the nodes at every level (relative
            // errors up to 1e-7 in zhat of the last pole)
            const double ihP = rcp_nr2(hP);
            const double v = fma(hT * ihP, xq[tid], (cT - cP) * ihP);
            double t0 = 1.0, t1 = v;
            Tv[tid][0] = 1.0;
            Tv[tid][1] = v;
            for (int n = 2; n < P; n++) {
                const double t2 = 2.0 * v * t1 - t0;
                Tv[tid][n] = t2;
                t0 = t1; t1 = t2;
            }
        }
        grp_sync<G>();
        for (int t = tid; t < P * nf; t += G) {
            const int n = t / nf, f = t % nf;
            double s = 0.0;
            for (int q = 0; q < P; q++) s = fma(Fs[q][f], Tx[q * P + n], s);
            Ac[n][f] = s * ((n == 0) ? (1.0 / P) : (2.0 / P));
        }
        grp_sync<G>();
        for (int t = tid; t < P * nf; t += G) {
            const int q = t / nf, f = t % nf;
            double s = pl.F[(g * P + q) * pl.nfield + f];
            for (int n = 0; n < P; n++) s = fma(Tv[q][n], Ac[n][f], s);
            Fs[q][f] = s;     // own row (q, f) only
        }
    } else {
        for (int t = tid; t < P * nf; t += G) Fs[t / nf][t % nf] = 0.0;
    }
    grp_sync<G>();
    // parent's node values -> coefficients -> this box's nodes; on the
    // leaves the field -> coefficients for the targets
    if (tid == 0 && pl.flops) {
        const int64_t v = (alln ? 0 : 2 * P * (P - 2) + 4 * P * P * nf) + ((l == 0) ? 2 * P * P * nf : 0);
        if (v > 0) atomicAdd(pl.flops, (unsigned long long)v);
    }
    if (l > 0) {
        for (int t = tid; t < P * nf; t += G) pl.F[(g * P + t / nf) * pl.nfield + t % nf] = Fs[t / nf][t % nf];
    } else {
        const int64_t gl = pl.leaf_base[p] + b;
        for (int t = tid; t < P * nf; t += G) {
            const int n = t / nf, f = t % nf;
            double s = 0.0;
            for (int q = 0; q < P; q++) s = fma(Fs[q][f], Tx[q * P + n], s);
            pl.coef[(gl * pl.nfield + f) * P + n] = s * ((n == 0) ? (1.0 / P) : (2.0 / P));
        }
    }
}

// Downward pass, launched per top-relative level t0 >= 1 (levels counted from
// each problem's top box, level L-1 of a problem with L levels), one CTA per
// box of level t0 (the parent is final: done by an earlier launch).
//   NARROW (fields of at most NARROW_NF columns: secular, b, Loewner): the
//     CTA also finishes the box's subtree DOWN_LEVELS - 1 levels further
//     down, level by level, a warp per box (the 1, 2, 4, 8 boxes of the four
//     levels take 1, 1, 1, 2 rounds of the four warps), so the narrow fields
//     take a quarter of the launches;
//   wide fields (the Cauchy-like ones, one field per column): one level per
//     launch, the whole CTA on one box.
// Same arithmetic per box either way.
constexpr int DOWN_LEVELS = 4;
constexpr int NARROW_NF = 4;

template <bool NARROW>
__global__ void __launch_bounds__(128) k_fmm_down(FmmDev pl, const int32_t *__restrict__ mk, int t0, int nf)
{
    constexpr int WF = NARROW ? NARROW_NF : WMAX;
    constexpr int NG = NARROW ? 4 : 1;               // box groups per CTA
    constexpr int G = 128 / NG;
    __shared__ double xq[P];
    __shared__ double Tx[P * P];
    __shared__ double Fs[NG][P][WF + 1];
    __shared__ double Ac[NG][P][WF + 1];
    __shared__ double Tv[NG][P][P + 1];
    cheb_tables(xq, Tx);
    const int grp = threadIdx.x / G, tid = threadIdx.x % G;
    const int nf_ = *pl.nfmm;
    const int64_t *lo = pl.top_off + (int64_t)t0 * (pl.cap_f + 1);
    const int64_t nu = lo[nf_];
    for (int64_t u = blockIdx.x; u < nu; u += gridDim.x) {
        const int64_t f = sdc_upper_index(lo, (int64_t)nf_, u);
        const int br = (int)(u - lo[f]);
        const int64_t p = pl.fprob[f];
        if (pl.fslot[p] < 0) continue;
        const int nb0 = (mk[p] + B - 1) / B;
        const int L = lev_count(nb0);
        const int lr = L - 1 - t0;
        if (lr < 0 || br >= lev_nb(nb0, lr)) continue;
        for (int k = 0; k < (NARROW ? DOWN_LEVELS : 1) && lr - k >= 0; k++) {
            const int l = lr - k;
            const int b0 = br << k, bend = min(lev_nb(nb0, l), (br + 1) << k);
            __syncthreads();                   // the parents (previous level) are written
            for (int bb = b0; bb < bend; bb += NG) {
                const int b = bb + grp;
                if (b < bend)
                    l2l_box<G, WF>(pl, p, nb0, l, b, pl.box_base[p] + lev_base(nb0, l) + b, nf, tid, Fs[grp],
                                   Ac[grp], Tv[grp], Tx, xq);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Secular roots of the FMM problems, one warp per leaf box: with boxes of 64
// a lane takes the next root of the box when its root has converged (the
// box's roots share the near list).  The near boxes' poles and weights (fixed
// during the iteration) are staged in shared memory once per box; each sweep
// sums them with shifted differences and evaluates the four far-field
// expansions at x = d_K + y.  Once no root is left to hand out and fewer than
// TAIL_X lanes are busy, the box's stragglers go to k_secular_tail.  The last
// root of each problem (outside the tree) is solved by k_secular_last.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64)
k_secular_fmm(FmmDev pl, const int64_t *__restrict__ off, R1Out o, double stop_c, int max_iter,
              unsigned long long *terms)
{
    __shared__ double sd[2][SPLIT_NEAR * B], sw[2][SPLIT_NEAR * B];
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = (int64_t)blockIdx.x * 2 + warp; gl < nleaf; gl += (int64_t)gridDim.x * 2) {
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int k0 = Tb * B;
        const int kend = min(k0 + B, m - 1);
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
        if (nnr < 0 || nnr >= SPLIT_NEAR) continue;     // long near list: k_secular_fmm_split
        int near_terms = 0;
        __syncwarp();
        for (int i = 0; i < nn; i++) {
            const int j0 = near_box_chk(pl, g, nnr, i, (m + B - 1) / B, o.status) * B;
            const int cnt = min(B, m - j0);
            near_terms += cnt;
            for (int jj = lane; jj < cnt; jj += 32) {
                sd[warp][i * B + jj] = dk[j0 + jj];
                const double z = zk[j0 + jj];
                sw[warp][i * B + jj] = z * z;
            }
        }
        __syncwarp();
        int k = k0 + lane;
        bool act = k < kend;
        int next = k0 + 32;
        Root R;
        R.dK = 0.0; R.y = 1.0; R.phase = 1;
        if (act) R.init(dk, zk, k, m, W, o.unshifted != 0);
        while (__any_sync(FULL, act)) {
            const int kwlo = __reduce_min_sync(FULL, act ? k : 0x7fffffff);
            const int kwhi = __reduce_max_sync(FULL, act ? k : -1);
            const int kk = act ? k : kwlo;
            const bool p0 = __all_sync(FULL, !act || R.phase == 0);
            const unsigned amask = __ballot_sync(FULL, act);
            if (terms && lane == 0) atomicAdd(terms, (unsigned long long)__popc(amask) * (unsigned long long)near_terms);
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
                const int j0 = near_box_chk(pl, g, nnr, i, (m + B - 1) / B, o.status) * B;
                const int cnt = min(B, m - j0);
                const double *bd = sd[warp] + i * B, *bw = sw[warp] + i * B;
                if (p0) sweep<false>(bd, bw, 0, cnt, j0, kk, kwlo, kwhi, R.dK, R.y, A);
                else    sweep<true>(bd, bw, 0, cnt, j0, kk, kwlo, kwhi, R.dK, R.y, A);
            }
            bool fin = false;
            if (act && R.update(A, tol, max_iter, o.status)) {
                o.org[b0 + k] = R.K;
                o.eta[b0 + k] = R.y;
                o.dorg[b0 + k] = R.dK;
                o.lamk[b0 + k] = R.dK + R.y;
                if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                fin = true;
            }
            const unsigned mask = __ballot_sync(FULL, fin);
            if (fin) {
                k = next + __popc(mask & ((1u << lane) - 1u));
                act = k < kend;
                if (act) R.init(dk, zk, k, m, W, o.unshifted != 0);
            }
            next += __popc(mask);
            // no root left to refill and fewer than TAIL_X lanes busy: the
            // stragglers go to k_secular_tail, which runs 32 of them per warp
            if (next >= kend) {
                const unsigned am = __ballot_sync(FULL, act);
                const int nact = __popc(am);
                if (nact > 0 && nact < TAIL_X) {
                    unsigned base = 0;
                    if (lane == 0) base = atomicAdd(pl.ntail, (unsigned)nact);
                    base = __shfl_sync(FULL, base, 0);
                    if (act) {
                        FmmTail tr;
                        tr.p = p; tr.k = k; tr.K = R.K; tr.phase = R.phase; tr.nsw = R.nsw;
                        tr.dK = R.dK; tr.y = R.y; tr.lo = R.lo; tr.hi = R.hi;
                        pl.tail[base + __popc(am & ((1u << lane) - 1u))] = tr;
                    }
                    break;
                }
            }
        }
    }
}

// The stragglers of k_secular_fmm: four lanes per root, each summing every
// fourth pole of each near box of the root's box (poles read through L1),
// combined by a fixed butterfly; the root's far field and update are computed
// by all four lanes alike.  The warps are persistent: a lane group whose root
// has converged claims the next straggler (ntail[1]), so lanes do not wait for
// the slowest root of a fixed batch.  A root's arithmetic does not depend on
// which group runs it.
constexpr int TAIL_LANES = 4;

__global__ void __launch_bounds__(128)
k_secular_tail(FmmDev pl, const int64_t *__restrict__ off, R1Out o, double stop_c, int max_iter,
               unsigned long long *terms)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, part = lane & (TAIL_LANES - 1), lead = lane & ~(TAIL_LANES - 1);
    const unsigned n = pl.ntail[0];
    unsigned *claim = pl.ntail + 1;
    bool act = false, dry = false;
    Root R;
    R.dK = 0.0; R.y = 1.0; R.phase = 1; R.k = 0;
    int64_t b0 = 0, g = 0, gl = 0;
    int m = 1, nnr = 0, nn = 0;
    unsigned nterm = 0;
    double cT = 0.0, ihT = 1.0, tol = 0.0;
    while (true) {
        // groups without a root claim the next one (warp-wide shuffle of the claim)
        const bool need = !act && !dry;
        unsigned idx = 0;
        if (need && part == 0) idx = atomicAdd(claim, 1u);
        idx = __shfl_sync(FULL, idx, lead);
        if (need) {
            if (idx < n) {
                const FmmTail tr = pl.tail[idx];
                const int64_t p = tr.p;
                b0 = off[p];
                m = o.mk[p];
                R.init(o.dk + b0, o.zk + b0, tr.k, m, o.wsum[p], o.unshifted != 0);
                R.K = tr.K; R.phase = tr.phase; R.nsw = tr.nsw;
                R.dK = tr.dK; R.y = tr.y; R.lo = tr.lo; R.hi = tr.hi;
                const int Tb = tr.k / B;
                g = pl.box_base[p] + Tb;
                gl = pl.leaf_base[p] + Tb;
                nnr = pl.nnear[g];
                nn = near_len(nnr, (m + B - 1) / B);
                nterm = 0;
                if (part == 0)
                    for (int i = 0; i < nn; i++) nterm += min(B, m - near_box(pl, g, nnr, i) * B);
                double hT;
                box_ch(pl.blo[g], pl.bhi[g], cT, hT);
                ihT = 1.0 / hT;
                tol = stop_c * (double)m * SDC_EPS;
                act = true;
            } else {
                dry = true;
            }
        }
        if (!__any_sync(FULL, act)) break;
        if (terms) {
            const unsigned nt = __reduce_add_sync(FULL, act ? nterm : 0u);
            if (lane == 0) atomicAdd(terms, (unsigned long long)nt);
        }
        Acc A = {0.0, 0.0, 0.0, 0.0};
        if (act) {
            for (int i = 0; i < nn; i++) {
                const int j0 = near_box_chk(pl, g, nnr, i, (m + B - 1) / B, o.status) * B;
                const int cnt = min(B, m - j0);
                const double *dd = o.dk + b0 + j0, *zz = o.zk + b0 + j0;
                for (int jj = part; jj < cnt; jj += TAIL_LANES) {
                    const double r = rcp_nr1(shifted_t(dd[jj], R.dK, R.y));
                    const double z = zz[jj];
                    const double a = (z * z) * r;
                    if (j0 + jj <= R.k) { A.psi += a; A.dpsi = fma(a, r, A.dpsi); }
                    else                { A.phi += a; A.dphi = fma(a, r, A.dphi); }
                }
            }
        }
        // the four lanes of a root are consecutive: butterfly over lane bits 0, 1
        for (int sh = 1; sh < TAIL_LANES; sh <<= 1) {
            A.psi += __shfl_xor_sync(FULL, A.psi, sh);
            A.phi += __shfl_xor_sync(FULL, A.phi, sh);
            A.dpsi += __shfl_xor_sync(FULL, A.dpsi, sh);
            A.dphi += __shfl_xor_sync(FULL, A.dphi, sh);
        }
        if (act) {
            const double *cf = pl.coef + gl * pl.nfield * P;
            const double uu = ((R.dK + R.y) - cT) * ihT;
            const double u2 = uu + uu;
            double a1 = 0, a2 = 0, b1 = 0, b2 = 0, c1 = 0, c2 = 0, e1 = 0, e2 = 0;
            for (int q = P - 1; q >= 1; q--) {
                double t;
                t = fma(u2, a1, cf[q] - a2);         a2 = a1; a1 = t;
                t = fma(u2, b1, cf[P + q] - b2);     b2 = b1; b1 = t;
                t = fma(u2, c1, cf[2 * P + q] - c2); c2 = c1; c1 = t;
                t = fma(u2, e1, cf[3 * P + q] - e2); e2 = e1; e1 = t;
            }
            A.psi += fma(uu, a1, cf[0] - a2);
            A.phi += fma(uu, b1, cf[P] - b2);
            A.dpsi += fma(uu, c1, cf[2 * P] - c2);
            A.dphi += fma(uu, e1, cf[3 * P] - e2);
            if (R.update(A, tol, max_iter, o.status)) {
                if (part == 0) {
                    const int k = R.k;
                    o.org[b0 + k] = R.K;
                    o.eta[b0 + k] = R.y;
                    o.dorg[b0 + k] = R.dK;
                    o.lamk[b0 + k] = R.dK + R.y;
                    if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                }
                act = false;
            }
        }
    }
}

// Leaf boxes with long near lists (SPLIT_NEAR boxes or more, or "all near"),
// one CTA of SPW warps per box: the warps hold the same 32 roots (replicated
// state), split the near boxes between them and reduce the partial sums
// through shared memory in a fixed order after every sweep; the box's roots
// run in groups of 32.
template <int SPW>
__global__ void __launch_bounds__(SPW * 32)
k_secular_fmm_split(FmmDev pl, const int64_t *__restrict__ off, R1Out o, double stop_c, int max_iter,
                    unsigned long long *terms)
{
    __shared__ double sd[SPW][B], sw[SPW][B];
    __shared__ double red[SPW][4][32];
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nsplit = *pl.nsplit;
    for (int u = blockIdx.x; u < nsplit; u += gridDim.x) {
        const int64_t gl = pl.split[u];                  // a leaf box with a long near list
        const int64_t p = sdc_upper_index(pl.leaf_base, pl.nprob, gl);
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int Tb = (int)(gl - pl.leaf_base[p]);
        const int64_t g = pl.box_base[p] + Tb;
        const int nnr = pl.nnear[g];
        const int nn = near_len(nnr, (m + B - 1) / B);
        const int k0b = Tb * B;
        const int kendb = min(k0b + B, m - 1);
        const double *dk = o.dk + b0, *zk = o.zk + b0;
        const double W = o.wsum[p];
        const double tol = stop_c * (double)m * SDC_EPS;
        double cT, hT;
        box_ch(pl.blo[g], pl.bhi[g], cT, hT);
        const double ihT = 1.0 / hT;
        const double *cf = pl.coef + gl * pl.nfield * P;
        int near_terms = 0;
        if (terms)
            for (int i = 0; i < nn; i++) near_terms += min(B, m - near_box(pl, g, nnr, i) * B);
        for (int k0 = k0b; k0 < kendb; k0 += 32) {
            const int k = k0 + lane;
            bool act = k < kendb;
            Root R;
            R.dK = 0.0; R.y = 1.0; R.phase = 1;
            if (act) R.init(dk, zk, k, m, W, o.unshifted != 0);
            while (__syncthreads_or(act)) {
                const int kwlo = __reduce_min_sync(FULL, act ? k : 0x7fffffff);
                const int kwhi = __reduce_max_sync(FULL, act ? k : -1);
                const int kk = act ? k : kwlo;
                const bool p0 = __all_sync(FULL, !act || R.phase == 0);
                const unsigned amask = __ballot_sync(FULL, act);
                if (terms && warp == 0 && lane == 0)
                    atomicAdd(terms, (unsigned long long)__popc(amask) * (unsigned long long)near_terms);
                Acc A = {0.0, 0.0, 0.0, 0.0};
                if (warp == 0 && act) {
                    const double uu = ((R.dK + R.y) - cT) * ihT;
                    A.psi = clenshaw(cf, uu);
                    A.phi = clenshaw(cf + P, uu);
                    A.dpsi = clenshaw(cf + 2 * P, uu);
                    A.dphi = clenshaw(cf + 3 * P, uu);
                }
                for (int i = warp; i < nn; i += SPW) {
                    const int S = near_box_chk(pl, g, nnr, i, (m + B - 1) / B, o.status);
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
                red[warp][0][lane] = A.psi;
                red[warp][1][lane] = A.phi;
                red[warp][2][lane] = A.dpsi;
                red[warp][3][lane] = A.dphi;
                __syncthreads();
                Acc T = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                for (int w = 0; w < SPW; w++) {      // same order in every warp
                    T.psi += red[w][0][lane];
                    T.phi += red[w][1][lane];
                    T.dpsi += red[w][2][lane];
                    T.dphi += red[w][3][lane];
                }
                __syncthreads();
                if (act && R.update(T, tol, max_iter, warp == 0 ? o.status : nullptr)) {
                    if (warp == 0) {
                        o.org[b0 + k] = R.K;
                        o.eta[b0 + k] = R.y;
                        o.dorg[b0 + k] = R.dK;
                        o.lamk[b0 + k] = R.dK + R.y;
                        if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                    }
                    act = false;
                }
            }
        }
    }
}

// The last root of every FMM problem (in (d_{m-1}, d_{m-1} + sum w]), one CTA
// per problem: boxes at least their own width to the left of the bracket are
// summed through their Chebyshev node weights at the plain position (far
// field), the leaf boxes next to the bracket directly with shifted
// differences; if the lists overflow, every pole directly.  Thread 0 holds
// the root state, the partial sums are reduced in a fixed order.
constexpr int SL_T = 256;

constexpr int LAST_FAR = 112;     // boxes summed through their node weights for the last root
constexpr int LAST_NEAR = 32;     // leaf boxes summed directly for it

__global__ void __launch_bounds__(SL_T)
k_secular_last(FmmDev pl, const int64_t *__restrict__ off, R1Out o, double stop_c, int max_iter,
               unsigned long long *terms)
{
    __shared__ double red[2][SL_T / 32];
    __shared__ double s_dK, s_y;
    __shared__ int s_done, s_p0;
    __shared__ double xq[P];
    __shared__ double fs[LAST_FAR * P], fw[LAST_FAR * P];      // far boxes: node positions, weights
    __shared__ int64_t s_far[LAST_FAR];
    __shared__ int s_near[LAST_NEAR], s_nfar, s_nnear, s_ok;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int q = tid; q < P; q += SL_T) xq[q] = cospi((double)(2 * q + 1) / (2.0 * P));
    const int nf = *pl.nfmm;
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        const int64_t p = pl.fprob[f];
        if (pl.fslot[p] < 0) continue;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const double *dk = o.dk + b0, *zk = o.zk + b0;
        const double tol = stop_c * (double)m * SDC_EPS;
        Root R;
        __syncthreads();
        if (tid == 0) {
            R.init(dk, zk, m - 1, m, o.wsum[p], o.unshifted != 0);
            s_dK = R.dK; s_y = R.y; s_done = 0; s_p0 = 1;
            // every pole lies to the left of the root's bracket [d_{m-1}, d_{m-1} + W]:
            // a box at least its own width away from the bracket is summed
            // through its node weights (multipole to point), the leaf boxes
            // next to it directly; walk the tree from the top
            const int nb0 = (m + B - 1) / B;
            const int L = lev_count(nb0);
            const double tlo = dk[m - 1];
            int nfar = 0, nnear = 0, ok = 1;
            int cand[2 * LAST_NEAR], nc = 1, ncand[2 * LAST_NEAR];
            cand[0] = 0;
            for (int l = L - 1; l >= 0 && ok; l--) {
                const int64_t gb = pl.box_base[p] + lev_base(nb0, l);
                int nn2 = 0;
                for (int i = 0; i < nc && ok; i++) {
                    const int bx = cand[i];
                    const double lo = pl.blo[gb + bx], hi = pl.bhi[gb + bx];
                    if (tlo - hi >= FMM_KAPPA * (hi - lo) && hi > lo) {
                        if (nfar < LAST_FAR) s_far[nfar++] = gb + bx; else ok = 0;
                    } else if (l == 0) {
                        if (nnear < LAST_NEAR) s_near[nnear++] = bx; else ok = 0;
                    } else {
                        const int nbc = lev_nb(nb0, l - 1);
                        for (int c = 2 * bx; c <= 2 * bx + 1 && c < nbc; c++) {
                            if (nn2 < 2 * LAST_NEAR) ncand[nn2++] = c; else ok = 0;
                        }
                    }
                }
                for (int i = 0; i < nn2; i++) cand[i] = ncand[i];
                nc = nn2;
            }
            s_nfar = nfar; s_nnear = nnear; s_ok = ok;
        }
        __syncthreads();
        const bool tree = s_ok != 0;
        const int nfar = s_nfar, nnear = s_nnear;
        int64_t nterms = m;
        if (tree) {
            for (int t = tid; t < nfar * P; t += SL_T) {
                const int64_t g = s_far[t / P];
                const int q = t % P;
                double c, h;
                box_ch(pl.blo[g], pl.bhi[g], c, h);
                fs[t] = c + h * xq[q];
                fw[t] = pl.W[(g * P + q) * pl.ncol];
            }
            nterms = (int64_t)nfar * P;
            for (int i = 0; i < nnear; i++) nterms += min(B, m - s_near[i] * B);
            __syncthreads();
        }
        while (!s_done) {
            const double dK = s_dK, y = s_y;
            const bool p0 = s_p0 != 0;
            double ps = 0.0, dps = 0.0;
            if (tree) {
                // far boxes at the plain position x = d_K + y (local shifting)
                const double x = dK + y;
                for (int t = tid; t < nfar * P; t += SL_T) {
                    const double r = rcp_nr1(fs[t] - x);
                    const double a = fw[t] * r;
                    ps += a;
                    if (!p0) dps = fma(a, r, dps);
                }
                for (int i = 0; i < nnear; i++) {
                    const int j0 = s_near[i] * B, cnt = min(B, m - j0);
                    for (int jj = tid; jj < cnt; jj += SL_T) {
                        const double r = rcp_nr1(shifted_t(dk[j0 + jj], dK, y));
                        const double z = zk[j0 + jj];
                        const double a = (z * z) * r;
                        ps += a;
                        if (!p0) dps = fma(a, r, dps);
                    }
                }
            } else {
                for (int j = tid; j < m; j += SL_T) {
                    const double r = rcp_nr1(shifted_t(dk[j], dK, y));
                    const double z = zk[j];
                    const double a = (z * z) * r;
                    ps += a;
                    if (!p0) dps = fma(a, r, dps);
                }
            }
            for (int sh = 16; sh > 0; sh >>= 1) {
                ps += __shfl_down_sync(FULL, ps, sh);
                dps += __shfl_down_sync(FULL, dps, sh);
            }
            if (lane == 0) { red[0][warp] = ps; red[1][warp] = dps; }
            __syncthreads();
            if (tid == 0) {
                Acc A = {0.0, 0.0, 0.0, 0.0};
                for (int w = 0; w < SL_T / 32; w++) { A.psi += red[0][w]; A.dpsi += red[1][w]; }
                const bool fin = R.update(A, tol, max_iter, o.status);
                if (terms) atomicAdd(terms, (unsigned long long)nterms);
                s_dK = R.dK; s_y = R.y; s_p0 = (R.phase == 0); s_done = fin;
                if (fin) {
                    const int k = m - 1;
                    o.org[b0 + k] = R.K;
                    o.eta[b0 + k] = R.y;
                    o.dorg[b0 + k] = R.dK;
                    o.lamk[b0 + k] = R.dK + R.y;
                    if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                }
            }
            __syncthreads();
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
        int64_t nsrc = 0;
        for (int s = 0; s < nn; s++) {
            const int S = near_box_chk(pl, g, nnr, s, (m + B - 1) / B, o.status);
            const int j0 = S * B;
            const int cnt = min(B, (m - 1) - j0);
            nsrc += max(cnt, 0);
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
        // near ratios (5 each, as the direct kernel), the far field's Clenshaw sum
        const int64_t nt = max(0, min(B, m - Tb * B));
        fl_add(pl, nt * (5 * (nsrc + 1) + 2 * P + 6));
    }
}

// b of the FMM problems, eq. (4.27): near boxes with the shifted entries of
// eq. (4.28), far boxes by expansion at lambda_j = d_{K_j} + eta_j.  The last
// target j = m-1 (outside the tree) is summed directly, spread over the leaf
// boxes: each box adds up its own sources in a fixed order into lastp, and
// k_fmm_lastsum combines the boxes (so no single CTA walks all m sources).
__global__ void __launch_bounds__(B) k_bnorm_fmm(FmmDev pl, const int64_t *__restrict__ off, R1Out o)
{
    __shared__ double sd[B], sv[B];
    __shared__ double red[B];
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = blockIdx.x; gl < nleaf; gl += gridDim.x) {
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
        int64_t nsrc = 0;
        for (int q = 0; q < nn; q++) {
            const int S = near_box_chk(pl, g, nnr, q, (m + B - 1) / B, o.status);
            const int i0 = S * B;
            const int cnt = min(B, m - i0);
            nsrc += max(cnt, 0);
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
        // this box's sources in the sum for the last target
        double t = 0.0;
        if (j < m) {
            const double r = rcp_nr2((o.dk[b0 + j] - o.dorg[b0 + m - 1]) - o.eta[b0 + m - 1]);
            const double vr = o.vhat[b0 + j] * r;
            t = vr * vr;
        }
        __syncthreads();
        red[tid] = t;
        __syncthreads();
        if (tid == 0) {
            double a = 0.0;
            for (int q = 0; q < B; q++) a += red[q];
            pl.lastp[gl * pl.ncol] = a;
        }
        // near terms (6 each, as the direct kernel), Clenshaw, the last target's share
        const int64_t nt = max(0, min(B, (m - 1) - Tb * B)), ns = max(0, min(B, m - Tb * B));
        fl_add(pl, nt * (6 * nsrc + 2 * P + 2) + ns * 7);
    }
}

// The last eigenvalue's sums from the leaf boxes' shares (lastp), one warp per
// (FMM problem, column), in a fixed order: lane-strided partial sums, then a
// butterfly.  MODE 0: b_{m-1} = sum^{-1/2} into bout.  MODE 1: row pinv_{m-1}
// of Y = Qhat^T X, b_{m-1} (from bnorm) times the sum.
template <int MODE>
__global__ void __launch_bounds__(128) k_fmm_lastsum(FmmDev pl, const int64_t *__restrict__ off,
                                                     const int32_t *__restrict__ mk, double *__restrict__ bout,
                                                     const double *__restrict__ bnorm,
                                                     const int32_t *__restrict__ pinv, double *__restrict__ Y,
                                                     int64_t ldy, int col0, int nc)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)(*pl.nfmm) * nc;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t p = pl.fprob[w / nc];
        const int q = (int)(w % nc);
        if (pl.fslot[p] < 0) continue;
        const int64_t l0 = pl.leaf_base[p], l1 = pl.leaf_base[p + 1];
        double a = 0.0;
        for (int64_t gl = l0 + lane; gl < l1; gl += 32) a += pl.lastp[gl * pl.ncol + q];
        for (int sh = 16; sh > 0; sh >>= 1) a += __shfl_xor_sync(0xffffffffu, a, sh);
        if (lane == 0) {
            const int64_t b0 = off[p];
            const int m = mk[p];
            if (MODE == 0) bout[b0 + m - 1] = 1.0 / sqrt(a);
            else Y[b0 + pinv[b0 + m - 1] + (int64_t)(col0 + q) * ldy] = bnorm[b0 + m - 1] * a;
        }
    }
}

// Y = Qhat^T X (columns [col0, col0+nc)) for the FMM problems:
//   y_{pinv_j} = b_j sum_i vhat_i x_{src_i} / ((d_i - d_{K_j}) - eta_j)
// The row of the last eigenvalue (outside the tree) is summed directly,
// spread over the leaf boxes (lastp, then k_fmm_lastsum).
template <int NC>
__global__ void __launch_bounds__(B)
k_cauchyT_fmm(FmmDev pl, FactorView f, const double *__restrict__ X, int64_t ldx, double *__restrict__ Y,
              int64_t ldy, int col0, int nc)
{
    __shared__ double sd[B];
    __shared__ double sx[NC][B + 1];
    const int tid = threadIdx.x;
    const int64_t nleaf = pl.leaf_base[pl.nprob];
    for (int64_t gl = blockIdx.x; gl < nleaf; gl += gridDim.x) {
        double acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) acc[q] = 0.0;
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
        int64_t nsrc = 0;
        for (int s = 0; s < nn; s++) {
            const int S = SDC_IDX(near_box(pl, g, nnr, s), (m + B - 1) / B, f.status);
            const int i0 = S * B;
            const int cnt = min(B, m - i0);
            nsrc += max(cnt, 0);
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
                // two sources per iteration: the next reciprocal's dependent
                // chain overlaps this one's column FMAs (same order per column)
#pragma unroll 2
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
        // this box's sources in the row of the last eigenvalue
        __syncthreads();
        if (j < m) {
            const double r = rcp_nr2((f.dk[b0 + j] - f.dorg[b0 + m - 1]) - f.eta[b0 + m - 1]);
            const double v = f.vhat[b0 + j] * r;
            const int64_t row = b0 + f.src[b0 + j];
#pragma unroll
            for (int q = 0; q < NC; q++) sx[q][tid] = (q < nc) ? v * X[row + (int64_t)(col0 + q) * ldx] : 0.0;
        } else {
#pragma unroll
            for (int q = 0; q < NC; q++) sx[q][tid] = 0.0;
        }
        __syncthreads();
        for (int q = tid; q < nc; q += B) {
            double t = 0.0;
            for (int i = 0; i < B; i++) t += sx[q][i];
            pl.lastp[gl * pl.ncol + q] = t;
        }
        // near terms (difference, reciprocal, one FMA per column), Clenshaw
        // and the scale by b per column, the last row's share per source
        const int64_t nt = max(0, min(B, (m - 1) - Tb * B)), ns = max(0, min(B, m - Tb * B));
        fl_add(pl, nt * (nsrc * (3 + 2 * nc) + (2 * P + 1) * nc) + ns * (4 + 2 * nc));
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
        int64_t nsrc = 0;
        for (int s = 0; s < nn; s++) {
            const int S = SDC_IDX(near_box(pl, g, nnr, s), (m + B - 1) / B, f.status);
            const int j0 = S * B;
            const int cnt = min(B, (m - 1) - j0);
            nsrc += max(cnt, 0);
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
#pragma unroll 2
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
        // near terms and the last source (difference, reciprocal, one FMA
        // per column), Clenshaw and the scale by vhat per column
        const int64_t nt = max(0, min(B, m - Tb * B));
        fl_add(pl, nt * ((nsrc + 1) * (3 + 2 * nc) + (2 * P + 1) * nc));
    }
}

unsigned fmm_grid() { return (unsigned)(sdc_num_sms() * 8); }

// As many CTAs of kernel K as the GPU holds at once (threads per CTA, static
// shared memory only), from the occupancy calculator, once per device: the
// grid of kernels whose CTAs take equal shares of the work (a second, partial
// wave would double the launch).
template <auto K>
unsigned resident_grid(int threads)
{
    static std::mutex mu;
    static int per_sm[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return (unsigned)sdc_num_sms();
    std::lock_guard<std::mutex> lk(mu);
    if (per_sm[dev] == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, K, threads, 0) != cudaSuccess) v = 1;
        per_sm[dev] = v > 0 ? v : 1;
    }
    return (unsigned)(sdc_num_sms() * per_sm[dev]);
}

template <int MODE>
unsigned up_grid() { return resident_grid<k_fmm_up<MODE>>(up_threads<MODE>()); }

// one warp per (FMM problem, column) of k_fmm_lastsum, 4 warps per CTA
unsigned lastsum_grid(const FmmPlan &pl, int nc)
{
    const int64_t w = std::max<int64_t>(1, pl.cap_f) * nc;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((w + 3) / 4, (int64_t)sdc_num_sms() * 8));
}

// grid of a downward-pass launch: at most one CTA per box that top-relative
// level t0 can hold (a problem has at most 2^t0 boxes there, and at most its
// leaf boxes)
unsigned down_grid(const FmmPlan &pl, int t0)
{
    const int64_t per = (t0 >= 30) ? (int64_t)pl.nb0max : std::min<int64_t>(pl.nb0max, (int64_t)1 << t0);
    const int64_t nb = per * std::max<int64_t>(1, pl.cap_f);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)sdc_num_sms() * 8));
}

SrcArgs src_from_r1(const int64_t *off, const R1Out &o)
{
    SrcArgs a{};
    a.off = off; a.mk = o.mk; a.dk = o.dk; a.zk = o.zk; a.vhat = o.vhat; a.bnorm = o.bnorm;
    a.dorg = o.dorg; a.eta = o.eta; a.src = o.src; a.pinv = o.pinv;
    return a;
}

template <int MODE, int KER>
superdc_status far_field(const FmmPlan &pl, const SrcArgs &a, int nw, int kmode, cudaStream_t st)
{
    const FmmDev &dv = pl.dv;
    const unsigned g = fmm_grid();
    const int nf = (KER == K_SEC) ? 4 : nw;
    PROF_LAUNCH("fmm_up", st, k_fmm_up<MODE><<<up_grid<MODE>(), up_threads<MODE>(), 0, st>>>(dv, a));
    PROF_LAUNCH("fmm_m2l", st, k_fmm_m2l<KER><<<g, 128, 0, st>>>(dv, a.mk, nw, dv.kslots > 0 ? kmode : 0));
    if (nf <= NARROW_NF) {
        for (int t0 = 1; t0 < pl.lmax; t0 += DOWN_LEVELS)
            PROF_LAUNCH("fmm_l2l", st, k_fmm_down<true><<<down_grid(pl, t0), 128, 0, st>>>(dv, a.mk, t0, nf));
    } else {
        for (int t0 = 1; t0 < pl.lmax; t0++)
            PROF_LAUNCH("fmm_l2l", st, k_fmm_down<false><<<down_grid(pl, t0), 128, 0, st>>>(dv, a.mk, t0, nf));
    }
    return SUPERDC_OK;
}

// grids: 8 CTAs per SM, or what fits when the column count's accumulators
// leave room for fewer
template <int NC>
void launch_ct(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y, int64_t ldy, int col0,
               int nc, cudaStream_t st)
{
    const unsigned g = std::min(fmm_grid(), resident_grid<k_cauchyT_fmm<NC>>(B));
    k_cauchyT_fmm<NC><<<g, B, 0, st>>>(pl.dv, f, X, ldx, Y, ldy, col0, nc);
}

template <int NC>
void launch_cn(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y, int64_t ldy, int col0,
               int nc, cudaStream_t st)
{
    const unsigned g = std::min(fmm_grid(), resident_grid<k_cauchyN_fmm<NC>>(B));
    k_cauchyN_fmm<NC><<<g, B, 0, st>>>(pl.dv, f, X, ldx, Y, ldy, col0, nc);
}

}  // namespace


superdc_status plan(FmmPlan &pl, int64_t nprob, const int64_t *off, int64_t total, int64_t max_m,
                        const int32_t *mk, const double *dk, int min_m, int ncol, int nfield, int32_t *used,
                        int kslots, cudaStream_t st)
{
    pl = FmmPlan();
    pl.box = B;
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
    pl.nb0max = nb0max;
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
    int64_t *nstart;
    double *blo, *bhi;
    SDC_CHECK(al(&box_base, nprob + 1));
    SDC_CHECK(al(&leaf_base, nprob + 1));
    SDC_CHECK(al(&fslot, nprob));
    SDC_CHECK(al(&fprob, nf_cap));
    SDC_CHECK(al(&nfmm, 1));
    SDC_CHECK(al(&blo, pl.cap_boxes));
    SDC_CHECK(al(&bhi, pl.cap_boxes));
    SDC_CHECK(al(&nnear, pl.cap_boxes));
    SDC_CHECK(al(&near, pl.cap_boxes * FMM_NPOOL));
    SDC_CHECK(al(&nstart, pl.cap_boxes));
    SDC_CHECK(al(&d.W, (size_t)pl.cap_boxes * P * ncol));
    SDC_CHECK(al(&d.coef, (size_t)pl.cap_leaves * nfield * P));
    SDC_CHECK(al(&d.F, (size_t)pl.cap_boxes * P * nfield));
    SDC_CHECK(al(&d.lastp, (size_t)pl.cap_leaves * ncol));
    SDC_CHECK(al(&d.tail, (size_t)std::max<int64_t>(1, total)));
    SDC_CHECK(al(&d.ntail, 2));
    SDC_CHECK(cudaMemsetAsync(d.ntail, 0, 2 * sizeof(unsigned int), st));
    // kernel matrices kept for the later far fields of this plan, if they fit
    // a few GB (otherwise every far field evaluates its own)
    const double kbytes = (double)pl.cap_boxes * kslots * P * P * sizeof(double);
    d.kslots = (kslots > 0 && kbytes <= 8.0e9) ? kslots : 0;
    d.kmat = nullptr;
    if (d.kslots > 0) SDC_CHECK(al(&d.kmat, (size_t)pl.cap_boxes * d.kslots * P * P));
    int64_t *lev_off, *top_off;
    SDC_CHECK(al(&lev_off, (size_t)pl.lmax * (nf_cap + 1)));
    SDC_CHECK(al(&top_off, (size_t)pl.lmax * (nf_cap + 1)));
    SDC_CHECK(al(&d.upcnt, pl.cap_boxes));
    SDC_CHECK(cudaMemsetAsync(d.upcnt, 0, (size_t)pl.cap_boxes * sizeof(int32_t), st));
    SDC_CHECK(al(&d.upq, 2));
    SDC_CHECK(al(&d.split, pl.cap_leaves));
    SDC_CHECK(al(&d.nsplit, 1));
    SDC_CHECK(cudaMemsetAsync(d.upq, 0, 2 * sizeof(unsigned long long), st));
    d.lev_off = lev_off;
    d.top_off = top_off;
    d.cap_f = nf_cap;

    d.flops = prof_counter("fmm_flops");
    d.box_base = box_base; d.leaf_base = leaf_base; d.fslot = fslot; d.fprob = fprob; d.nfmm = nfmm;
    d.blo = blo; d.bhi = bhi; d.nnear = nnear; d.near = near; d.nstart = nstart;
    PROF_LAUNCH("fmm_plan", st, k_fmm_plan<<<1, 1024, 0, st>>>(nprob, mk, min_m, pl.cap_boxes, pl.cap_leaves,
                                                               pl.cap_f, box_base, leaf_base, fslot, fprob, nfmm));
    // one CTA per problem; a batch of fewer problems than SMs (the top tree
    // levels) gives each tree 1024 threads instead of 256
    const unsigned gt = (unsigned)std::min<int64_t>(nprob, (int64_t)sdc_num_sms() * 4);
    const int tt = (nprob < sdc_num_sms()) ? 1024 : 256;
    SDC_CHECK(cudaMemsetAsync(d.nsplit, 0, sizeof(int32_t), st));
    PROF_LAUNCH("fmm_tree", st, k_fmm_tree<<<gt, tt, 0, st>>>(nprob, off, mk, dk, box_base, fslot, blo, bhi,
                                                               nnear, nstart, near, used, leaf_base, d.split,
                                                               d.nsplit));
    PROF_LAUNCH("fmm_plan", st, k_fmm_levoff<<<pl.lmax, 1024, 0, st>>>(mk, fprob, nfmm, nf_cap, lev_off,
                                                                   top_off));
    SDC_CHECK(cudaGetLastError());
    pl.on = true;
    return SUPERDC_OK;
}

void free_plan(FmmPlan &pl, cudaStream_t st)
{
    for (void *p : pl.bufs) cudaFreeAsync(p, st);
    pl.bufs.clear();
    pl.on = false;
}

superdc_status secular(const FmmPlan &pl, const int64_t *off, const R1Out &o, double stop_c, int max_iter,
                           cudaStream_t st)
{
    if (!pl.on) return SUPERDC_OK;
    far_field<M_SEC, K_SEC>(pl, src_from_r1(off, o), 1, 1, st);      // keeps the kernel matrices
    const unsigned gl = (unsigned)std::max<int64_t>(1, std::min<int64_t>(pl.cap_f, (int64_t)sdc_num_sms() * 2));
    unsigned long long *terms = prof_counter("fmm_secular_terms");
    unsigned long long *lterms = prof_counter("fmm_secular_last_terms");
    PROF_LAUNCH("fmm_secular_last", st, k_secular_last<<<gl, SL_T, 0, st>>>(pl.dv, off, o, stop_c, max_iter,
                                                                             lterms));
    PROF_LAUNCH("fmm_secular", st, k_secular_fmm<<<fmm_grid(), 64, 0, st>>>(pl.dv, off, o, stop_c, max_iter,
                                                                             terms));
    PROF_LAUNCH("fmm_secular", st, k_secular_tail<<<(unsigned)(sdc_num_sms() * 4), 128, 0, st>>>(
                                       pl.dv, off, o, stop_c, max_iter, terms));
    PROF_LAUNCH("fmm_secular", st, (k_secular_fmm_split<8><<<fmm_grid(), 256, 0, st>>>(pl.dv, off, o, stop_c,
                                                                                      max_iter, terms)));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

superdc_status lowner(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st)
{
    if (!pl.on) return SUPERDC_OK;
    far_field<M_LOW, K_LOG>(pl, src_from_r1(off, o), 1, 2, st);      // reads them
    PROF_LAUNCH("fmm_lowner", st, k_lowner_fmm<<<fmm_grid(), B, 0, st>>>(pl.dv, off, o));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

superdc_status bnorm(const FmmPlan &pl, const int64_t *off, const R1Out &o, cudaStream_t st)
{
    if (!pl.on) return SUPERDC_OK;
    far_field<M_BN, K_2>(pl, src_from_r1(off, o), 1, 2, st);
    PROF_LAUNCH("fmm_bnorm", st, k_bnorm_fmm<<<fmm_grid(), B, 0, st>>>(pl.dv, off, o));
    PROF_LAUNCH("fmm_bnorm", st, k_fmm_lastsum<0><<<lastsum_grid(pl, 1), 128, 0, st>>>(
                                     pl.dv, off, o.mk, o.bnorm, nullptr, nullptr, nullptr, 0, 0, 1));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

superdc_status cauchy(const FmmPlan &pl, const FactorView &f, const double *X, int64_t ldx, double *Y,
                          int64_t ldy, int col0, int nc, bool trans, cudaStream_t st)
{
    if (!pl.on || nc <= 0) return SUPERDC_OK;
    if (nc > WMAX || nc > pl.dv.ncol || nc > pl.dv.nfield) return SUPERDC_ERR_ARG;
    SrcArgs a{};
    a.off = f.off; a.mk = f.mk; a.dk = f.dk; a.vhat = f.vhat; a.bnorm = f.bnorm; a.dorg = f.dorg; a.eta = f.eta;
    a.src = f.src; a.pinv = f.pinv; a.X = X; a.ldx = ldx; a.col0 = col0; a.nc = nc;
    // a plan kept from the factor's rank-one step holds its M2L kernel matrices
    if (trans) far_field<M_CT, K_1>(pl, a, nc, 2, st);
    else far_field<M_CN, K_1N>(pl, a, nc, 2, st);
    typedef void (*Fn)(const FmmPlan &, const FactorView &, const double *, int64_t, double *, int64_t, int, int,
                       cudaStream_t);
    Fn fn;
    // the inner loops run all NC columns: even widths up to 20 (the ranks of
    // typical HSS generators) waste at most one FMA per term
#define SDC_FMM_NC(W) else if (nc <= W) fn = trans ? launch_ct<W> : launch_cn<W>;
    if (false) {}
    SDC_FMM_NC(2) SDC_FMM_NC(4) SDC_FMM_NC(6) SDC_FMM_NC(8) SDC_FMM_NC(10) SDC_FMM_NC(12)
    SDC_FMM_NC(14) SDC_FMM_NC(16) SDC_FMM_NC(18) SDC_FMM_NC(20) SDC_FMM_NC(24)
    else fn = trans ? launch_ct<32> : launch_cn<32>;
#undef SDC_FMM_NC
    PROF_LAUNCH("fmm_cauchy", st, fn(pl, f, X, ldx, Y, ldy, col0, nc, st));
    if (trans)
        PROF_LAUNCH("fmm_cauchy", st, k_fmm_lastsum<1><<<lastsum_grid(pl, nc), 128, 0, st>>>(
                                          pl.dv, f.off, f.mk, nullptr, f.bnorm, f.pinv, Y, ldy, col0, nc));
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}

}  // namespace FMM_NS
