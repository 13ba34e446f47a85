// SuperDC eigendecomposition of a symmetric HSS matrix on sm_103a (FP64).
//
//   superdc_build_hss -- library-owned copy of the generators + tree levels;
//   superdc_eig       -- Algorithm 1 (dividing, balanced form eqs. (3.11)/(3.12),
//                        accumulated generator updates of Lemma 2.1), leaf
//                        eigendecompositions, then Algorithm 3 level by level:
//                        every node of a level is one problem of the batched
//                        rank-one pipeline (rank1.cu), so a whole level runs
//                        in one launch per kernel;
//   superdc_apply_Q   -- Algorithm 4 at the root (Q or Q^T times a block).
//
// Zhat_p = diag(Q_c1^T, Q_c2^T) Z_p (eq. (2.8)) is formed from W_c = Q_c^T U_c:
// with Z_p = [U_c1 Bt/sqrt(beta); sqrt(beta) U_c2] (eq. (3.12)),
// Zhat_p = [W_c1 Bt/sqrt(beta); sqrt(beta) W_c2], and W_p = Qhat_p^T P_p
// [W_c1 R_c1; W_c2 R_c2] is carried through the r rank-one steps of node p
// as r extra columns.  This equals Algorithm 3's superdcmv route in exact
// arithmetic and avoids re-applying whole subtrees.
#include <algorithm>
#include <string>
#include <cmath>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "rank1.cuh"
#include "cauchy.cuh"
#include "fmm.cuh"
#include "prof.cuh"

#include <mutex>
#include "handles.cuh"

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t n, std::vector<char *> *own)
{
    cudaError_t e = sdc_malloc(p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess && own) own->push_back((char *)*p);
    return e;
}

// ---------------------------------------------------------------------------
// Dividing stage, one CTA per non-leaf node of a level (top-down); with
// balanced = 0 the original dividing (beta replaced by 1; ablation).
// For node i with children c1, c2 and accumulated update H_i (D_i -> D_i - U_i H_i U_i^T):
//   Bt = B_c1 - R_c1 H_i R_c2^T                    (Lemma 2.1)
//   beta = ||Bt||_2
//   H_c1 = R_c1 H_i R_c1^T + Bt Bt^T / beta,  H_c2 = R_c2 H_i R_c2^T + beta I   (eq. (3.12))
//   Zhat scale: Bts = Bt / sqrt(beta), sqb = sqrt(beta)
// H_root = 0 (the R generators of the root's children are never read).
// ---------------------------------------------------------------------------
__device__ void jacobi_small_maxeig(double *G, int r, double *out, double *V)
{
    // cyclic Jacobi on the r x r symmetric matrix G (column-major, shared
    // memory), called by all 32 lanes of one warp (r <= 32): the rotation
    // parameters are computed by every lane alike, the row, column and V
    // updates one index per lane, the norms by lane 0 in the serial order, so
    // every entry sees the same operations in the same order as in a one-thread
    // sweep (a lone thread spent ~1 ms per node on these dependent chains).
    // V (r x r, may be NULL) accumulates the rotations; *out = largest
    // eigenvalue, V's first column is overwritten with its eigenvector
    const unsigned FULL = 0xffffffffu;
    const int k = threadIdx.x & 31;
    double fro = 0;
    if (k == 0) {
        for (int i = 0; i < r * r; i++) fro += G[i] * G[i];
        fro = sqrt(fro);
    }
    fro = __shfl_sync(FULL, fro, 0);
    if (V && k < r)
        for (int i = 0; i < r; i++) V[i + r * k] = (i == k) ? 1.0 : 0.0;
    __syncwarp();
    for (int sw = 0; sw < 60; sw++) {
        double off = 0;
        if (k == 0)
            for (int j = 0; j < r; j++)
                for (int i = 0; i < r; i++)
                    if (i != j) off += G[i + r * j] * G[i + r * j];
        off = __shfl_sync(FULL, off, 0);
        if (sqrt(off) <= SDC_EPS * fro) break;
        for (int p = 0; p < r - 1; p++)
            for (int q = p + 1; q < r; q++) {
                const double apq = G[p + r * q];
                if (apq == 0.0) continue;
                const double app = G[p + r * p], aqq = G[q + r * q];
                const double zeta = (aqq - app) / (2.0 * apq);
                const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                                      : ((zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta)));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                __syncwarp();
                if (k < r) {
                    const double gp = G[p + r * k], gq = G[q + r * k];
                    G[p + r * k] = c * gp - sn * gq;
                    G[q + r * k] = sn * gp + c * gq;
                }
                __syncwarp();
                if (k < r) {
                    const double gp = G[k + r * p], gq = G[k + r * q];
                    G[k + r * p] = c * gp - sn * gq;
                    G[k + r * q] = sn * gp + c * gq;
                    if (V) {
                        const double vp = V[k + r * p], vq = V[k + r * q];
                        V[k + r * p] = c * vp - sn * vq;
                        V[k + r * q] = sn * vp + c * vq;
                    }
                }
                __syncwarp();
            }
    }
    double mx = G[0];
    int im = 0;
    for (int i = 1; i < r; i++) if (G[i + r * i] > mx) { mx = G[i + r * i]; im = i; }
    *out = fmax(mx, 0.0);
    if (V && im != 0 && k < r) V[k] = V[k + r * im];
    __syncwarp();
}

__global__ void k_divide(const int32_t *__restrict__ nodes, int root, int r, const int32_t *__restrict__ lch,
                         const int32_t *__restrict__ rch, const double *__restrict__ R,
                         const double *__restrict__ B, double *__restrict__ H, double *__restrict__ Bts,
                         double *__restrict__ sqb, int32_t *status, double *__restrict__ tBt,
                         double *__restrict__ tbeta, double *__restrict__ tu1, double *__restrict__ tv1,
                         int balanced, double *__restrict__ bnrm)
{
    extern __shared__ double sm[];
    const int rr = r * r;
    double *Hi = sm, *R1 = sm + rr, *R2 = sm + 2 * rr, *Bt = sm + 3 * rr, *T1 = sm + 4 * rr, *T2 = sm + 5 * rr,
           *G = sm + 6 * rr, *Vg = sm + 7 * rr;
    __shared__ double s_beta;
    const int i = nodes[blockIdx.x];
    const int c1 = lch[i], c2 = rch[i];
    const bool isroot = (i == root);
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        Hi[e] = isroot ? 0.0 : H[(int64_t)i * rr + e];
        R1[e] = isroot ? 0.0 : R[(int64_t)c1 * rr + e];
        R2[e] = isroot ? 0.0 : R[(int64_t)c2 * rr + e];
        Bt[e] = B[(int64_t)c1 * rr + e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {      // T1 = R1 Hi, T2 = R2 Hi
        int a = e % r, b = e / r;
        double s1 = 0, s2 = 0;
        for (int k = 0; k < r; k++) { s1 += R1[a + r * k] * Hi[k + r * b]; s2 += R2[a + r * k] * Hi[k + r * b]; }
        T1[e] = s1;
        T2[e] = s2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {      // Bt - T1 R2^T, staged in G
        int a = e % r, b = e / r;
        double s = 0;
        for (int k = 0; k < r; k++) s += T1[a + r * k] * R2[b + r * k];
        G[e] = Bt[e] - s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += blockDim.x) Bt[e] = G[e];
    __syncthreads();
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {       // G = Bt^T Bt
        int a = e % r, b = e / r;
        double s = 0;
        for (int k = 0; k < r; k++) s += Bt[k + r * a] * Bt[k + r * b];
        G[e] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double mx;
        jacobi_small_maxeig(G, r, &mx, Vg);
        if (threadIdx.x == 0) {
            s_beta = sqrt(fmax(mx, 0.0));
            if (!isfinite(s_beta)) sdc_latch(status, SUPERDC_DEV_NONFINITE);
        }
    }
    __syncthreads();
    // balanced dividing (eqs. (3.11)/(3.12)) scales by beta = ||Bt||_2; the
    // original one (eqs. (2.4)/(2.5)) by 1: H_c1 += Bt Bt^T, H_c2 += I
    const double beta = balanced ? s_beta : 1.0;
    if (bnrm && threadIdx.x == 0) bnrm[i] = s_beta;
    if (tBt) {      // forward tape for the adjoint: Bt, beta, top singular pair u1 = Bt v1 / beta, v1
        for (int e = threadIdx.x; e < rr; e += blockDim.x) tBt[(int64_t)i * rr + e] = Bt[e];
        for (int a = threadIdx.x; a < r; a += blockDim.x) {
            double sv = 0;
            for (int k = 0; k < r; k++) sv += Bt[a + r * k] * Vg[k];
            tu1[(int64_t)i * r + a] = (beta > 0) ? sv / beta : 0.0;
            tv1[(int64_t)i * r + a] = Vg[a];
        }
        if (threadIdx.x == 0) tbeta[i] = beta;
    }
    const double sb = sqrt(beta);
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        int a = e % r, b = e / r;
        double h1 = 0, h2 = 0, bb = 0;
        for (int k = 0; k < r; k++) {
            h1 += T1[a + r * k] * R1[b + r * k];
            h2 += T2[a + r * k] * R2[b + r * k];
            bb += Bt[a + r * k] * Bt[b + r * k];
        }
        if (beta > 0) h1 += bb / beta;
        if (a == b) h2 += beta;
        H[(int64_t)c1 * rr + e] = h1;
        H[(int64_t)c2 * rr + e] = h2;
        Bts[(int64_t)i * rr + e] = (beta > 0) ? Bt[e] / sb : 0.0;
    }
    if (threadIdx.x == 0) sqb[i] = sb;
}

// ---------------------------------------------------------------------------
constexpr int LEAF_T = 256;

// Leaf eigendecompositions Dhat = D - U H U^T = Q diag(lambda) Q^T (Lemma 2.1).
//   k_leaf_tri    one CTA per leaf: Dhat, Householder reduction to tridiagonal
//                 form (d, e), the orthogonal factor formed in place from the
//                 reflectors; Q (row-major, unsorted) to the leaf's output slot.
// Then implicit QL iterations with the usual shift from the leading 2x2 block
// on (d, e).  A QL sweep is one chain of dependent scalar steps, and on this
// GPU a scalar FP64 chain is slow, so the chains run in parallel:
//   large leaves (one CTA per SM): k_leaf_ql runs one leaf per lane and
//                 records every sweep's rotations; k_leaf_rot applies them to
//                 the rows of Q (each row independently, a leaf's rows split
//                 over several CTAs), k_leaf_out sorts and emits;
//   small leaves: k_leaf_qlcta, in each leaf's CTA, thread 0 computes one
//                 sweep while the other warps apply the previous one, and
//                 several CTAs share an SM.
// Outputs: eigenvalues ascending (ties by index), Q columns in that order,
// W = Q^T U.  The FP64 work is about 4 m^3 per leaf (cyclic Jacobi needs about
// 10 sweeps of 4 m^3).
__global__ void __launch_bounds__(LEAF_T)
k_leaf_tri(int r, const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ leaf_m,
           const int64_t *__restrict__ leaf_doff, const int64_t *__restrict__ leaf_uoff,
           const int32_t *__restrict__ leaf_id, const double *__restrict__ D, const double *__restrict__ U,
           const double *__restrict__ H, double *__restrict__ Qleaf, const int64_t *__restrict__ qoff,
           double *__restrict__ dout, double *__restrict__ eout)
{
    extern __shared__ double sm[];
    __shared__ double dg[128], ee[128], hh[128];
    __shared__ double red[LEAF_T / 32];
    __shared__ double s_ih;
    const int L = blockIdx.x;
    const int m = (int)leaf_m[L];
    const int lda = m | 1;
    double *A = sm;                              // m x lda, row-major: A[i * lda + j]
    double *T = sm + (size_t)m * lda;            // m x r = U H, then scratch of length m
    const double *Dl = D + leaf_doff[L];
    const double *Ul = U + leaf_uoff[L];
    const double *Hl = H + (int64_t)leaf_id[L] * r * r;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < m * r; e += LEAF_T) {
        const int i = e % m, k = e / m;
        double s = 0;
        for (int q = 0; q < r; q++) s += Ul[i + (int64_t)m * q] * Hl[q + r * k];
        T[i + m * k] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += LEAF_T) {
        const int i = e % m, j = e / m;
        if (i > j) continue;
        double s = 0;
        for (int q = 0; q < r; q++) s += T[i + m * q] * Ul[j + (int64_t)m * q];
        const double v = Dl[i + (int64_t)m * j] - s;
        A[i * lda + j] = v;
        A[j * lda + i] = v;
    }
    __syncthreads();
    // block-wide sum; every thread gets the same value
    auto bsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        double t = 0;
        for (int w = 0; w < LEAF_T / 32; w++) t += red[w];
        __syncthreads();
        return t;
    };
    // Householder reduction: step i zeroes A[i][0 .. i-2] (and the column)
    for (int i = m - 1; i >= 1; i--) {
        const int l = i - 1;
        double sig = 0;
        for (int k = tid; k < l; k += LEAF_T) sig += A[i * lda + k] * A[i * lda + k];
        sig = bsum(sig);                                     // without the subdiagonal entry
        const double f = A[i * lda + l];
        if (l == 0 || sig == 0.0) {
            if (tid == 0) { ee[i] = f; hh[i] = 0.0; }
            __syncthreads();
            continue;
        }
        const double full = sig + f * f;
        const double g = (f >= 0.0) ? -sqrt(full) : sqrt(full);
        const double h = full - f * g;                       // = ||u||^2 / 2
        __syncthreads();
        if (tid == 0) { ee[i] = g; hh[i] = h; s_ih = 1.0 / h; A[i * lda + l] = f - g; }
        __syncthreads();
        const double ih = s_ih;
        // p = A u / h on the leading (l+1) x (l+1) block, u = A[i][0..l]
        double up = 0;
        for (int j = tid; j <= l; j += LEAF_T) {
            double s = 0;
            for (int k = 0; k <= l; k++) s += A[j * lda + k] * A[i * lda + k];
            const double pj = s * ih;
            dg[j] = pj;                                      // p kept in dg until the reduction ends
            up += A[i * lda + j] * pj;
        }
        const double K = bsum(up) * (0.5 * ih);
        for (int j = tid; j <= l; j += LEAF_T) dg[j] -= K * A[i * lda + j];   // q = p - K u
        __syncthreads();
        for (int e2 = tid; e2 < (l + 1) * (l + 1); e2 += LEAF_T) {
            const int j = e2 / (l + 1), k = e2 % (l + 1);
            A[j * lda + k] -= A[i * lda + j] * dg[k] + dg[j] * A[i * lda + k];
        }
        __syncthreads();
        for (int j = tid; j <= l; j += LEAF_T) A[j * lda + i] = A[i * lda + j] * ih;  // u / h in column i
        __syncthreads();
    }
    // diagonal of the tridiagonal matrix, then the orthogonal factor in place
    for (int i = tid; i < m; i += LEAF_T) dg[i] = A[i * lda + i];
    __syncthreads();
    for (int i = 0; i < m; i++) {
        const int l = i - 1;
        if (l >= 0 && hh[i] != 0.0) {
            // Q[0..l][0..l] <- (I - u u^T / h) Q: g_j = sum_k u_k Q[k][j], Q[k][j] -= g_j (u_k / h)
            for (int j = tid; j <= l; j += LEAF_T) {
                double g = 0;
                for (int k = 0; k <= l; k++) g += A[i * lda + k] * A[k * lda + j];
                T[j] = g;
            }
            __syncthreads();
            for (int e2 = tid; e2 < (l + 1) * (l + 1); e2 += LEAF_T) {
                const int k = e2 / (l + 1), j = e2 % (l + 1);
                A[k * lda + j] -= T[j] * A[k * lda + i];
            }
            __syncthreads();
        }
        for (int j = tid; j < i; j += LEAF_T) { A[i * lda + j] = 0.0; A[j * lda + i] = 0.0; }
        if (tid == 0) A[i * lda + i] = 1.0;
        __syncthreads();
    }
    // outputs: Q row-major into the leaf's slot; d; e shifted so that e[i]
    // couples d[i] and d[i+1]
    double *Q = Qleaf + qoff[L];
    for (int e = tid; e < m * m; e += LEAF_T) Q[e] = A[(e / m) * lda + (e % m)];
    const int64_t o = leaf_off[L];
    for (int i = tid; i < m; i += LEAF_T) {
        dout[o + i] = dg[i];
        eout[o + i] = (i + 1 < m) ? ee[i + 1] : 0.0;
    }
}

// Givens pair of a QL step: rr = sqrt(f^2 + g^2), c = g / rr, s = f / rr.  In
// the usual range x^(-1/2) of q = f^2 + g^2 comes from an FP32 seed and two
// Newton steps y <- y + y (1 - q y^2) / 2 (relative error 2^-22 -> 2^-44 ->
// below one ulp), which replaces a square root and a division in the chain of
// dependent operations; elsewhere hypot and one division.
// q^(-1/2) to about 2^-22 for a normal q > 0: the FP32 approximate reciprocal
// square root of the leading mantissa bits (scaled into [1, 4) to make the
// exponent even), the exponent halved by integer arithmetic; no conversion
// between FP64 and FP32 in the chain of dependent steps
__device__ __forceinline__ double rsqrt_seed(double q)
{
    const int hi = __double2hiint(q);
    const unsigned lo = (unsigned)__double2loint(q);
    const int e = ((hi >> 20) & 0x7FF) - 1023;
    const int odd = e & 1;
    const unsigned mb = (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__uint_as_float(((unsigned)(127 + odd) << 23) | mb)));
    const unsigned rb = __float_as_uint(r);                  // in (0.5, 1]
    const int E = (int)(rb >> 23) - 127 - (e - odd) / 2 + 1023;
    const unsigned rm = rb & 0x7FFFFFu;
    return __hiloint2double((int)(((unsigned)E << 20) | (rm >> 3)), (int)(rm << 29));
}

__device__ __forceinline__ void ql_pair(double f, double g, double &c, double &s, double &rr)
{
    const double q = fma(f, f, g * g);
    if (q > 1e-36 && q < 1e36) {
        double y = rsqrt_seed(q);
        double e = fma(-q * y, y, 1.0);
        y = fma(0.5 * y, e, y);
        e = fma(-q * y, y, 1.0);
        y = fma(0.5 * y, e, y);
        rr = q * y;
        c = g * y;
        s = f * y;
    } else {
        rr = hypot(f, g);
        const double inv = (rr != 0.0) ? 1.0 / rr : 0.0;
        c = g * inv;
        s = f * inv;
    }
}

// One implicit QL sweep on the unreduced block [l, h] of a symmetric
// tridiagonal matrix (diagonal a[i * S], off-diagonal b[i * S] coupling i and
// i + 1): the implicit symmetric QR step with Wilkinson's shift of Golub and
// Van Loan (Section 8.3), in its QL orientation.  The shift mu is the
// eigenvalue of the leading 2 x 2 block nearer to a_l; the first rotation, in
// plane (h-1, h), has its second column along the last column of T - mu I
// restricted to rows h-1, h, i.e. along (b_{h-1}, a_h - mu); every later
// rotation, in plane (i, i+1), removes the bulge at (i, i+2) that the
// previous one left, against the entry b_{i+1}.  A rotation G with G(i,i) =
// G(i+1,i+1) = c, G(i,i+1) = s, G(i+1,i) = -s acts as T <- G^T T G:
//   a_i     <- c^2 a_i - 2 c s b_i + s^2 a_{i+1}
//   a_{i+1} <- s^2 a_i + 2 c s b_i + c^2 a_{i+1}
//   b_i     <- c s (a_i - a_{i+1}) + (c^2 - s^2) b_i
//   b_{i-1} <- c b_{i-1}, and the new bulge at (i-1, i+1) is s b_{i-1}.
// rec(q, c, s) records rotation q (plane (h-1-q, h-q)): the eigenvectors are
// Q <- Q G, i.e. columns (x_i, x_{i+1}) <- (c x_i - s x_{i+1}, s x_i + c x_{i+1}).
// Returns the number of rotations (h - l).
template <int S, typename Rec>
__device__ __forceinline__ int ql_sweep_tri(double *a, double *b, int l, int h, Rec rec)
{
    const double al = a[l * S], bl = b[l * S];
    const double del = 0.5 * (a[(l + 1) * S] - al);
    const double mu = al - bl * bl / (del + copysign(hypot(del, bl), del));
    double x = a[h * S] - mu, z = b[(h - 1) * S];
    int q = 0;
    for (int i = h - 1; i >= l; i--, q++) {
        double c, s, r;
        ql_pair(z, x, c, s, r);                 // c = x / r, s = z / r
        if (!(r > 0.0)) { c = 1.0; s = 0.0; r = x; }
        if (i < h - 1) b[(i + 1) * S] = r;      // the bulge is gone
        const double ai = a[i * S], ai1 = a[(i + 1) * S], bi = b[i * S];
        const double cc = c * c, ss = s * s, cs = c * s;
        const double t2 = 2.0 * cs * bi;
        a[i * S] = fma(cc, ai, fma(ss, ai1, -t2));
        a[(i + 1) * S] = fma(ss, ai, fma(cc, ai1, t2));
        const double bn = fma(cs, ai - ai1, (cc - ss) * bi);
        b[i * S] = bn;
        rec(q, c, s);
        if (i > l) {
            const double bm = b[(i - 1) * S];
            z = s * bm;                         // bulge at (i-1, i+1)
            b[(i - 1) * S] = c * bm;
            x = bn;
        }
    }
    return q;
}

// Implicit QL on the tridiagonal (d, e) of every leaf, one lane per leaf and
// LPW leaves per warp (lanes LPW.. idle); d and e staged in shared memory
// ([index][lane]).  A chain of dependent FP64 steps advances at the pipe's
// latency whatever the number of lanes that share it, so a batch of fewer
// leaves than the GPU has warp schedulers spreads them thin (LPW = 2 puts the
// 1024 leaves of n = 131072 on 512 warps instead of 32).  Sweep t of leaf L
// records its first column and count in hdr[L * caps + t] and its rotations
// (c, s) in rot[L * cap + ...] (rotation q of the sweep acts on columns
// (first - q, first - q + 1)).  A leaf whose iterations or records exceed the
// caps latches SUPERDC_DEV_NOCONV.
template <int LPW>
__global__ void __launch_bounds__(32)
k_leaf_ql(int nleaves, int mmax, const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ leaf_m,
          double *__restrict__ dd, const double *__restrict__ ein, double2 *__restrict__ rot, int2 *__restrict__ hdr,
          int32_t *__restrict__ nsw, int64_t cap, int caps, int32_t *status)
{
    extern __shared__ double sq[];
    const int lane = threadIdx.x;
    if (lane >= LPW) return;
    const int L = blockIdx.x * LPW + lane;
    double *sd = sq, *se = sq + (size_t)mmax * LPW;
    const bool act = L < nleaves;
    const int m = act ? (int)leaf_m[L] : 0;
    const int64_t o = act ? leaf_off[L] : 0;
    for (int i = 0; i < m; i++) { sd[i * LPW + lane] = dd[o + i]; se[i * LPW + lane] = ein[o + i]; }
    int64_t nrot = 0;
    int nsweep = 0;
    bool bad = false;
    double2 *R = rot + (int64_t)(act ? L : 0) * cap;
    int2 *Hd = hdr + (int64_t)(act ? L : 0) * caps;
    for (int l = 0; l < m && !bad; l++) {
        for (int iter = 0;; iter++) {
            int mm = l;
            for (; mm < m - 1; mm++) {
                const double s2 = fabs(sd[mm * LPW + lane]) + fabs(sd[(mm + 1) * LPW + lane]);
                if (fabs(se[mm * LPW + lane]) <= SDC_EPS * s2) break;
            }
            if (mm == l) break;
            if (iter >= 64 || nsweep >= caps || nrot + (mm - l) > cap) { bad = true; break; }
            double2 *Rs = R + nrot;
            const int cnt = ql_sweep_tri<LPW>(sd + lane, se + lane, l, mm,
                                             [&](int q, double c, double s) { Rs[q] = make_double2(c, s); });
            Hd[nsweep] = make_int2(mm - 1, cnt);
            nsweep++;
            nrot += cnt;
        }
    }
    if (act) {
        nsw[L] = nsweep;
        for (int i = 0; i < m; i++) dd[o + i] = sd[i * LPW + lane];
        if (bad) sdc_latch(status, SUPERDC_DEV_NOCONV);
    }
}

// eigenvalues ascending (ties by index), Q columns in that order (column-major
// into the leaf's slot), W = Q^T U; A holds Q row-major (ld lda), dd the
// eigenvalues (leaf-local); block-wide
__device__ void leaf_emit(int L, int r, int64_t n, int m, const double *A, int lda, const double *dd,
                          const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ leaf_uoff,
                          const double *__restrict__ U, double *__restrict__ Q, double *__restrict__ lam,
                          double *__restrict__ W, int32_t *status, int *rank)
{
    const int tid = threadIdx.x;
    const int64_t o = leaf_off[L];
    for (int i = tid; i < m; i += blockDim.x) {
        const double li = dd[i];
        int rk = 0;
        for (int j = 0; j < m; j++) {
            const double lj = dd[j];
            rk += (lj < li) || (lj == li && j < i);
        }
        rank[i] = rk;
        lam[o + rk] = li;
        if (!isfinite(li)) sdc_latch(status, SUPERDC_DEV_NONFINITE);
    }
    __syncthreads();
    const double *Ul = U + leaf_uoff[L];
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int row = e % m, i = e / m;
        Q[(int64_t)rank[i] * m + row] = A[row * lda + i];
    }
    for (int e = tid; e < m * r; e += blockDim.x) {
        const int i = e % m, k = e / m;
        double s = 0;
        for (int row = 0; row < m; row++) s += A[row * lda + i] * Ul[row + (int64_t)m * k];
        W[o + rank[i] + n * k] = s;
    }
}

// Rows [y * LEAF_R, ...) of every leaf's Q get the recorded rotations, one
// thread per row (rows are independent): rotation q of a sweep acts on columns
// (i, i+1), i = first - q, and the entry at i + 1 is final after it (carry
// form).  A leaf's Q (128 x 129 doubles) fills the shared memory of an SM, so
// its rows are split over several CTAs, several of which share an SM.
constexpr int LEAF_R = 32;

__global__ void __launch_bounds__(LEAF_R)
k_leaf_rot(const int64_t *__restrict__ leaf_m, double *__restrict__ Qleaf, const int64_t *__restrict__ qoff,
           const double2 *__restrict__ rot, const int2 *__restrict__ hdr, const int32_t *__restrict__ nsw,
           int64_t cap, int caps)
{
    extern __shared__ double sm[];
    const int L = blockIdx.x;
    const int m = (int)leaf_m[L];
    const int r0 = blockIdx.y * LEAF_R;
    if (r0 >= m) return;
    const int nr = min(LEAF_R, m - r0);
    const int lda = m | 1;
    double *Q = Qleaf + qoff[L] + (int64_t)r0 * m;
    const int tid = threadIdx.x;
    for (int e = tid; e < nr * m; e += LEAF_R) sm[(e / m) * lda + (e % m)] = Q[e];
    __syncthreads();
    if (tid < nr) {
        const double2 *R = rot + (int64_t)L * cap;
        const int2 *Hd = hdr + (int64_t)L * caps;
        const int ns = nsw[L];
        double *qr = sm + tid * lda;
        int64_t k = 0;
        for (int t = 0; t < ns; t++) {
            const int2 h = Hd[t];
            const int first = h.x, cnt = h.y;
            double carry = qr[first + 1];
            for (int q = 0; q < cnt; q++) {
                const int i = first - q;
                const double2 cs = R[k + q];
                const double x = qr[i];
                qr[i + 1] = cs.y * x + cs.x * carry;
                carry = cs.x * x - cs.y * carry;
            }
            qr[first - cnt + 1] = carry;
            k += cnt;
        }
    }
    __syncthreads();
    for (int e = tid; e < nr * m; e += LEAF_R) Q[e] = sm[(e / m) * lda + (e % m)];
}

// Q (rotations applied) to the outputs: see leaf_emit
__global__ void __launch_bounds__(LEAF_T)
k_leaf_out(int r, int64_t n, const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ leaf_m,
           const int64_t *__restrict__ leaf_uoff, const double *__restrict__ U, double *__restrict__ Qleaf,
           const int64_t *__restrict__ qoff, const double *__restrict__ dd, double *__restrict__ lam,
           double *__restrict__ W, int32_t *status)
{
    extern __shared__ double sm[];
    __shared__ int rank[128];
    const int L = blockIdx.x;
    const int m = (int)leaf_m[L];
    const int lda = m | 1;
    double *A = sm;
    const int tid = threadIdx.x;
    double *Q = Qleaf + qoff[L];
    for (int e = tid; e < m * m; e += LEAF_T) A[(e / m) * lda + (e % m)] = Q[e];
    __syncthreads();
    leaf_emit(L, r, n, m, A, lda, dd + leaf_off[L], leaf_off, leaf_uoff, U, Q, lam, W, status, rank);
}

// Small leaves (several CTAs per SM): QL on (d, e) inside the leaf's CTA.
// Thread 0 computes the rotations of one QL sweep into one of two buffers
// while warps 1.. apply the previous sweep's rotations to the rows of Q
// (double buffering, one barrier per phase; the sweeps depend only on d, e,
// which thread 0 alone updates).
__global__ void __launch_bounds__(LEAF_T)
k_leaf_qlcta(int r, int64_t n, const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ leaf_m,
             const int64_t *__restrict__ leaf_uoff, const double *__restrict__ U, double *__restrict__ Qleaf,
             const int64_t *__restrict__ qoff, const double *__restrict__ din, const double *__restrict__ ein,
             double *__restrict__ lam, double *__restrict__ W, int32_t *status)
{
    extern __shared__ double sm[];
    __shared__ double dg[128], ee[128];
    __shared__ int s_cnt_b[2], s_first_b[2], s_flag;
    __shared__ int rank[128];
    const int L = blockIdx.x;
    const int m = (int)leaf_m[L];
    const int lda = m | 1;
    double *A = sm;
    double *rc = sm + (size_t)m * lda, *rs = rc + 2 * m;     // two buffers of m each
    const int tid = threadIdx.x;
    double *Q = Qleaf + qoff[L];
    const int64_t o = leaf_off[L];
    for (int e = tid; e < m * m; e += LEAF_T) A[(e / m) * lda + (e % m)] = Q[e];
    for (int i = tid; i < m; i += LEAF_T) { dg[i] = din[o + i]; ee[i] = ein[o + i]; }
    if (tid == 0) s_flag = 0;
    __syncthreads();
    int ql_l = 0, ql_iter = 0;
    auto ql_sweep = [&](int b) -> int {
        double *bc = rc + b * m, *bs = rs + b * m;
        while (ql_l < m) {
            const int l = ql_l;
            int mm = l;
            for (; mm < m - 1; mm++) {
                const double dd2 = fabs(dg[mm]) + fabs(dg[mm + 1]);
                if (fabs(ee[mm]) <= SDC_EPS * dd2) break;
            }
            if (mm == l || ql_iter >= 64) {
                if (mm != l) s_flag = 1;
                ql_l++;
                ql_iter = 0;
                continue;
            }
            ql_iter++;
            const int cnt = ql_sweep_tri<1>(dg, ee, l, mm, [&](int q, double c, double s) { bc[q] = c; bs[q] = s; });
            s_first_b[b] = mm - 1;
            return cnt;
        }
        return -1;
    };
    if (tid == 0) s_cnt_b[0] = ql_sweep(0);
    __syncthreads();
    for (int t = 0;; t++) {
        const int b = t & 1;
        const int cnt = s_cnt_b[b];
        if (cnt < 0) break;                          // uniform: read after the barrier
        if (tid == 0) {
            s_cnt_b[b ^ 1] = ql_sweep(b ^ 1);
        } else if (tid >= 32) {
            const int first = s_first_b[b];
            const double *bc = rc + b * m, *bs = rs + b * m;
            for (int k = tid - 32; k < m; k += LEAF_T - 32) {
                double *qr = A + k * lda;
                double carry = qr[first + 1];
                for (int q = 0; q < cnt; q++) {
                    const int i = first - q;
                    const double x = qr[i];
                    qr[i + 1] = bs[q] * x + bc[q] * carry;
                    carry = bc[q] * x - bs[q] * carry;
                }
                qr[first - cnt + 1] = carry;
            }
        }
        __syncthreads();
    }
    if (tid == 0 && s_flag) sdc_latch(status, SUPERDC_DEV_NOCONV);
    leaf_emit(L, r, n, m, A, lda, dg, leaf_off, leaf_uoff, U, Q, lam, W, status, rank);
}

// ---------------------------------------------------------------------------
// Level setup: merge the children's eigenvalues (stable, left child first on
// ties) -> d^(0) and P_p; rows of Zhat_p (r columns) and of [W_c1 R_c1; W_c2 R_c2]
// (r more columns, not at the root) in merged order.
// ---------------------------------------------------------------------------
__global__ void k_build(int64_t n, int r, int nl, const int64_t *__restrict__ loff, const int32_t *__restrict__ lnodes,
                        int root, const int32_t *__restrict__ lch, const int32_t *__restrict__ rch,
                        const int64_t *__restrict__ size, const double *__restrict__ R,
                        const double *__restrict__ Bts, const double *__restrict__ sqb,
                        const double *__restrict__ lam_prev, const double *__restrict__ Wp,
                        double *__restrict__ d0, int32_t *__restrict__ P, double *__restrict__ WK)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = sdc_upper_index(loff, (int64_t)nl, x);
        const int64_t o = loff[q];
        const int node = lnodes[q];
        const int c1 = lch[node], c2 = rch[node];
        const int m = (int)(loff[q + 1] - o);
        const int m1 = (int)size[c1];
        const int i = (int)(x - o);
        const double *l1 = lam_prev + o, *l2 = lam_prev + o + m1;
        const double val = lam_prev[x];
        int pos;
        if (i < m1) {             // + number of right-child values strictly smaller
            int lo = 0, hi = m - m1;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (l2[mid] < val) lo = mid + 1; else hi = mid; }
            pos = i + lo;
        } else {                  // + number of left-child values smaller or equal
            int lo = 0, hi = m1;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (l1[mid] <= val) lo = mid + 1; else hi = mid; }
            pos = (i - m1) + lo;
        }
        const int64_t y = o + pos;
        d0[y] = val;
        P[y] = i;
        const int rr = r * r;
        const bool top = i < m1;
        const double *Rc = R + (int64_t)(top ? c1 : c2) * rr;
        const double *Bs = Bts + (int64_t)node * rr;
        const double sb = sqb[node];
        for (int col = 0; col < r; col++) {
            double zv = 0.0, xv = 0.0;
            for (int k = 0; k < r; k++) {
                const double w = Wp[x + n * k];
                if (top) zv += w * Bs[k + r * col];
                xv += w * Rc[k + r * col];
            }
            if (!top) zv = sb * Wp[x + n * col];
            WK[y + n * col] = zv;
            if (node != root) WK[y + n * (r + col)] = xv;
        }
    }
}

// row permutations inside every node of a level: gather (Y[o+pos] = X[o+P[o+pos]])
// or scatter (Y[o+P[o+pos]] = X[o+pos])
__global__ void k_permute(int64_t n, int nl, const int64_t *__restrict__ loff, const int32_t *__restrict__ P,
                          const double *__restrict__ X, int64_t ldx, double *__restrict__ Y, int64_t ldy,
                          int ncols, int scatter)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ncols;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % n;
        const int col = (int)(t / n);
        const int64_t q = sdc_upper_index(loff, (int64_t)nl, x);
        const int64_t o = loff[q];
        const int64_t src = o + P[x];
        if (scatter) Y[src + ldy * col] = X[x + ldx * col];
        else         Y[x + ldy * col] = X[src + ldx * col];
    }
}

// dense leaf blocks: Y_leaf = Q_leaf^T X_leaf (trans) or Q_leaf X_leaf
__global__ void k_leaf_apply(int64_t n, const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ leaf_m,
                             const double *__restrict__ Qleaf, const int64_t *__restrict__ qoff,
                             const double *__restrict__ X, int64_t ldx, double *__restrict__ Y, int64_t ldy,
                             int ncols, int trans)
{
    const int L = blockIdx.x;
    const int m = (int)leaf_m[L];
    const int64_t o = leaf_off[L];
    const double *Q = Qleaf + qoff[L];
    for (int e = threadIdx.x; e < m * ncols; e += blockDim.x) {
        const int i = e % m, col = e / m;
        const double *x = X + o + ldx * col;
        double s = 0.0;
        if (trans) for (int k = 0; k < m; k++) s += Q[(int64_t)i * m + k] * x[k];
        else       for (int k = 0; k < m; k++) s += Q[i + (int64_t)k * m] * x[k];
        Y[o + i + ldy * col] = s;
    }
}

__global__ void k_copy_cols(int64_t n, int ncols, const double *__restrict__ X, int64_t ldx, double *__restrict__ Y,
                            int64_t ldy)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ncols;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % n;
        const int col = (int)(t / n);
        Y[x + ldy * col] = X[x + ldx * col];
    }
}

// *out = max(*out, max_i |v_i|) (non-negative doubles compare as their bit patterns)
__global__ void k_maxabs(int64_t n, const double *__restrict__ v, double *out)
{
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(v[i]));
    for (int sh = 16; sh > 0; sh >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, sh));
    if ((threadIdx.x & 31) == 0)
        atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong(isnan(m) ? INFINITY : m));
}

// Y(:, col) = fv .* Y(:, col) (rows scaled by the function values)
__global__ void k_scale_rows(int64_t n, int ncols, const double *__restrict__ fv, double *__restrict__ Y, int64_t ldy)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ncols;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % n;
        const int col = (int)(t / n);
        Y[x + ldy * col] *= fv[x];
    }
}

__global__ void k_stats(int64_t nprob, const int64_t *__restrict__ off, const int32_t *__restrict__ mk,
                        const int32_t *__restrict__ sweeps, unsigned long long *acc)
{
    // acc[0] += deflated, acc[1] += sweeps, acc[2] = max sweeps
    for (int64_t p = blockIdx.x; p < nprob; p += gridDim.x) {
        const int64_t o = off[p];
        const int m = (int)(off[p + 1] - o), k = mk[p];
        unsigned long long s = 0, mx = 0;
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            unsigned long long v = (unsigned long long)sweeps[o + i];
            s += v;
            mx = v > mx ? v : mx;
        }
        for (int w = 16; w > 0; w >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, w);
            unsigned long long o2 = __shfl_xor_sync(0xffffffffu, mx, w);
            mx = o2 > mx ? o2 : mx;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&acc[1], s);
            atomicMax(&acc[2], mx);
        }
        if (threadIdx.x == 0) atomicAdd(&acc[0], (unsigned long long)(m - k));
    }
}

superdc_status status_from_word(int32_t w)
{
    if (w & SUPERDC_DEV_NONFINITE) return SUPERDC_ERR_NONFINITE;
    if (w & SUPERDC_DEV_NOCONV) return SUPERDC_ERR_NOCONV;
    if (w & SUPERDC_DEV_INDEX) return SUPERDC_ERR_CUDA;
    return SUPERDC_OK;
}

FactorView view(const superdc_eigfact *f, int l, int j)
{
    const superdc_hss *h = f->h;
    const StepF &S = f->F[l][j];
    FactorView v;
    v.nprob = (int64_t)h->lev_nodes[l].size();
    v.off = h->d_lev_off[l];
    v.mk = S.mk; v.ngiv = S.ngiv;
    v.dk = S.dk; v.eta = S.eta; v.dorg = S.dorg; v.vhat = S.vhat; v.bnorm = S.bnorm;
    v.src = S.src; v.perm = nullptr; v.pinv = S.pinv; v.giv_ab = S.giv_ab; v.giv_cs = S.giv_cs;
    v.fmm_min_m = f->fmm_min_m;
#ifdef SUPERDC_CHECK
    v.status = f->status;
#endif
    int64_t mx = 0;
    for (int i : h->lev_nodes[l]) mx = std::max<int64_t>(mx, h->size[i]);
    v.max_m = mx;
    return v;
}

// ---------------------------------------------------------------------------
// Leaves of 128 rows: divide and conquer on the tridiagonal form (the
// method's own rank-one machinery applied inside the leaves).  The QL chase
// of a 128-row leaf is one chain of about 12,000 dependent rotations; torn into
// blocks of 32 (Cuppen's splitting T = diag(T_1', ..., T_4') + sum of rank-one
// couplings), the chains are 16 times shorter, and the two merge levels are
// batched rank-one steps (deflation, secular roots, Loewner zhat, b) whose
// eigenvector products go through the Cauchy-like application.
//   k_dc_tear      per leaf: scale (d, e) by a power of two >= ||T||_inf (so an
//                  absolute deflation tolerance of a few eps serves every
//                  leaf), then tear at every block boundary j: the coupling
//                  beta = e_{j-1} leaves the tridiagonal, d_{j-1} and d_j lose
//                  |beta|, and T = blocks + |beta| v v^T, v = e_{j-1} +
//                  sign(beta) e_j;
//   k_leaf_ql / k_leaf_rot on the 32-row blocks (identity start);
//   k_dc_base      block eigenvalues ascending, eigenvector j of a block as
//                  row (block start + j) of an n x 32 column-major array;
//   k_dc_merge_in  per merge problem: the children's eigenvalues merged
//                  (stable, left child first on ties), z = sqrt|beta| (last
//                  row of the left eigenvectors; sign(beta) first row of the
//                  right ones), and X = (blkdiag(Q_1, Q_2) P)^T with P the merge;
//   then the batched rank-one step and Y = Qhat^T X (eigenvectors of the
//   merged block as rows, in ascending eigenvalue order);
//   k_dc_gemm      Q_leaf = Q_householder Q_tridiagonal (row-major, into the
//                  leaf's slot), eigenvalues scaled back.
// ---------------------------------------------------------------------------
constexpr int DC_B = 32;        // rows of a block solved by QL
constexpr int DC_M = 128;       // leaf rows of the divide-and-conquer path

__global__ void k_dc_tear(const int64_t *__restrict__ leaf_off, double *__restrict__ d, double *__restrict__ e,
                          double *__restrict__ scale, double *__restrict__ beta_at)
{
    __shared__ double red[4];
    const int L = blockIdx.x, tid = threadIdx.x;            // DC_M threads
    const int64_t o = leaf_off[L];
    const double di = d[o + tid], ei = (tid + 1 < DC_M) ? e[o + tid] : 0.0;
    const double em = (tid > 0) ? e[o + tid - 1] : 0.0;
    double rowsum = fabs(di) + fabs(ei) + fabs(em);
    for (int sh = 16; sh > 0; sh >>= 1) rowsum = fmax(rowsum, __shfl_xor_sync(0xffffffffu, rowsum, sh));
    if ((tid & 31) == 0) red[tid >> 5] = rowsum;
    __syncthreads();
    const double nrm = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
    // the power of two at or above the norm (1 for a zero block), exact scaling
    int ex = 0;
    const double fr = frexp(nrm > 0.0 && isfinite(nrm) ? nrm : 1.0, &ex);
    const double s = ldexp(1.0, fr == 0.5 ? ex - 1 : ex);
    const double is = 1.0 / s;
    double dn = di * is;
    // couplings torn at the block boundaries (block starts j = 32, 64, 96)
    if ((tid % DC_B) == DC_B - 1 && tid + 1 < DC_M) dn -= fabs(ei * is);
    if ((tid % DC_B) == 0 && tid > 0) {
        dn -= fabs(em * is);
        beta_at[o + tid] = em * is;
    }
    d[o + tid] = dn;
    e[o + tid] = ((tid % DC_B) == DC_B - 1) ? 0.0 : ei * is;
    if (tid == 0) scale[L] = s;
}

// QB (row-major 32 x 32 per block, identity before k_leaf_rot)
__global__ void k_dc_eye(int64_t nblk, double *__restrict__ QB)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nblk * DC_B * DC_B;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % (DC_B * DC_B));
        QB[t] = (e / DC_B == e % DC_B) ? 1.0 : 0.0;
    }
}

// block eigenvalues ascending (ties by index) into lam, eigenvector j of
// block b as row (o_b + j) of Y (n x 32, column-major, ld n); one warp per block
__global__ void k_dc_base(int64_t nblk, int64_t n, const double *__restrict__ dd, const double *__restrict__ QB,
                          double *__restrict__ lam, double *__restrict__ Y)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nblk) return;
    const int64_t o = b * DC_B;
    const double li = dd[o + lane];
    int rk = 0;
    for (int j = 0; j < DC_B; j++) {
        const double lj = __shfl_sync(0xffffffffu, li, j);
        rk += (lj < li) || (lj == li && j < lane);
    }
    lam[o + rk] = li;
    const double *Q = QB + b * DC_B * DC_B;
    for (int c = 0; c < DC_B; c++) Y[(o + rk) + (int64_t)c * n] = Q[c * DC_B + lane];
}

// merge problem p of size s (children of h = s/2 rows): merged d, z and X
__global__ void k_dc_merge_in(int64_t n, int s, const double *__restrict__ lam, const double *__restrict__ beta_at,
                              const double *__restrict__ Yin, double *__restrict__ din, double *__restrict__ zin,
                              double *__restrict__ X)
{
    const int h = s / 2;
    const int64_t o = (int64_t)blockIdx.x * s;
    const int t = threadIdx.x;                    // s threads
    const double beta = beta_at[o + h];
    const double sb = sqrt(fabs(beta));
    const bool left = t < h;
    const int j = left ? t : t - h;
    const int64_t ro = left ? o : o + h;          // the child's first row
    const double *other = lam + (left ? o + h : o);
    const double lj = lam[ro + j];
    // elements of the other child before this one: strictly smaller (left
    // child) or smaller or equal (right child): left first on ties
    int lo = 0, hi = h;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (left ? (other[mid] < lj) : (other[mid] <= lj)) lo = mid + 1; else hi = mid;
    }
    const int64_t pos = o + j + lo;
    din[pos] = lj;
    zin[pos] = left ? sb * Yin[(ro + j) + (int64_t)(h - 1) * n] : copysign(sb, beta) * Yin[(ro + j)];
    for (int c = 0; c < s; c++) {
        const bool mine = left ? (c < h) : (c >= h);
        X[pos + (int64_t)c * n] = mine ? Yin[(ro + j) + (int64_t)(left ? c : c - h) * n] : 0.0;
    }
}

// Q_leaf = Q_householder Q_tridiagonal for every leaf (row-major, into the
// leaf's slot), with Q_tridiagonal(c, k) = Y(o + k, c); 64 x 64 tiles, 256
// threads, 4 x 4 outputs per thread, k-chunks of 16 staged in shared memory.
// Eigenvalues (lam, ascending) scaled back into dd.
__global__ void __launch_bounds__(256)
k_dc_gemm(int64_t n, const int64_t *__restrict__ leaf_off, const int64_t *__restrict__ qoff,
          const double *__restrict__ Qh, const double *__restrict__ Y, double *__restrict__ Qleaf,
          const double *__restrict__ lam, const double *__restrict__ scale, double *__restrict__ dd)
{
    __shared__ double As[16][64 + 1], Bs[16][64 + 1];
    const int L = blockIdx.x, tr = blockIdx.y * 64, tc = blockIdx.z * 64;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int64_t o = leaf_off[L];
    const double *A = Qh + qoff[L];
    double acc[4][4] = {};
    for (int k0 = 0; k0 < DC_M; k0 += 16) {
        __syncthreads();
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e % 16, rr = e / 16;
            As[kk][rr] = A[(int64_t)(tr + rr) * DC_M + k0 + kk];          // Q_h(row, k)
            const int cc = e % 64, kb = e / 64;
            Bs[kb][cc] = Y[(o + tc + cc) + (int64_t)(k0 + kb) * n];         // Q_tri(k, col)
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    double *C = Qleaf + qoff[L];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) C[(int64_t)(tr + ty * 4 + i) * DC_M + tc + tx * 4 + j] = acc[i][j];
    if (blockIdx.y == 0 && blockIdx.z == 0)
        for (int k = tid; k < DC_M; k += 256) dd[o + k] = lam[o + k] * scale[L];
}

}  // namespace

extern "C" {

// Real form of complex blocks: a complex rows x cols block M (column-major,
// entries as (re, im) pairs) becomes the real 2rows x 2cols block
// [[Re M, -Im M], [Im M, Re M]] (column-major).  One launch covers nblk
// blocks; block b starts at in + 2 ioff[b], out + ooff[b], with rows[b] rows
// and cols columns (cols = 0: square, cols = rows[b]).
__global__ void k_realify(int nblk, const int64_t *__restrict__ ioff, const int64_t *__restrict__ ooff,
                          const int32_t *__restrict__ rows, int cols_in, const double *__restrict__ in,
                          double *__restrict__ out)
{
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
        const int m = rows[b];
        const int cols = cols_in > 0 ? cols_in : m;
        const double *M = in + 2 * ioff[b];
        double *Rm = out + ooff[b];
        const int64_t ld = 2 * (int64_t)m;
        for (int t = threadIdx.x; t < m * cols; t += blockDim.x) {
            const int i = t % m, j = t / m;
            const double re = M[2 * (i + (int64_t)m * j)], im = M[2 * (i + (int64_t)m * j) + 1];
            Rm[i + ld * j] = re;
            Rm[(i + m) + ld * j] = im;
            Rm[i + ld * (j + cols)] = -im;
            Rm[(i + m) + ld * (j + cols)] = re;
        }
    }
}

superdc_status superdc_build_hss(const superdc_tree *tree, const double *D, const double *U, const double *R,
                                 const double *B, cudaStream_t stream, superdc_hss **out)
{
    if (!tree || !out || !D || !U || !B || !tree->lchild || !tree->rchild || !tree->leaf_size) return SUPERDC_ERR_ARG;
    const int nn = tree->nnodes, r = tree->rank;
    if (nn < 1 || (nn % 2) == 0 || r < 1 || r > 32 || tree->n < 1) return SUPERDC_ERR_ARG;
    if (nn > 1 && !R) return SUPERDC_ERR_ARG;
    bool big = false;
    for (int i = 0; i < nn; i++) if (tree->lchild[i] < 0 && tree->leaf_size[i] > 128) big = true;
    if (big && nn > 1) {
        // leaves above 128 rows: refine them into exact rank-r subtrees first
        std::vector<int32_t> lch2, rch2;
        std::vector<int64_t> ls2;
        double *D2 = nullptr, *U2 = nullptr, *R2 = nullptr, *B2 = nullptr;
        superdc_status s = refine_leaves(tree, D, U, R, B, stream, lch2, rch2, ls2, &D2, &U2, &R2, &B2);
        if (s != SUPERDC_OK) return s;
        superdc_tree t2 = *tree;
        t2.nnodes = (int32_t)lch2.size();
        t2.lchild = lch2.data();
        t2.rchild = rch2.data();
        t2.leaf_size = ls2.data();
        s = superdc_build_hss(&t2, D2, U2, R2, B2, stream, out);      // synchronises the stream
        cudaFree(D2); cudaFree(U2); cudaFree(R2); cudaFree(B2);
        return s;
    }
    superdc_hss *h = new superdc_hss();
    h->nnodes = nn; h->r = r; h->n = tree->n;
    h->lch.assign(tree->lchild, tree->lchild + nn);
    h->rch.assign(tree->rchild, tree->rchild + nn);
    h->level.assign(nn, -1);
    h->size.assign(nn, 0);
    h->off.assign(nn, 0);
    // postorder: children precede parents; every non-root has one parent
    std::vector<int> parent(nn, -1);
    bool ok = true;
    for (int i = 0; i < nn && ok; i++) {
        int a = h->lch[i], b = h->rch[i];
        if ((a < 0) != (b < 0)) ok = false;
        if (a >= 0) {
            if (a >= i || b >= i || parent[a] >= 0 || parent[b] >= 0) ok = false;
            else { parent[a] = i; parent[b] = i; }
        }
    }
    for (int i = 0; i < nn - 1 && ok; i++) if (parent[i] < 0) ok = false;
    if (!ok) { delete h; return SUPERDC_ERR_ARG; }
    // levels top-down, sizes bottom-up, offsets top-down
    h->level[nn - 1] = 0;
    for (int i = nn - 1; i >= 0; i--)
        if (h->lch[i] >= 0) { h->level[h->lch[i]] = h->level[i] + 1; h->level[h->rch[i]] = h->level[i] + 1; }
    int lmax = 0;
    for (int i = 0; i < nn; i++) lmax = std::max(lmax, h->level[i]);
    int64_t ntot = 0;
    int mmax = 0;
    for (int i = 0; i < nn; i++) {
        if (h->lch[i] < 0) {
            if (h->level[i] != lmax) ok = false;          // perfect tree
            int64_t m = tree->leaf_size[i];
            if (m < 1 || m > 128) ok = false;
            h->size[i] = m;
            ntot += m;
            mmax = std::max<int>(mmax, (int)m);
        } else {
            h->size[i] = h->size[h->lch[i]] + h->size[h->rch[i]];
        }
    }
    if (!ok || ntot != tree->n) { delete h; return SUPERDC_ERR_ARG; }
    h->off[nn - 1] = 0;
    for (int i = nn - 1; i >= 0; i--)
        if (h->lch[i] >= 0) { h->off[h->lch[i]] = h->off[i]; h->off[h->rch[i]] = h->off[i] + h->size[h->lch[i]]; }
    h->lmax = lmax;
    h->mmax = mmax;
    h->lev_nodes.assign(lmax + 1, {});
    for (int i = 0; i < nn; i++) h->lev_nodes[h->level[i]].push_back(i);
    for (auto &v : h->lev_nodes) std::sort(v.begin(), v.end(), [&](int a, int b) { return h->off[a] < h->off[b]; });
    h->leaves = h->lev_nodes[lmax];
    h->nleaves = (int)h->leaves.size();
    // device copies
    int64_t dsz = 0, usz = 0;
    std::vector<int64_t> loff, lm, ldo, luo;
    std::vector<int32_t> lid;
    for (int L : h->leaves) {
        loff.push_back(h->off[L]);
        lm.push_back(h->size[L]);
        ldo.push_back(dsz);
        luo.push_back(usz);
        lid.push_back(L);
        dsz += h->size[L] * h->size[L];
        usz += h->size[L] * r;
    }
    // the caller's D and U are packed in postorder; leaves in postorder are left to right
    const int rr = r * r;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    chk(sdc_malloc(&h->D, dsz * sizeof(double)));
    chk(sdc_malloc(&h->U, usz * sizeof(double)));
    chk(sdc_malloc(&h->R, (size_t)nn * rr * sizeof(double)));
    chk(sdc_malloc(&h->B, (size_t)nn * rr * sizeof(double)));
    chk(sdc_malloc(&h->d_lch, nn * sizeof(int32_t)));
    chk(sdc_malloc(&h->d_rch, nn * sizeof(int32_t)));
    chk(sdc_malloc(&h->d_size, nn * sizeof(int64_t)));
    chk(sdc_malloc(&h->d_leaf_off, h->nleaves * sizeof(int64_t)));
    chk(sdc_malloc(&h->d_leaf_m, h->nleaves * sizeof(int64_t)));
    chk(sdc_malloc(&h->d_leaf_doff, h->nleaves * sizeof(int64_t)));
    chk(sdc_malloc(&h->d_leaf_uoff, h->nleaves * sizeof(int64_t)));
    chk(sdc_malloc(&h->d_leaf_id, h->nleaves * sizeof(int32_t)));
    if (e != cudaSuccess) { superdc_hss_free(h); return e == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA; }
    chk(cudaMemcpyAsync(h->D, D, dsz * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    chk(cudaMemcpyAsync(h->U, U, usz * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    if (R) chk(cudaMemcpyAsync(h->R, R, (size_t)nn * rr * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    else chk(cudaMemsetAsync(h->R, 0, (size_t)nn * rr * sizeof(double), stream));
    chk(cudaMemcpyAsync(h->B, B, (size_t)nn * rr * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    chk(cudaMemcpyAsync(h->d_lch, h->lch.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_rch, h->rch.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_size, h->size.data(), nn * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_leaf_off, loff.data(), loff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_leaf_m, lm.data(), lm.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_leaf_doff, ldo.data(), ldo.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_leaf_uoff, luo.data(), luo.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    chk(cudaMemcpyAsync(h->d_leaf_id, lid.data(), lid.size() * sizeof(int32_t), cudaMemcpyHostToDevice, stream));
    h->d_lev_off.assign(lmax + 1, nullptr);
    h->d_lev_nodes.assign(lmax + 1, nullptr);
    for (int l = 0; l <= lmax; l++) {
        std::vector<int64_t> lo;
        for (int i : h->lev_nodes[l]) lo.push_back(h->off[i]);
        lo.push_back(h->n);
        chk(sdc_malloc(&h->d_lev_off[l], lo.size() * sizeof(int64_t)));
        chk(sdc_malloc(&h->d_lev_nodes[l], h->lev_nodes[l].size() * sizeof(int32_t)));
        if (e != cudaSuccess) break;
        chk(cudaMemcpyAsync(h->d_lev_off[l], lo.data(), lo.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
        chk(cudaMemcpyAsync(h->d_lev_nodes[l], h->lev_nodes[l].data(), h->lev_nodes[l].size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, stream));
    }
    // host vectors passed to async copies must live until the copies ran
    chk(cudaStreamSynchronize(stream));
    if (e != cudaSuccess) { superdc_hss_free(h); return e == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA; }
    *out = h;
    return SUPERDC_OK;
}

superdc_status superdc_build_hss_hermitian(const superdc_tree *tree, const double *D, const double *U,
                                           const double *R, const double *B, cudaStream_t stream,
                                           superdc_hss **out)
{
    if (!tree || !out || !D || !U || !B || !tree->lchild || !tree->rchild || !tree->leaf_size) return SUPERDC_ERR_ARG;
    const int nn = tree->nnodes, r = tree->rank;
    if (nn < 1 || (nn % 2) == 0 || r < 1 || 2 * r > 32 || tree->n < 1) return SUPERDC_ERR_ARG;
    if (nn > 1 && !R) return SUPERDC_ERR_ARG;
    // leaves in postorder, their sizes doubled; block offsets (complex entries
    // in, real entries out)
    std::vector<int64_t> sz2(nn);
    std::vector<int64_t> dio, doo, uio, uoo, rio, roo;
    std::vector<int32_t> drow, urow, rrow;
    int64_t di = 0, dr = 0, ui = 0, ur = 0, n2 = 0;
    for (int i = 0; i < nn; i++) {
        const bool leaf = tree->lchild[i] < 0;
        const int64_t m = leaf ? tree->leaf_size[i] : 0;
        if (leaf && (m < 1 || 2 * m > 128)) return SUPERDC_ERR_ARG;
        sz2[i] = 2 * m;
        if (leaf) {
            dio.push_back(di); doo.push_back(dr); drow.push_back((int32_t)m);
            uio.push_back(ui); uoo.push_back(ur); urow.push_back((int32_t)m);
            di += m * m; dr += 4 * m * m; ui += m * r; ur += 4 * m * r; n2 += 2 * m;
        }
        rio.push_back((int64_t)i * r * r); roo.push_back((int64_t)i * 4 * r * r); rrow.push_back(r);
    }
    if (n2 != 2 * tree->n) return SUPERDC_ERR_ARG;
    const int nl = (int)dio.size();
    // one device slab: the real generators and the block tables
    const size_t nd = (size_t)dr + ur + 2 * (size_t)nn * 4 * r * r;
    const size_t ni = dio.size() * 4 + rio.size() * 2, n32 = drow.size() * 2 + rrow.size();
    char *slab = nullptr;
    SDC_CHECK(sdc_alloc(&slab, nd * 8 + ni * 8 + n32 * 4, stream));
    double *RD = (double *)slab, *RU = RD + dr, *RR = RU + ur, *RB = RR + (size_t)nn * 4 * r * r;
    int64_t *tab = (int64_t *)(RB + (size_t)nn * 4 * r * r);
    int32_t *rows = (int32_t *)(tab + ni);
    std::vector<int64_t> htab;
    for (auto *v : {&dio, &doo, &uio, &uoo, &rio, &roo}) htab.insert(htab.end(), v->begin(), v->end());
    std::vector<int32_t> hrows;
    for (auto *v : {&drow, &urow, &rrow}) hrows.insert(hrows.end(), v->begin(), v->end());
    cudaError_t e = cudaMemcpyAsync(tab, htab.data(), htab.size() * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rows, hrows.data(), hrows.size() * 4, cudaMemcpyHostToDevice, stream);
    const unsigned g = (unsigned)(sdc_num_sms() * 4);
    superdc_status st = SUPERDC_OK;
    if (e == cudaSuccess) {
        k_realify<<<g, 256, 0, stream>>>(nl, tab, tab + nl, rows, 0, D, RD);           // square leaf blocks
        k_realify<<<g, 256, 0, stream>>>(nl, tab + 2 * nl, tab + 3 * nl, rows + nl, r, U, RU);
        if (R) k_realify<<<g, 256, 0, stream>>>(nn, tab + 4 * nl, tab + 4 * nl + nn, rows + 2 * nl, r, R, RR);
        else e = cudaMemsetAsync(RR, 0, (size_t)nn * 4 * r * r * sizeof(double), stream);
        k_realify<<<g, 256, 0, stream>>>(nn, tab + 4 * nl, tab + 4 * nl + nn, rows + 2 * nl, r, B, RB);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        superdc_tree t2 = *tree;
        t2.n = 2 * tree->n;
        t2.rank = 2 * r;
        t2.leaf_size = sz2.data();
        st = superdc_build_hss(&t2, RD, RU, RR, RB, stream, out);   // synchronises the stream
    }
    cudaFreeAsync(slab, stream);
    if (e != cudaSuccess) return SUPERDC_ERR_CUDA;
    return st;
}

superdc_status superdc_hss_get(const superdc_hss *h, const char *field, void *dst)
{
    if (!h || !field || !dst) return SUPERDC_ERR_ARG;
    size_t dsz = 0, usz = 0;
    for (int k : h->leaves) { dsz += (size_t)h->size[k] * h->size[k]; usz += (size_t)h->size[k] * h->r; }
    const size_t rr = (size_t)h->nnodes * h->r * h->r;
    const std::string f(field);
    const void *src = nullptr;
    size_t bytes = 0;
    if (f == "D") { src = h->D; bytes = dsz * 8; }
    else if (f == "U") { src = h->U; bytes = usz * 8; }
    else if (f == "R") { src = h->R; bytes = rr * 8; }
    else if (f == "B") { src = h->B; bytes = rr * 8; }
    else return SUPERDC_ERR_ARG;
    return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}

void superdc_hss_free(superdc_hss *h)
{
    if (!h) return;
    cudaFree(h->D); cudaFree(h->U); cudaFree(h->R); cudaFree(h->B);
    cudaFree(h->d_lch); cudaFree(h->d_rch); cudaFree(h->d_size);
    cudaFree(h->d_leaf_off); cudaFree(h->d_leaf_m); cudaFree(h->d_leaf_doff); cudaFree(h->d_leaf_uoff);
    cudaFree(h->d_leaf_id);
    for (auto p : h->d_lev_off) cudaFree(p);
    for (auto p : h->d_lev_nodes) cudaFree(p);
    delete h;
}

void superdc_eigfact_free(superdc_eigfact *f)
{
    if (!f) return;
    for (auto p : f->slabs) cudaFree(p);
    delete f;
}

// The leaf kernels' dynamic shared-memory limits, raised once per device to
// what the largest leaf (128 rows) and rank (32) need; a launch uses only what
// its own leaves need.
cudaError_t leaf_attrs()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    const size_t mm = 128, rmax = 32;
    const struct { const void *fn; size_t bytes; } at[] = {
        {(const void *)k_leaf_tri, (mm * (mm | 1) + std::max(mm * rmax, mm)) * sizeof(double)},
        {(const void *)k_leaf_ql<32>, 2 * mm * 32 * sizeof(double)},
        {(const void *)k_leaf_out, mm * (mm | 1) * sizeof(double)},
        {(const void *)k_leaf_qlcta, (mm * (mm | 1) + 4 * mm) * sizeof(double)},
        {(const void *)k_divide, 8 * rmax * rmax * sizeof(double)}};   // 64 KiB at the largest rank
    for (const auto &a : at) {
        e = cudaFuncSetAttribute(a.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.bytes);
        if (e != cudaSuccess) return e;
    }
    done[dev] = true;
    return cudaSuccess;
}

superdc_status superdc_eig_plan(const superdc_hss *h, const superdc_opts *opts, superdc_eigfact **fact)
{
    superdc_opts def;
    if (!opts) { superdc_opts_default(&def); opts = &def; }
    if (!h || !fact || !(opts->tau >= 0) || !(opts->stop_c > 0) || opts->max_iter < 1 || opts->sched < 0 ||
        opts->sched > 2 || (opts->shifted != 0 && opts->shifted != 1) || (opts->balanced != 0 && opts->balanced != 1) ||
        (opts->tape && !opts->balanced))
        return SUPERDC_ERR_ARG;
    const int64_t n = h->n;
    const int r = h->r, lmax = h->lmax, rr = r * r, nn = h->nnodes;
    superdc_eigfact *f = new superdc_eigfact();
    f->h = h; f->n = n; f->r = r; f->lmax = lmax;
    f->opts = *opts;
    f->fmm_min_m = fmm_resolve(opts->fmm_min_m);
    auto fail = [&](cudaError_t e) {
        superdc_eigfact_free(f);
        return e == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA;
    };
#define EIG_CHECK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return fail(e_); } while (0)
    // ---- storage of the structured Q
    std::vector<int64_t> qoff(h->nleaves + 1, 0);
    for (int k = 0; k < h->nleaves; k++) qoff[k + 1] = qoff[k] + h->size[h->leaves[k]] * h->size[h->leaves[k]];
    EIG_CHECK(dalloc(&f->Qleaf, qoff.back(), &f->slabs));
    EIG_CHECK(dalloc(&f->d_qoff, qoff.size(), &f->slabs));
    EIG_CHECK(dalloc(&f->status, 1, &f->slabs));
    EIG_CHECK(cudaMemcpy(f->d_qoff, qoff.data(), qoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    f->P.assign(lmax, nullptr);
    f->F.assign(lmax, std::vector<StepF>(r));
    for (int l = 0; l < lmax; l++) {
        EIG_CHECK(dalloc(&f->P[l], n, &f->slabs));
        const int64_t np = (int64_t)h->lev_nodes[l].size();
        for (int j = 0; j < r; j++) {
            StepF &S = f->F[l][j];
            // one slab per step: 9 double arrays (dk, eta, dorg, vhat, bnorm, giv_cs x2, din, zin),
            // int arrays
            double *dslab;
            EIG_CHECK(dalloc(&dslab, 9 * n, &f->slabs));
            S.dk = dslab; S.eta = dslab + n; S.dorg = dslab + 2 * n; S.vhat = dslab + 3 * n;
            S.bnorm = dslab + 4 * n; S.giv_cs = dslab + 5 * n; S.din = dslab + 7 * n; S.zin = dslab + 8 * n;
            int32_t *islab;
            EIG_CHECK(dalloc(&islab, 5 * n + 3 * np, &f->slabs));
            S.src = islab; S.pinv = islab + n; S.giv_ab = islab + 2 * n; S.sweeps = islab + 4 * n;
            S.mk = islab + 5 * n; S.ngiv = islab + 5 * n + np; S.fmm = islab + 5 * n + 2 * np;
        }
    }
    // ---- work buffers of the run (kept with the handle so that a run
    // allocates nothing but the stream-ordered scratch of its steps)
    EigWork &w = f->work;
    Tape &T = f->tape;
    T.on = opts->tape != 0;
    EIG_CHECK(dalloc(&w.H, (size_t)nn * rr, &f->slabs));
    EIG_CHECK(dalloc(&w.Bts, (size_t)nn * rr, &f->slabs));
    EIG_CHECK(dalloc(&w.sqb, nn, &f->slabs));
    if (T.on) {
        EIG_CHECK(dalloc(&T.Bt, (size_t)nn * rr, &f->slabs));
        EIG_CHECK(dalloc(&T.beta, nn, &f->slabs));
        EIG_CHECK(dalloc(&T.u1, (size_t)nn * r, &f->slabs));
        EIG_CHECK(dalloc(&T.v1, (size_t)nn * r, &f->slabs));
        T.H = w.H; T.Bts = w.Bts; T.sqb = w.sqb;
        T.lam_prev.assign(lmax, nullptr);
        T.Wprev.assign(lmax, nullptr);
        T.WKb.assign(lmax, std::vector<double *>(r, nullptr));
        for (int l = 0; l < lmax; l++) {
            const int ctot = (l == 0) ? r : 2 * r;
            EIG_CHECK(dalloc(&T.lam_prev[l], n, &f->slabs));
            EIG_CHECK(dalloc(&T.Wprev[l], (size_t)n * r, &f->slabs));
            for (int j = 0; j < r; j++) EIG_CHECK(dalloc(&T.WKb[l][j], (size_t)n * (ctot - j), &f->slabs));
        }
    }
    EIG_CHECK(dalloc(&w.lamA, n, &f->slabs));
    EIG_CHECK(dalloc(&w.lamB, n, &f->slabs));
    EIG_CHECK(dalloc(&w.Wp, (size_t)n * r, &f->slabs));
    EIG_CHECK(dalloc(&w.WK, (size_t)n * 2 * r, &f->slabs));
    EIG_CHECK(dalloc(&w.WK2, (size_t)n * 2 * r, &f->slabs));
    EIG_CHECK(dalloc(&w.zk, n, &f->slabs));
    EIG_CHECK(dalloc(&w.wsum, nn, &f->slabs));
    EIG_CHECK(dalloc(&w.org, n, &f->slabs));
    EIG_CHECK(dalloc(&w.perm, n, &f->slabs));
    EIG_CHECK(dalloc(&w.dq, n, &f->slabs));
    EIG_CHECK(dalloc(&w.bnrm, nn, &f->slabs));
    EIG_CHECK(dalloc(&w.rho_d, 1, &f->slabs));
    EIG_CHECK(cudaMemset(w.bnrm, 0, nn * sizeof(double)));
    EIG_CHECK(dalloc(&w.eq, n, &f->slabs));
    // leaf eigensolver layout and kernel attributes (set here, not in the run)
    const size_t mm = (size_t)h->mmax;
    w.leaf_batched = mm >= 96;
    w.smem1 = (mm * (mm | 1) + std::max(mm * (size_t)r, mm)) * sizeof(double);
    w.smem2 = 2 * mm * 32 * sizeof(double);
    // leaves per warp of the QL chase: about one warp per scheduler (4 per SM)
    w.ql_lpw = 1;
    while (w.ql_lpw < 32 && (int64_t)w.ql_lpw * 4 * sdc_num_sms() < h->nleaves) w.ql_lpw *= 2;
    w.smem3 = mm * (mm | 1) * sizeof(double);
    w.smem4 = (mm * (mm | 1) + 4 * mm) * sizeof(double);
    w.smem5 = (size_t)LEAF_R * (mm | 1) * sizeof(double);
    w.cap = 3 * (int64_t)mm * mm;
    w.caps = 16 * (int64_t)mm;
    // leaves all of 128 rows: divide and conquer inside the leaves (blocks of
    // 32, two merge levels); its QL records fit the leaves' record buffers
    w.leaf_dc = (mm == DC_M);
    for (int L : h->leaves) w.leaf_dc = w.leaf_dc && h->size[L] == DC_M;
    const int64_t nblk = n / DC_B;
    if (w.leaf_batched) {
        EIG_CHECK(dalloc(&w.rot, (size_t)h->nleaves * w.cap, &f->slabs));
        EIG_CHECK(dalloc(&w.hdr, (size_t)h->nleaves * w.caps, &f->slabs));
        EIG_CHECK(dalloc(&w.nsw, std::max<int64_t>(h->nleaves, w.leaf_dc ? nblk : 0), &f->slabs));
    }
    if (w.leaf_dc) {
        std::vector<int64_t> bo(nblk), bm(nblk, DC_B), bq(nblk);
        for (int64_t b = 0; b < nblk; b++) { bo[b] = b * DC_B; bq[b] = b * DC_B * DC_B; }
        EIG_CHECK(dalloc(&w.dc_boff, nblk, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_bm, nblk, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_bq, nblk, &f->slabs));
        EIG_CHECK(cudaMemcpy(w.dc_boff, bo.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
        EIG_CHECK(cudaMemcpy(w.dc_bm, bm.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
        EIG_CHECK(cudaMemcpy(w.dc_bq, bq.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
        for (int lv = 0; lv < 2; lv++) {
            const int64_t sz = 64 << lv, np = n / sz;
            std::vector<int64_t> po(np + 1);
            for (int64_t p = 0; p <= np; p++) po[p] = p * sz;
            EIG_CHECK(dalloc(&w.dc_off[lv], np + 1, &f->slabs));
            EIG_CHECK(cudaMemcpy(w.dc_off[lv], po.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        }
        EIG_CHECK(dalloc(&w.dc_scale, h->nleaves, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_beta, n, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_QB, (size_t)n * DC_B, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_Ya, (size_t)n * DC_M, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_Yb, (size_t)n * DC_M, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_X, (size_t)n * DC_M, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_Qh, (size_t)n * DC_M, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_lam, n, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_din, n, &f->slabs));
        EIG_CHECK(dalloc(&w.dc_zin, n, &f->slabs));
        R1Out &o = w.dc_o;
        for (double **x : {&o.dk, &o.zk, &o.eta, &o.vhat, &o.bnorm, &o.dorg}) EIG_CHECK(dalloc(x, n, &f->slabs));
        EIG_CHECK(dalloc(&o.giv_cs, 2 * (size_t)n, &f->slabs));
        for (int32_t **x : {&o.org, &o.src, &o.perm, &o.sweeps, &o.pinv}) EIG_CHECK(dalloc(x, n, &f->slabs));
        EIG_CHECK(dalloc(&o.giv_ab, 2 * (size_t)n, &f->slabs));
        EIG_CHECK(dalloc(&o.mk, n / 64, &f->slabs));
        EIG_CHECK(dalloc(&o.ngiv, n / 64, &f->slabs));
        EIG_CHECK(dalloc(&o.wsum, n / 64, &f->slabs));
        o.lam = w.dc_lam;
        o.status = f->status;
        o.fmm_used = nullptr;
        o.unshifted = 0;
    }
    EIG_CHECK(leaf_attrs());
    EIG_CHECK(r1_prepare());
#undef EIG_CHECK
    *fact = f;
    return SUPERDC_OK;
}

// Leaves of 128 rows, divide and conquer (see k_dc_tear): from the
// tridiagonal forms (w.dq, w.eq) and the Householder factors (w.dc_Qh) to
// the eigenvalues (w.dq) and row-major eigenvectors in the leaves' slots.
static superdc_status leaf_dc_run(superdc_eigfact *f, cudaStream_t st)
{
    const superdc_hss *h = f->h;
    const int64_t n = f->n, nblk = n / DC_B;
    EigWork &w = f->work;
    PROF_LAUNCH("leaf", st, k_dc_tear<<<(unsigned)h->nleaves, DC_M, 0, st>>>(h->d_leaf_off, w.dq, w.eq, w.dc_scale,
                                                                            w.dc_beta));
    // blocks of 32: QL chases (about one warp per scheduler), rotations onto identities
    int lpw = 1;
    while (lpw < 32 && (int64_t)lpw * 4 * sdc_num_sms() < nblk) lpw *= 2;
    const unsigned gq = (unsigned)((nblk + lpw - 1) / lpw);
    const size_t sq = 2 * (size_t)DC_B * lpw * sizeof(double);
    const int64_t capb = 3 * DC_B * DC_B, capsb = 16 * DC_B;
#define SDC_QL(W) \
    if (lpw == W) \
        PROF_LAUNCH("leaf", st, k_leaf_ql<W><<<gq, 32, sq, st>>>((int)nblk, DC_B, w.dc_boff, w.dc_bm, w.dq, w.eq, \
                                                                w.rot, w.hdr, w.nsw, capb, (int)capsb, f->status));
    SDC_QL(1) SDC_QL(2) SDC_QL(4) SDC_QL(8) SDC_QL(16) SDC_QL(32)
#undef SDC_QL
    const unsigned g = (unsigned)(sdc_num_sms() * 8);
    PROF_LAUNCH("leaf", st, k_dc_eye<<<g, 256, 0, st>>>(nblk, w.dc_QB));
    PROF_LAUNCH("leaf", st, k_leaf_rot<<<dim3((unsigned)nblk, 1), LEAF_R, (size_t)LEAF_R * (DC_B | 1) * sizeof(double),
                                         st>>>(w.dc_bm, w.dc_QB, w.dc_bq, w.rot, w.hdr, w.nsw, capb, (int)capsb));
    PROF_LAUNCH("leaf", st, k_dc_base<<<(unsigned)((nblk * 32 + 255) / 256), 256, 0, st>>>(nblk, n, w.dq, w.dc_QB,
                                                                                          w.dc_lam, w.dc_Ya));
    // two merge levels: 64 and 128 rows
    double *Yin = w.dc_Ya, *Yout = w.dc_Yb;
    for (int lv = 0; lv < 2; lv++) {
        const int sz = 64 << lv;
        const int64_t np = n / sz;
        PROF_LAUNCH("leaf", st, k_dc_merge_in<<<(unsigned)np, sz, 0, st>>>(n, sz, w.dc_lam, w.dc_beta, Yin, w.dc_din,
                                                                           w.dc_zin, w.dc_X));
        R1Args a;
        a.nprob = np;
        a.total = n;
        a.off = w.dc_off[lv];
        a.d = w.dc_din;
        a.z = w.dc_zin;
        a.sqrt_rho = 1.0;
        a.tau = 16.0 * SDC_EPS;                 // the leaves are scaled to norm <= 1
        a.stop_c = f->opts.stop_c;
        a.max_iter = f->opts.max_iter;
        a.tile_roots = 0;
        a.sched = 0;
        a.fmm_min_m = 0;
        a.max_m = sz;
        a.o = w.dc_o;
        superdc_status s = r1_run(a, st);
        if (s != SUPERDC_OK) return s;
        FactorView fv;
        fv.nprob = np; fv.off = w.dc_off[lv]; fv.mk = w.dc_o.mk; fv.ngiv = w.dc_o.ngiv; fv.dk = w.dc_o.dk;
        fv.eta = w.dc_o.eta; fv.dorg = w.dc_o.dorg; fv.vhat = w.dc_o.vhat; fv.bnorm = w.dc_o.bnorm;
        fv.src = w.dc_o.src; fv.perm = w.dc_o.perm; fv.pinv = w.dc_o.pinv; fv.giv_ab = w.dc_o.giv_ab;
        fv.giv_cs = w.dc_o.giv_cs; fv.fmm_min_m = 0; fv.max_m = sz;
#ifdef SUPERDC_CHECK
        fv.status = w.dc_o.status;
#endif
        s = cauchy_apply_T(fv, n, w.dc_X, n, Yout, n, sz, st);
        if (s != SUPERDC_OK) return s;
        std::swap(Yin, Yout);
    }
    PROF_LAUNCH("leaf", st, k_dc_gemm<<<dim3((unsigned)h->nleaves, DC_M / 64, DC_M / 64), 256, 0, st>>>(
                                n, h->d_leaf_off, f->d_qoff, w.dc_Qh, Yin, f->Qleaf, w.dc_lam, w.dc_scale, w.dq));
    return cudaGetLastError() == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}

superdc_status superdc_eig_run(superdc_eigfact *f, cudaStream_t st, double *lambda)
{
    if (!f || !lambda) return SUPERDC_ERR_ARG;
    const superdc_hss *h = f->h;
    const superdc_opts *opts = &f->opts;
    const int64_t n = f->n;
    const int r = f->r, lmax = f->lmax, rr = r * r, nn = h->nnodes;
    EigWork &w = f->work;
    Tape &T = f->tape;
    double *H = w.H, *Bts = w.Bts, *sqb = w.sqb;
    double *Wp = w.Wp, *WK = w.WK, *WK2 = w.WK2, *zk = w.zk, *wsum = w.wsum;
    int32_t *org = w.org, *perm = w.perm;
#define RUN_CHECK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) \
        return e_ == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA; } while (0)
    RUN_CHECK(cudaMemsetAsync(f->status, 0, sizeof(int32_t), st));
    RUN_CHECK(cudaMemsetAsync(H, 0, (size_t)nn * rr * sizeof(double), st));
    if (T.on) {
        RUN_CHECK(cudaMemsetAsync(T.Bt, 0, (size_t)nn * rr * sizeof(double), st));
        RUN_CHECK(cudaMemsetAsync(T.beta, 0, nn * sizeof(double), st));
    }
    const int nsm = sdc_num_sms();
    // ---- 1. dividing stage, top-down
    for (int l = 0; l < lmax; l++) {
        int nnodes_l = 0;
        for (int i : h->lev_nodes[l]) if (h->lch[i] >= 0) nnodes_l++;
        if (nnodes_l == 0) continue;
        PROF_LAUNCH("divide", st, k_divide<<<(unsigned)nnodes_l, 128, 8 * rr * sizeof(double), st>>>(
            h->d_lev_nodes[l], nn - 1, r, h->d_lch, h->d_rch, h->R, h->B, H, Bts, sqb, f->status,
            T.on ? T.Bt : nullptr, T.beta, T.u1, T.v1, opts->balanced, w.bnrm));
    }
    // ---- 2. leaves: large leaves (one CTA per SM) batch the QL chases one
    // lane per leaf; small leaves chase inside each leaf's CTA, several CTAs per SM
    {
        const int mm = h->mmax;
        PROF_LAUNCH("leaf", st, k_leaf_tri<<<(unsigned)h->nleaves, LEAF_T, w.smem1, st>>>(
            r, h->d_leaf_off, h->d_leaf_m, h->d_leaf_doff, h->d_leaf_uoff, h->d_leaf_id, h->D, h->U, H,
            w.leaf_dc ? w.dc_Qh : f->Qleaf, f->d_qoff, w.dq, w.eq));
        if (w.leaf_dc) {
            const superdc_status ls = leaf_dc_run(f, st);
            if (ls != SUPERDC_OK) return ls;
            PROF_LAUNCH("leaf", st, k_leaf_out<<<(unsigned)h->nleaves, LEAF_T, w.smem3, st>>>(
                r, n, h->d_leaf_off, h->d_leaf_m, h->d_leaf_uoff, h->U, f->Qleaf, f->d_qoff, w.dq, w.lamA, Wp,
                f->status));
        } else if (w.leaf_batched) {
            const int lpw = w.ql_lpw;
            const unsigned gq = (unsigned)((h->nleaves + lpw - 1) / lpw);
            const size_t sq = 2 * (size_t)mm * lpw * sizeof(double);
#define SDC_QL(W) \
            if (lpw == W) \
                PROF_LAUNCH("leaf", st, k_leaf_ql<W><<<gq, 32, sq, st>>>(h->nleaves, mm, h->d_leaf_off, h->d_leaf_m, \
                                                                        w.dq, w.eq, w.rot, w.hdr, w.nsw, w.cap, \
                                                                        (int)w.caps, f->status));
            SDC_QL(1) SDC_QL(2) SDC_QL(4) SDC_QL(8) SDC_QL(16) SDC_QL(32)
#undef SDC_QL
            PROF_LAUNCH("leaf", st, k_leaf_rot<<<dim3((unsigned)h->nleaves, (unsigned)((mm + LEAF_R - 1) / LEAF_R)),
                                                 LEAF_R, w.smem5, st>>>(h->d_leaf_m, f->Qleaf, f->d_qoff, w.rot, w.hdr,
                                                                        w.nsw, w.cap, (int)w.caps));
            PROF_LAUNCH("leaf", st, k_leaf_out<<<(unsigned)h->nleaves, LEAF_T, w.smem3, st>>>(
                r, n, h->d_leaf_off, h->d_leaf_m, h->d_leaf_uoff, h->U, f->Qleaf, f->d_qoff, w.dq, w.lamA, Wp,
                f->status));
        } else {
            PROF_LAUNCH("leaf", st, k_leaf_qlcta<<<(unsigned)h->nleaves, LEAF_T, w.smem4, st>>>(
                r, n, h->d_leaf_off, h->d_leaf_m, h->d_leaf_uoff, h->U, f->Qleaf, f->d_qoff, w.dq, w.eq, w.lamA, Wp,
                f->status));
        }
    }
    // largest |eigenvalue| of the updated leaf blocks, ||Dhat_k||_2 (Table 6's rho)
    RUN_CHECK(cudaMemsetAsync(w.rho_d, 0, sizeof(double), st));
    k_maxabs<<<(unsigned)nsm, 256, 0, st>>>(n, w.lamA, w.rho_d);
    // ---- 3. conquering stage, bottom-up over levels
    double *dcur = w.lamA, *dnxt = w.lamB;
    for (int l = lmax - 1; l >= 0; l--) {
        const int nl = (int)h->lev_nodes[l].size();
        const bool root = (l == 0);
        const int ctot = root ? r : 2 * r;
        int64_t lev_max = 0;
        for (int i : h->lev_nodes[l]) lev_max = std::max<int64_t>(lev_max, h->size[i]);
        if (T.on) {
            RUN_CHECK(cudaMemcpyAsync(T.lam_prev[l], dcur, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            RUN_CHECK(cudaMemcpyAsync(T.Wprev[l], Wp, (size_t)n * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        PROF_LAUNCH("build", st, k_build<<<(unsigned)(nsm * 4), 256, 0, st>>>(
            n, r, nl, h->d_lev_off[l], h->d_lev_nodes[l], nn - 1, h->d_lch, h->d_rch, h->d_size, h->R, Bts, sqb,
            dcur, Wp, dnxt, f->P[l], WK));
        std::swap(dcur, dnxt);
        for (int j = 0; j < r; j++) {
            StepF &S = f->F[l][j];
            if (T.on)
                RUN_CHECK(cudaMemcpyAsync(T.WKb[l][j], WK + (int64_t)j * n, (size_t)n * (ctot - j) * sizeof(double),
                                          cudaMemcpyDeviceToDevice, st));
            // the step's inputs (poles and z column), kept for inspection
            RUN_CHECK(cudaMemcpyAsync(S.din, dcur, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            RUN_CHECK(cudaMemcpyAsync(S.zin, WK + (int64_t)j * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            // level-batched (default): every node of the level is one problem of
            // one launch sequence; unbatched baseline: one sequence per node
            const int nseg = opts->batching ? 1 : nl;
            for (int q = 0; q < nseg; q++) {
                const int np = opts->batching ? nl : 1;
                R1Args a;
                a.nprob = np; a.total = n; a.off = h->d_lev_off[l] + q;
                a.rows = opts->batching ? n : h->size[h->lev_nodes[l][q]];
                a.d = dcur; a.z = WK + (int64_t)j * n;
                a.sqrt_rho = 1.0; a.tau = opts->tau; a.stop_c = opts->stop_c; a.max_iter = opts->max_iter;
                a.tile_roots = opts->tile_roots; a.sched = opts->sched;
                a.fmm_min_m = f->fmm_min_m;
                a.max_m = opts->batching ? lev_max : a.rows;
                a.o.lam = dnxt; a.o.dk = S.dk; a.o.zk = zk; a.o.eta = S.eta; a.o.vhat = S.vhat;
                a.o.bnorm = S.bnorm; a.o.org = org; a.o.src = S.src; a.o.perm = perm; a.o.giv_ab = S.giv_ab;
                a.o.giv_cs = S.giv_cs; a.o.mk = S.mk + q; a.o.ngiv = S.ngiv + q; a.o.sweeps = S.sweeps;
                a.o.status = f->status; a.o.dorg = S.dorg; a.o.pinv = S.pinv; a.o.wsum = wsum + q;
                a.o.fmm_used = S.fmm + q;
                a.o.unshifted = opts->shifted ? 0 : 1;
                const int c = ctot - (j + 1);
                // the step's FMM plan (tree, near lists, M2L kernel matrices)
                // also serves the Cauchy-like update of the remaining columns
                FmmPlan keep;
                if (opts->batching && c > 0 && c <= 24) { a.keep = &keep; a.keep_width = c; }
                superdc_status s1 = r1_run(a, st);
                if (s1 != SUPERDC_OK) { fmm_free(keep, st); return s1; }
                if (c > 0) {
                    FactorView v = view(f, l, j);
                    if (!opts->batching) {
                        v.nprob = 1; v.off += q; v.mk += q; v.ngiv += q;
                        v.max_m = h->size[h->lev_nodes[l][q]];
                    }
                    superdc_status s2 = cauchy_apply_T(v, n, WK + (int64_t)(j + 1) * n, n,
                                                       WK2 + (int64_t)(j + 1) * n, n, c, st,
                                                       a.keep ? &keep : nullptr);
                    if (s2 != SUPERDC_OK) { fmm_free(keep, st); return s2; }
                }
                fmm_free(keep, st);
            }
            if (ctot - (j + 1) > 0) std::swap(WK, WK2);
            std::swap(dcur, dnxt);
        }
        if (!root) RUN_CHECK(cudaMemcpyAsync(Wp, WK + (int64_t)r * n, (size_t)n * r * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
    }
    RUN_CHECK(cudaMemcpyAsync(lambda, dcur, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    RUN_CHECK(cudaGetLastError());
#undef RUN_CHECK
    f->last_stream = st;
    f->ran = true;
    return SUPERDC_OK;
}

superdc_status superdc_eig(const superdc_hss *h, const superdc_opts *opts, cudaStream_t st, double *lambda,
                           superdc_eigfact **fact)
{
    if (!h || !lambda || !fact) return SUPERDC_ERR_ARG;
    superdc_eigfact *f = nullptr;
    superdc_status s = superdc_eig_plan(h, opts, &f);
    if (s != SUPERDC_OK) return s;
    s = superdc_eig_run(f, st, lambda);
    if (s != SUPERDC_OK) {
        cudaStreamSynchronize(st);
        superdc_eigfact_free(f);
        return s;
    }
    int32_t word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, f->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { superdc_eigfact_free(f); return SUPERDC_ERR_CUDA; }
    *fact = f;
    return status_from_word(word);
}

superdc_status superdc_apply_Q(const superdc_eigfact *f, int32_t trans, int64_t ncols, const double *X, int64_t ldx,
                               double *Y, int64_t ldy, cudaStream_t st)
{
    if (!f || !X || !Y || ncols < 0 || (trans != 0 && trans != 1)) return SUPERDC_ERR_ARG;
    const superdc_hss *h = f->h;
    const int64_t n = f->n;
    if (ldx < n || ldy < n || ncols > INT32_MAX) return SUPERDC_ERR_ARG;
    if (ncols == 0) return SUPERDC_OK;
    const int nc = (int)ncols;
    const int nsm = sdc_num_sms();
    double *B0 = nullptr, *B1 = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&B0, (size_t)n * nc));
    SDC_CHECK(sc.get(&B1, (size_t)n * nc));
    const unsigned g = (unsigned)(nsm * 8);
    superdc_status s = SUPERDC_OK;
    if (trans) {
        PROF_LAUNCH("leafapply", st, k_leaf_apply<<<(unsigned)h->nleaves, 256, 0, st>>>(
            n, h->d_leaf_off, h->d_leaf_m, f->Qleaf, f->d_qoff, X, ldx, B0, n, nc, 1));
        for (int l = f->lmax - 1; l >= 0 && s == SUPERDC_OK; l--) {
            const int nl = (int)h->lev_nodes[l].size();
            PROF_LAUNCH("permute", st, k_permute<<<g, 256, 0, st>>>(n, nl, h->d_lev_off[l], f->P[l], B0, n, B1, n,
                                                                    nc, 0));
            std::swap(B0, B1);
            for (int j = 0; j < f->r && s == SUPERDC_OK; j++) {
                s = cauchy_apply_T(view(f, l, j), n, B0, n, B1, n, nc, st);
                std::swap(B0, B1);
            }
        }
        k_copy_cols<<<g, 256, 0, st>>>(n, nc, B0, n, Y, ldy);
    } else {
        k_copy_cols<<<g, 256, 0, st>>>(n, nc, X, ldx, B0, n);
        for (int l = 0; l < f->lmax && s == SUPERDC_OK; l++) {
            const int nl = (int)h->lev_nodes[l].size();
            for (int j = f->r - 1; j >= 0 && s == SUPERDC_OK; j--) {
                s = cauchy_apply_N(view(f, l, j), n, B0, n, B1, n, nc, st);
                std::swap(B0, B1);
            }
            PROF_LAUNCH("permute", st, k_permute<<<g, 256, 0, st>>>(n, nl, h->d_lev_off[l], f->P[l], B0, n, B1, n,
                                                                    nc, 1));
            std::swap(B0, B1);
        }
        PROF_LAUNCH("leafapply", st, k_leaf_apply<<<(unsigned)h->nleaves, 256, 0, st>>>(
            n, h->d_leaf_off, h->d_leaf_m, f->Qleaf, f->d_qoff, B0, n, Y, ldy, nc, 0));
    }
    cudaError_t e = cudaGetLastError();
    if (s != SUPERDC_OK) return s;
    return e == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}

superdc_status superdc_apply_function(const superdc_eigfact *f, const double *fvals, int64_t ncols,
                                      const double *X, int64_t ldx, double *Y, int64_t ldy, cudaStream_t st)
{
    if (!f || !fvals || !X || !Y || ncols < 0 || ncols > INT32_MAX) return SUPERDC_ERR_ARG;
    const int64_t n = f->n;
    if (ldx < n || ldy < n) return SUPERDC_ERR_ARG;
    if (ncols == 0) return SUPERDC_OK;
    double *T = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&T, (size_t)n * ncols));
    superdc_status s = superdc_apply_Q(f, 1, ncols, X, ldx, T, n, st);
    if (s != SUPERDC_OK) return s;
    PROF_LAUNCH("scale", st, k_scale_rows<<<(unsigned)(sdc_num_sms() * 8), 256, 0, st>>>(n, (int)ncols, fvals, T, n));
    return superdc_apply_Q(f, 0, ncols, T, n, Y, ldy, st);
}

superdc_status superdc_eigfact_set_fmm_min_m(superdc_eigfact *f, int32_t fmm_min_m)
{
    if (!f) return SUPERDC_ERR_ARG;
    f->fmm_min_m = fmm_resolve(fmm_min_m);
    return SUPERDC_OK;
}

superdc_status superdc_sync_status(const superdc_eigfact *f)
{
    if (!f) return SUPERDC_ERR_ARG;
    int32_t word = 0;
    if (cudaMemcpy(&word, f->status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return SUPERDC_ERR_CUDA;
    return status_from_word(word);
}

superdc_status superdc_eigfact_stats(const superdc_eigfact *f, int64_t *deflated, int64_t *sweeps, int32_t *max_sweeps)
{
    if (!f) return SUPERDC_ERR_ARG;
    unsigned long long *acc = nullptr;
    if (cudaMalloc(&acc, 3 * sizeof(unsigned long long)) != cudaSuccess) return SUPERDC_ERR_OOM;
    cudaMemset(acc, 0, 3 * sizeof(unsigned long long));
    for (int l = 0; l < f->lmax; l++)
        for (int j = 0; j < f->r; j++)
            k_stats<<<256, 128>>>((int64_t)f->h->lev_nodes[l].size(), f->h->d_lev_off[l], f->F[l][j].mk,
                                  f->F[l][j].sweeps, acc);
    unsigned long long hv[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpy(hv, acc, sizeof(hv), cudaMemcpyDeviceToHost);
    cudaFree(acc);
    if (e != cudaSuccess) return SUPERDC_ERR_CUDA;
    if (deflated) *deflated = (int64_t)hv[0];
    if (sweeps) *sweeps = (int64_t)hv[1];
    if (max_sweeps) *max_sweeps = (int32_t)hv[2];
    return SUPERDC_OK;
}

superdc_status superdc_eigfact_get(const superdc_eigfact *f, int32_t level, int32_t step, const char *field,
                                   void *dst)
{
    if (!f || !field || !dst || level < 0 || level >= f->lmax || step < 0 || step >= f->r) return SUPERDC_ERR_ARG;
    const StepF &S = f->F[level][step];
    const int64_t n = f->n, np = (int64_t)f->h->lev_nodes[level].size();
    const void *src = nullptr;
    size_t bytes = 0;
    std::string fld(field);
    if (fld == "dk") { src = S.dk; bytes = n * 8; }
    else if (fld == "eta") { src = S.eta; bytes = n * 8; }
    else if (fld == "dorg") { src = S.dorg; bytes = n * 8; }
    else if (fld == "vhat") { src = S.vhat; bytes = n * 8; }
    else if (fld == "bnorm") { src = S.bnorm; bytes = n * 8; }
    else if (fld == "din") { src = S.din; bytes = n * 8; }
    else if (fld == "zin") { src = S.zin; bytes = n * 8; }
    else if (fld == "src") { src = S.src; bytes = n * 4; }
    else if (fld == "pinv") { src = S.pinv; bytes = n * 4; }
    else if (fld == "sweeps") { src = S.sweeps; bytes = n * 4; }
    else if (fld == "P") { src = f->P[level]; bytes = n * 4; }
    else if (fld == "giv_cs") { src = S.giv_cs; bytes = 2 * n * 8; }
    else if (fld == "giv_ab") { src = S.giv_ab; bytes = 2 * n * 4; }
    else if (fld == "mk") { src = S.mk; bytes = np * 4; }
    else if (fld == "ngiv") { src = S.ngiv; bytes = np * 4; }
    else if (fld == "fmm") { src = S.fmm; bytes = np * 4; }
    else return SUPERDC_ERR_ARG;
    return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}

superdc_status superdc_eigfact_norms(const superdc_eigfact *f, double *rho_bt, double *rho_dt)
{
    if (!f || !f->ran) return f ? SUPERDC_ERR_STATE : SUPERDC_ERR_ARG;
    const int nn = f->h->nnodes;
    std::vector<double> b(nn);
    double d = 0.0;
    if (cudaMemcpy(b.data(), f->work.bnrm, nn * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&d, f->work.rho_d, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SUPERDC_ERR_CUDA;
    double mb = 0.0;
    for (int i = 0; i < nn; i++) mb = std::isnan(b[i]) ? INFINITY : std::max(mb, b[i]);
    if (rho_bt) *rho_bt = mb;
    if (rho_dt) *rho_dt = d;
    return SUPERDC_OK;
}

superdc_status superdc_eigfact_shape(const superdc_eigfact *f, int32_t *lmax, int32_t *r, int64_t *n)
{
    if (!f) return SUPERDC_ERR_ARG;
    if (lmax) *lmax = f->lmax;
    if (r) *r = f->r;
    if (n) *n = f->n;
    return SUPERDC_OK;
}

}  // extern "C"

FactorView factor_view(const superdc_eigfact *f, int l, int j) { return view(f, l, j); }

superdc_status leaves_apply(const superdc_eigfact *f, int trans, int ncols, const double *X, int64_t ldx, double *Y,
                            int64_t ldy, cudaStream_t st)
{
    const superdc_hss *h = f->h;
    k_leaf_apply<<<(unsigned)h->nleaves, 256, 0, st>>>(f->n, h->d_leaf_off, h->d_leaf_m, f->Qleaf, f->d_qoff, X, ldx,
                                                       Y, ldy, ncols, trans);
    return cudaGetLastError() == cudaSuccess ? SUPERDC_OK : SUPERDC_ERR_CUDA;
}
