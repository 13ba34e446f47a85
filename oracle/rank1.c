/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, slow, FP64 C implementation of one rank-one update step of the
 * SuperDC conquering stage (Ou & Xia, "SuperDC: stable superfast
 * divide-and-conquer eigenvalue decomposition"), plus a dense cyclic Jacobi
 * eigensolver used for the leaf blocks.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may call this code; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * Problem: diag(d) + z z^T with d ascending (length m).
 *   1. deflation, Remark 4.1 (|z_k| < tau first; then a left-to-right Givens
 *      scan over the survivors with the test |(d_a-d_b) z_a z_b| < (z_a^2+z_b^2) tau);
 *   2. secular roots in shifted form, Section 4.2 (eqs. (4.13), (4.14), (4.17)):
 *      origin d_k or d_{k+1} chosen by the sign of f at the midpoint,
 *      gap eta = lambda - d_K; the sums are split into the triangular parts
 *      psi (j <= k) and phi (j > k) of eqs. (4.7)-(4.10);
 *      mode 0 = bisection of g_K to adjacent doubles ("exact"),
 *      mode 1 = middle-way modified Newton (Section 4.1.3, following Li's
 *      rational interpolation) with the stopping test eq. (4.12) and a
 *      bisection safeguard;
 *   3. Loewner's formula eq. (4.23) for zhat (paired ratios, shifted differences);
 *   4. normalisation b, eq. (4.27), with shifted differences eq. (4.28);
 *   5. the new eigenvalues sorted by (value, input index).
 * Plus the application of the Cauchy-like factor eqs. (4.26)/(4.29) and its
 * transpose (Algorithms 3 and 4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define EPS DBL_EPSILON

/* ------------------------------------------------------------------ */
/* 1. Deflation (Remark 4.1)                                            */
/* ------------------------------------------------------------------ */
/* in : m, d[m] ascending, z[m], tau
 * out: dd[m] values after the rotations, zz[m] z after rotations,
 *      kept[m] 1 if entry stays in the secular problem,
 *      giv_a/giv_b (input indices), giv_c/giv_s: rotations in scan order.
 * returns the number of rotations. */
int orc_deflate(int m, const double *d, const double *z, double tau,
                double *dd, double *zz, int *kept,
                int *giv_a, int *giv_b, double *giv_c, double *giv_s)
{
    int ng = 0;
    for (int i = 0; i < m; i++) {
        dd[i] = d[i];
        zz[i] = z[i];
        kept[i] = fabs(z[i]) < tau ? 0 : 1;   /* step 1: small z */
        if (!kept[i]) zz[i] = 0.0;
    }
    int a = -1;                               /* step 2: Givens scan */
    for (int b = 0; b < m; b++) {
        if (!kept[b]) continue;
        if (a >= 0) {
            double za = zz[a], zb = zz[b];
            double lhs = fabs((dd[a] - dd[b]) * za * zb);
            double rhs = (za * za + zb * zb) * tau;
            if (lhs < rhs) {
                double rho = sqrt(za * za + zb * zb);
                double c = zb / rho, s = za / rho;
                double da = dd[a], db = dd[b];
                dd[a] = c * c * da + s * s * db;
                dd[b] = s * s * da + c * c * db;
                zz[a] = 0.0;
                zz[b] = rho;
                kept[a] = 0;
                giv_a[ng] = a; giv_b[ng] = b; giv_c[ng] = c; giv_s[ng] = s;
                ng++;
            }
        }
        a = b;
    }
    return ng;
}

/* ------------------------------------------------------------------ */
/* 2. Secular equation g_K(y) = 1 + sum_j w_j / ((d_j - d_K) - y)        */
/* ------------------------------------------------------------------ */
/* Evaluates g and the triangular parts at y in the frame of origin K,
 * splitting the sum at index k (j <= k: psi, j > k: phi). */
static double geval(int m, const double *d, const double *w, int K, int k, double y,
                    double *psi, double *phi, double *dpsi, double *dphi)
{
    double p = 0, q = 0, dp = 0, dq = 0;
    double dK = d[K];
    for (int j = 0; j < m; j++) {
        double t = (d[j] - dK) - y;
        double a = w[j] / t;
        if (j <= k) { p += a; dp += a / t; }
        else        { q += a; dq += a / t; }
    }
    if (psi) *psi = p;
    if (phi) *phi = q;
    if (dpsi) *dpsi = dp;
    if (dphi) *dphi = dq;
    return 1.0 + p + q;
}

/* the root of a*y^2 + b*y + c = 0 lying strictly inside (lo, hi); if none,
 * the middle of the bracket */
static double quad_in(double a, double b, double c, double lo, double hi)
{
    double mid = 0.5 * (lo + hi);
    if (a == 0.0) {
        if (b == 0.0) return mid;
        double y = -c / b;
        return (y > lo && y < hi) ? y : mid;
    }
    double disc = b * b - 4.0 * a * c;
    if (!(disc >= 0.0)) return mid;
    double sq = sqrt(disc);
    double q = -0.5 * (b + (b >= 0 ? sq : -sq));
    double y1 = q / a;
    double y2 = (q != 0.0) ? c / q : y1;
    if (y1 > lo && y1 < hi) return y1;
    if (y2 > lo && y2 < hi) return y2;
    return mid;
}

/* one root.  d, w: kept problem (m entries, d ascending, w = z^2 > 0).
 * out: *K origin index, *eta gap, *iters sweeps used.
 * returns 0 on success, 1 when mode 1 did not meet the stopping test. */
int orc_secular_root(int m, const double *d, const double *w, int k, int mode,
                     double stop_c, int max_iter, int *Kout, double *etaout, int *iters)
{
    int last = (k == m - 1);
    int K;
    double lo, hi, y, glo, ghi;
    double W = 0;
    for (int j = 0; j < m; j++) W += w[j];
    int sweeps = 0;
    double rest;      /* frozen non-adjacent part at the midpoint (initial guess) */
    double fmid;
    double ym;
    if (!last) {
        double D = d[k + 1] - d[k];
        double h = 0.5 * D;
        fmid = geval(m, d, w, k, k, h, NULL, NULL, NULL, NULL);
        sweeps++;
        rest = fmid + w[k] / h - w[k + 1] / (D - h);
        if (fmid >= 0.0) { K = k;     lo = 0.0; hi = h;  glo = -INFINITY; ghi = fmid; }
        else             { K = k + 1; lo = -h;  hi = 0.0; glo = fmid;     ghi = INFINITY; }
        (void)ym;
    } else {
        K = k;
        ym = 0.5 * W;
        fmid = geval(m, d, w, K, k, ym, NULL, NULL, NULL, NULL);
        sweeps++;
        if (fmid >= 0.0) { lo = 0.0; hi = ym; glo = -INFINITY; ghi = fmid; }
        else             { lo = ym;  hi = W;  glo = fmid;      ghi = geval(m, d, w, K, k, W, NULL, NULL, NULL, NULL); sweeps++; }
        rest = fmid + w[k] / ym;
        /* g(W) >= 0 in exact arithmetic; widen if rounding says otherwise */
        int guard = 0;
        while (ghi < 0.0 && guard < 64) {
            lo = hi; glo = ghi; hi = 2.0 * hi;
            ghi = geval(m, d, w, K, k, hi, NULL, NULL, NULL, NULL);
            sweeps++; guard++;
        }
    }

    if (mode == 0) {
        /* bisection of the increasing function g_K on (lo, hi) */
        for (int it = 0; it < 5000; it++) {
            double mid = lo + 0.5 * (hi - lo);
            if (!(mid > lo && mid < hi)) break;
            double g = geval(m, d, w, K, k, mid, NULL, NULL, NULL, NULL);
            sweeps++;
            if (g < 0.0) { lo = mid; glo = g; } else { hi = mid; ghi = g; }
        }
        y = (fabs(glo) < fabs(ghi)) ? lo : hi;
        *Kout = K; *etaout = y; if (iters) *iters = sweeps;
        return 0;
    }

    /* mode 1: initial guess by freezing the non-adjacent terms (Li's scheme) */
    if (!last) {
        double a = d[k] - d[K], b = d[k + 1] - d[K];
        double A2 = rest;
        double B2 = -(rest * (a + b) + w[k] + w[k + 1]);
        double C2 = w[k] * b + w[k + 1] * a;
        y = quad_in(A2, B2, C2, lo, hi);
    } else {
        y = (rest > 0.0) ? w[k] / rest : 0.5 * (lo + hi);
        if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
    }
    double eps_tol = stop_c * (double)m * EPS;
    for (int it = 0; it < max_iter; it++) {
        double psi, phi, dpsi, dphi;
        double f = geval(m, d, w, K, k, y, &psi, &phi, &dpsi, &dphi);
        sweeps++;
        if (fabs(f) < eps_tol * (1.0 + fabs(psi) + fabs(phi))) {      /* eq. (4.12) */
            *Kout = K; *etaout = y; if (iters) *iters = sweeps;
            return 0;
        }
        if (f < 0.0) lo = y; else hi = y;
        double ynew;
        if (!last) {
            double Dk  = (d[k] - d[K]) - y;       /* d_k - x     */
            double Dk1 = (d[k + 1] - d[K]) - y;   /* d_{k+1} - x */
            double c = f - Dk * dpsi - Dk1 * dphi;
            double A = (Dk + Dk1) * f - Dk * Dk1 * (dpsi + dphi);
            double Bq = Dk * Dk1 * f;
            double corr;
            if (c == 0.0) {
                corr = (A != 0.0) ? Bq / A : 0.0;
            } else {
                double disc = A * A - 4.0 * Bq * c;
                if (disc < 0.0) disc = 0.0;
                double s = sqrt(disc);
                double den = A + (A >= 0 ? s : -s);
                corr = (den != 0.0) ? 2.0 * Bq / den : 0.0;
            }
            ynew = y + corr;
        } else {
            double Dl = (d[k] - d[K]) - y;
            double den = f - Dl * dpsi;
            double corr = (den != 0.0) ? Dl + Dl * Dl * dpsi / den : 0.0;
            ynew = y + corr;
        }
        if (!(ynew > lo && ynew < hi)) ynew = lo + 0.5 * (hi - lo);
        if (ynew == y || !(ynew > lo && ynew < hi)) {
            /* bracket exhausted at double resolution */
            *Kout = K; *etaout = y; if (iters) *iters = sweeps;
            return 0;
        }
        y = ynew;
    }
    *Kout = K; *etaout = y; if (iters) *iters = sweeps;
    return 1;
}

/* all roots of a kept problem; returns the number of roots that failed */
int orc_secular_all(int m, const double *d, const double *z, int mode, double stop_c,
                    int max_iter, int *K, double *eta, int *iters)
{
    double *w = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int j = 0; j < m; j++) w[j] = z[j] * z[j];
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+:bad)
    for (int k = 0; k < m; k++)
        bad += orc_secular_root(m, d, w, k, mode, stop_c, max_iter, &K[k], &eta[k],
                                iters ? &iters[k] : NULL);
    free(w);
    return bad;
}

/* ------------------------------------------------------------------ */
/* 3. Loewner's formula, eq. (4.23), paired as in Gu & Eisenstat         */
/* ------------------------------------------------------------------ */
/* lambda_j - d_i evaluated as (d_{K_j} - d_i) + eta_j */
void orc_lowner(int m, const double *d, const double *z, const int *K, const double *eta,
                double *vhat)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < m; i++) {
        double di = d[i];
        double prod = (d[K[m - 1]] - di) + eta[m - 1];
        for (int j = 0; j < i; j++)
            prod *= ((d[K[j]] - di) + eta[j]) / (d[j] - di);
        for (int j = i; j < m - 1; j++)
            prod *= ((d[K[j]] - di) + eta[j]) / (d[j + 1] - di);
        double v = sqrt(prod);
        vhat[i] = (z[i] < 0) ? -v : v;
    }
}

/* ------------------------------------------------------------------ */
/* 4. b_j = (sum_i vhat_i^2 / ((d_i - d_{K_j}) - eta_j)^2)^(-1/2), eq. (4.27) */
/* ------------------------------------------------------------------ */
void orc_bnorm(int m, const double *d, const double *vhat, const int *K, const double *eta,
               double *b)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < m; j++) {
        double s = 0.0;
        double dK = d[K[j]];
        for (int i = 0; i < m; i++) {
            double t = (d[i] - dK) - eta[j];
            s += (vhat[i] * vhat[i]) / (t * t);
        }
        b[j] = 1.0 / sqrt(s);
    }
}

/* ------------------------------------------------------------------ */
/* Cauchy-like factor Qc(i,j) = vhat_i b_j / ((d_i - d_{K_j}) - eta_j)  */
/* X, Y: m x c row-major.  trans=1: Y = Qc^T X, trans=0: Y = Qc X      */
/* ------------------------------------------------------------------ */
void orc_cauchy_apply(int m, int c, const double *d, const double *vhat, const double *b,
                      const int *K, const double *eta, int trans,
                      const double *X, double *Y)
{
    #pragma omp parallel for schedule(static)
    for (int o = 0; o < m; o++) {
        for (int col = 0; col < c; col++) Y[(size_t)o * c + col] = 0.0;
        for (int q = 0; q < m; q++) {
            int i = trans ? q : o;   /* row index of Qc */
            int j = trans ? o : q;   /* column index    */
            double e = vhat[i] * b[j] / ((d[i] - d[K[j]]) - eta[j]);
            for (int col = 0; col < c; col++)
                Y[(size_t)o * c + col] += e * X[(size_t)q * c + col];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Dense cyclic Jacobi (row-cyclic order), A symmetric n x n row-major.  */
/* On exit lam ascending, V columns the eigenvectors (row-major n x n).  */
/* Stops when off(A) <= eps * ||A||_F or after maxsweep sweeps.           */
/* Each rotation J (c, s on (p, q)) forms J^T A J: rows p, q first; by    */
/* symmetry the new columns p, q are the new rows p, q.  The rotations    */
/* are accumulated into W = V^T (rows), transposed at the end.            */
/* ------------------------------------------------------------------ */
int orc_jacobi(int n, double *A, double *V, double *lam, int maxsweep)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) W[i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0;
    for (int i = 0; i < n * n; i++) fro += A[i] * A[i];
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep < maxsweep; sweep++) {
        double off = 0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if (i != j) off += A[i * n + j] * A[i * n + j];
        if (sqrt(off) <= EPS * fro) break;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double zeta = (aqq - app) / (2.0 * apq);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* J = [[c, s], [-s, c]] on (p, q): rows of J^T A */
                double *rp = A + (size_t)p * n, *rq = A + (size_t)q * n;
                for (int k = 0; k < n; k++) {
                    double apk = rp[k], aqk = rq[k];
                    rp[k] = c * apk - s * aqk;
                    rq[k] = s * apk + c * aqk;
                }
                /* 2x2 block of (J^T A) J */
                double bpp = rp[p], bpq = rp[q], bqp = rq[p], bqq = rq[q];
                rp[p] = c * bpp - s * bpq;
                rp[q] = s * bpp + c * bpq;
                rq[p] = c * bqp - s * bqq;
                rq[q] = s * bqp + c * bqq;
                /* columns p, q mirror rows p, q */
                for (int k = 0; k < n; k++) {
                    if (k == p || k == q) continue;
                    A[(size_t)k * n + p] = rp[k];
                    A[(size_t)k * n + q] = rq[k];
                }
                double *wp = W + (size_t)p * n, *wq = W + (size_t)q * n;
                for (int k = 0; k < n; k++) {
                    double vp = wp[k], vq = wq[k];
                    wp[k] = c * vp - s * vq;
                    wq[k] = s * vp + c * vq;
                }
            }
        }
    }
    /* sort ascending (selection sort, eigenvector rows of W follow) */
    for (int i = 0; i < n; i++) lam[i] = A[i * n + i];
    for (int i = 0; i < n; i++) {
        int mi = i;
        for (int j = i + 1; j < n; j++) if (lam[j] < lam[mi]) mi = j;
        if (mi != i) {
            double t = lam[i]; lam[i] = lam[mi]; lam[mi] = t;
            for (int k = 0; k < n; k++) {
                double u = W[(size_t)i * n + k]; W[(size_t)i * n + k] = W[(size_t)mi * n + k]; W[(size_t)mi * n + k] = u;
            }
        }
    }
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++) V[(size_t)k * n + i] = W[(size_t)i * n + k];
    free(W);
    return sweep;
}
