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

/* Rational model of Section 4.1.3 ("middle way", after Li): near the
 * bracket (delta_k, delta_{k+1}) of root k, in the frame of origin K
 * (delta_j = d_j - d_K), the secular function is modelled as
 *     h(xi) = C + beta1 / (delta_k - xi) + beta2 / (delta_{k+1} - xi),
 * which is strictly increasing between its two poles and therefore has
 * exactly one zero there.  Written with the step s = xi - y from the current
 * point y, p = delta_k - y < 0 < q = delta_{k+1} - y, the zero solves
 *     C s^2 - (C (p + q) + beta1 + beta2) s + p q h(y) = 0
 * (multiply h by (p - s)(q - s); the constant term C p q + beta1 q + beta2 p
 * equals p q h(y), which the iteration passes as such: it tends to 0 with
 * h(y) instead of cancelling).  model_step returns the zero lying in (p, q): both roots
 * of the quadratic are formed without cancellation (the one of larger
 * magnitude from the sign-matched sum, the other as the product over it),
 * and the one between the poles is kept.  Returns 0 when rounding leaves no
 * root strictly inside (p, q); the caller then bisects. */
static int model_step(double C, double beta1, double beta2, double p, double q, double cst,
                      double *s_out)
{
    double lin = -(C * (p + q) + beta1 + beta2);     /* coefficient of s   */
    double r1, r2;
    if (C == 0.0) {                                    /* linear model       */
        if (lin == 0.0) return 0;
        r1 = r2 = -cst / lin;
    } else {
        double disc = lin * lin - 4.0 * C * cst;
        if (disc < 0.0) disc = 0.0;                    /* rounding only: one zero is between the poles */
        double big = -0.5 * (lin + copysign(sqrt(disc), lin));
        if (big == 0.0) { r1 = r2 = 0.0; }
        else { r1 = big / C; r2 = cst / big; }
    }
    int in1 = (r1 > p && r1 < q), in2 = (r2 > p && r2 < q);
    if (in1 && in2) { *s_out = (fabs(r1) <= fabs(r2)) ? r1 : r2; return 1; }
    if (in1) { *s_out = r1; return 1; }
    if (in2) { *s_out = r2; return 1; }
    return 0;
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
    double ymid, fmid;
    if (!last) {
        /* origin (Section 4.2.1): the sign of f at the middle of (d_k, d_{k+1})
         * says which pole the root is closer to */
        ymid = 0.5 * (d[k + 1] - d[k]);
        fmid = geval(m, d, w, k, k, ymid, NULL, NULL, NULL, NULL);
        sweeps++;
        if (fmid >= 0.0) { K = k;     lo = 0.0;   hi = ymid; glo = -INFINITY; ghi = fmid; }
        else             { K = k + 1; lo = -ymid; hi = 0.0;  glo = fmid;      ghi = INFINITY; }
    } else {
        /* last root: lambda in (d_{m-1}, d_{m-1} + sum w); test the middle */
        K = k;
        ymid = 0.5 * W;
        fmid = geval(m, d, w, K, k, ymid, NULL, NULL, NULL, NULL);
        sweeps++;
        if (fmid >= 0.0) { lo = 0.0;  hi = ymid; glo = -INFINITY; ghi = fmid; }
        else             { lo = ymid; hi = W;    glo = fmid;      ghi = geval(m, d, w, K, k, W, NULL, NULL, NULL, NULL); sweeps++; }
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

    /* mode 1.  Start (after Li): keep the poles next to the root exactly
     * and freeze every other term at its value at the middle point,
     *   h0(xi) = rest + w_k/(delta_k - xi) [+ w_{k+1}/(delta_{k+1} - xi)],
     * with rest = f(ymid) minus the adjacent terms at ymid (evaluated in the
     * frame of d_k, where f(ymid) was taken), and start from h0's zero. */
    double dlo = d[k] - d[K];                          /* delta_k in the chosen frame     */
    double dhi = last ? 0.0 : d[k + 1] - d[K];         /* delta_{k+1} in the chosen frame */
    double rest;
    if (!last) rest = fmid + w[k] / ymid - w[k + 1] / ((d[k + 1] - d[k]) - ymid);
    else       rest = fmid + w[k] / ymid;
    y = lo + 0.5 * (hi - lo);
    if (!last) {
        /* step from xi = 0; one of dlo, dhi is 0 (the origin pole), so the
         * constant term is the limit w_k dhi + w_{k+1} dlo (+ rest dlo dhi = 0) */
        double s0;
        if (model_step(rest, w[k], w[k + 1], dlo, dhi, rest * dlo * dhi + w[k] * dhi + w[k + 1] * dlo, &s0)
            && s0 > lo && s0 < hi)
            y = s0;
    } else if (rest > 0.0) {
        /* one-pole model rest + w_k/(0 - xi) = 0 */
        double x0 = w[k] / rest;
        if (x0 > lo && x0 < hi) y = x0;
    }

    double tol_c = stop_c * (double)m * EPS;
    for (int it = 0; it < max_iter; it++) {
        double psi, phi, dpsi, dphi;
        double f = geval(m, d, w, K, k, y, &psi, &phi, &dpsi, &dphi);
        sweeps++;
        /* stopping test, eq. (4.12) */
        if (fabs(f) < tol_c * (1.0 + fabs(psi) + fabs(phi))) {
            *Kout = K; *etaout = y; if (iters) *iters = sweeps;
            return 0;
        }
        /* g_K increases on the bracket: shrink it to the side of the root */
        if (f > 0.0) hi = y; else lo = y;
        /* match value and slope of psi at y by alpha1 + beta1/(delta_k - xi)
         * and of phi by alpha2 + beta2/(delta_{k+1} - xi) */
        double p = dlo - y;
        double beta1 = dpsi * p * p;
        double alpha1 = psi - dpsi * p;
        double xi;
        int ok;
        if (!last) {
            double q = dhi - y;
            double beta2 = dphi * q * q;
            double alpha2 = phi - dphi * q;
            double s;
            ok = model_step(1.0 + alpha1 + alpha2, beta1, beta2, p, q, p * q * f, &s);
            xi = y + s;
        } else {
            /* no pole to the right: 1 + alpha1 + beta1/(delta_k - xi) = 0 */
            double C = 1.0 + alpha1;
            ok = (C != 0.0);
            xi = ok ? dlo + beta1 / C : y;
        }
        if (!ok || !(xi > lo && xi < hi)) xi = lo + 0.5 * (hi - lo);   /* safeguard: bisect */
        if (!(xi > lo && xi < hi) || xi == y) {
            /* the bracket holds no other double */
            *Kout = K; *etaout = y; if (iters) *iters = sweeps;
            return 0;
        }
        y = xi;
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

/* the roots ks[0..nk-1] of a kept problem only (same per-root routine);
 * returns the number of roots that failed */
int orc_secular_some(int m, const double *d, const double *z, int nk, const int *ks, int mode,
                     double stop_c, int max_iter, int *K, double *eta, int *iters)
{
    double *w = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int j = 0; j < m; j++) w[j] = z[j] * z[j];
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 4) reduction(+:bad)
    for (int t = 0; t < nk; t++)
        bad += orc_secular_root(m, d, w, ks[t], mode, stop_c, max_iter, &K[t], &eta[t],
                                iters ? &iters[t] : NULL);
    free(w);
    return bad;
}

/* f = g_K(y) and its triangular parts at given points: root ks[t] in the
 * frame of origin Ks[t] at gap ys[t] (direct sums, the same evaluation as the
 * iteration).  Outputs per point: f, psi, phi and f' = psi' + phi'. */
void orc_secular_eval(int m, const double *d, const double *z, int nk, const int *ks, const int *Ks,
                      const double *ys, double *f, double *psi, double *phi, double *df)
{
    double *w = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int j = 0; j < m; j++) w[j] = z[j] * z[j];
    #pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < nk; t++) {
        double p, q, dp, dq;
        f[t] = geval(m, d, w, Ks[t], ks[t], ys[t], &p, &q, &dp, &dq);
        psi[t] = p; phi[t] = q; df[t] = dp + dq;
    }
    free(w);
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
