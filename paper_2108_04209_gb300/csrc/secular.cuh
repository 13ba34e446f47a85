// Device building blocks of the secular-equation solver shared by the
// direct tiled evaluator (rank1.cu) and the triangular FMM path (fmm.cu):
// the FP64 reciprocal, the bracketed quadratic root, the triangular sweep
// over staged poles (eqs. (4.7)-(4.10), shifted differences of eq. (4.14))
// and the per-root iteration state (Algorithm 2, stopping test eq. (4.12)).
#pragma once
#include "common.cuh"

namespace {

// ---------------------------------------------------------------------------
// FP64 reciprocal without the FP64 divide sequence.  The GB300 FP64 pipe
// retires ~2 DFMA per clock per SM, so every FP64 instruction of the inner
// loops counts, while integer and MUFU pipes are nearly free.  Seed: the
// leading 23 mantissa bits of |t| as a float in [1,2), reciprocal on the MUFU
// (rcp.approx.f32, relative error < 2^-22 after the truncation), exponent and
// sign rebuilt with integer arithmetic (valid for every normal double).  Then
// Newton-Raphson r <- r + r (1 - t r), which squares the relative error:
// one step -> < 2^-44, two steps -> correctly rounded up to ~1 ulp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mufu_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ double rcp_seed(double t)
{
    const int hi = __double2hiint(t);
    const unsigned lo = (unsigned)__double2loint(t);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int e = (hi >> 20) & 0x7FF;
    const unsigned mb = (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
    const float rm = mufu_rcp(__uint_as_float(0x3F800000u | mb));   // in (0.5, 1]
    const unsigned rb = __float_as_uint(rm);
    const int E = (int)(rb >> 23) - 127 - (e - 1023) + 1023;
    const unsigned rmant = rb & 0x7FFFFFu;
    return __hiloint2double((int)(sign | ((unsigned)E << 20) | (rmant >> 3)), (int)(rmant << 29));
}

// one Newton step: relative error < 2^-44 (secular sweeps: every term of psi
// (phi) has the same sign, so the sum inherits the per-term bound, which is
// below the stopping tolerance of eq. (4.12) for m >= 32)
__device__ __forceinline__ double rcp_nr1(double t)
{
    double r = rcp_seed(t);
    double e = fma(-t, r, 1.0);
    return fma(r, e, r);
}

// two Newton steps: full FP64 accuracy (b, Cauchy-like applications)
__device__ __forceinline__ double rcp_nr2(double t)
{
    double r = rcp_seed(t);
    double e = fma(-t, r, 1.0);
    r = fma(r, e, r);
    e = fma(-t, r, 1.0);
    return fma(r, e, r);
}

// root of a*y^2 + b*y + c = 0 strictly inside (lo, hi), else the bracket middle
__device__ double quad_in(double a, double b, double c, double lo, double hi)
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

// ---------------------------------------------------------------------------
// Secular roots.
// ---------------------------------------------------------------------------
struct Acc { double psi, phi, dpsi, dphi; };

// Accumulate the triangular parts over poles [j0, j1) of a staged chunk whose
// first pole has global index jg0.  Pole j goes to psi if j <= k, else to phi.
// The warp's roots are consecutive (kwlo..kwhi), so the loop runs in three
// warp-uniform regions; only the middle one selects per lane.
__device__ __forceinline__ int fexp(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

// Every term uses the shifted difference (d_j - d_K) - y of eq. (4.14).  (The
// local-shifting variant that takes d_j - x for far poles, eqs. (4.19)-(4.21),
// saves one FP64 subtraction per term but measured slower on GB300: the
// integer exponent test and branch cost more than the subtraction.)
__device__ __forceinline__ double shifted_t(double dj, double dK, double y)
{
    return (dj - dK) - y;
}

template <bool DERIV>
__device__ __forceinline__ void sweep(const double *__restrict__ sd, const double *__restrict__ sw,
                                      int j0, int j1, int jg0, int k, int kwlo, int kwhi,
                                      double dK, double y, Acc &A)
{
    // region A: global j <= kwlo -> psi for every lane
    int ea = min(j1, max(j0, kwlo - jg0 + 1));
#pragma unroll 4
    for (int j = j0; j < ea; j++) {
        double t = shifted_t(sd[j], dK, y);
        double r = rcp_nr1(t);
        if (DERIV) {
            double a = sw[j] * r;
            A.psi += a;
            A.dpsi = fma(a, r, A.dpsi);
        } else {
            A.psi = fma(sw[j], r, A.psi);
        }
    }
    // region B: kwlo < j <= kwhi -> per lane
    int eb = min(j1, max(ea, kwhi - jg0 + 1));
    for (int j = ea; j < eb; j++) {
        double t = shifted_t(sd[j], dK, y);
        double r = rcp_nr1(t);
        double a = sw[j] * r;
        if (jg0 + j <= k) { A.psi += a; if (DERIV) A.dpsi = fma(a, r, A.dpsi); }
        else              { A.phi += a; if (DERIV) A.dphi = fma(a, r, A.dphi); }
    }
    // region C: j > kwhi -> phi for every lane
#pragma unroll 4
    for (int j = eb; j < j1; j++) {
        double t = shifted_t(sd[j], dK, y);
        double r = rcp_nr1(t);
        if (DERIV) {
            double a = sw[j] * r;
            A.phi += a;
            A.dphi = fma(a, r, A.dphi);
        } else {
            A.phi = fma(sw[j], r, A.phi);
        }
    }
}

struct Root {
    int k, m, K, phase, nsw;
    bool last, plain;
    double dK, y, lo, hi;
    double d0, d1, w0, w1, W;   // d_k, d_{k+1}, w_k, w_{k+1}, sum w

    // plain (ablation of the local shifting): the origin is 0 instead of a
    // pole, so y is the root's position itself and every difference
    // (d_j - dK) - y is d_j - lambda formed from rounded values
    __device__ void init(const double *__restrict__ dk, const double *__restrict__ zk, int k_, int m_, double W_,
                         bool plain_ = false)
    {
        k = k_; m = m_; W = W_; plain = plain_;
        last = (k == m - 1);
        d0 = dk[k];
        double z0 = zk[k];
        w0 = z0 * z0;
        if (!last) { d1 = dk[k + 1]; double z1 = zk[k + 1]; w1 = z1 * z1; }
        else       { d1 = d0; w1 = 0.0; }
        phase = 0; nsw = 0;
        K = k; dK = plain ? 0.0 : d0;
        y = last ? 0.5 * W : 0.5 * (d1 - d0);     // midpoint sweep
        if (plain) y += d0;
        lo = hi = 0.0;
    }

    // returns true when the root is final
    __device__ bool update(const Acc &A, double tol, int max_iter, int32_t *status)
    {
        nsw++;
        double f = 1.0 + A.psi + A.phi;
        if (!isfinite(f)) { sdc_latch(status, SUPERDC_DEV_NONFINITE); return true; }
        if (phase == 0) {
            // origin choice (Section 4.2.1) and initial guess: freeze the
            // non-adjacent terms at the midpoint, solve the two-pole model
            if (!last) {
                double D = d1 - d0, h = 0.5 * D;
                double rest = f + w0 / h - w1 / (D - h);
                if (f >= 0.0) { K = k;     lo = 0.0; hi = h;   dK = d0; }
                else          { K = k + 1; lo = -h;  hi = 0.0; dK = d1; }
                if (plain) { lo += dK; hi += dK; dK = 0.0; }
                double a = d0 - dK, b = d1 - dK;     // one of them is 0 unless plain
                y = quad_in(rest, -(rest * (a + b) + w0 + w1), w0 * b + w1 * a + rest * a * b, lo, hi);
            } else {
                double ym = 0.5 * W;
                if (f >= 0.0) { lo = 0.0; hi = ym; } else { lo = ym; hi = W; }
                double rest = f + w0 / ym;
                y = (rest > 0.0) ? w0 / rest : 0.5 * (lo + hi);
                if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
                if (plain) { y += d0; lo += d0; hi += d0; }
            }
            phase = 1;
            return false;
        }
        if (fabs(f) < tol * (1.0 + fabs(A.psi) + fabs(A.phi))) return true;   // eq. (4.12)
        if (f < 0.0) lo = y; else hi = y;
        double ynew;
        if (!last) {
            // middle-way step: psi ~ a1 + b1/(d_k - x), phi ~ a2 + b2/(d_{k+1} - x)
            double Dk = (d0 - dK) - y, Dk1 = (d1 - dK) - y;
            double c = f - Dk * A.dpsi - Dk1 * A.dphi;
            double Aq = (Dk + Dk1) * f - Dk * Dk1 * (A.dpsi + A.dphi);
            double Bq = Dk * Dk1 * f;
            double corr;
            if (c == 0.0) {
                corr = (Aq != 0.0) ? Bq / Aq : 0.0;
            } else {
                double disc = Aq * Aq - 4.0 * Bq * c;
                if (disc < 0.0) disc = 0.0;
                double s = sqrt(disc);
                double den = Aq + (Aq >= 0 ? s : -s);
                corr = (den != 0.0) ? 2.0 * Bq / den : 0.0;
            }
            ynew = y + corr;
        } else {
            double Dl = (d0 - dK) - y;
            double den = f - Dl * A.dpsi;
            double corr = (den != 0.0) ? Dl + Dl * Dl * A.dpsi / den : 0.0;
            ynew = y + corr;
        }
        if (!(ynew > lo && ynew < hi)) ynew = lo + 0.5 * (hi - lo);
        if (ynew == y || !(ynew > lo && ynew < hi)) return true;   // bracket at double resolution
        y = ynew;
        if (nsw - 1 >= max_iter) { sdc_latch(status, SUPERDC_DEV_NOCONV); return true; }
        return false;
    }
};

}  // namespace
