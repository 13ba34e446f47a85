// Batched rank-one update step of the SuperDC conquering stage on sm_103a.
//
// For every problem p of a batch (independent problems, or all nodes of one
// HSS tree level), with poles d ascending and update vector z:
//   k_deflate   -- Remark 4.1: |z_k| < tau, then the sequential Givens scan
//                  over the survivors (one thread per problem: each test
//                  depends on the z produced by the previous rotation);
//                  compaction into kept / deflated slots.
//   k_tiles     -- prefix of root tiles per problem (device-side, so a level
//                  can be launched without a host round trip).
//   k_secular   -- Algorithm 2 with the shifted secular equation eq. (4.13):
//                  every root iterates on its gap eta = lambda - d_K (eq. (4.17))
//                  with shifted differences (d_j - d_K) - y (eq. (4.14)); the
//                  sums are split at the root's index into the lower part psi
//                  (j <= k) and the upper part phi (j > k), eqs. (4.7)-(4.10);
//                  middle-way rational step, stopping test eq. (4.12).  Direct
//                  tiled evaluator: poles and weights staged in shared memory,
//                  one root per thread.
//   k_lowner    -- eq. (4.23) (paired ratios, shifted differences).
//   k_bnorm     -- eq. (4.27) with the shifted entries of eq. (4.28).
//   k_merge     -- new eigenvalues (eq. (4.21)) and deflated values sorted by
//                  (value, input index).
// Everything is FP64: the root iteration, the shifted differences and zhat
// need it for stability.
#include "common.cuh"
#include "rank1.cuh"
#include "prof.cuh"

namespace {

constexpr int SEC_CHUNK = 2048;   // poles staged per shared-memory chunk

__device__ __forceinline__ double rcp(double t) { return 1.0 / t; }

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
// Deflation (Remark 4.1), one thread per problem.
// ---------------------------------------------------------------------------
__global__ void k_deflate(int64_t nprob, const int64_t *__restrict__ off,
                          const double *__restrict__ d, const double *__restrict__ z,
                          double sqrt_rho, double tau,
                          double *__restrict__ wd, double *__restrict__ wz, int8_t *__restrict__ kept,
                          R1Out o)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    const int64_t b0 = off[p];
    const int m = (int)(off[p + 1] - b0);
    bool bad = false;
    for (int i = 0; i < m; i++) {
        double di = d[b0 + i], zi = z[b0 + i] * sqrt_rho;
        if (!isfinite(di) || !isfinite(zi)) bad = true;
        wd[b0 + i] = di;
        bool keep = !(fabs(zi) < tau);
        wz[b0 + i] = keep ? zi : 0.0;
        kept[b0 + i] = keep ? 1 : 0;
    }
    if (bad) sdc_latch(o.status, SUPERDC_DEV_NONFINITE);
    // Givens scan over the survivors (left to right, candidate a)
    int ng = 0;
    int a = -1;
    for (int bb = 0; bb < m; bb++) {
        if (!kept[b0 + bb]) continue;
        if (a >= 0) {
            // the test and the rotation use explicitly rounded operations (no
            // fused multiply-add), so decisions and rotated values are
            // reproducible bit for bit by any IEEE evaluation in this order
            double za = wz[b0 + a], zb = wz[b0 + bb];
            double da = wd[b0 + a], db = wd[b0 + bb];
            double lhs = fabs(__dmul_rn(__dmul_rn(__dsub_rn(da, db), za), zb));
            double nrm2 = __dadd_rn(__dmul_rn(za, za), __dmul_rn(zb, zb));
            double rhs = __dmul_rn(nrm2, tau);
            if (lhs < rhs) {
                double r = __dsqrt_rn(nrm2);
                double c = __ddiv_rn(zb, r), s = __ddiv_rn(za, r);
                double cc = __dmul_rn(c, c), ss = __dmul_rn(s, s);
                wd[b0 + a] = __dadd_rn(__dmul_rn(cc, da), __dmul_rn(ss, db));
                wd[b0 + bb] = __dadd_rn(__dmul_rn(ss, da), __dmul_rn(cc, db));
                wz[b0 + a] = 0.0;
                wz[b0 + bb] = r;
                kept[b0 + a] = 0;
                o.giv_ab[2 * (b0 + ng)] = a;
                o.giv_ab[2 * (b0 + ng) + 1] = bb;
                o.giv_cs[2 * (b0 + ng)] = c;
                o.giv_cs[2 * (b0 + ng) + 1] = s;
                ng++;
            }
        }
        a = bb;
    }
    // compaction: kept slots first (ascending), then deflated sorted by (value, index)
    int mk = 0;
    double W = 0.0;
    for (int i = 0; i < m; i++) {
        if (!kept[b0 + i]) continue;
        double zi = wz[b0 + i];
        o.dk[b0 + mk] = wd[b0 + i];
        o.zk[b0 + mk] = zi;
        o.src[b0 + mk] = i;
        W = __dadd_rn(W, __dmul_rn(zi, zi));
        mk++;
    }
    int nd = 0;
    for (int i = 0; i < m; i++) {
        if (kept[b0 + i]) continue;
        double v = wd[b0 + i];
        int s = mk + nd;
        // insertion: shift larger keys right (src increases with i, so ties keep order)
        while (s > mk && o.dk[b0 + s - 1] > v) {
            o.dk[b0 + s] = o.dk[b0 + s - 1];
            o.src[b0 + s] = o.src[b0 + s - 1];
            s--;
        }
        o.dk[b0 + s] = v;
        o.src[b0 + s] = i;
        nd++;
    }
    for (int s = mk; s < m; s++) {
        o.zk[b0 + s] = 0.0;
        o.org[b0 + s] = -1;
        o.eta[b0 + s] = 0.0;
        o.dorg[b0 + s] = o.dk[b0 + s];
        o.vhat[b0 + s] = 0.0;
        o.bnorm[b0 + s] = 1.0;
        if (o.sweeps) o.sweeps[b0 + s] = 0;
    }
    o.mk[p] = mk;
    o.ngiv[p] = ng;
    o.wsum[p] = W;
}

// ---------------------------------------------------------------------------
// Prefix of root tiles per problem (single CTA).
// ---------------------------------------------------------------------------
__global__ void k_tiles(int64_t nprob, const int32_t *__restrict__ mk, int tr, int64_t *__restrict__ tile_off)
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

// ---------------------------------------------------------------------------
// Secular roots.
// ---------------------------------------------------------------------------
struct Acc { double psi, phi, dpsi, dphi; };

// Accumulate the triangular parts over poles [j0, j1) of a staged chunk whose
// first pole has global index jg0.  Pole j goes to psi if j <= k, else to phi.
// The warp's roots are consecutive (kwlo..kwhi), so the loop runs in three
// warp-uniform regions; only the middle one selects per lane.
__device__ __forceinline__ void sweep(const double *__restrict__ sd, const double *__restrict__ sw,
                                      int j0, int j1, int jg0, int k, int kwlo, int kwhi,
                                      double dK, double y, Acc &A)
{
    // region A: global j <= kwlo -> psi for every lane
    int ea = min(j1, max(j0, kwlo - jg0 + 1));
    for (int j = j0; j < ea; j++) {
        double t = (sd[j] - dK) - y;
        double r = rcp(t);
        double a = sw[j] * r;
        A.psi += a;
        A.dpsi = fma(a, r, A.dpsi);
    }
    // region B: kwlo < j <= kwhi -> per lane
    int eb = min(j1, max(ea, kwhi - jg0 + 1));
    for (int j = ea; j < eb; j++) {
        double t = (sd[j] - dK) - y;
        double r = rcp(t);
        double a = sw[j] * r;
        if (jg0 + j <= k) { A.psi += a; A.dpsi = fma(a, r, A.dpsi); }
        else              { A.phi += a; A.dphi = fma(a, r, A.dphi); }
    }
    // region C: j > kwhi -> phi for every lane
    for (int j = eb; j < j1; j++) {
        double t = (sd[j] - dK) - y;
        double r = rcp(t);
        double a = sw[j] * r;
        A.phi += a;
        A.dphi = fma(a, r, A.dphi);
    }
}

struct Root {
    int k, m, K, phase, nsw;
    bool last;
    double dK, y, lo, hi;
    double d0, d1, w0, w1, W;   // d_k, d_{k+1}, w_k, w_{k+1}, sum w

    __device__ void init(const double *__restrict__ dk, const double *__restrict__ zk, int k_, int m_, double W_)
    {
        k = k_; m = m_; W = W_;
        last = (k == m - 1);
        d0 = dk[k];
        double z0 = zk[k];
        w0 = z0 * z0;
        if (!last) { d1 = dk[k + 1]; double z1 = zk[k + 1]; w1 = z1 * z1; }
        else       { d1 = d0; w1 = 0.0; }
        phase = 0; nsw = 0;
        K = k; dK = d0;
        y = last ? 0.5 * W : 0.5 * (d1 - d0);     // midpoint sweep
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
                double a = d0 - dK, b = d1 - dK;
                y = quad_in(rest, -(rest * (a + b) + w0 + w1), w0 * b + w1 * a, lo, hi);
            } else {
                double ym = 0.5 * W;
                if (f >= 0.0) { lo = 0.0; hi = ym; } else { lo = ym; hi = W; }
                double rest = f + w0 / ym;
                y = (rest > 0.0) ? w0 / rest : 0.5 * (lo + hi);
                if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
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

template <int TR>
__global__ void __launch_bounds__(TR)
k_secular(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off,
          R1Out o, double stop_c, int max_iter)
{
    __shared__ double sd[SEC_CHUNK];
    __shared__ double sw[SEC_CHUNK];
    const int64_t ntiles = tile_off[nprob];
    const int lane = threadIdx.x & 31;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const double *dk = o.dk + b0, *zk = o.zk + b0;
        const int k = (int)(tile - tile_off[p]) * TR + threadIdx.x;
        const bool active = k < m;
        const int kc = min(k, m - 1);
        const int kwlo = __shfl_sync(0xffffffffu, kc, 0);
        const int kwhi = __shfl_sync(0xffffffffu, kc, 31);
        (void)lane;
        const double tol = stop_c * (double)m * SDC_EPS;
        Root R;
        bool done = true;
        if (active) { R.init(dk, zk, k, m, o.wsum[p]); done = false; }
        __syncthreads();   // previous tile finished with the shared arrays
        if (m <= SEC_CHUNK) {
            for (int j = threadIdx.x; j < m; j += TR) {
                sd[j] = dk[j];
                double zj = zk[j];
                sw[j] = zj * zj;
            }
            __syncthreads();
            // every root iterates on its own: no block-wide barrier inside
            while (!done) {
                Acc A = {0.0, 0.0, 0.0, 0.0};
                sweep(sd, sw, 0, m, 0, kc, kwlo, kwhi, R.dK, R.y, A);
                done = R.update(A, tol, max_iter, o.status);
            }
        } else {
            // lock-step sweeps, poles streamed through shared memory in chunks
            while (__syncthreads_or(!done)) {
                Acc A = {0.0, 0.0, 0.0, 0.0};
                for (int c0 = 0; c0 < m; c0 += SEC_CHUNK) {
                    const int cn = min(SEC_CHUNK, m - c0);
                    __syncthreads();
                    for (int j = threadIdx.x; j < cn; j += TR) {
                        sd[j] = dk[c0 + j];
                        double zj = zk[c0 + j];
                        sw[j] = zj * zj;
                    }
                    __syncthreads();
                    if (!done) sweep(sd, sw, 0, cn, c0, kc, kwlo, kwhi, R.dK, R.y, A);
                }
                if (!done) done = R.update(A, tol, max_iter, o.status);
            }
        }
        if (active) {
            o.org[b0 + k] = R.K;
            o.eta[b0 + k] = R.y;
            o.dorg[b0 + k] = R.dK;
            if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
        }
    }
}

// ---------------------------------------------------------------------------
// Loewner zhat, eq. (4.23):
//   vhat_i^2 = (lambda_{m-1} - d_i) prod_{j<i} (lambda_j - d_i)/(d_j - d_i)
//                                   prod_{i<=j<m-1} (lambda_j - d_i)/(d_{j+1} - d_i)
// with lambda_j - d_i = (d_{K_j} - d_i) + eta_j.
// ---------------------------------------------------------------------------
template <int TR>
__global__ void __launch_bounds__(TR)
k_lowner(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off, R1Out o)
{
    const int64_t ntiles = tile_off[nprob];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int i = (int)(tile - tile_off[p]) * TR + threadIdx.x;
        if (i >= m) continue;
        const double *dk = o.dk + b0, *dorg = o.dorg + b0, *eta = o.eta + b0;
        const double di = dk[i];
        double prod = (dorg[m - 1] - di) + eta[m - 1];
        for (int j = 0; j < m - 1; j++) {
            double num = (dorg[j] - di) + eta[j];
            double den = ((j < i) ? dk[j] : dk[j + 1]) - di;
            prod *= num / den;
        }
        double v = sqrt(prod);
        if (!isfinite(v)) sdc_latch(o.status, SUPERDC_DEV_NONFINITE);
        o.vhat[b0 + i] = (o.zk[b0 + i] < 0.0) ? -v : v;
    }
}

// ---------------------------------------------------------------------------
// b_j = (sum_i vhat_i^2 / ((d_i - d_{K_j}) - eta_j)^2)^(-1/2), eq. (4.27)
// ---------------------------------------------------------------------------
template <int TR>
__global__ void __launch_bounds__(TR)
k_bnorm(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off, R1Out o)
{
    const int64_t ntiles = tile_off[nprob];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int j = (int)(tile - tile_off[p]) * TR + threadIdx.x;
        if (j >= m) continue;
        const double *dk = o.dk + b0, *v = o.vhat + b0;
        const double dK = o.dorg[b0 + j], e = o.eta[b0 + j];
        double s = 0.0;
        for (int i = 0; i < m; i++) {
            double t = (dk[i] - dK) - e;
            double r = rcp(t);
            double vr = v[i] * r;
            s = fma(vr, vr, s);
        }
        o.bnorm[b0 + j] = 1.0 / sqrt(s);
    }
}

// ---------------------------------------------------------------------------
// Merge: new eigenvalue list per problem, ascending by (value, input index).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool key_less(double v1, int s1, double v2, int s2)
{
    return v1 < v2 || (v1 == v2 && s1 < s2);
}

__global__ void k_merge(int64_t nprob, const int64_t *__restrict__ off, int64_t total, R1Out o)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = sdc_upper_index(off, nprob, x);
        const int64_t b0 = off[p];
        const int m = (int)(off[p + 1] - b0);
        const int mk = o.mk[p];
        const int s = (int)(x - b0);
        const double *dk = o.dk + b0, *dorg = o.dorg + b0, *eta = o.eta + b0;
        const int32_t *src = o.src + b0;
        int pos;
        double val;
        if (s < mk) {
            val = dorg[s] + eta[s];                      // eq. (4.21)
            // deflated slots with a smaller key
            int lo = mk, hi = m;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (key_less(dk[mid], src[mid], val, src[s])) lo = mid + 1; else hi = mid;
            }
            pos = s + (lo - mk);
        } else {
            val = dk[s];
            int lo = 0, hi = mk;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                double lm = dorg[mid] + eta[mid];
                if (key_less(lm, src[mid], val, src[s])) lo = mid + 1; else hi = mid;
            }
            pos = (s - mk) + lo;
        }
        o.lam[b0 + pos] = val;
        o.perm[b0 + pos] = s;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------
superdc_status r1_run(const R1Args &a, cudaStream_t st)
{
    const int nsm = sdc_num_sms();
    double *wd = nullptr, *wz = nullptr;
    int8_t *kept = nullptr;
    int64_t *tile_off = nullptr;
    SDC_CHECK(sdc_alloc(&wd, a.total, st));
    SDC_CHECK(sdc_alloc(&wz, a.total, st));
    SDC_CHECK(sdc_alloc(&kept, a.total, st));
    SDC_CHECK(sdc_alloc(&tile_off, a.nprob + 1, st));

    const int tpb = 128;
    PROF_LAUNCH("deflate", st, k_deflate<<<(unsigned)((a.nprob + tpb - 1) / tpb), tpb, 0, st>>>(
        a.nprob, a.off, a.d, a.z, a.sqrt_rho, a.tau, wd, wz, kept, a.o));
    const int TR = 128;
    PROF_LAUNCH("tiles", st, k_tiles<<<1, 1024, 0, st>>>(a.nprob, a.o.mk, TR, tile_off));
    const unsigned grid = (unsigned)(nsm * 8);
    PROF_LAUNCH("secular", st, k_secular<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o, a.stop_c, a.max_iter));
    PROF_LAUNCH("lowner", st, k_lowner<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o));
    PROF_LAUNCH("bnorm", st, k_bnorm<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o));
    PROF_LAUNCH("merge", st, k_merge<<<(unsigned)(nsm * 8), 256, 0, st>>>(a.nprob, a.off, a.total, a.o));
    SDC_CHECK(cudaGetLastError());

    SDC_CHECK(cudaFreeAsync(wd, st));
    SDC_CHECK(cudaFreeAsync(wz, st));
    SDC_CHECK(cudaFreeAsync(kept, st));
    SDC_CHECK(cudaFreeAsync(tile_off, st));
    return SUPERDC_OK;
}
