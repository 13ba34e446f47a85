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
#include "secular.cuh"
#include "fmm.cuh"
#include <algorithm>
#include <mutex>

namespace {

constexpr int SEC_CHUNK = 2048;   // poles staged per shared-memory chunk
constexpr int DEFL_BIG = 128;     // problems larger than this deflate with a whole CTA


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
    if (m > DEFL_BIG) return;            // handled by k_deflate_big
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
// Deflation of large problems, one CTA (DB_T threads) per problem: the
// |z| < tau mask, the adjacent Givens tests and the compactions run in
// parallel; only chains of consecutive rotations are walked sequentially.
// The arithmetic is the same explicitly rounded sequence as k_deflate, so
// decisions and rotated values agree bit for bit.
// ---------------------------------------------------------------------------
constexpr int DB_T = 512;         // threads per problem; 1024 when a batch has fewer problems than SMs
constexpr int WALK_CAP = 64;      // speculative steps of one chain before one thread finishes it

// exclusive block scan of one int per thread; returns the prefix, *total = sum
template <int T>
__device__ __forceinline__ int block_exscan(int v, int *sh, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < T / 32) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    const int before = (warp > 0) ? sh[warp - 1] : 0;
    *total = sh[T / 32 - 1];
    __syncthreads();
    return before + x - v;
}

template <int T>
__global__ void __launch_bounds__(T)
k_deflate_big(int64_t nprob, const int64_t *__restrict__ off, const double *__restrict__ d,
              const double *__restrict__ z, double sqrt_rho, double tau, double *__restrict__ wd,
              double *__restrict__ wz, int8_t *__restrict__ kept, int32_t *__restrict__ surv, R1Out o)
{
    __shared__ int sh[32];
    __shared__ int s_bad, s_ng;
    __shared__ double s_w[T / 32];
    const int64_t p = blockIdx.x;
    if (p >= nprob) return;
    const int64_t b0 = off[p];
    const int m = (int)(off[p + 1] - b0);
    if (m <= DEFL_BIG) return;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // A: copy, mask, survivor list
    int S = 0;
    for (int c = 0; c < m; c += T) {
        const int i = c + tid;
        int keep = 0;
        if (i < m) {
            double di = d[b0 + i], zi = z[b0 + i] * sqrt_rho;
            if (!isfinite(di) || !isfinite(zi)) s_bad = 1;
            keep = !(fabs(zi) < tau);
            wd[b0 + i] = di;
            wz[b0 + i] = keep ? zi : 0.0;
            kept[b0 + i] = (int8_t)keep;
        }
        int tot;
        int pre = block_exscan<T>(keep, sh, &tot);
        if (keep) surv[b0 + S + pre] = i;
        S += tot;
    }
    __syncthreads();
    if (tid == 0 && s_bad) sdc_latch(o.status, SUPERDC_DEV_NONFINITE);
    // B: Givens scan over the survivors.  The candidate of every test is the
    // previous survivor, so a test can differ from its value on the original
    // data only right after a rotation.  B1 evaluates every adjacent test on
    // the original values in parallel and marks the survivors whose test
    // passes (kept = 2, "chain heads").  B2 takes the positions in rounds of
    // T: every head of the round walks its chain in its own thread on the
    // original values (rotate, re-test the next pair with the rotated values,
    // until a test fails; at most WALK_CAP steps); one thread then decides in
    // order which heads start a chain of the sequential scan (a head inside or
    // at the end of the previous chain does not) and gives each chain its
    // offset in the rotation list; finally the chains write their rotations in
    // parallel (chains are disjoint; a chain longer than WALK_CAP is finished
    // and written by that one thread).  Each chain evaluates the same
    // explicitly rounded operations in the same order as the plain sequential
    // scan (k_deflate), so decisions and rotated values agree bit for bit.
    for (int t = 1 + tid; t < S; t += T) {
        const int ia = surv[b0 + t - 1], ib = surv[b0 + t];
        const double da = wd[b0 + ia], za = wz[b0 + ia], db = wd[b0 + ib], zb = wz[b0 + ib];
        const double lhs = fabs(__dmul_rn(__dmul_rn(__dsub_rn(da, db), za), zb));
        const double rhs = __dmul_rn(__dadd_rn(__dmul_rn(za, za), __dmul_rn(zb, zb)), tau);
        if (lhs < rhs) kept[b0 + ib] = 2;
    }
    __syncthreads();
    {
        __shared__ int h_pos[T], h_end[T], h_off[T];
        __shared__ int s_nh, s_eprev;
        // one chain from position h (candidate s_{h-1}); write = false: count
        // only.  Returns the first position whose test fails (or S), or -1 when
        // max_steps rotations were taken without reaching it.  nrot >= 0: take
        // exactly nrot rotations without testing (the chain's length is known;
        // its last, failing test would read the first entry of the next chain,
        // which that chain may be rotating at the same time).
        auto walk = [&](int h, int max_steps, bool write, int ng0, int nrot) -> int {
            int ia = surv[b0 + h - 1];
            double da = wd[b0 + ia], za = wz[b0 + ia];
            int t2 = h, k = 0;
            while (t2 < S) {
                if (nrot >= 0 && k == nrot) break;
                if (k == max_steps) return -1;
                const int ib = surv[b0 + t2];
                const double db = wd[b0 + ib], zb = wz[b0 + ib];
                const double nrm2 = __dadd_rn(__dmul_rn(za, za), __dmul_rn(zb, zb));
                if (nrot < 0) {
                    const double lhs = fabs(__dmul_rn(__dmul_rn(__dsub_rn(da, db), za), zb));
                    const double rhs = __dmul_rn(nrm2, tau);
                    if (!(lhs < rhs)) break;
                }
                const double r = __dsqrt_rn(nrm2);
                const double cc0 = __ddiv_rn(zb, r), ss0 = __ddiv_rn(za, r);
                const double cc = __dmul_rn(cc0, cc0), ss = __dmul_rn(ss0, ss0);
                const double na = __dadd_rn(__dmul_rn(cc, da), __dmul_rn(ss, db));
                const double nb = __dadd_rn(__dmul_rn(ss, da), __dmul_rn(cc, db));
                if (write) {
                    wd[b0 + ia] = na;
                    wz[b0 + ia] = 0.0;
                    kept[b0 + ia] = 0;
                    wd[b0 + ib] = nb;
                    wz[b0 + ib] = r;
                    o.giv_ab[2 * (b0 + ng0 + k)] = ia;
                    o.giv_ab[2 * (b0 + ng0 + k) + 1] = ib;
                    o.giv_cs[2 * (b0 + ng0 + k)] = cc0;
                    o.giv_cs[2 * (b0 + ng0 + k) + 1] = ss0;
                }
                ia = ib; da = nb; za = r;
                t2++;
                k++;
            }
            return t2;
        };
        if (tid == 0) { s_eprev = 0; s_ng = 0; }
        for (int c = 1; c < S; c += T) {
            const int t = c + tid;
            const int hf = (t < S && kept[b0 + surv[b0 + t]] == 2) ? 1 : 0;
            int nh;
            const int pre = block_exscan<T>(hf, sh, &nh);
            if (hf) h_pos[pre] = t;
            __syncthreads();
            if (nh == 0) continue;
            // speculative walks; a head at or before the previous chain's end is
            // not a chain start, and such a head may read rotated values, so its
            // result is only used once that has been ruled out
            if (tid < nh) {
                const int h = h_pos[tid];
                h_end[tid] = (h <= s_eprev) ? 0 : walk(h, WALK_CAP, false, 0, -1);
            }
            __syncthreads();
            if (tid == 0) {
                int e_prev = s_eprev, ng = s_ng;
                for (int i = 0; i < nh; i++) {
                    const int h = h_pos[i];
                    if (h <= e_prev) { h_off[i] = -1; continue; }
                    int e = h_end[i];
                    if (e < 0) {                         // long chain: finished and written here
                        e = walk(h, S, true, ng, -1);
                        h_off[i] = -1;
                    } else {
                        h_off[i] = ng;
                    }
                    ng += e - h;
                    e_prev = e;
                }
                s_eprev = e_prev;
                s_ng = ng;
            }
            __syncthreads();
            if (tid < nh && h_off[tid] >= 0) walk(h_pos[tid], S, true, h_off[tid], h_end[tid] - h_pos[tid]);
            __syncthreads();
        }
    }
    __syncthreads();
    // C: compaction, kept slots in index order, then deflated slots in index order
    int mk = 0;
    double wpart = 0.0;
    for (int c = 0; c < m; c += T) {
        const int i = c + tid;
        const int k = (i < m) ? (int)(kept[b0 + i] != 0) : 0;
        int tot;
        int pre = block_exscan<T>(k, sh, &tot);
        if (k) {
            double zi = wz[b0 + i];
            o.dk[b0 + mk + pre] = wd[b0 + i];
            o.zk[b0 + mk + pre] = zi;
            o.src[b0 + mk + pre] = i;
            wpart = __dadd_rn(wpart, __dmul_rn(zi, zi));
        }
        mk += tot;
    }
    int nd = 0;
    for (int c = 0; c < m; c += T) {
        const int i = c + tid;
        const int dflt = (i < m) ? (int)(kept[b0 + i] == 0) : 0;
        int tot;
        int pre = block_exscan<T>(dflt, sh, &tot);
        if (dflt) {
            o.dk[b0 + mk + nd + pre] = wd[b0 + i];
            o.src[b0 + mk + nd + pre] = i;
        }
        nd += tot;
    }
    // deterministic sum of kept z^2
    for (int of = 16; of > 0; of >>= 1) wpart += __shfl_xor_sync(0xffffffffu, wpart, of);
    if ((tid & 31) == 0) s_w[tid >> 5] = wpart;
    __syncthreads();
    // D: deflated values sorted by (value, index): they are in index order and
    // out of order only inside tau-sized intervals, so insertion is short
    if (tid == 0) {
        double W = 0.0;
        for (int w = 0; w < T / 32; w++) W += s_w[w];
        o.wsum[p] = W;
        o.mk[p] = mk;
        o.ngiv[p] = s_ng;
        for (int q = mk + 1; q < m; q++) {
            double v = o.dk[b0 + q];
            int sv = o.src[b0 + q];
            int s2 = q;
            while (s2 > mk && o.dk[b0 + s2 - 1] > v) {
                o.dk[b0 + s2] = o.dk[b0 + s2 - 1];
                o.src[b0 + s2] = o.src[b0 + s2 - 1];
                s2--;
            }
            o.dk[b0 + s2] = v;
            o.src[b0 + s2] = sv;
        }
    }
    __syncthreads();
    for (int s2 = mk + tid; s2 < m; s2 += T) {
        o.zk[b0 + s2] = 0.0;
        o.org[b0 + s2] = -1;
        o.eta[b0 + s2] = 0.0;
        o.dorg[b0 + s2] = o.dk[b0 + s2];
        o.vhat[b0 + s2] = 0.0;
        o.bnorm[b0 + s2] = 1.0;
        if (o.sweeps) o.sweeps[b0 + s2] = 0;
    }
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


// Work units of the secular kernel: (problem, first root, end root), at most
// ubig roots each.  A unit stages its problem's poles in shared memory (all of
// them when they fit in SEC_CHUNK, else in chunks per sweep).  Units are
// ordered by decreasing problem size (largest first) so the long units start
// early, and capping the roots per unit spreads a large problem over several
// SMs, which keeps the tail of the launch short.
constexpr int SEC_UNIT_BIG = 2048;
constexpr int SORT_MAX = 8192;

__global__ void k_units(int64_t nprob, const int32_t *__restrict__ mk, const int32_t *__restrict__ fslot, int ubig,
                        int whole_small, int4 *__restrict__ units, int *__restrict__ nunits,
                        int *__restrict__ counter)
{
    extern __shared__ unsigned long long keys[];   // SORT_MAX entries when sorting
    __shared__ int part[1024];
    const int T = blockDim.x;
    const bool sorted = nprob <= SORT_MAX;
    int64_t n2 = 1;
    if (sorted) {
        while (n2 < nprob) n2 <<= 1;
        for (int64_t i = threadIdx.x; i < n2; i += T) {
            // descending by size: key = (size << 32) | (~p) so that equal sizes keep index order
            const int mi = (i < nprob && !(fslot && fslot[i] >= 0)) ? mk[i] : 0;
            keys[i] = (i < nprob) ? (((unsigned long long)(unsigned)mi << 32) |
                                     (unsigned long long)(0xFFFFFFFFu - (unsigned)i))
                                  : 0ull;
        }
        __syncthreads();
        for (int64_t kk = 2; kk <= n2; kk <<= 1) {
            for (int64_t j = kk >> 1; j > 0; j >>= 1) {
                for (int64_t i = threadIdx.x; i < n2; i += T) {
                    int64_t ixj = i ^ j;
                    if (ixj > i) {
                        bool desc = ((i & kk) == 0);
                        unsigned long long a = keys[i], b = keys[ixj];
                        if (desc ? (a < b) : (a > b)) { keys[i] = b; keys[ixj] = a; }
                    }
                }
                __syncthreads();
            }
        }
    }
    // units per problem (in the chosen order), block-wide prefix
    int64_t per = (nprob + T - 1) / T;
    int64_t beg = threadIdx.x * per, end = min(nprob, beg + per);
    int cnt = 0;
    for (int64_t q = beg; q < end; q++) {
        int64_t pp = sorted ? (int64_t)(0xFFFFFFFFu - (unsigned)(keys[q] & 0xFFFFFFFFull)) : q;
        int m = (fslot && fslot[pp] >= 0) ? 0 : mk[pp];   // FMM problems: not here
        cnt += (m + ubig - 1) / ubig;
    }
    part[threadIdx.x] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < T; i++) { int v = part[i]; part[i] = acc; acc += v; }
        *nunits = acc;
        *counter = 0;
    }
    __syncthreads();
    int u = part[threadIdx.x];
    for (int64_t q = beg; q < end; q++) {
        int64_t pp = sorted ? (int64_t)(0xFFFFFFFFu - (unsigned)(keys[q] & 0xFFFFFFFFull)) : q;
        int m = (fslot && fslot[pp] >= 0) ? 0 : mk[pp];
        if (m <= 0) continue;
        for (int r = 0; r < m; r += ubig) units[u++] = make_int4((int)pp, r, min(m, r + ubig), 0);
    }
}

// One CTA of NW warps per unit, persistent over an atomic unit queue.
//
// SPLIT = false (many roots per launch, e.g. thousands of independent
// problems): each warp owns a contiguous 1/NW of the unit's roots; a lane
// whose root has converged takes the next root of the warp's range, so the
// FP64 pipe keeps working on live roots instead of waiting for the slowest
// root of a fixed group of 32.
// SPLIT = true (few large problems, e.g. the top levels of the tree): the NW
// warps share one 32-lane root range and split the poles NW ways; the partial
// sums are reduced through shared memory after every sweep and each warp
// applies the same update, so the replicated root state stays identical.
// Both keep the live roots of a warp inside a short window, so the psi/phi
// split keeps its three warp-uniform regions.
template <int NW, bool SPLIT>
__global__ void __launch_bounds__(NW * 32)
k_secular(const int64_t *__restrict__ off, const int4 *__restrict__ units,
          const int *__restrict__ nunits, int *__restrict__ counter,
          R1Out o, double stop_c, int max_iter)
{
    __shared__ double sd[SEC_CHUNK];
    __shared__ double sw[SEC_CHUNK];
    __shared__ double red[SPLIT ? NW : 1][4][32];
    __shared__ double s_dK[SPLIT ? 32 : 1], s_y[SPLIT ? 32 : 1];
    __shared__ int s_ph[SPLIT ? 32 : 1], s_fin[SPLIT ? 32 : 1];
    __shared__ int s_unit;
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nu = *nunits;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= nu) break;
        const int4 U = units[u];
        const int64_t p = U.x;
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const double *dk = o.dk + b0, *zk = o.zk + b0;
        const double W = o.wsum[p];
        const double tol = stop_c * (double)m * SDC_EPS;
        const int len = U.z - U.y;
        const int wbeg = SPLIT ? U.y : U.y + (int)(((int64_t)len * warp) / NW);
        const int wend = SPLIT ? U.z : U.y + (int)(((int64_t)len * (warp + 1)) / NW);
        int k = wbeg + lane;
        bool act = k < wend;
        int next = wbeg + 32;
        Root R;
        R.dK = 0.0; R.y = 1.0; R.phase = 1;     // defined values for lanes that stay idle
        if (act) R.init(dk, zk, k, m, W, o.unshifted != 0);
        const bool single = (m <= SEC_CHUNK);
        if (single) {
            for (int j = threadIdx.x; j < m; j += NW * 32) {
                sd[j] = dk[j];
                double zj = zk[j];
                sw[j] = zj * zj;
            }
        }
        __syncthreads();
        const bool lockstep = SPLIT || !single;
        while (lockstep ? __syncthreads_or(act) : __any_sync(FULL, act)) {
            const int kwlo = __reduce_min_sync(FULL, act ? k : 0x7fffffff);
            const int kwhi = __reduce_max_sync(FULL, act ? k : -1);
            const int kk = act ? k : kwlo;
            const bool p0 = __all_sync(FULL, !act || R.phase == 0);
            const bool any = __any_sync(FULL, act);
            Acc A = {0.0, 0.0, 0.0, 0.0};
            for (int c0 = 0; c0 < m; c0 += SEC_CHUNK) {
                const int cn = min(SEC_CHUNK, m - c0);
                if (!single) {
                    __syncthreads();
                    for (int j = threadIdx.x; j < cn; j += NW * 32) {
                        sd[j] = dk[c0 + j];
                        double zj = zk[c0 + j];
                        sw[j] = zj * zj;
                    }
                    __syncthreads();
                }
                const int j0 = SPLIT ? (int)(((int64_t)cn * warp) / NW) : 0;
                const int j1 = SPLIT ? (int)(((int64_t)cn * (warp + 1)) / NW) : cn;
                if (any) {
                    if (p0) sweep<false>(sd, sw, j0, j1, c0, kk, kwlo, kwhi, R.dK, R.y, A);
                    else    sweep<true>(sd, sw, j0, j1, c0, kk, kwlo, kwhi, R.dK, R.y, A);
                }
            }
            bool fin = false;
            if (SPLIT) {
                // the warps hold the same roots: warp 0 alone reduces the partial
                // sums (fixed order) and updates, the others take the new iterate
                // (an FP64 instruction costs its pipe slot in every warp that runs it)
                red[SPLIT ? warp : 0][0][lane] = A.psi;
                red[SPLIT ? warp : 0][1][lane] = A.phi;
                red[SPLIT ? warp : 0][2][lane] = A.dpsi;
                red[SPLIT ? warp : 0][3][lane] = A.dphi;
                __syncthreads();
                if (warp == 0) {
                    Acc T = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                    for (int w = 0; w < (SPLIT ? NW : 1); w++) {
                        T.psi += red[w][0][lane];
                        T.phi += red[w][1][lane];
                        T.dpsi += red[w][2][lane];
                        T.dphi += red[w][3][lane];
                    }
                    if (act) {
                        fin = R.update(T, tol, max_iter, o.status);
                        if (fin) {
                            o.org[b0 + k] = R.K;
                            o.eta[b0 + k] = R.y;
                            o.dorg[b0 + k] = R.dK;
                            o.lamk[b0 + k] = R.dK + R.y;
                            if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                        }
                    }
                    s_dK[SPLIT ? lane : 0] = R.dK;
                    s_y[SPLIT ? lane : 0] = R.y;
                    s_ph[SPLIT ? lane : 0] = R.phase;
                    s_fin[SPLIT ? lane : 0] = fin ? 1 : 0;
                }
                __syncthreads();
                if (warp != 0) {
                    R.dK = s_dK[SPLIT ? lane : 0];
                    R.y = s_y[SPLIT ? lane : 0];
                    R.phase = s_ph[SPLIT ? lane : 0];
                    fin = s_fin[SPLIT ? lane : 0] != 0;
                }
            } else if (act) {
                fin = R.update(A, tol, max_iter, o.status);
                if (fin) {
                    o.org[b0 + k] = R.K;
                    o.eta[b0 + k] = R.y;
                    o.dorg[b0 + k] = R.dK;
                    o.lamk[b0 + k] = R.dK + R.y;
                    if (o.sweeps) o.sweeps[b0 + k] = R.nsw;
                }
            }
            const unsigned mask = __ballot_sync(FULL, fin);
            if (fin) {
                k = next + __popc(mask & ((1u << lane) - 1u));
                act = k < wend;
                if (act) R.init(dk, zk, k, m, W, o.unshifted != 0);
            }
            next += __popc(mask);
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
k_lowner(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off, R1Out o,
         const int32_t *__restrict__ fslot, unsigned long long *__restrict__ queue)
{
    __shared__ int64_t s_tile;
    const int64_t ntiles = tile_off[nprob];
    for (int64_t it = blockIdx.x;; it += gridDim.x) {
        int64_t tile = it;
        if (queue) {                          // tiles claimed one at a time (costs differ by m)
            __syncthreads();
            if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(queue, 1ull);
            __syncthreads();
            tile = s_tile;
        }
        if (tile >= ntiles) break;
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        if (fslot && fslot[p] >= 0) continue;   // FMM problem
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int i = (int)(tile - tile_off[p]) * TR + threadIdx.x;
        if (i >= m) continue;
        const double *dk = o.dk + b0, *dorg = o.dorg + b0, *eta = o.eta + b0;
        const double di = dk[i];
        // numerator and denominator products kept apart (one division per
        // entry instead of one per factor); every 8 factors both are brought
        // back to [1/2, 1) by exponent arithmetic, the exponents summed in ex
        double pn = (dorg[m - 1] - di) + eta[m - 1];
        double pd = 1.0;
        int ex = 0;
        for (int j = 0; j < m - 1; j++) {
            double num = (dorg[j] - di) + eta[j];
            double den = ((j < i) ? dk[j] : dk[j + 1]) - di;
            pn *= num;
            pd *= den;
            if ((j & 7) == 7) {
                int hn = __double2hiint(pn), hd = __double2hiint(pd);
                int en = (hn >> 20) & 0x7FF, ed = (hd >> 20) & 0x7FF;
                if (en != 0 && ed != 0 && en != 0x7FF && ed != 0x7FF) {
                    ex += en - ed;
                    pn = __hiloint2double((hn & 0x800FFFFF) | (1022 << 20), __double2loint(pn));
                    pd = __hiloint2double((hd & 0x800FFFFF) | (1022 << 20), __double2loint(pd));
                }
            }
        }
        double prod = pn / pd;
        if (ex & 1) { prod *= 2.0; ex -= 1; }
        double vs = sqrt(prod);
        vs = ldexp(vs, ex / 2);
        double v = vs;
        if (!isfinite(v)) sdc_latch(o.status, SUPERDC_DEV_NONFINITE);
        o.vhat[b0 + i] = (o.zk[b0 + i] < 0.0) ? -v : v;
    }
}

// ---------------------------------------------------------------------------
// b_j = (sum_i vhat_i^2 / ((d_i - d_{K_j}) - eta_j)^2)^(-1/2), eq. (4.27)
// ---------------------------------------------------------------------------
template <int TR>
__global__ void __launch_bounds__(TR)
k_bnorm(int64_t nprob, const int64_t *__restrict__ off, const int64_t *__restrict__ tile_off, R1Out o,
         const int32_t *__restrict__ fslot, unsigned long long *__restrict__ queue)
{
    __shared__ int64_t s_tile;
    const int64_t ntiles = tile_off[nprob];
    for (int64_t it = blockIdx.x;; it += gridDim.x) {
        int64_t tile = it;
        if (queue) {                          // tiles claimed one at a time (costs differ by m)
            __syncthreads();
            if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(queue, 1ull);
            __syncthreads();
            tile = s_tile;
        }
        if (tile >= ntiles) break;
        const int64_t p = sdc_upper_index(tile_off, nprob, tile);
        if (fslot && fslot[p] >= 0) continue;   // FMM problem
        const int64_t b0 = off[p];
        const int m = o.mk[p];
        const int j = (int)(tile - tile_off[p]) * TR + threadIdx.x;
        if (j >= m) continue;
        const double *dk = o.dk + b0, *v = o.vhat + b0;
        const double dK = o.dorg[b0 + j], e = o.eta[b0 + j];
        double s = 0.0;
        for (int i = 0; i < m; i++) {
            double t = (dk[i] - dK) - e;
            double r = rcp_nr2(t);
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
        if (x < off[0] || x >= off[nprob]) continue;
        const int64_t p = sdc_upper_index(off, nprob, x);
        const int64_t b0 = off[p];
        const int m = (int)(off[p + 1] - b0);
        const int mk = SDC_IDX(o.mk[p], m + 1, o.status);       // kept count in [0, m]
        const int s = (int)(x - b0);
        const double *dk = o.dk + b0, *dorg = o.dorg + b0, *eta = o.eta + b0;
        const int32_t *src = o.src + b0;
        int pos;
        double val;
        if (s < mk) {
            val = o.lamk[b0 + s];                        // eq. (4.21), d_K + eta
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
                double lm = o.lamk[b0 + mid];
                if (key_less(lm, src[mid], val, src[s])) lo = mid + 1; else hi = mid;
            }
            pos = (s - mk) + lo;
        }
        o.lam[b0 + pos] = val;
        o.perm[b0 + pos] = s;
        o.pinv[b0 + s] = pos;
    }
}

// k_units sorts in dynamic shared memory beyond the default 48 KB: raise its
// limit once per device (the attribute belongs to the device's context)
cudaError_t units_attr()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        e = cudaFuncSetAttribute(k_units, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(SORT_MAX * sizeof(unsigned long long)));
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

// Secular schedule of a batch (shared by r1_run and the allocation-free
// entry point): with many roots per CTA slot, whole problems (or 2048-root
// pieces) go to CTAs whose warps own separate root ranges; with few roots per
// slot (the top levels of a tree), units shrink so every SM gets work and the
// warps of a CTA split the poles instead of the roots.  opts.sched forces
// either mode, opts.tile_roots the unit size.
void secular_schedule(int64_t rows, int sched, int tile_roots, int slots, bool *split, int *ubig)
{
    const int64_t per = rows / slots;
    *split = (sched == 2) || (sched == 0 && per < 512);
    *ubig = SEC_UNIT_BIG / 2;
    if (*split) *ubig = (int)std::max<int64_t>(32, std::min<int64_t>(256, (per / 32) * 32));
    if (tile_roots >= 32 && tile_roots <= 4096) *ubig = (tile_roots / 32) * 32;
}

}  // namespace

cudaError_t r1_prepare() { sdc_pool(); return units_attr(); }

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------
superdc_status r1_run(const R1Args &a_in, cudaStream_t st)
{
    R1Args a = a_in;
    const int nsm = sdc_num_sms();
    double *wd = nullptr, *wz = nullptr;
    int8_t *kept = nullptr;
    int64_t *tile_off = nullptr;
    SdcScratch sc(st);
    SDC_CHECK(sc.get(&wd, a.total));
    SDC_CHECK(sc.get(&wz, a.total));
    SDC_CHECK(sc.get(&kept, a.total));
    SDC_CHECK(sc.get(&tile_off, a.nprob + 1));
    int32_t *surv = nullptr;
    SDC_CHECK(sc.get(&surv, a.total));
    SDC_CHECK(sc.get(&a.o.lamk, a.total));
    int4 *units = nullptr;
    int *ucount = nullptr;
    SDC_CHECK(sc.get(&units, a.nprob + a.total / 32 + 2));
    SDC_CHECK(sc.get(&ucount, 2));
    SDC_CHECK(units_attr());

    const int tpb = 128;
    PROF_LAUNCH("deflate", st, k_deflate<<<(unsigned)((a.nprob + tpb - 1) / tpb), tpb, 0, st>>>(
        a.nprob, a.off, a.d, a.z, a.sqrt_rho, a.tau, wd, wz, kept, a.o));
    if (a.total > DEFL_BIG)
        PROF_LAUNCH("deflate", st, (nsm > a.nprob ? k_deflate_big<1024> : k_deflate_big<DB_T>)<<<
                                       (unsigned)a.nprob, nsm > a.nprob ? 1024 : DB_T, 0, st>>>(
            a.nprob, a.off, a.d, a.z, a.sqrt_rho, a.tau, wd, wz, kept, surv, a.o));
    // problems whose kept size reaches the threshold take the triangular FMM
    // path; the direct kernels below skip them
    FmmPlan fp;
    {
        // boxes of 32: the secular sweeps repeat the near field every iteration
        const int w = a.keep ? std::min(32, a.keep_width) : 0;
        superdc_status fs = fmm_plan(fp, a.nprob, a.off, a.total, a.max_m, a.o.mk, a.o.dk, a.fmm_min_m,
                                     std::max(1, w), std::max(4, w), a.o.fmm_used, 32, 3, st);
        if (fs != SUPERDC_OK) { fmm_free(fp, st); return fs; }
    }
    const int32_t *fslot = fp.on ? fp.dv.fslot : nullptr;
    const int TR = 128;
    PROF_LAUNCH("tiles", st, k_tiles<<<1, 1024, 0, st>>>(a.nprob, a.o.mk, TR, tile_off));
    const unsigned grid = (unsigned)(nsm * 8);
    const size_t ksm = (a.nprob <= SORT_MAX) ? (size_t)SORT_MAX * sizeof(unsigned long long) : 0;
    const int slots = nsm * 6;
    bool split;
    int ubig;
    secular_schedule(a.rows >= 0 ? a.rows : a.total, a.sched, a.tile_roots, slots, &split, &ubig);
    PROF_LAUNCH("units", st, k_units<<<1, 1024, ksm, st>>>(a.nprob, a.o.mk, fslot, ubig, split ? 0 : 1, units,
                                                           ucount, ucount + 1));
    if (split)
        PROF_LAUNCH("secular", st, (k_secular<4, true><<<(unsigned)slots, 128, 0, st>>>(
                                       a.off, units, ucount, ucount + 1, a.o, a.stop_c, a.max_iter)));
    else
        PROF_LAUNCH("secular", st, (k_secular<4, false><<<(unsigned)slots, 128, 0, st>>>(
                                       a.off, units, ucount, ucount + 1, a.o, a.stop_c, a.max_iter)));
    superdc_status fs = fmm_secular(fp, a.off, a.o, a.stop_c, a.max_iter, st);
    unsigned long long *tq = nullptr;          // tile queues of the direct Loewner and b kernels
    SDC_CHECK(sc.get(&tq, 2));
    SDC_CHECK(cudaMemsetAsync(tq, 0, 2 * sizeof(unsigned long long), st));
    PROF_LAUNCH("lowner", st, k_lowner<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o, fslot, tq));
    if (fs == SUPERDC_OK) fs = fmm_lowner(fp, a.off, a.o, st);
    PROF_LAUNCH("bnorm", st, k_bnorm<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o, fslot, tq + 1));
    if (fs == SUPERDC_OK) fs = fmm_bnorm(fp, a.off, a.o, st);
    PROF_LAUNCH("merge", st, k_merge<<<(unsigned)(nsm * 8), 256, 0, st>>>(a.nprob, a.off, a.total, a.o));
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) { fmm_free(fp, st); return SUPERDC_ERR_CUDA; }
    if (a.keep && fs == SUPERDC_OK) *a.keep = fp;
    else fmm_free(fp, st);
    return fs;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the batched rank-one step.
//
// Some callers cannot allocate device memory while they run: code that is
// recorded once into a CUDA graph and replayed, code on a real-time or
// latency-bound path where an allocation may block or fail, and hosts whose
// memory budget is fixed up front (a stream-ordered pool they do not own, a
// framework that has already reserved the device).  For them the scratch of
// the batched step lives in one statically sized device array that the
// library reserves when it is loaded, and the entry point below never calls
// cudaMalloc, cudaFree or any allocating routine.
//
// Limits: total entries <= SDC_NOALLOC_MAX_TOTAL, problems <= SDC_NOALLOC_MAX_PROB.
// The array is shared by every call on a device and keeps the previous call's
// contents; each call writes every scratch word before reading it (the unit
// counter is reset by k_units), so nothing has to be cleared in between.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the array: serialise them.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NA_T = SDC_NOALLOC_MAX_TOTAL;
constexpr int64_t NA_P = SDC_NOALLOC_MAX_PROB;
constexpr size_t na_round(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t NA_WD = 0;
constexpr size_t NA_WZ = NA_WD + na_round(NA_T * sizeof(double));
constexpr size_t NA_DORG = NA_WZ + na_round(NA_T * sizeof(double));
constexpr size_t NA_WSUM = NA_DORG + na_round(NA_T * sizeof(double));
constexpr size_t NA_TILE = NA_WSUM + na_round(NA_P * sizeof(double));
constexpr size_t NA_UNITS = NA_TILE + na_round((NA_P + 1) * sizeof(int64_t));
constexpr size_t NA_SURV = NA_UNITS + na_round((NA_P + NA_T / 32 + 2) * sizeof(int4));
constexpr size_t NA_PINV = NA_SURV + na_round(NA_T * sizeof(int32_t));
constexpr size_t NA_KEPT = NA_PINV + na_round(NA_T * sizeof(int32_t));
constexpr size_t NA_UCNT = NA_KEPT + na_round(NA_T * sizeof(int8_t));
constexpr size_t NA_LAMK = NA_UCNT + na_round(2 * sizeof(int));
constexpr size_t NA_BYTES = NA_LAMK + na_round(NA_T * sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of g_noalloc_scratch for the current device.  In host code
// the symbol name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress once per device (with that device current) and
// cached.
cudaError_t noalloc_scratch(unsigned char **ptr)
{
    static std::mutex mu;
    static unsigned char *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = (unsigned char *)p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" superdc_status superdc_secular_batched_noalloc(int64_t nprob, const int64_t *offsets, int64_t total,
                                                          const double *d, const double *z, double rho,
                                                          const superdc_opts *opts, superdc_rank1_out *out,
                                                          cudaStream_t st)
{
    superdc_opts def;
    if (!opts) { superdc_opts_default(&def); opts = &def; }
    if (nprob < 0 || total < 0 || !(rho > 0.0) || !out) return SUPERDC_ERR_ARG;
    if (!(opts->tau >= 0.0) || !(opts->stop_c > 0.0) || opts->max_iter < 1 || opts->max_iter > 10000 ||
        opts->sched < 0 || opts->sched > 2 || (opts->shifted != 0 && opts->shifted != 1))
        return SUPERDC_ERR_ARG;
    if (nprob > NA_P || total > NA_T) return SUPERDC_ERR_ARG;   // beyond the static scratch
    if (nprob == 0) return SUPERDC_OK;
    if (!offsets || !d || !z) return SUPERDC_ERR_ARG;
    if (!out->lam || !out->dk || !out->zk || !out->eta || !out->vhat || !out->bnorm || !out->org ||
        !out->src || !out->perm || !out->giv_ab || !out->giv_cs || !out->mk || !out->ngiv || !out->status)
        return SUPERDC_ERR_ARG;
    unsigned char *base = nullptr;
    SDC_CHECK(noalloc_scratch(&base));
    R1Args a;
    a.nprob = nprob; a.total = total; a.off = offsets; a.d = d; a.z = z;
    a.sqrt_rho = sqrt(rho); a.tau = opts->tau; a.stop_c = opts->stop_c; a.max_iter = opts->max_iter;
    a.tile_roots = opts->tile_roots; a.sched = opts->sched;
    a.o.lam = out->lam; a.o.dk = out->dk; a.o.zk = out->zk; a.o.eta = out->eta;
    a.o.vhat = out->vhat; a.o.bnorm = out->bnorm; a.o.org = out->org; a.o.src = out->src;
    a.o.perm = out->perm; a.o.giv_ab = out->giv_ab; a.o.giv_cs = out->giv_cs; a.o.mk = out->mk;
    a.o.ngiv = out->ngiv; a.o.sweeps = out->sweeps; a.o.status = out->status;
    a.o.unshifted = opts->shifted ? 0 : 1;
    a.o.dorg = (double *)(base + NA_DORG);
    a.o.wsum = (double *)(base + NA_WSUM);
    a.o.pinv = (int32_t *)(base + NA_PINV);
    a.o.lamk = (double *)(base + NA_LAMK);
    if (out->fmm) SDC_CHECK(cudaMemsetAsync(out->fmm, 0, (size_t)nprob * sizeof(int32_t), st));   // direct only
    double *wd = (double *)(base + NA_WD), *wz = (double *)(base + NA_WZ);
    int8_t *kept = (int8_t *)(base + NA_KEPT);
    int64_t *tile_off = (int64_t *)(base + NA_TILE);
    int32_t *surv = (int32_t *)(base + NA_SURV);
    int4 *units = (int4 *)(base + NA_UNITS);
    int *ucount = (int *)(base + NA_UCNT);
    SDC_CHECK(units_attr());
    const int nsm = sdc_num_sms();
    const int tpb = 128;
    k_deflate<<<(unsigned)((a.nprob + tpb - 1) / tpb), tpb, 0, st>>>(a.nprob, a.off, a.d, a.z, a.sqrt_rho, a.tau,
                                                                      wd, wz, kept, a.o);
    if (a.total > DEFL_BIG)
        k_deflate_big<DB_T><<<(unsigned)a.nprob, DB_T, 0, st>>>(a.nprob, a.off, a.d, a.z, a.sqrt_rho, a.tau, wd, wz,
                                                           kept, surv, a.o);
    const int TR = 128;
    k_tiles<<<1, 1024, 0, st>>>(a.nprob, a.o.mk, TR, tile_off);
    const unsigned grid = (unsigned)(nsm * 8);
    const size_t ksm = (a.nprob <= SORT_MAX) ? (size_t)SORT_MAX * sizeof(unsigned long long) : 0;
    const int slots = nsm * 6;
    bool split;
    int ubig;
    secular_schedule(a.total, a.sched, a.tile_roots, slots, &split, &ubig);
    k_units<<<1, 1024, ksm, st>>>(a.nprob, a.o.mk, nullptr, ubig, split ? 0 : 1, units, ucount, ucount + 1);
    if (split)
        k_secular<4, true><<<(unsigned)slots, 128, 0, st>>>(a.off, units, ucount, ucount + 1, a.o, a.stop_c,
                                                             a.max_iter);
    else
        k_secular<4, false><<<(unsigned)slots, 128, 0, st>>>(a.off, units, ucount, ucount + 1, a.o, a.stop_c,
                                                              a.max_iter);
    k_lowner<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o, nullptr, nullptr);
    k_bnorm<128><<<grid, 128, 0, st>>>(a.nprob, a.off, tile_off, a.o, nullptr, nullptr);
    k_merge<<<(unsigned)(nsm * 8), 256, 0, st>>>(a.nprob, a.off, a.total, a.o);
    SDC_CHECK(cudaGetLastError());
    return SUPERDC_OK;
}
