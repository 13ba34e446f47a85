// HSS construction by off-diagonal compression (the HSS input the paper's
// Example 4 needs: "direct off-diagonal compression" of a kernel matrix,
// Section 5).  A symmetric matrix given by its entries (a dense device array
// or a kernel evaluated at points) is approximated by a symmetric HSS matrix
// with a perfect tree of leaves of `leaf` rows and one rank r at every node,
// the form superdc_build_hss takes.
//
// Method (randomized range finding on the off-diagonal block rows, one sample
// matrix for the whole tree; the caller passes the Gaussian sample Omega):
//   Y = A Omega; for a leaf i, Y_i^off = Y(I_i) - A(I_i, I_i) Omega(I_i) samples
//   the block row A(I_i, I_i^c); U_i = its leading r left singular vectors.
//   Projections carried up the tree: P_i = U_i^T Y_i^off, W_i = U_i^T Omega(I_i)
//   (r x s each, with U_i the explicit nested basis of node i).
//   At a node i with children c1, c2: B_c1 = U_c1^T A(I_c1, I_c2) U_c2 (exact
//   block product), the children's samples restricted to i's complement,
//     V_c1 = P_c1 - B_c1 W_c2,  V_c2 = P_c2 - B_c1^T W_c1,
//   and [R_c1; R_c2] = the leading r left singular vectors of [V_c1; V_c2], so
//   U_i = diag(U_c1, U_c2) [R_c1; R_c2]; P_i = R_c1^T V_c1 + R_c2^T V_c2,
//   W_i = R_c1^T W_c1 + R_c2^T W_c2.  Leaves keep D_i = A(I_i, I_i).
// The leading singular vectors of a q x s sample M come from the
// eigenvectors of M^T M (cyclic Jacobi, s <= 64), U = M v / sigma, then two
// passes of Gram-Schmidt; the ratio sigma_{r+1} / sigma_1 of every node is
// returned (largest over the tree) as the estimate of the relative
// truncation error.
#include <algorithm>
#include <functional>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "handles.cuh"

namespace {

struct EntrySrc {
    int kind;              // 0 dense, 1 sqrt|x_i - x_j|, 2 exp(-|x_i - x_j| / param)
    const double *A;
    int64_t lda;
    const double *x;
    double param;
};

__device__ __forceinline__ double entry(const EntrySrc &e, int64_t i, int64_t j, double xi, double xj)
{
    if (e.kind == 0) return e.A[i + j * e.lda];
    const double d = fabs(xi - xj);
    if (e.kind == 1) return sqrt(d);
    return exp(-d / e.param);
}

// One block product per blockIdx.z:  out(r, :) (+)= sum_{j in cols} A(r0 + r, c0 + j) M(j, :)
// over the column split blockIdx.y of the block's columns; rows one per
// thread (blockIdx.x tiles of 128), K columns of M (K <= KT) staged 32 at a
// time.  Partial sums of the splits go to part[split] (reduced in order by
// k_reduce_splits); block b: rows [r0[b], r0[b] + nr[b]), columns
// [c0[b], c0[b] + nc[b]), M_b = Mbase + moff[b] (ld ldm), out rows at
// orow[b] in part (ld ldo).
struct BlockSet {
    const int64_t *r0, *nr, *c0, *nc, *moff, *orow;
};

template <int KT>
__global__ void __launch_bounds__(128) k_blockprod(EntrySrc e, BlockSet bs, const double *__restrict__ M, int64_t ldm,
                                                   int K, double *__restrict__ part, int64_t ldo, int64_t split_stride)
{
    __shared__ double sm[32][KT];
    __shared__ double sx[32];
    const int b = blockIdx.z;
    const int64_t nr = bs.nr[b], nc = bs.nc[b];
    const int64_t row = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if ((int64_t)blockIdx.x * 128 >= nr) return;
    const int64_t r0 = bs.r0[b], c0 = bs.c0[b];
    const int nsplit = gridDim.y;
    const int64_t jb = nc * blockIdx.y / nsplit, je = nc * (blockIdx.y + 1) / nsplit;
    const double *Mb = M + bs.moff[b];
    const bool act = row < nr;
    const double xi = (act && e.kind != 0) ? e.x[r0 + row] : 0.0;
    double acc[KT];
#pragma unroll
    for (int q = 0; q < KT; q++) acc[q] = 0.0;
    for (int64_t j0 = jb; j0 < je; j0 += 32) {
        const int cnt = (int)(je - j0 < 32 ? je - j0 : 32);
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * KT; t += 128) {
            const int jj = t / KT, q = t % KT;
            sm[jj][q] = (jj < cnt && q < K) ? Mb[(j0 + jj) + (int64_t)q * ldm] : 0.0;
        }
        if (threadIdx.x < 32) sx[threadIdx.x] = (threadIdx.x < cnt && e.kind != 0) ? e.x[c0 + j0 + threadIdx.x] : 0.0;
        __syncthreads();
        if (act) {
            for (int jj = 0; jj < cnt; jj++) {
                const double a = entry(e, r0 + row, c0 + j0 + jj, xi, sx[jj]);
#pragma unroll
                for (int q = 0; q < KT; q++) acc[q] = fma(a, sm[jj][q], acc[q]);
            }
        }
    }
    if (act) {
        double *o = part + (int64_t)blockIdx.y * split_stride + bs.orow[b] + row;
#pragma unroll
        for (int q = 0; q < KT; q++)
            if (q < K) o[(int64_t)q * ldo] = acc[q];
    }
}

// out(i, q) = sum over splits of part[split](i, q) (fixed order); n rows, K columns
__global__ void k_reduce_splits(int64_t n, int K, int nsplit, const double *__restrict__ part, int64_t ldo,
                                int64_t split_stride, double *__restrict__ out, int64_t ldout, double sign,
                                const double *__restrict__ base)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % n;
        const int q = (int)(t / n);
        double s = 0.0;
        for (int sp = 0; sp < nsplit; sp++) s += part[sp * split_stride + i + q * ldo];
        out[i + q * ldout] = (base ? base[i + q * ldout] : 0.0) + sign * s;
    }
}

// D blocks of the leaves: D_k = A(I_k, I_k), column-major m x m
__global__ void k_leaf_blocks(EntrySrc e, int nleaves, int m, double *__restrict__ D)
{
    const int64_t mm = (int64_t)m * m;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nleaves * mm;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / mm, w = t % mm;
        const int64_t i = k * m + w % m, j = k * m + w / m;
        const double xi = e.kind ? e.x[i] : 0.0, xj = e.kind ? e.x[j] : 0.0;
        D[t] = entry(e, i, j, xi, xj);
    }
}

// Leading r left singular vectors of one q x s sample per CTA (q <= 128,
// r <= s <= 64): G = M^T M, cyclic Jacobi for its eigenpairs, the r largest,
// U(:, t) = M v_t / sqrt(lambda_t), two passes of modified Gram-Schmidt.
// Sample b at M + mo[b] (ld ldm), output at U + uo[b] (ld ldu); ratio[b] =
// sigma_{r+1} / sigma_1 (0 when s == r).  Rank-deficient samples (sigma_t = 0)
// get zero columns before the Gram-Schmidt passes, which then complete them
// from unit vectors.
constexpr int RQ = 128, RS = 64;

__global__ void __launch_bounds__(256) k_range(const int64_t *__restrict__ mo, const int64_t *__restrict__ uo,
                                               const double *__restrict__ M, int64_t ldm, int q, int s, int r,
                                               double *__restrict__ U, int64_t ldu, double *__restrict__ ratio,
                                               int32_t *status)
{
    extern __shared__ double sh[];
    double *Ms = sh;                       // q x s   (ld RQ)
    double *G = Ms + RQ * RS;              // s x s   (ld RS)
    double *V = G + RS * RS;               // s x s
    double *Us = V + RS * RS;              // q x r   (ld RQ)
    __shared__ double s_c, s_s, s_off, s_fro;
    __shared__ int s_top[RS];
    const int b = blockIdx.x, tid = threadIdx.x;
    const double *Mb = M + mo[b];
    for (int t = tid; t < q * s; t += blockDim.x) Ms[(t % q) + RQ * (t / q)] = Mb[(t % q) + ldm * (t / q)];
    __syncthreads();
    for (int t = tid; t < s * s; t += blockDim.x) {
        const int a = t % s, c = t / s;
        double v = 0.0;
        for (int i = 0; i < q; i++) v = fma(Ms[i + RQ * a], Ms[i + RQ * c], v);
        G[a + RS * c] = v;
        V[a + RS * c] = (a == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double f = 0.0;
        for (int a = 0; a < s; a++)
            for (int c = 0; c < s; c++) f += G[a + RS * c] * G[a + RS * c];
        s_fro = sqrt(f);
    }
    __syncthreads();
    for (int sweep = 0; sweep < 40; sweep++) {
        if (tid == 0) {
            double o = 0.0;
            for (int c = 0; c < s; c++)
                for (int a = 0; a < s; a++)
                    if (a != c) o += G[a + RS * c] * G[a + RS * c];
            s_off = sqrt(o);
        }
        __syncthreads();
        if (!(s_off > SDC_EPS * s_fro)) break;
        for (int p = 0; p < s - 1; p++)
            for (int w = p + 1; w < s; w++) {
                if (tid == 0) {
                    const double apq = G[p + RS * w];
                    double c = 1.0, sn = 0.0;
                    if (apq != 0.0) {
                        const double zeta = (G[w + RS * w] - G[p + RS * p]) / (2.0 * apq);
                        const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                                              : ((zeta >= 0 ? 1.0 : -1.0) /
                                                                 (fabs(zeta) + sqrt(1.0 + zeta * zeta)));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                    }
                    s_c = c;
                    s_s = sn;
                }
                __syncthreads();
                const double c = s_c, sn = s_s;
                if (sn != 0.0) {
                    // rows p, w of G, then columns p, w (two phases), and V's columns
                    if (tid < s) {
                        const double gp = G[p + RS * tid], gw = G[w + RS * tid];
                        G[p + RS * tid] = c * gp - sn * gw;
                        G[w + RS * tid] = sn * gp + c * gw;
                    }
                    __syncthreads();
                    if (tid < s) {
                        const double gp = G[tid + RS * p], gw = G[tid + RS * w];
                        G[tid + RS * p] = c * gp - sn * gw;
                        G[tid + RS * w] = sn * gp + c * gw;
                    } else if (tid >= 64 && tid < 64 + s) {
                        const int k = tid - 64;
                        const double vp = V[k + RS * p], vw = V[k + RS * w];
                        V[k + RS * p] = c * vp - sn * vw;
                        V[k + RS * w] = sn * vp + c * vw;
                    }
                    __syncthreads();
                }
            }
    }
    if (tid == 0) {
        // the r largest eigenvalues (selection, ties by index)
        bool used[RS];
        for (int a = 0; a < s; a++) used[a] = false;
        for (int t = 0; t < r; t++) {
            int best = -1;
            for (int a = 0; a < s; a++)
                if (!used[a] && (best < 0 || G[a + RS * a] > G[best + RS * best])) best = a;
            used[best] = true;
            s_top[t] = best;
        }
        const double l1 = fmax(G[s_top[0] + RS * s_top[0]], 0.0);
        if (!isfinite(l1)) sdc_latch(status, SUPERDC_DEV_NONFINITE);
    }
    __syncthreads();
    for (int t = tid; t < q * r; t += blockDim.x) {
        const int i = t % q, c = t / q;
        const int a = s_top[c];
        const double lam = G[a + RS * a];
        double v = 0.0;
        for (int k = 0; k < s; k++) v = fma(Ms[i + RQ * k], V[k + RS * a], v);
        Us[i + RQ * c] = (lam > 0.0) ? v / sqrt(lam) : 0.0;
    }
    __syncthreads();
    // two passes of modified Gram-Schmidt; a column that vanishes is replaced
    // by the first unit vector not yet in the span
    __shared__ double s_dot;
    for (int pass = 0; pass < 2; pass++) {
        for (int c = 0; c < r; c++) {
            for (int c2 = 0; c2 < c; c2++) {
                if (tid == 0) {
                    double d = 0.0;
                    for (int i = 0; i < q; i++) d = fma(Us[i + RQ * c2], Us[i + RQ * c], d);
                    s_dot = d;
                }
                __syncthreads();
                for (int i = tid; i < q; i += blockDim.x) Us[i + RQ * c] -= s_dot * Us[i + RQ * c2];
                __syncthreads();
            }
            if (tid == 0) {
                double nn = 0.0;
                for (int i = 0; i < q; i++) nn = fma(Us[i + RQ * c], Us[i + RQ * c], nn);
                s_dot = sqrt(nn);
            }
            __syncthreads();
            if (s_dot > 1e-8) {
                for (int i = tid; i < q; i += blockDim.x) Us[i + RQ * c] /= s_dot;
            } else if (pass == 0) {
                // completion: e_(c) orthogonalised on the next pass
                for (int i = tid; i < q; i += blockDim.x) Us[i + RQ * c] = (i == (c % q)) ? 1.0 : 0.0;
            }
            __syncthreads();
        }
    }
    for (int t = tid; t < q * r; t += blockDim.x) U[uo[b] + (t % q) + ldu * (t / q)] = Us[(t % q) + RQ * (t / q)];
    // relative residual of the sample's projection, ||M - U U^T M||_F / ||M||_F
    // (what the rank-r basis leaves out; exact to rounding, unlike the Gram
    // matrix's eigenvalues, which cannot resolve ratios below sqrt(eps))
    __shared__ double s_res[RS], s_nrm[RS];
    if (tid < s) {
        double cf[32];
        for (int t = 0; t < r; t++) {
            double v = 0.0;
            for (int i = 0; i < q; i++) v = fma(Us[i + RQ * t], Ms[i + RQ * tid], v);
            cf[t] = v;
        }
        double rs = 0.0, nm = 0.0;
        for (int i = 0; i < q; i++) {
            double v = Ms[i + RQ * tid];
            nm = fma(v, v, nm);
            for (int t = 0; t < r; t++) v = fma(-Us[i + RQ * t], cf[t], v);
            rs = fma(v, v, rs);
        }
        s_res[tid] = rs;
        s_nrm[tid] = nm;
    }
    __syncthreads();
    if (tid == 0) {
        double rs = 0.0, nm = 0.0;
        for (int c = 0; c < s; c++) { rs += s_res[c]; nm += s_nrm[c]; }
        ratio[b] = (nm > 0.0) ? sqrt(rs / nm) : 0.0;
    }
}

// small dense products per node (column-major), one CTA per node:
//   C_b = op(A_b) B_b (+ beta C_b), op = transpose when ta
struct SmallMM {
    const int64_t *ao, *bo, *co;
};
__global__ void k_small_mm(SmallMM o, const double *__restrict__ A, int64_t lda, const double *__restrict__ Bm,
                           int64_t ldb, double *__restrict__ C, int64_t ldc, int m, int n, int k, int ta,
                           double alpha, double beta)
{
    const int b = blockIdx.x;
    const double *Ab = A + o.ao[b], *Bb = Bm + o.bo[b];
    double *Cb = C + o.co[b];
    for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
        const int i = t % m, j = t / m;
        double s = 0.0;
        for (int p = 0; p < k; p++) s = fma(ta ? Ab[p + lda * i] : Ab[i + lda * p], Bb[p + ldb * j], s);
        Cb[i + ldc * j] = alpha * s + (beta != 0.0 ? beta * Cb[i + ldc * j] : 0.0);
    }
}

// leaf bases: rows k m .. k m + m - 1 of the n x r matrix Ul -> the k-th
// column-major m x r block of Up
__global__ void k_pack_leaves(int64_t n, int m, int r, const double *__restrict__ Ul, double *__restrict__ Up)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * r; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t % n, j = t / n;
        const int64_t k = row / m, i = row % m;
        Up[k * (int64_t)m * r + i + (int64_t)m * j] = Ul[t];
    }
}

int sel_kt(int K) { return K <= 16 ? 16 : K <= 32 ? 32 : K <= 48 ? 48 : 64; }

// out rows (ld ldout, K columns) = sum over the blocks of A-block * M-block, with
// nsplit column splits reduced in order; base/sign: out = base + sign * product
cudaError_t block_products(const EntrySrc &e, const std::vector<int64_t> &hr0, const std::vector<int64_t> &hnr,
                           const std::vector<int64_t> &hc0, const std::vector<int64_t> &hnc,
                           const std::vector<int64_t> &hmoff, const std::vector<int64_t> &horow, int64_t nrows,
                           const double *M, int64_t ldm, int K, double *out, int64_t ldout, double sign,
                           const double *base, int nsplit, SdcScratch &sc, cudaStream_t st)
{
    const int nb = (int)hr0.size();
    if (nb == 0) return cudaSuccess;
    int64_t *tab = nullptr;
    cudaError_t err = sc.get(&tab, 6 * (size_t)nb);
    if (err != cudaSuccess) return err;
    std::vector<int64_t> h;
    for (auto *v : {&hr0, &hnr, &hc0, &hnc, &hmoff, &horow}) h.insert(h.end(), v->begin(), v->end());
    err = cudaMemcpyAsync(tab, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return err;
    // the host table must live until the copy ran
    err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return err;
    BlockSet bs{tab, tab + nb, tab + 2 * nb, tab + 3 * nb, tab + 4 * nb, tab + 5 * nb};
    double *part = nullptr;
    err = sc.get(&part, (size_t)nsplit * nrows * K);
    if (err != cudaSuccess) return err;
    int64_t maxr = 1;
    for (int64_t v : hnr) maxr = std::max(maxr, v);
    dim3 grid((unsigned)((maxr + 127) / 128), (unsigned)nsplit, (unsigned)nb);
    const int kt = sel_kt(K);
    const int64_t ss = nrows * K;
    if (kt == 16) k_blockprod<16><<<grid, 128, 0, st>>>(e, bs, M, ldm, K, part, nrows, ss);
    else if (kt == 32) k_blockprod<32><<<grid, 128, 0, st>>>(e, bs, M, ldm, K, part, nrows, ss);
    else if (kt == 48) k_blockprod<48><<<grid, 128, 0, st>>>(e, bs, M, ldm, K, part, nrows, ss);
    else k_blockprod<64><<<grid, 128, 0, st>>>(e, bs, M, ldm, K, part, nrows, ss);
    k_reduce_splits<<<(unsigned)(sdc_num_sms() * 8), 256, 0, st>>>(nrows, K, nsplit, part, nrows, ss, out, ldout, sign,
                                                                    base);
    return cudaGetLastError();
}

// Perfect tree over n = m 2^L rows in postorder: node ids, children, offsets,
// sizes, and the nodes of every level left to right.
struct PTree {
    int L = 0, nn = 0;
    std::vector<std::vector<int>> lev;
    std::vector<int32_t> lch, rch;
    std::vector<int64_t> lsize, off, sz;
};

PTree make_ptree(int64_t n, int m)
{
    PTree t;
    const int64_t nleaves = n / m;
    while ((int64_t(1) << t.L) < nleaves) t.L++;
    t.nn = 2 * (int)nleaves - 1;
    t.lev.assign(t.L + 1, {});
    t.lch.assign(t.nn, -1); t.rch.assign(t.nn, -1);
    t.lsize.assign(t.nn, 0); t.off.assign(t.nn, 0); t.sz.assign(t.nn, 0);
    int counter = 0;
    std::function<int(int, int64_t)> build = [&](int l, int64_t o) -> int {
        if (l == t.L) {
            const int id = counter++;
            t.lsize[id] = m; t.off[id] = o; t.sz[id] = m; t.lev[l].push_back(id);
            return id;
        }
        const int64_t half = (int64_t)m << (t.L - l - 1);
        const int a = build(l + 1, o), b2 = build(l + 1, o + half);
        const int id = counter++;
        t.lch[id] = a; t.rch[id] = b2; t.off[id] = o; t.sz[id] = 2 * half; t.lev[l].push_back(id);
        return id;
    };
    build(0, 0);
    return t;
}

// Counter-based N(0,1) sample for callers that pass none: splitmix64 of the
// entry index gives two uniforms, Box-Muller one normal.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_gauss(int64_t cnt, uint64_t seed, double *__restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix64(seed ^ (2 * (uint64_t)t)), b = splitmix64(seed ^ (2 * (uint64_t)t + 1));
        const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
        out[t] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// Outputs of one compression: device arrays the caller owns (D: leaves m x m,
// U: leaves m x r packed per leaf, R, B: nn blocks r x r; all in postorder).
struct CompressOut {
    double *D, *U, *R, *B;
};

// The compression of one matrix (the method of the file comment).  Ext
// (optional, n x re, ld lde): exact extra columns appended to every node's
// sample, for a matrix that is one leaf of a larger HSS matrix whose coupling
// to the rest is Ext; with Ext the top split takes R_c = U_c^T Ext(I_c, :), so
// the tree's top basis is Ext itself.  *ratio_max: largest relative
// projection residual over the nodes' samples.
superdc_status compress_core(const EntrySrc &e, int64_t n, int m, int r, const double *Omega, int s,
                             const double *Ext, int64_t lde, int re, const CompressOut &co, double *ratio_max,
                             cudaStream_t st)
{
    const PTree pt = make_ptree(n, m);
    const int L = pt.L, nn = pt.nn;
    const int64_t nleaves = n / m;
    const std::vector<std::vector<int>> &lev = pt.lev;
    const std::vector<int32_t> &lch = pt.lch, &rch = pt.rch;
    const std::vector<int64_t> &off = pt.off, &sz = pt.sz;
    const int sx = s + re;              // sample columns carried up the tree
    SdcScratch sc(st);
    const int nsplit_full = 8;
#define CB_CHECK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) \
        return e_ == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA; } while (0)
    double *Y = nullptr, *Yoff = nullptr, *Ul = nullptr;
    double *P = nullptr, *W = nullptr, *Vb = nullptr, *Ub0 = nullptr, *Ub1 = nullptr, *T = nullptr, *ratio = nullptr;
    double *Rtmp = nullptr;
    int32_t *status = nullptr;
    double *D = co.D, *Rg = co.R, *Bg = co.B;
    CB_CHECK(sc.get(&Y, (size_t)n * s));
    CB_CHECK(sc.get(&Yoff, (size_t)n * sx));
    CB_CHECK(sc.get(&Ul, (size_t)n * r));
    CB_CHECK(sc.get(&P, (size_t)nn * r * sx));
    CB_CHECK(sc.get(&W, (size_t)nn * r * s));
    CB_CHECK(sc.get(&Vb, (size_t)nn * 2 * r * sx));
    CB_CHECK(sc.get(&Ub0, (size_t)n * r));
    CB_CHECK(sc.get(&Ub1, (size_t)n * r));
    CB_CHECK(sc.get(&T, (size_t)n * r));
    CB_CHECK(sc.get(&ratio, 2 * (size_t)nn));
    CB_CHECK(sc.get(&Rtmp, (size_t)nn * 2 * r * r));
    CB_CHECK(sc.get(&status, 1));
    CB_CHECK(cudaMemsetAsync(Rg, 0, (size_t)nn * r * r * sizeof(double), st));
    CB_CHECK(cudaMemsetAsync(Bg, 0, (size_t)nn * r * r * sizeof(double), st));
    CB_CHECK(cudaMemsetAsync(ratio, 0, 2 * (size_t)nn * sizeof(double), st));
    CB_CHECK(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    int64_t roff = nleaves;      // ratio slots: leaves first, then every level's nodes
    const size_t rsm = (size_t)(RQ * RS + 2 * RS * RS + RQ * 32) * sizeof(double);
    CB_CHECK(cudaFuncSetAttribute(k_range, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    // 1. Y = A Omega (row tiles, 8 column splits)
    {
        std::vector<int64_t> r0{0}, nr{n}, c0{0}, nc{n}, mo{0}, orow{0};
        CB_CHECK(block_products(e, r0, nr, c0, nc, mo, orow, n, Omega, n, s, Y, n, 1.0, nullptr, nsplit_full, sc, st));
    }
    // 2. leaves: Y_off = Y - A(I,I) Omega(I) (+ the exact columns); D blocks; U = range
    {
        std::vector<int64_t> r0, nr, c0, nc, mo, orow;
        for (int64_t k = 0; k < nleaves; k++) {
            r0.push_back(k * m); nr.push_back(m); c0.push_back(k * m); nc.push_back(m);
            mo.push_back(k * m); orow.push_back(k * m);
        }
        CB_CHECK(block_products(e, r0, nr, c0, nc, mo, orow, n, Omega, n, s, Yoff, n, -1.0, Y, 1, sc, st));
        if (re > 0)
            CB_CHECK(cudaMemcpy2DAsync(Yoff + (int64_t)n * s, n * sizeof(double), Ext, lde * sizeof(double),
                                       n * sizeof(double), re, cudaMemcpyDeviceToDevice, st));
        k_leaf_blocks<<<(unsigned)(sdc_num_sms() * 8), 256, 0, st>>>(e, (int)nleaves, m, D);
        std::vector<int64_t> h;
        for (int64_t k = 0; k < nleaves; k++) h.push_back(k * m);
        for (int64_t k = 0; k < nleaves; k++) h.push_back(k * m);
        int64_t *tab = nullptr;
        CB_CHECK(sc.get(&tab, h.size()));
        CB_CHECK(cudaMemcpyAsync(tab, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
        CB_CHECK(cudaStreamSynchronize(st));
        k_range<<<(unsigned)nleaves, 256, rsm, st>>>(tab, tab + nleaves, Yoff, n, m, sx, r, Ul, n, ratio, status);
        CB_CHECK(cudaGetLastError());
        CB_CHECK(cudaMemcpyAsync(Ub0, Ul, (size_t)n * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // P_leaf = U^T [Y_off(I), Ext(I)] (r x sx), W_leaf = U^T Omega(I) (r x s)
        std::vector<int64_t> hh;
        for (int64_t k = 0; k < nleaves; k++) hh.push_back(k * m);
        for (int64_t k = 0; k < nleaves; k++) hh.push_back(k * m);
        for (int64_t k = 0; k < nleaves; k++) hh.push_back((int64_t)lev[L][k] * r * sx);
        for (int64_t k = 0; k < nleaves; k++) hh.push_back((int64_t)lev[L][k] * r * s);
        int64_t *mt = nullptr;
        CB_CHECK(sc.get(&mt, hh.size()));
        CB_CHECK(cudaMemcpyAsync(mt, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice, st));
        CB_CHECK(cudaStreamSynchronize(st));
        SmallMM o{mt, mt + nleaves, mt + 2 * nleaves}, ow{mt, mt + nleaves, mt + 3 * nleaves};
        k_small_mm<<<(unsigned)nleaves, 256, 0, st>>>(o, Ul, n, Yoff, n, P, r, r, sx, m, 1, 1.0, 0.0);
        k_small_mm<<<(unsigned)nleaves, 256, 0, st>>>(ow, Ul, n, Omega, n, W, r, r, s, m, 1, 1.0, 0.0);
        CB_CHECK(cudaGetLastError());
    }
    // 3. up the tree: level l's nodes from their children's bases (Ub0: the
    // children's explicit bases, rows at their offsets)
    for (int l = L - 1; l >= 0; l--) {
        const std::vector<int> &nodes = lev[l];
        const int nl = (int)nodes.size();
        const int64_t ch = sz[lch[nodes[0]]];
        // B_c1 = U_c1^T (A(I_c1, I_c2) U_c2)
        {
            std::vector<int64_t> r0, nr, c0, nc, mo, orow;
            for (int i : nodes) {
                const int a = lch[i], b2 = rch[i];
                r0.push_back(off[a]); nr.push_back(sz[a]); c0.push_back(off[b2]); nc.push_back(sz[b2]);
                mo.push_back(off[b2]); orow.push_back(off[a]);
            }
            const int nsp = std::max(1, (int)std::min<int64_t>(8, ch / 1024));
            CB_CHECK(block_products(e, r0, nr, c0, nc, mo, orow, n, Ub0, n, r, T, n, 1.0, nullptr, nsp, sc, st));
            std::vector<int64_t> h;
            for (int i : nodes) h.push_back(off[lch[i]]);
            for (int i : nodes) h.push_back(off[lch[i]]);
            for (int i : nodes) h.push_back((int64_t)lch[i] * r * r);
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, h.size()));
            CB_CHECK(cudaMemcpyAsync(mt, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            SmallMM o{mt, mt + nl, mt + 2 * nl};
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(o, Ub0, n, T, n, Bg, r, r, r, (int)ch, 1, 1.0, 0.0);
            CB_CHECK(cudaGetLastError());
        }
        if (l == 0) {
            // the top split of a leaf refinement: R_c = U_c^T Ext(I_c, :), the
            // exact columns of the children's projected samples
            if (re > 0) {
                const int i = nodes[0];
                for (int c : {lch[i], rch[i]})
                    CB_CHECK(cudaMemcpy2DAsync(Rg + (int64_t)c * r * r, r * sizeof(double),
                                               P + (int64_t)c * r * sx + (int64_t)r * s, r * sizeof(double),
                                               r * sizeof(double), re, cudaMemcpyDeviceToDevice, st));
            }
            break;
        }
        // V = [P_c1 - B_c1 W_c2; P_c2 - B_c1^T W_c1] on the sampled columns, the
        // exact columns carried unchanged (2r x sx per node at node id * 2 r sx)
        {
            std::vector<int64_t> hh;
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * 2 * r * sx);
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * 2 * r * sx + r);
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, hh.size()));
            CB_CHECK(cudaMemcpyAsync(mt, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            for (int i : nodes) {
                const int a = lch[i], b2 = rch[i];
                CB_CHECK(cudaMemcpy2DAsync(Vb + (int64_t)i * 2 * r * sx, 2 * r * sizeof(double),
                                           P + (int64_t)a * r * sx, r * sizeof(double), r * sizeof(double), sx,
                                           cudaMemcpyDeviceToDevice, st));
                CB_CHECK(cudaMemcpy2DAsync(Vb + (int64_t)i * 2 * r * sx + r, 2 * r * sizeof(double),
                                           P + (int64_t)b2 * r * sx, r * sizeof(double), r * sizeof(double), sx,
                                           cudaMemcpyDeviceToDevice, st));
            }
            SmallMM o1{mt, mt + nl, mt + 2 * nl};
            SmallMM o2{mt + 3 * nl, mt + 4 * nl, mt + 5 * nl};
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(o1, Bg, r, W, r, Vb, 2 * r, r, s, r, 0, -1.0, 1.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(o2, Bg, r, W, r, Vb, 2 * r, r, s, r, 1, -1.0, 1.0);
            CB_CHECK(cudaGetLastError());
        }
        // [R_c1; R_c2] = range(V) (2r x r, into Rtmp at node id * 2 r r)
        {
            std::vector<int64_t> h;
            for (int i : nodes) h.push_back((int64_t)i * 2 * r * sx);
            for (int i : nodes) h.push_back((int64_t)i * 2 * r * r);
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, h.size()));
            CB_CHECK(cudaMemcpyAsync(mt, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            k_range<<<(unsigned)nl, 256, rsm, st>>>(mt, mt + nl, Vb, 2 * r, 2 * r, sx, r, Rtmp, 2 * r,
                                                    ratio + roff, status);
            CB_CHECK(cudaGetLastError());
            roff += nl;
        }
        // split into R_c1, R_c2; P_i, W_i; explicit U_i = [U_c1 R_c1; U_c2 R_c2]
        {
            for (int i : nodes) {
                const int a = lch[i], b2 = rch[i];
                CB_CHECK(cudaMemcpy2DAsync(Rg + (int64_t)a * r * r, r * sizeof(double), Rtmp + (int64_t)i * 2 * r * r,
                                           2 * r * sizeof(double), r * sizeof(double), r, cudaMemcpyDeviceToDevice, st));
                CB_CHECK(cudaMemcpy2DAsync(Rg + (int64_t)b2 * r * r, r * sizeof(double),
                                           Rtmp + (int64_t)i * 2 * r * r + r, 2 * r * sizeof(double), r * sizeof(double),
                                           r, cudaMemcpyDeviceToDevice, st));
            }
            std::vector<int64_t> hh;
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)i * 2 * r * sx);
            for (int i : nodes) hh.push_back((int64_t)i * r * sx);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)i * 2 * r * sx + r);
            for (int i : nodes) hh.push_back((int64_t)i * r * sx);
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * r * s);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * r * s);
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, hh.size()));
            CB_CHECK(cudaMemcpyAsync(mt, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            SmallMM p1{mt, mt + nl, mt + 2 * nl}, p2{mt + 3 * nl, mt + 4 * nl, mt + 5 * nl};
            SmallMM w1{mt + 6 * nl, mt + 7 * nl, mt + 8 * nl}, w2{mt + 9 * nl, mt + 10 * nl, mt + 11 * nl};
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(p1, Rg, r, Vb, 2 * r, P, r, r, sx, r, 1, 1.0, 0.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(p2, Rg, r, Vb, 2 * r, P, r, r, sx, r, 1, 1.0, 1.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(w1, Rg, r, W, r, W, r, r, s, r, 1, 1.0, 0.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(w2, Rg, r, W, r, W, r, r, s, r, 1, 1.0, 1.0);
            CB_CHECK(cudaGetLastError());
            std::vector<int64_t> u;
            for (int i : nodes) for (int c : {lch[i], rch[i]}) u.push_back(off[c]);
            for (int i : nodes) for (int c : {lch[i], rch[i]}) u.push_back((int64_t)c * r * r);
            for (int i : nodes) for (int c : {lch[i], rch[i]}) u.push_back(off[c]);
            int64_t *ut = nullptr;
            CB_CHECK(sc.get(&ut, u.size()));
            CB_CHECK(cudaMemcpyAsync(ut, u.data(), u.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            SmallMM uo{ut, ut + 2 * nl, ut + 4 * nl};
            k_small_mm<<<(unsigned)(2 * nl), 256, 0, st>>>(uo, Ub0, n, Rg, r, Ub1, n, (int)ch, r, r, 0, 1.0, 0.0);
            CB_CHECK(cudaGetLastError());
            std::swap(Ub0, Ub1);
        }
    }
    // 4. leaf bases packed m x r per leaf (they were rows of an n x r matrix)
    k_pack_leaves<<<(unsigned)(sdc_num_sms() * 8), 256, 0, st>>>(n, m, r, Ul, co.U);
    CB_CHECK(cudaGetLastError());
    std::vector<double> hr(2 * nn);
    int32_t word = 0;
    CB_CHECK(cudaMemcpyAsync(hr.data(), ratio, 2 * nn * sizeof(double), cudaMemcpyDeviceToHost, st));
    CB_CHECK(cudaMemcpyAsync(&word, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CB_CHECK(cudaStreamSynchronize(st));
#undef CB_CHECK
    double mx = 0.0;
    for (double v : hr) mx = std::max(mx, v);
    if (ratio_max) *ratio_max = mx;
    if (word & SUPERDC_DEV_NONFINITE) return SUPERDC_ERR_NONFINITE;
    return SUPERDC_OK;
}

}  // namespace

// Leaves above 128 rows (superdc_build_hss): every such leaf block is turned
// into a subtree with leaves of at most 128 rows whose top basis is the leaf's
// U, by the compression above applied to the leaf block with U as exact
// columns; it must be exact at rank r (relative projection residual of every
// sample at most 1e-12, as for the banded and tridiagonal leaf blocks of
// Section 5's Examples 1-2), else SUPERDC_ERR_ARG.  Outputs the refined tree
// and generators in new device arrays (freed by the caller with cudaFree).
superdc_status refine_leaves(const superdc_tree *tree, const double *D, const double *U, const double *R,
                             const double *B, cudaStream_t st, std::vector<int32_t> &lch2,
                             std::vector<int32_t> &rch2, std::vector<int64_t> &lsize2, double **D2, double **U2,
                             double **R2, double **B2)
{
    const int nn = tree->nnodes, r = tree->rank;
    // the big leaves' common size and their subtree shape
    int64_t M = 0;
    for (int i = 0; i < nn; i++)
        if (tree->lchild[i] < 0) {
            if (M == 0) M = tree->leaf_size[i];
            else if (tree->leaf_size[i] != M) return SUPERDC_ERR_ARG;
        }
    int k = 0;
    while ((M >> k) > 128) k++;
    const int64_t ms = M >> k;
    if ((ms << k) != M || ms < r || M > 4096) return SUPERDC_ERR_ARG;
    const int nsub = 1 << k, nloc = 2 * nsub - 1;
    const PTree lt = make_ptree(M, (int)ms);
    // the new tree: every leaf i becomes the root of a copy of lt
    std::vector<int> newid(nn, -1);
    std::vector<std::pair<int, int>> origin;         // new node -> (old leaf or -1, local id) / old internal
    lch2.clear(); rch2.clear(); lsize2.clear();
    std::vector<int> leafidx(nn, -1);
    int nleaves = 0;
    for (int i = 0; i < nn; i++) {
        if (tree->lchild[i] < 0) {
            leafidx[i] = nleaves++;
            const int base = (int)lch2.size();
            for (int j = 0; j < nloc; j++) {
                lch2.push_back(lt.lch[j] < 0 ? -1 : base + lt.lch[j]);
                rch2.push_back(lt.rch[j] < 0 ? -1 : base + lt.rch[j]);
                lsize2.push_back(lt.lsize[j]);
                origin.push_back({i, j});
            }
            newid[i] = base + nloc - 1;
        } else {
            lch2.push_back(newid[tree->lchild[i]]);
            rch2.push_back(newid[tree->rchild[i]]);
            lsize2.push_back(0);
            origin.push_back({i, -1});
            newid[i] = (int)lch2.size() - 1;
        }
    }
    const int nn2 = (int)lch2.size();
    const size_t rr = (size_t)r * r;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    chk(sdc_malloc(D2, (size_t)nleaves * nsub * ms * ms * sizeof(double)));
    chk(sdc_malloc(U2, (size_t)nleaves * M * r * sizeof(double)));
    chk(sdc_malloc(R2, (size_t)nn2 * rr * sizeof(double)));
    chk(sdc_malloc(B2, (size_t)nn2 * rr * sizeof(double)));
    double *lR = nullptr, *lB = nullptr, *Om = nullptr;
    const int s = std::min(64 - r, r + 10);
    chk(sdc_malloc(&lR, (size_t)nleaves * nloc * rr * sizeof(double)));
    chk(sdc_malloc(&lB, (size_t)nleaves * nloc * rr * sizeof(double)));
    chk(sdc_malloc(&Om, (size_t)M * s * sizeof(double)));
    auto cleanup = [&]() {
        cudaFree(lR); cudaFree(lB); cudaFree(Om);
    };
    if (e != cudaSuccess) {
        cleanup(); cudaFree(*D2); cudaFree(*U2); cudaFree(*R2); cudaFree(*B2);
        return e == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA;
    }
    k_gauss<<<(unsigned)(sdc_num_sms() * 4), 256, 0, st>>>((int64_t)M * s, 0x5DC0FFEEull, Om);
    superdc_status status = SUPERDC_OK;
    double worst = 0.0;
    // leaf blocks in postorder = left to right
    int64_t doff = 0, uoff = 0;
    for (int i = 0; i < nn && status == SUPERDC_OK; i++) {
        if (tree->lchild[i] >= 0) continue;
        const int li = leafidx[i];
        EntrySrc src{0, D + doff, M, nullptr, 0.0};
        CompressOut co{*D2 + (size_t)li * nsub * ms * ms, *U2 + (size_t)li * M * r, lR + (size_t)li * nloc * rr,
                       lB + (size_t)li * nloc * rr};
        double ratio = 0.0;
        status = compress_core(src, M, (int)ms, r, Om, s, U + uoff, M, r, co, &ratio, st);
        worst = std::max(worst, ratio);
        doff += M * M;
        uoff += M * r;
    }
    if (status == SUPERDC_OK && !(worst <= 1e-12)) status = SUPERDC_ERR_ARG;
    if (status == SUPERDC_OK) {
        // R, B of the new nodes: the old ones for the old nodes (a refined leaf
        // keeps its own R, B), the local ones inside the subtrees
        for (int j = 0; j < nn2 && e == cudaSuccess; j++) {
            const int oi = origin[j].first, lj = origin[j].second;
            if (lj < 0 || lj == nloc - 1) {
                chk(cudaMemcpyAsync(*R2 + j * rr, R + (size_t)oi * rr, rr * sizeof(double), cudaMemcpyDeviceToDevice, st));
                chk(cudaMemcpyAsync(*B2 + j * rr, B + (size_t)oi * rr, rr * sizeof(double), cudaMemcpyDeviceToDevice, st));
            } else {
                const size_t lo = ((size_t)leafidx[oi] * nloc + lj) * rr;
                chk(cudaMemcpyAsync(*R2 + j * rr, lR + lo, rr * sizeof(double), cudaMemcpyDeviceToDevice, st));
                chk(cudaMemcpyAsync(*B2 + j * rr, lB + lo, rr * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
        }
        chk(cudaStreamSynchronize(st));
        if (e != cudaSuccess) status = SUPERDC_ERR_CUDA;
    }
    cleanup();
    if (status != SUPERDC_OK) {
        cudaFree(*D2); cudaFree(*U2); cudaFree(*R2); cudaFree(*B2);
        *D2 = *U2 = *R2 = *B2 = nullptr;
    }
    return status;
}

extern "C" superdc_status superdc_build_hss_compress(int64_t n, int32_t leaf, int32_t rank,
                                                     const superdc_matrix_entries *src, const double *Omega,
                                                     int32_t nsamp, cudaStream_t st, superdc_hss **out,
                                                     double *err_est)
{
    if (!src || !Omega || !out || n < 2 || leaf < 1 || leaf > 128 || rank < 1 || rank > 32 || nsamp < rank ||
        nsamp > 64)
        return SUPERDC_ERR_ARG;
    if (src->kind < 0 || src->kind > 2) return SUPERDC_ERR_ARG;
    if (src->kind == 0 && (!src->A || src->lda < n)) return SUPERDC_ERR_ARG;
    if (src->kind != 0 && !src->x) return SUPERDC_ERR_ARG;
    if (src->kind == 2 && !(src->param > 0.0)) return SUPERDC_ERR_ARG;
    const int64_t nleaves = n / leaf;
    if (nleaves * leaf != n || nleaves < 2 || (nleaves & (nleaves - 1)) != 0 || rank > leaf) return SUPERDC_ERR_ARG;
    const int r = rank, m = leaf;
    const PTree pt = make_ptree(n, m);
    const int nn = pt.nn;
    SdcScratch sc(st);
    double *D = nullptr, *Up = nullptr, *Rg = nullptr, *Bg = nullptr;
    SDC_CHECK(sc.get(&D, (size_t)nleaves * m * m));
    SDC_CHECK(sc.get(&Up, (size_t)n * r));
    SDC_CHECK(sc.get(&Rg, (size_t)nn * r * r));
    SDC_CHECK(sc.get(&Bg, (size_t)nn * r * r));
    EntrySrc e{src->kind, src->A, src->lda, src->x, src->param};
    double ratio = 0.0;
    superdc_status s0 = compress_core(e, n, m, r, Omega, nsamp, nullptr, 0, 0, CompressOut{D, Up, Rg, Bg}, &ratio, st);
    if (s0 != SUPERDC_OK) return s0;
    superdc_tree tree;
    tree.n = n;
    tree.nnodes = nn;
    tree.lchild = pt.lch.data();
    tree.rchild = pt.rch.data();
    tree.leaf_size = pt.lsize.data();
    tree.rank = r;
    superdc_status s1 = superdc_build_hss(&tree, D, Up, Rg, Bg, st, out);   // synchronises the stream
    if (err_est) *err_est = ratio;
    return s1;
}
