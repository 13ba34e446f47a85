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
        double next = 0.0;
        for (int a = 0; a < s; a++)
            if (!used[a]) next = fmax(next, G[a + RS * a]);
        const double l1 = fmax(G[s_top[0] + RS * s_top[0]], 0.0);
        ratio[b] = (s > r && l1 > 0.0) ? sqrt(fmax(next, 0.0) / l1) : 0.0;
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

}  // namespace

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
    int L = 0;
    while ((int64_t(1) << L) < nleaves) L++;
    const int r = rank, s = nsamp, m = leaf;
    EntrySrc e{src->kind, src->A, src->lda, src->x, src->param};
    // perfect tree in postorder: node ids by level, level l has 2^l nodes left to right
    std::vector<std::vector<int>> lev(L + 1);
    const int nn = 2 * (int)nleaves - 1;
    std::vector<int32_t> lch(nn, -1), rch(nn, -1);
    std::vector<int64_t> lsize(nn, 0), off(nn, 0), sz(nn, 0);
    {
        int counter = 0;
        std::function<int(int, int64_t)> build = [&](int l, int64_t o) -> int {
            if (l == L) {
                const int id = counter++;
                lsize[id] = m; off[id] = o; sz[id] = m; lev[l].push_back(id);
                return id;
            }
            const int64_t half = (int64_t)m << (L - l - 1);
            const int a = build(l + 1, o), b2 = build(l + 1, o + half);
            const int id = counter++;
            lch[id] = a; rch[id] = b2; off[id] = o; sz[id] = 2 * half; lev[l].push_back(id);
            return id;
        };
        build(0, 0);
    }
    SdcScratch sc(st);
    const int nsplit_full = 8;
#define CB_CHECK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) \
        return e_ == cudaErrorMemoryAllocation ? SUPERDC_ERR_OOM : SUPERDC_ERR_CUDA; } while (0)
    double *Y = nullptr, *Yoff = nullptr, *D = nullptr, *Ul = nullptr, *Rg = nullptr, *Bg = nullptr;
    double *P = nullptr, *W = nullptr, *Vb = nullptr, *Ub0 = nullptr, *Ub1 = nullptr, *T = nullptr, *ratio = nullptr;
    int32_t *status = nullptr;
    CB_CHECK(sc.get(&Y, (size_t)n * s));
    CB_CHECK(sc.get(&Yoff, (size_t)n * s));
    CB_CHECK(sc.get(&D, (size_t)nleaves * m * m));
    CB_CHECK(sc.get(&Ul, (size_t)n * r));
    CB_CHECK(sc.get(&Rg, (size_t)nn * r * r));
    CB_CHECK(sc.get(&Bg, (size_t)nn * r * r));
    CB_CHECK(sc.get(&P, (size_t)nn * r * s));
    CB_CHECK(sc.get(&W, (size_t)nn * r * s));
    CB_CHECK(sc.get(&Vb, (size_t)nn * 2 * r * s));
    CB_CHECK(sc.get(&Ub0, (size_t)n * r));
    CB_CHECK(sc.get(&Ub1, (size_t)n * r));
    CB_CHECK(sc.get(&T, (size_t)n * r));
    double *Rtmp = nullptr;
    CB_CHECK(sc.get(&ratio, 2 * (size_t)nn));
    CB_CHECK(sc.get(&Rtmp, (size_t)nn * 2 * r * r));
    CB_CHECK(sc.get(&status, 1));
    CB_CHECK(cudaMemsetAsync(Rg, 0, (size_t)nn * r * r * sizeof(double), st));
    CB_CHECK(cudaMemsetAsync(Bg, 0, (size_t)nn * r * r * sizeof(double), st));
    CB_CHECK(cudaMemsetAsync(ratio, 0, 2 * (size_t)nn * sizeof(double), st));
    int64_t roff = nleaves;      // ratio slots: leaves first, then every level's nodes
    CB_CHECK(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    const size_t rsm = (size_t)(RQ * RS + 2 * RS * RS + RQ * 32) * sizeof(double);
    CB_CHECK(cudaFuncSetAttribute(k_range, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    // 1. Y = A Omega (row tiles, 8 column splits)
    {
        std::vector<int64_t> r0{0}, nr{n}, c0{0}, nc{n}, mo{0}, orow{0};
        CB_CHECK(block_products(e, r0, nr, c0, nc, mo, orow, n, Omega, n, s, Y, n, 1.0, nullptr, nsplit_full, sc, st));
    }
    // 2. leaves: Y_off = Y - A(I,I) Omega(I); D blocks; U = range(Y_off)
    {
        std::vector<int64_t> r0, nr, c0, nc, mo, orow;
        for (int64_t k = 0; k < nleaves; k++) {
            r0.push_back(k * m); nr.push_back(m); c0.push_back(k * m); nc.push_back(m);
            mo.push_back(k * m); orow.push_back(k * m);
        }
        CB_CHECK(block_products(e, r0, nr, c0, nc, mo, orow, n, Omega, n, s, Yoff, n, -1.0, Y, 1, sc, st));
        k_leaf_blocks<<<(unsigned)(sdc_num_sms() * 8), 256, 0, st>>>(e, (int)nleaves, m, D);
        std::vector<int64_t> hmo, huo;
        for (int64_t k = 0; k < nleaves; k++) { hmo.push_back(k * m); huo.push_back(k * m); }
        int64_t *tab = nullptr;
        CB_CHECK(sc.get(&tab, 2 * (size_t)nleaves));
        std::vector<int64_t> h(hmo);
        h.insert(h.end(), huo.begin(), huo.end());
        CB_CHECK(cudaMemcpyAsync(tab, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
        CB_CHECK(cudaStreamSynchronize(st));
        k_range<<<(unsigned)nleaves, 256, rsm, st>>>(tab, tab + nleaves, Yoff, n, m, s, r, Ul, n, ratio, status);
        CB_CHECK(cudaGetLastError());
        CB_CHECK(cudaMemcpyAsync(Ub0, Ul, (size_t)n * r * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // P_leaf = U^T Y_off(I), W_leaf = U^T Omega(I)   (r x s, per leaf at node id * r * s)
        std::vector<int64_t> ao, bo, co;
        for (int64_t k = 0; k < nleaves; k++) {
            ao.push_back(k * m); bo.push_back(k * m); co.push_back((int64_t)lev[L][k] * r * s);
        }
        int64_t *mt = nullptr;
        CB_CHECK(sc.get(&mt, 3 * (size_t)nleaves));
        std::vector<int64_t> hh(ao);
        hh.insert(hh.end(), bo.begin(), bo.end());
        hh.insert(hh.end(), co.begin(), co.end());
        CB_CHECK(cudaMemcpyAsync(mt, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice, st));
        CB_CHECK(cudaStreamSynchronize(st));
        SmallMM o{mt, mt + nleaves, mt + 2 * nleaves};
        k_small_mm<<<(unsigned)nleaves, 256, 0, st>>>(o, Ul, n, Yoff, n, P, r, r, s, m, 1, 1.0, 0.0);
        k_small_mm<<<(unsigned)nleaves, 256, 0, st>>>(o, Ul, n, Omega, n, W, r, r, s, m, 1, 1.0, 0.0);
        CB_CHECK(cudaGetLastError());
    }
    // 3. up the tree: level l's nodes from their children's bases (Ub0: the
    // children's explicit bases, rows at their offsets)
    for (int l = L - 1; l >= 0; l--) {
        const std::vector<int> &nodes = lev[l];
        const int nl = (int)nodes.size();
        // B_c1 = U_c1^T (A(I_c1, I_c2) U_c2)
        {
            std::vector<int64_t> r0, nr, c0, nc, mo, orow;
            for (int i : nodes) {
                const int a = lch[i], b2 = rch[i];
                r0.push_back(off[a]); nr.push_back(sz[a]); c0.push_back(off[b2]); nc.push_back(sz[b2]);
                mo.push_back(off[b2]); orow.push_back(off[a]);
            }
            const int nsp = std::max(1, (int)std::min<int64_t>(8, sz[lch[nodes[0]]] / 1024));
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
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(o, Ub0, n, T, n, Bg, r, r, r, (int)sz[lch[nodes[0]]], 1, 1.0, 0.0);
            CB_CHECK(cudaGetLastError());
        }
        if (l == 0) break;
        // V = [P_c1 - B_c1 W_c2; P_c2 - B_c1^T W_c1]  (2r x s per node at node id * 2 r s)
        {
            std::vector<int64_t> h1, h2;
            // first block rows: C = P_c1 - B_c1 W_c2
            std::vector<int64_t> ao, bo, co, ao2, bo2, co2;
            for (int i : nodes) {
                const int a = lch[i], b2 = rch[i];
                ao.push_back((int64_t)a * r * r); bo.push_back((int64_t)b2 * r * s); co.push_back((int64_t)i * 2 * r * s);
                ao2.push_back((int64_t)a * r * r); bo2.push_back((int64_t)a * r * s); co2.push_back((int64_t)i * 2 * r * s + r);
            }
            // copy P children into V, then subtract
            std::vector<int64_t> hh(ao);
            hh.insert(hh.end(), bo.begin(), bo.end());
            hh.insert(hh.end(), co.begin(), co.end());
            hh.insert(hh.end(), ao2.begin(), ao2.end());
            hh.insert(hh.end(), bo2.begin(), bo2.end());
            hh.insert(hh.end(), co2.begin(), co2.end());
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, hh.size()));
            CB_CHECK(cudaMemcpyAsync(mt, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            // V rows: P_c (r x s, ld r) placed at rows 0..r-1 / r..2r-1 of V (ld 2r)
            for (int i : nodes) {
                const int a = lch[i], b2 = rch[i];
                CB_CHECK(cudaMemcpy2DAsync(Vb + (int64_t)i * 2 * r * s, 2 * r * sizeof(double), P + (int64_t)a * r * s,
                                           r * sizeof(double), r * sizeof(double), s, cudaMemcpyDeviceToDevice, st));
                CB_CHECK(cudaMemcpy2DAsync(Vb + (int64_t)i * 2 * r * s + r, 2 * r * sizeof(double),
                                           P + (int64_t)b2 * r * s, r * sizeof(double), r * sizeof(double), s,
                                           cudaMemcpyDeviceToDevice, st));
            }
            SmallMM o1{mt, mt + nl, mt + 2 * nl};
            SmallMM o2{mt + 3 * nl, mt + 4 * nl, mt + 5 * nl};
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(o1, Bg, r, W, r, Vb, 2 * r, r, s, r, 0, -1.0, 1.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(o2, Bg, r, W, r, Vb, 2 * r, r, s, r, 1, -1.0, 1.0);
            CB_CHECK(cudaGetLastError());
        }
        // [R_c1; R_c2] = range(V) (2r x r, written into Rtmp at node id * 2 r r)
        {
            std::vector<int64_t> h;
            for (int i : nodes) h.push_back((int64_t)i * 2 * r * s);
            for (int i : nodes) h.push_back((int64_t)i * 2 * r * r);
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, h.size()));
            CB_CHECK(cudaMemcpyAsync(mt, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            k_range<<<(unsigned)nl, 256, rsm, st>>>(mt, mt + nl, Vb, 2 * r, 2 * r, s, r, Rtmp, 2 * r,
                                                    ratio + roff, status);
            roff += nl;
            CB_CHECK(cudaGetLastError());
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
            // P_i = R_c1^T V_c1 + R_c2^T V_c2 with V rows of the node (ld 2r)
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)i * 2 * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * r * s);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)i * 2 * r * s + r);
            for (int i : nodes) hh.push_back((int64_t)i * r * s);
            // W_i = R_c1^T W_c1 + R_c2^T W_c2
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)lch[i] * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * r * s);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * r);
            for (int i : nodes) hh.push_back((int64_t)rch[i] * r * s);
            for (int i : nodes) hh.push_back((int64_t)i * r * s);
            // U_i rows: U_c1 R_c1 at off[c1], U_c2 R_c2 at off[c2] (into Ub1, ld n)
            int64_t *mt = nullptr;
            CB_CHECK(sc.get(&mt, hh.size()));
            CB_CHECK(cudaMemcpyAsync(mt, hh.data(), hh.size() * 8, cudaMemcpyHostToDevice, st));
            CB_CHECK(cudaStreamSynchronize(st));
            SmallMM p1{mt, mt + nl, mt + 2 * nl}, p2{mt + 3 * nl, mt + 4 * nl, mt + 5 * nl};
            SmallMM w1{mt + 6 * nl, mt + 7 * nl, mt + 8 * nl}, w2{mt + 9 * nl, mt + 10 * nl, mt + 11 * nl};
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(p1, Rg, r, Vb, 2 * r, P, r, r, s, r, 1, 1.0, 0.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(p2, Rg, r, Vb, 2 * r, P, r, r, s, r, 1, 1.0, 1.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(w1, Rg, r, W, r, W, r, r, s, r, 1, 1.0, 0.0);
            k_small_mm<<<(unsigned)nl, 256, 0, st>>>(w2, Rg, r, W, r, W, r, r, s, r, 1, 1.0, 1.0);
            CB_CHECK(cudaGetLastError());
            std::vector<int64_t> u;
            const int64_t ch = sz[lch[nodes[0]]];
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
    // 4. the handle: leaf bases packed m x r per leaf (they were rows of an n x r matrix)
    double *Up = Yoff;       // Y_off is no longer needed (n x s >= n x r)
    k_pack_leaves<<<(unsigned)(sdc_num_sms() * 8), 256, 0, st>>>(n, m, r, Ul, Up);
    CB_CHECK(cudaGetLastError());
    superdc_tree tree;
    tree.n = n;
    tree.nnodes = nn;
    tree.lchild = lch.data();
    tree.rchild = rch.data();
    tree.leaf_size = lsize.data();
    tree.rank = r;
    // superdc_build_hss reads B as nnodes blocks r x r and R likewise
    superdc_status s1 = superdc_build_hss(&tree, D, Up, Rg, Bg, st, out);   // synchronises the stream
    if (s1 != SUPERDC_OK) return s1;
    std::vector<double> hr(2 * nn);
    int32_t word = 0;
    CB_CHECK(cudaMemcpy(hr.data(), ratio, 2 * nn * sizeof(double), cudaMemcpyDeviceToHost));
    CB_CHECK(cudaMemcpy(&word, status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    double mx = 0.0;
    for (double v : hr) mx = std::max(mx, v);
    if (err_est) *err_est = mx;
#undef CB_CHECK
    if (word & SUPERDC_DEV_NONFINITE) {
        superdc_hss_free(*out);
        *out = nullptr;
        return SUPERDC_ERR_NONFINITE;
    }
    return SUPERDC_OK;
}
