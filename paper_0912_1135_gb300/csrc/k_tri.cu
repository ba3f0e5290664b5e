// Triangular solves and the Cholesky factorization of X (float64, FP64 pipe).
//
// Section 4 forms Y = X^{-1} explicitly (Eq. 16). This library factors X = L L^*
// instead (X is symmetric positive definite with kappa(X) = kappa(P^{-1}A)^2, small)
// and folds R and L into T1 = L^{-1} R^{-*}, so that steps 3-5 of the apply become
// two dense triangular products: P^{-*} Y P^{-1} c = Pi^* T1^* T1 Pi c.
#include "rtproj_internal.cuh"

#include <algorithm>

namespace rtp {
namespace {

constexpr int TRSM_NB = 4;        // right-hand-side columns per CTA
constexpr int TRSM_THREADS = 256;
constexpr int TRSM_BS = 32;       // rows per diagonal block

// Inverse of each 32 x 32 diagonal block of T (lower or upper), one warp per block:
// lane j forms column j by substitution. Dinv[b] is row-major 32 x 32.
template <bool lower>
__global__ void tri_diag_inv_kernel(const double* T, int64_t t_rs, int64_t t_cs, int m, double* Dinv, int* status) {
    const int b = blockIdx.x, j = threadIdx.x;
    const int r0 = b * TRSM_BS;
    const int bs = min(TRSM_BS, m - r0);
    double* out = Dinv + (size_t)b * TRSM_BS * TRSM_BS;
    double col[TRSM_BS];
#pragma unroll
    for (int i = 0; i < TRSM_BS; ++i) col[i] = 0.0;
    auto D = [&](int i, int k) { return T[(int64_t)(r0 + i) * t_rs + (int64_t)(r0 + k) * t_cs]; };
    if (j < bs) {
        if (lower) {
#pragma unroll
            for (int i = 0; i < TRSM_BS; ++i) {
                if (i < j || i >= bs) continue;
                double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < TRSM_BS; ++k)
                    if (k >= j && k < i) s = fma(-D(i, k), col[k], s);
                double d = D(i, i);
                if (!(d != 0.0) || !isfinite(d)) { set_status(status, RTPROJ_ENONFINITE); d = 1.0; }
                col[i] = s / d;
            }
        } else {
#pragma unroll
            for (int ii = TRSM_BS - 1; ii >= 0; --ii) {
                const int i = ii;
                if (i > j) continue;
                double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < TRSM_BS; ++k)
                    if (k > i && k <= j) s = fma(-D(i, k), col[k], s);
                double d = D(i, i);
                if (!(d != 0.0) || !isfinite(d)) { set_status(status, RTPROJ_ENONFINITE); d = 1.0; }
                col[i] = s / d;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < TRSM_BS; ++i) out[i * TRSM_BS + j] = col[i];
}

// Solves op(T) X = B for TRSM_NB columns of B per CTA, block by block: the 32 rows of a
// diagonal block are obtained at once from the precomputed block inverse (a small
// matrix product, no sequential chain), then all threads subtract that block's
// contribution from the rows still to be solved. Three barriers per block.
template <bool lower>
__global__ void __launch_bounds__(TRSM_THREADS) trsm_kernel(const double* T, int64_t t_rs, int64_t t_cs, int m,
                                                            double* B, int64_t b_rs, int ncols, const double* Dinv) {
    extern __shared__ double x[];   // m * TRSM_NB
    const int j0 = blockIdx.x * TRSM_NB;
    const int nc = min(TRSM_NB, ncols - j0);
    const int t = threadIdx.x;
    for (int e = t; e < m * TRSM_NB; e += TRSM_THREADS) {
        const int i = e / TRSM_NB, jj = e % TRSM_NB;
        x[e] = jj < nc ? B[(int64_t)i * b_rs + j0 + jj] : 0.0;
    }
    __syncthreads();
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    for (int bi = 0; bi < nblk; ++bi) {
        const int blk = lower ? bi : nblk - 1 - bi;
        const int r0 = blk * TRSM_BS;
        const int bs = min(TRSM_BS, m - r0);
        // x_blk = Dinv_blk x_blk
        double y = 0.0;
        const int i = t / TRSM_NB, jj = t % TRSM_NB;
        const bool act = t < TRSM_BS * TRSM_NB && i < bs;
        if (act) {
            const double* drow = Dinv + (size_t)blk * TRSM_BS * TRSM_BS + (size_t)i * TRSM_BS;
#pragma unroll 8
            for (int k = 0; k < TRSM_BS; ++k)
                if (k < bs) y = fma(drow[k], x[(r0 + k) * TRSM_NB + jj], y);
        }
        __syncthreads();
        if (act) x[(r0 + i) * TRSM_NB + jj] = y;
        __syncthreads();
        // rows not yet solved: below the block (lower) or above it (upper)
        const int rbeg = lower ? r0 + bs : 0;
        const int rend = lower ? m : r0;
        for (int r = rbeg + t; r < rend; r += TRSM_THREADS) {
            double acc[TRSM_NB];
#pragma unroll
            for (int q = 0; q < TRSM_NB; ++q) acc[q] = x[r * TRSM_NB + q];
            const double* trow = T + (int64_t)r * t_rs + (int64_t)r0 * t_cs;
            if (bs == TRSM_BS) {
#pragma unroll
                for (int k0 = 0; k0 < TRSM_BS; k0 += 8) {
                    double tv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) tv[q] = trow[(int64_t)(k0 + q) * t_cs];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
#pragma unroll
                        for (int c = 0; c < TRSM_NB; ++c)
                            acc[c] = fma(-tv[q], x[(r0 + k0 + q) * TRSM_NB + c], acc[c]);
                }
            } else {
                for (int k = 0; k < bs; ++k) {
                    const double tv = trow[(int64_t)k * t_cs];
#pragma unroll
                    for (int c = 0; c < TRSM_NB; ++c) acc[c] = fma(-tv, x[(r0 + k) * TRSM_NB + c], acc[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < TRSM_NB; ++c) x[r * TRSM_NB + c] = acc[c];
        }
        __syncthreads();
    }
    for (int e = t; e < m * TRSM_NB; e += TRSM_THREADS) {
        const int i = e / TRSM_NB, jj = e % TRSM_NB;
        if (jj < nc) B[(int64_t)i * b_rs + j0 + jj] = x[e];
    }
}

constexpr int CH_NB = 32;

// Unblocked Cholesky of the nb x nb diagonal block at (p0, p0), in shared memory.
__global__ void chol_diag_kernel(double* X, int m, int p0, int nb, int* status) {
    __shared__ double a[CH_NB][CH_NB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        a[i][j] = X[(int64_t)(p0 + i) * m + p0 + j];
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        if (t == 0) {
            double d = a[c][c];
            if (!(d > 0.0) || !isfinite(d)) {
                set_status(status, RTPROJ_ENOTSPD);
                d = 1.0;
            }
            a[c][c] = sqrt(d);
        }
        __syncthreads();
        const double inv = 1.0 / a[c][c];
        for (int r = c + 1 + t; r < nb; r += blockDim.x) a[r][c] *= inv;
        __syncthreads();
        for (int e = t; e < nb * nb; e += blockDim.x) {
            const int r = e / nb, q = e % nb;
            if (q > c && r >= q) a[r][q] = fma(-a[r][c], a[q][c], a[r][q]);
        }
        __syncthreads();
    }
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        X[(int64_t)(p0 + i) * m + p0 + j] = (j <= i) ? a[i][j] : 0.0;
    }
}

// Rows below the diagonal block: x L_pp^* = X[r][p0..p0+nb), one thread per row.
__global__ void chol_panel_kernel(double* X, int m, int p0, int nb) {
    __shared__ double L[CH_NB][CH_NB + 1];
    __shared__ double inv[CH_NB];
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        L[i][j] = X[(int64_t)(p0 + i) * m + p0 + j];
    }
    __syncthreads();
    if (t < nb) inv[t] = 1.0 / L[t][t];
    __syncthreads();
    const int r = p0 + nb + blockIdx.x * blockDim.x + t;
    if (r >= m) return;
    double x[CH_NB];
    double* row = X + (int64_t)r * m + p0;
#pragma unroll
    for (int c = 0; c < CH_NB; ++c) x[c] = c < nb ? row[c] : 0.0;
#pragma unroll
    for (int c = 0; c < CH_NB; ++c) {
        if (c < nb) {
            double s = x[c];
#pragma unroll
            for (int q = 0; q < CH_NB; ++q)
                if (q < c) s = fma(-x[q], L[c][q], s);
            x[c] = s * inv[c];
        }
    }
#pragma unroll
    for (int c = 0; c < CH_NB; ++c)
        if (c < nb) row[c] = x[c];
}

// Trailing update of the blocked Cholesky: X[r][q] -= sum_t L[r][p0+t] L[q][p0+t] for
// p0 + nb <= q <= r < m, on 32 x 32 tiles of the lower triangle (one CTA per tile).
__global__ void __launch_bounds__(256) chol_update_kernel(double* X, int m, int p0, int nb) {
    __shared__ double Pr[32][CH_NB + 1];
    __shared__ double Pq[32][CH_NB + 1];
    const int base = p0 + nb;
    // tile index -> (tr, tq), tq <= tr
    int u = blockIdx.x, tr = 0;
    while (u > tr) { u -= tr + 1; ++tr; }
    const int tq = u;
    const int r0 = base + tr * 32, q0 = base + tq * 32;
    const int t = threadIdx.x;
    for (int e = t; e < 32 * nb; e += 256) {
        const int i = e / nb, c = e % nb;
        Pr[i][c] = (r0 + i < m) ? X[(int64_t)(r0 + i) * m + p0 + c] : 0.0;
        Pq[i][c] = (q0 + i < m) ? X[(int64_t)(q0 + i) * m + p0 + c] : 0.0;
    }
    __syncthreads();
    const int i = t >> 3, jb = (t & 7) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < nb; ++c) {
        const double a = Pr[i][c];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(a, Pq[jb + q][c], acc[q]);
    }
    const int r = r0 + i;
    if (r >= m) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int col = q0 + jb + q;
        if (col < m && col <= r) X[(int64_t)r * m + col] -= acc[q];
    }
}

}  // namespace

cudaError_t trsm(const double* T, int64_t t_rs, int64_t t_cs, bool lower, int m,
                 double* Bm, int64_t b_rs, int ncols, double* dinv_work, int* status, cudaStream_t s) {
    if (m <= 0 || ncols <= 0) return cudaSuccess;
    const size_t smem = (size_t)m * TRSM_NB * sizeof(double);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    const unsigned grid = (unsigned)((ncols + TRSM_NB - 1) / TRSM_NB);
    if (lower) {
        tri_diag_inv_kernel<true><<<nblk, TRSM_BS, 0, s>>>(T, t_rs, t_cs, m, dinv_work, status);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(trsm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        trsm_kernel<true><<<grid, TRSM_THREADS, smem, s>>>(T, t_rs, t_cs, m, Bm, b_rs, ncols, dinv_work);
    } else {
        tri_diag_inv_kernel<false><<<nblk, TRSM_BS, 0, s>>>(T, t_rs, t_cs, m, dinv_work, status);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(trsm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        trsm_kernel<false><<<grid, TRSM_THREADS, smem, s>>>(T, t_rs, t_cs, m, Bm, b_rs, ncols, dinv_work);
    }
    note_launch(2);
    return cudaGetLastError();
}

size_t trsm_work_doubles(int m) { return (size_t)((m + TRSM_BS - 1) / TRSM_BS) * TRSM_BS * TRSM_BS; }

cudaError_t cholesky(double* X, int m, double* part, size_t part_elems, int* status, cudaStream_t s) {
    for (int p0 = 0; p0 < m; p0 += CH_NB) {
        const int nb = std::min(CH_NB, m - p0);
        chol_diag_kernel<<<1, 256, 0, s>>>(X, m, p0, nb, status);
        note_launch();
        const int rest = m - p0 - nb;
        if (rest <= 0) break;
        chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(X, m, p0, nb);
        note_launch();
        const int nt = (rest + 31) / 32;
        chol_update_kernel<<<nt * (nt + 1) / 2, 256, 0, s>>>(X, m, p0, nb);
        note_launch();
    }
    (void)part;
    (void)part_elems;
    return zero_upper(X, m, s);
}

}  // namespace rtp
