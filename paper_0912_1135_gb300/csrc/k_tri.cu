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

// Solves op(T) X = B for TRSM_NB columns of B per CTA, in blocks of 32 rows: warp 0
// solves the 32 x 32 diagonal block with register shuffles, then all threads subtract
// that block's contribution from the rows still to be solved. Two barriers per block.
template <bool lower>
__global__ void __launch_bounds__(TRSM_THREADS) trsm_kernel(const double* T, int64_t t_rs, int64_t t_cs, int m,
                                                            double* B, int64_t b_rs, int ncols, int* status) {
    extern __shared__ double x[];   // m * TRSM_NB
    const int j0 = blockIdx.x * TRSM_NB;
    const int nc = min(TRSM_NB, ncols - j0);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int e = t; e < m * TRSM_NB; e += TRSM_THREADS) {
        const int i = e / TRSM_NB, jj = e % TRSM_NB;
        x[e] = jj < nc ? B[(int64_t)i * b_rs + j0 + jj] : 0.0;
    }
    __syncthreads();
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    for (int bi = 0; bi < nblk; ++bi) {
        // block rows [r0, r0 + bs)
        const int blk = lower ? bi : nblk - 1 - bi;
        const int r0 = blk * TRSM_BS;
        const int bs = min(TRSM_BS, m - r0);
        if (warp == 0) {
            // lane holds row r0 + lane of the block: its 4 right-hand-side values and its
            // row of the diagonal block T(r0 + lane, r0 + 0..bs)
            double xv[TRSM_NB];
            double trow[TRSM_BS];
            const bool in = lane < bs;
#pragma unroll
            for (int jj = 0; jj < TRSM_NB; ++jj) xv[jj] = in ? x[(r0 + lane) * TRSM_NB + jj] : 0.0;
#pragma unroll
            for (int k = 0; k < TRSM_BS; ++k)
                trow[k] = (in && k < bs) ? T[(int64_t)(r0 + lane) * t_rs + (int64_t)(r0 + k) * t_cs] : 0.0;
#pragma unroll
            for (int step = 0; step < TRSM_BS; ++step) {
                const int i = lower ? step : TRSM_BS - 1 - step;
                if (i < bs) {
                    if (lane == i) {
                        double d = trow[i];
                        if (!(d != 0.0) || !isfinite(d)) {
                            set_status(status, RTPROJ_ENONFINITE);
                            d = 1.0;
                        }
#pragma unroll
                        for (int jj = 0; jj < TRSM_NB; ++jj) xv[jj] /= d;
                    }
                    double xi[TRSM_NB];
#pragma unroll
                    for (int jj = 0; jj < TRSM_NB; ++jj) xi[jj] = __shfl_sync(0xffffffffu, xv[jj], i);
                    const bool after = lower ? (lane > i) : (lane < i);
                    if (after && in) {
#pragma unroll
                        for (int jj = 0; jj < TRSM_NB; ++jj) xv[jj] = fma(-trow[i], xi[jj], xv[jj]);
                    }
                }
            }
            if (in) {
#pragma unroll
                for (int jj = 0; jj < TRSM_NB; ++jj) x[(r0 + lane) * TRSM_NB + jj] = xv[jj];
            }
        }
        __syncthreads();
        // rows not yet solved: below the block (lower) or above it (upper)
        const int rbeg = lower ? r0 + bs : 0;
        const int rend = lower ? m : r0;
        for (int r = rbeg + t; r < rend; r += TRSM_THREADS) {
            double acc[TRSM_NB];
#pragma unroll
            for (int jj = 0; jj < TRSM_NB; ++jj) acc[jj] = x[r * TRSM_NB + jj];
            const double* trow = T + (int64_t)r * t_rs + (int64_t)r0 * t_cs;
            if (bs == TRSM_BS) {
                // full block: issue the 32 loads of T's row segment before the FMAs
#pragma unroll
                for (int k0 = 0; k0 < TRSM_BS; k0 += 8) {
                    double tv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) tv[q] = trow[(int64_t)(k0 + q) * t_cs];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
#pragma unroll
                        for (int jj = 0; jj < TRSM_NB; ++jj)
                            acc[jj] = fma(-tv[q], x[(r0 + k0 + q) * TRSM_NB + jj], acc[jj]);
                }
            } else {
                for (int k = 0; k < bs; ++k) {
                    const double tv = trow[(int64_t)k * t_cs];
#pragma unroll
                    for (int jj = 0; jj < TRSM_NB; ++jj) acc[jj] = fma(-tv, x[(r0 + k) * TRSM_NB + jj], acc[jj]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < TRSM_NB; ++jj) x[r * TRSM_NB + jj] = acc[jj];
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
        for (int r = c + 1 + t; r < nb; r += blockDim.x) a[r][c] /= a[c][c];
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
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        L[i][j] = X[(int64_t)(p0 + i) * m + p0 + j];
    }
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
            x[c] = s / L[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < CH_NB; ++c)
        if (c < nb) row[c] = x[c];
}

}  // namespace

cudaError_t trsm(const double* T, int64_t t_rs, int64_t t_cs, bool lower, int m,
                 double* Bm, int64_t b_rs, int ncols, int* status, cudaStream_t s) {
    if (m <= 0 || ncols <= 0) return cudaSuccess;
    const size_t smem = (size_t)m * TRSM_NB * sizeof(double);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)((ncols + TRSM_NB - 1) / TRSM_NB);
    if (lower) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(trsm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        trsm_kernel<true><<<grid, TRSM_THREADS, smem, s>>>(T, t_rs, t_cs, m, Bm, b_rs, ncols, status);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(trsm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        trsm_kernel<false><<<grid, TRSM_THREADS, smem, s>>>(T, t_rs, t_cs, m, Bm, b_rs, ncols, status);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t cholesky(double* X, int m, double* part, size_t part_elems, int* status, cudaStream_t s) {
    for (int p0 = 0; p0 < m; p0 += CH_NB) {
        const int nb = std::min(CH_NB, m - p0);
        chol_diag_kernel<<<1, 256, 0, s>>>(X, m, p0, nb, status);
        note_launch();
        const int rest = m - p0 - nb;
        if (rest <= 0) break;
        chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(X, m, p0, nb);
        note_launch();
        Gemm64 g;
        g.M = rest; g.N = rest; g.K = nb;
        g.A = X + (int64_t)(p0 + nb) * m + p0; g.a_rs = m; g.a_cs = 1;
        g.B = X + (int64_t)(p0 + nb) * m + p0; g.b_rs = 1; g.b_cs = m;
        g.C = X + (int64_t)(p0 + nb) * m + (p0 + nb); g.c_rs = m; g.c_cs = 1;
        g.alpha = -1.0; g.beta = 1.0;
        g.Cin = g.C; g.cin_rs = m; g.cin_cs = 1;
        g.lower_only = true;
        cudaError_t e = gemm64(g, part, part_elems, s);
        if (e != cudaSuccess) return e;
    }
    return zero_upper(X, m, s);
}

}  // namespace rtp
