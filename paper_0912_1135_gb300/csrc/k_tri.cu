// Triangular solves and the Cholesky factorization of X: float64 kernels (FP64 pipe) and
// float-float forms of the lower solve and the Cholesky for the mixed form (FP32 pipe).
//
// Section 4 forms Y = X^{-1} explicitly (Eq. 16). This library factors X = L L^*
// instead (X is symmetric positive definite with kappa(X) = kappa(P^{-1}A)^2, small)
// and folds R and L into T1 = L^{-1} R^{-*}, so that steps 3-5 of the apply become
// two dense products with T1: P^{-*} Y P^{-1} c = Pi^* T1^* T1 Pi c (triangular float64
// products in the float64 form, digit-sliced tensor-core products in the mixed form).
#include "rtproj_internal.cuh"
#include "ff.cuh"

#include <algorithm>

namespace rtp {
namespace {

constexpr int TRSM_THREADS = 512;
constexpr int TRSM_BS = 32;       // rows per diagonal block
constexpr int TRSM_DPARTS = 4;    // partial sums per entry of the diagonal-block product (4 warps)

// Inverse of each 32 x 32 diagonal block of T (lower or upper), one CTA of four warps per
// block, in two levels: with the block written lower triangular as D = [A 0; B C] (the
// transpose of an upper block), D^{-1} = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}]. One warp
// inverts A (lanes 0-15) and C (lanes 16-31) at once, lane j forming column j of its
// 16 x 16 block by right-looking substitution (once entry i is known it is removed from
// the rows below, so each float64 instruction is an independent update); then all four
// warps form F = B A^{-1} and -C^{-1} F as small products. The GB300 float64 pipe takes
// 64 cycles per warp instruction, so the 16-step chains and the products spread over four
// sub-partitions cost far less than one warp's 32 x 32 substitution. A block past the
// end of T (bs < 32) is padded with the identity. Dinv[b] is row-major 32 x 32, zero
// outside the block's triangle and outside bs x bs.
constexpr int TDI_THREADS = 128;
template <bool lower>
__global__ void __launch_bounds__(TDI_THREADS) tri_diag_inv_kernel(const double* T, int64_t t_rs, int64_t t_cs,
                                                                   int m, double* Dinv, int* status,
                                                                   const int* run_if) {
    if (run_if && *run_if == 0) return;   // a float-float solve ran instead
    constexpr int H = TRSM_BS / 2;
    __shared__ double a[TRSM_BS][TRSM_BS + 1];     // the block, lower triangular
    __shared__ double inv[TRSM_BS][TRSM_BS + 1];   // its inverse (lower triangle)
    __shared__ double f[H][H + 1];
    __shared__ double rd[TRSM_BS];
    const int b = blockIdx.x, t = threadIdx.x;
    const int r0 = b * TRSM_BS;
    const int bs = min(TRSM_BS, m - r0);
    for (int e = t; e < TRSM_BS * TRSM_BS; e += TDI_THREADS) {
        const int i = e / TRSM_BS, k = e % TRSM_BS;
        double v = i == k ? 1.0 : 0.0;
        if (i < bs && k <= i) {
            const int64_t ti = r0 + (lower ? i : k), tk = r0 + (lower ? k : i);
            v = T[ti * t_rs + tk * t_cs];
        }
        a[i][k] = v;
    }
    __syncthreads();
    if (t < TRSM_BS) {
        double d = a[t][t];
        if (!(d != 0.0) || !isfinite(d)) {
            set_status(status, RTPROJ_ENONFINITE);
            d = 1.0;
        }
        rd[t] = 1.0 / d;
    }
    __syncthreads();
    if (t < TRSM_BS) {   // A^{-1} on lanes 0-15, C^{-1} on lanes 16-31
        const int off = (t / H) * H, jj = t % H;
        double col[H];   // partial sums, then column jj
#pragma unroll
        for (int i = 0; i < H; ++i) col[i] = i == jj ? 1.0 : 0.0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            col[i] = i >= jj ? col[i] * rd[off + i] : 0.0;
#pragma unroll
            for (int r = i + 1; r < H; ++r) col[r] = fma(-a[off + r][off + i], col[i], col[r]);
        }
#pragma unroll
        for (int i = 0; i < H; ++i) inv[off + i][off + jj] = col[i];
    }
    __syncthreads();
    for (int e = t; e < H * H; e += TDI_THREADS) {   // F = B A^{-1} (A^{-1} is zero above its diagonal)
        const int i = e / H, j = e % H;
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int k = 0; k < H; k += 2) {
            s0 = fma(a[H + i][k], inv[k][j], s0);
            s1 = fma(a[H + i][k + 1], inv[k + 1][j], s1);
        }
        f[i][j] = s0 + s1;
    }
    __syncthreads();
    for (int e = t; e < H * H; e += TDI_THREADS) {   // lower-left block -C^{-1} F
        const int i = e / H, j = e % H;
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int k = 0; k < H; k += 2) {
            s0 = fma(inv[H + i][H + k], f[k][j], s0);
            s1 = fma(inv[H + i][H + k + 1], f[k + 1][j], s1);
        }
        inv[H + i][j] = -(s0 + s1);
    }
    __syncthreads();
    double* out = Dinv + (size_t)b * TRSM_BS * TRSM_BS;
    for (int e = t; e < TRSM_BS * TRSM_BS; e += TDI_THREADS) {
        const int i = e / TRSM_BS, j = e % TRSM_BS;
        const int li = lower ? i : j, lj = lower ? j : i;
        out[e] = (i < bs && j < bs && lj <= li) ? inv[li][lj] : 0.0;
    }
}

// Solves op(T) x = b for one column of B at a time. The CTAs (one per SM) take columns
// from a shared counter in increasing order: with a lower-triangular right-hand side the
// first columns carry the most rows, so the longest solves start first and the short ones
// fill in behind them. Per diagonal block: the block's rows are obtained at once from the
// precomputed block inverse (four partial sums per entry on four warps, so the float64
// pipes of all four sub-partitions share the product), then every thread subtracts that
// block's contribution from one row still to be solved, with the 32 entries of its row of
// T loaded before the products. Two barriers per block.
template <bool lower>
__global__ void __launch_bounds__(TRSM_THREADS, 1) trsm_kernel(const double* __restrict__ T, int64_t t_rs, int64_t t_cs,
                                                            int m, double* B, int64_t b_rs, int ncols,
                                                            const double* __restrict__ Dinv, int rhs_lower,
                                                            unsigned int* next_col, const int* run_if) {
    if (run_if && *run_if == 0) return;   // a float-float solve ran instead
    extern __shared__ double x[];   // m: the column being solved
    __shared__ int col_s;
    const int t = threadIdx.x;
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    for (;;) {
        if (t == 0) col_s = (int)atomicAdd(next_col, 1u);
        __syncthreads();
        const int j = col_s;
        if (j >= ncols) break;
        // A lower-triangular right-hand side (zero above its diagonal) gives a lower-triangular
        // solution of a lower system: the rows above column j's diagonal block stay zero.
        const int bi0 = (lower && rhs_lower) ? min(j, m) / TRSM_BS : 0;
        const int row0 = bi0 * TRSM_BS;
        for (int i = row0 + t; i < m; i += TRSM_THREADS) x[i] = B[(int64_t)i * b_rs + j];
        __syncthreads();
        for (int bi = bi0; bi < nblk; ++bi) {
            const int blk = lower ? bi : nblk - 1 - bi;
            const int r0 = blk * TRSM_BS;
            const int bs = min(TRSM_BS, m - r0);
            // x_blk = Dinv_blk x_blk: entry i on lanes 4i .. 4i+3 (k = part, part + 4, ...)
            const int di = t / TRSM_DPARTS, part = t % TRSM_DPARTS;
            double y = 0.0;
            if (t < TRSM_BS * TRSM_DPARTS) {
                const double* drow = Dinv + ((size_t)blk * TRSM_BS + di) * TRSM_BS;
                double y0 = 0.0, y1 = 0.0;
#pragma unroll
                for (int k0 = 0; k0 < TRSM_BS; k0 += 2 * TRSM_DPARTS) {
                    const int k = k0 + part;
                    if (k < bs) y0 = fma(drow[k], x[r0 + k], y0);
                    if (k + TRSM_DPARTS < bs) y1 = fma(drow[k + TRSM_DPARTS], x[r0 + k + TRSM_DPARTS], y1);
                }
                y = y0 + y1;
                y += __shfl_xor_sync(0xffffffffu, y, 1);
                y += __shfl_xor_sync(0xffffffffu, y, 2);
            }
            __syncthreads();
            if (t < TRSM_BS * TRSM_DPARTS && part == 0 && di < bs) x[r0 + di] = y;
            __syncthreads();
            // rows not yet solved: below the block (lower) or above it (upper)
            const int rbeg = lower ? r0 + bs : 0;
            const int rend = lower ? m : r0;
            for (int r = rbeg + t; r < rend; r += TRSM_THREADS) {
                const double* trow = T + (int64_t)r * t_rs + (int64_t)r0 * t_cs;
                double a0 = x[r], a1 = 0.0;
                if (bs == TRSM_BS) {
                    double tv[TRSM_BS];
#pragma unroll
                    for (int k = 0; k < TRSM_BS; ++k) tv[k] = trow[(int64_t)k * t_cs];
#pragma unroll
                    for (int k = 0; k < TRSM_BS; k += 2) {
                        a0 = fma(-tv[k], x[r0 + k], a0);
                        a1 = fma(-tv[k + 1], x[r0 + k + 1], a1);
                    }
                } else {
                    for (int k = 0; k < bs; ++k) a0 = fma(-trow[(int64_t)k * t_cs], x[r0 + k], a0);
                }
                x[r] = a0 + a1;
            }
            __syncthreads();
        }
        for (int i = row0 + t; i < m; i += TRSM_THREADS) B[(int64_t)i * b_rs + j] = x[i];
        __syncthreads();   // x and col_s are reused by the next column
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

// ---------------------------------------------------------------------------------
// Persistent blocked Cholesky: one cooperative launch for all panels of CHP_NB columns.
// Per panel p0: (A) CTA 0 factors the diagonal block in shared memory and forms its
// inverse Z = L_pp^{-1} in the same right-looking sweep (Gauss-Jordan on the identity);
// (B) every warp of the grid solves panel rows: L[r][p0..] = X[r][p0..] Z^*; (C) all CTAs
// update the trailing lower triangle on 16 x 16 tiles, CTA 0 taking the tiles of the next
// diagonal block and factoring it at once (lookahead). A grid-wide counter separates the
// phases; every wait is bounded (RTPROJ_ETIMEOUT).
constexpr int CHP_THREADS = 256;
constexpr int CHP_NB = 16;                 // panel width: the diagonal block's pivots run on one CTA
constexpr int CHP_TILE = 16;

struct CholPDev {
    double* X; int m;
    double* zbuf;            // 32 x 32: Z of the current panel
    unsigned int* counter;
    int* abort_flag;
    int* status;
    long long timeout;
    const int* run_if;       // non-null: run only when *run_if != 0 (the float-float form gave up)
};

__device__ __forceinline__ unsigned int chp_ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `k` (1, 2, ...): returns false when a wait expired or another CTA
// aborted; then every CTA leaves.
__device__ bool chp_grid_sync(const CholPDev& p, unsigned int k, int* ok_s) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(p.counter, 1u);
        const unsigned int target = k * gridDim.x;
        const long long t0 = clock64();
        int ok = 1;
        for (unsigned int it = 1;; ++it) {
            if (chp_ld_acquire(p.counter) >= target) break;
            if (clock64() - t0 > p.timeout) {
                atomicExch(p.abort_flag, 1);
                set_status(p.status, RTPROJ_ETIMEOUT);
                ok = 0;
                break;
            }
            if ((it & 63) == 0 && *(volatile int*)p.abort_flag) { ok = 0; break; }
        }
        *ok_s = ok;
    }
    __syncthreads();
    return *ok_s != 0;
}

// 1 / sqrt(d) for a pivot d: the float32 estimate and one Newton step in float64,
// y <- y (3 - d y^2) / 2, which squares the estimate's relative error (about 2^-45 after
// the step: ample for a preconditioner factor that the refinement corrects). Outside
// [2^-100, 2^100] the float64 library square root is used. A pivot that is not positive
// and finite latches RTPROJ_ENOTSPD and is replaced by 1.
__device__ __forceinline__ double pivot_rsqrt(double d, int* status) {
    const long long bits = __double_as_longlong(d);
    if (!(bits > 0 && bits < 0x7FF0000000000000ll)) {
        set_status(status, RTPROJ_ENOTSPD);
        return 1.0;
    }
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex <= 1023 - 100 || ex >= 1023 + 100) return 1.0 / sqrt(d);
    const double y = (double)rsqrtf((float)d);
    return y * fma(-0.5 * d, y * y, 1.5);
}

// Reciprocal 1/d of a pivot d: the float32 estimate and one Newton step in float64,
// r <- r + r (1 - d r), which squares the estimate's relative error (about 2^-46 after the
// step). Outside [2^-100, 2^100] the float64 division is used. A pivot that is not
// positive and finite latches RTPROJ_ENOTSPD and is replaced by 1.
__device__ __forceinline__ double pivot_rcp(double d, int* status) {
    const long long bits = __double_as_longlong(d);
    if (!(bits > 0 && bits < 0x7FF0000000000000ll)) {
        set_status(status, RTPROJ_ENOTSPD);
        return 1.0;
    }
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex <= 1023 - 100 || ex >= 1023 + 100) return 1.0 / d;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)d));
    const double r = (double)rf;
    return fma(r, fma(-d, r, 1.0), r);
}

// CTA-wide: factors the nb x nb diagonal block at (p0, p0) of X in shared memory (a) and
// forms Z = L_pp^{-1} (z) in the same right-looking sweep (a_loaded: the block's lower
// triangle is already in a, left there by the lookahead tile), then writes L_pp (upper part
// zero) back to X and Z to zbuf. The sweep is the unscaled elimination X = L' D L'^*
// (L' unit lower, D the pivots): per column c, with the multiplier L'[r][c] = a[r][c] / d_c,
// row r of the trailing block loses L'[r][c] times column c (a) and row r of Z' = L'^{-1}
// loses L'[r][c] times row c of Z' (z). Only 1/d_c is on the pivot chain: the lane that
// updates the next pivot takes its reciprocal at once, and one barrier separates columns.
// At the end L = L' D^{1/2} and Z = D^{-1/2} Z', with the reciprocal square roots of all
// pivots formed in parallel.
__device__ void chp_factor_diag(const CholPDev& p, int p0, int nb, double (*a)[CHP_NB + 1], double (*z)[CHP_NB + 1],
                                double* ys, bool a_loaded) {
    const int m = p.m, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int e = t; e < CHP_NB * CHP_NB; e += CHP_THREADS) {
        const int i = e / CHP_NB, j = e % CHP_NB;
        if (!a_loaded) a[i][j] = (i < nb && j <= i) ? __ldcg(p.X + (int64_t)(p0 + i) * m + p0 + j) : 0.0;
        z[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (t == 0) ys[0] = pivot_rcp(a[0][0], p.status);      // 1 / d_0
    __syncthreads();
    for (int c = 0; c + 1 < nb; ++c) {
        const double rc = ys[c];
        for (int r = c + 1 + warp; r < nb; r += CHP_THREADS / 32) {
            const double mrc = a[r][c] * rc;                 // L'[r][c]
            const int j = lane;
            if (j <= r) {
                double* dst = j <= c ? &z[r][j] : &a[r][j];
                const double src = j <= c ? z[c][j] : a[j][c];
                const double upd = fma(-mrc, src, *dst);
                *dst = upd;
                if (r == c + 1 && j == r) ys[r] = pivot_rcp(upd, p.status);   // the next pivot, now final
            }
        }
        __syncthreads();
    }
    // 1 / sqrt(d_c) for every pivot, then L and Z scaled by them
    const double yc = t < nb ? pivot_rsqrt(a[t][t], p.status) : 0.0;
    __syncthreads();
    if (t < nb) ys[t] = yc;
    __syncthreads();
    for (int e = t; e < CHP_NB * CHP_NB; e += CHP_THREADS) {
        const int i = e / CHP_NB, j = e % CHP_NB;
        if (i < nb && j < nb) p.X[(int64_t)(p0 + i) * m + p0 + j] = j <= i ? a[i][j] * ys[j] : 0.0;
        p.zbuf[e] = (i < nb) ? z[i][j] * ys[i] : z[i][j];
    }
}

// Trailing update tile `tile` of the panel at p0 (16 x 16, lower triangle of rows/columns
// [base, m)): X[r][q] -= sum_c L[r][p0+c] L[q][p0+c]. With `out` the updated entries go to
// out[i][j] (tile-local indices) instead of X.
__device__ void chp_update_tile(const CholPDev& p, int p0, int nb, int base, int tile, double (*pr)[CHP_NB + 1],
                                double (*pq)[CHP_NB + 1], double (*out)[CHP_NB + 1] = nullptr) {
    const int m = p.m, t = threadIdx.x;
    int u = tile, tr = 0;
    while (u > tr) { u -= tr + 1; ++tr; }
    const int r0 = base + tr * CHP_TILE, q0 = base + u * CHP_TILE;
    for (int e = t; e < CHP_TILE * CHP_NB; e += CHP_THREADS) {
        const int i = e / CHP_NB, c = e % CHP_NB;
        pr[i][c] = (r0 + i < m && c < nb) ? __ldcg(p.X + (int64_t)(r0 + i) * m + p0 + c) : 0.0;
        pq[i][c] = (q0 + i < m && c < nb) ? __ldcg(p.X + (int64_t)(q0 + i) * m + p0 + c) : 0.0;
    }
    __syncthreads();
    const int i = t / CHP_TILE, j = t % CHP_TILE;
    const int r = r0 + i, q = q0 + j;
    if (r < m && q <= r) {
        double* xp = p.X + (int64_t)r * m + q;
        const double x0 = __ldcg(xp);
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;   // independent partial sums
#pragma unroll
        for (int c = 0; c < CHP_NB; c += 4) {
            acc0 = fma(pr[i][c], pq[j][c], acc0);
            acc1 = fma(pr[i][c + 1], pq[j][c + 1], acc1);
            acc2 = fma(pr[i][c + 2], pq[j][c + 2], acc2);
            acc3 = fma(pr[i][c + 3], pq[j][c + 3], acc3);
        }
        const double xn = x0 - ((acc0 + acc1) + (acc2 + acc3));
        if (out) out[i][j] = xn;
        else *xp = xn;
    }
    __syncthreads();
}

// Panels with lookahead: CTA 0 updates the tile that covers the next diagonal block first
// (into shared memory) and factors that block while the other CTAs finish the trailing
// update, so that a
// panel costs two grid exchanges: (L_pp, Z ready) -> panel rows -> (panel rows ready) ->
// trailing update and the next diagonal block.
__global__ void __launch_bounds__(CHP_THREADS, 1) chol_persistent_kernel(CholPDev p) {
    __shared__ double a[CHP_NB][CHP_NB + 1];
    __shared__ double z[CHP_NB][CHP_NB + 1];
    __shared__ double pr[CHP_TILE][CHP_NB + 1];
    __shared__ double pq[CHP_TILE][CHP_NB + 1];
    __shared__ double ys[CHP_NB];
    __shared__ int ok_s;
    const int m = p.m, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int G = gridDim.x;
    unsigned int nsync = 0;
    if (p.run_if && *p.run_if == 0) return;
    if (blockIdx.x == 0) chp_factor_diag(p, 0, min(CHP_NB, m), a, z, ys, false);
    for (int p0 = 0; p0 < m; p0 += CHP_NB) {
        const int nb = min(CHP_NB, m - p0);
        const int base = p0 + nb, rest = m - base;
        if (rest <= 0) break;
        if (!chp_grid_sync(p, ++nsync, &ok_s)) return;
        // panel rows: x_c = sum_{k <= c} b_k Z[c][k], one warp per row
        for (int e = t; e < CHP_NB * CHP_NB; e += CHP_THREADS) z[e / CHP_NB][e % CHP_NB] = __ldcg(p.zbuf + e);
        __syncthreads();
        for (int r = base + blockIdx.x * (CHP_THREADS / 32) + warp; r < m; r += G * (CHP_THREADS / 32)) {
            double* row = p.X + (int64_t)r * m + p0;
            const double b = lane < nb ? __ldcg(row + lane) : 0.0;
            double x0 = 0.0, x1 = 0.0;                          // independent partial sums
#pragma unroll
            for (int k = 0; k < CHP_NB; k += 2) {
                const double bk0 = __shfl_sync(0xffffffffu, b, k);
                const double bk1 = __shfl_sync(0xffffffffu, b, k + 1);
                if (lane < CHP_NB && k <= lane) x0 = fma(bk0, z[lane][k], x0);
                if (lane < CHP_NB && k + 1 <= lane) x1 = fma(bk1, z[lane][k + 1], x1);
            }
            if (lane < nb) row[lane] = x0 + x1;
        }
        if (!chp_grid_sync(p, ++nsync, &ok_s)) return;
        // trailing update; tile 0 (the next diagonal block) on CTA 0, which updates it into
        // shared memory and factors it from there
        const int nt = (rest + CHP_TILE - 1) / CHP_TILE;
        const int ntiles = nt * (nt + 1) / 2;
        static_assert(CHP_NB == CHP_TILE, "the next diagonal block is one tile");
        const int lead = 1;
        if (blockIdx.x == 0) {
            chp_update_tile(p, p0, nb, base, 0, pr, pq, a);
            chp_factor_diag(p, base, min(CHP_NB, rest), a, z, ys, true);
            if (G == 1)
                for (int tile = lead; tile < ntiles; ++tile) chp_update_tile(p, p0, nb, base, tile, pr, pq);
        } else {
            for (int tile = lead + blockIdx.x - 1; tile < ntiles; tile += G - 1)
                chp_update_tile(p, p0, nb, base, tile, pr, pq);
        }
    }
}

}  // namespace

cudaError_t trsm(const double* T, int64_t t_rs, int64_t t_cs, bool lower, int m,
                 double* Bm, int64_t b_rs, int ncols, double* dinv_work, int* status, cudaStream_t s, bool rhs_lower,
                 const int* run_if) {
    if (m <= 0 || ncols <= 0) return cudaSuccess;
    const size_t smem = (size_t)m * sizeof(double);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    unsigned int* next_col = (unsigned int*)(dinv_work + (size_t)nblk * TRSM_BS * TRSM_BS);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min(ncols, std::max(sms, 1));
    cudaError_t e = cudaMemsetAsync(next_col, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (lower) {
        tri_diag_inv_kernel<true><<<nblk, TDI_THREADS, 0, s>>>(T, t_rs, t_cs, m, dinv_work, status, run_if);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(trsm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        trsm_kernel<true><<<grid, TRSM_THREADS, smem, s>>>(T, t_rs, t_cs, m, Bm, b_rs, ncols, dinv_work,
                                                             rhs_lower ? 1 : 0, next_col, run_if);
    } else {
        tri_diag_inv_kernel<false><<<nblk, TDI_THREADS, 0, s>>>(T, t_rs, t_cs, m, dinv_work, status, run_if);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(trsm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        trsm_kernel<false><<<grid, TRSM_THREADS, smem, s>>>(T, t_rs, t_cs, m, Bm, b_rs, ncols, dinv_work, 0,
                                                              next_col, run_if);
    }
    note_launch(2);
    return cudaGetLastError();
}

// the diagonal-block inverses, then one word for the column counter
size_t trsm_work_doubles(int m) { return (size_t)((m + TRSM_BS - 1) / TRSM_BS) * TRSM_BS * TRSM_BS + 2; }

cudaError_t cholesky(double* X, int m, double* part, size_t part_elems, int* status, cudaStream_t s,
                     long long spin_limit, const int* run_if) {
    // Persistent cooperative form; the per-panel launches below when it cannot run.
    int dev = 0, sms = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop && sms > 0 && part_elems >= CHP_NB * CHP_NB + 2) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_persistent_kernel, CHP_THREADS, 0);
        if (per_sm >= 1) {
            CholPDev p;
            p.X = X; p.m = m; p.zbuf = part;
            p.counter = (unsigned int*)(part + CHP_NB * CHP_NB);
            p.abort_flag = (int*)(p.counter + 1);
            p.status = status;
            p.timeout = spin_limit;
            p.run_if = run_if;
            cudaError_t e = cudaMemsetAsync(p.counter, 0, 2 * sizeof(unsigned int), s);
            if (e != cudaSuccess) return e;
            void* args[] = {&p};
            // a grid sized to the work: about two trailing tiles per CTA for small matrices
            // (so that a batch of small instances does not hold the whole GPU), one CTA per
            // SM from m = 256 up
            const int nt = (m + CHP_TILE - 1) / CHP_TILE;
            const int G = std::max(2, std::min(sms * per_sm, std::min(sms, nt * (nt + 1) / 4)));
            e = cudaLaunchCooperativeKernel((const void*)chol_persistent_kernel, dim3(m >= 256 ? sms : G),
                                            dim3(CHP_THREADS), args, 0, s);
            note_launch();
            if (e == cudaSuccess) return zero_upper(X, m, s);
            cudaGetLastError();   // clear and fall back
        }
    }
    // the per-panel kernels below are unconditional: a conditional call must not get here
    if (run_if) return cudaErrorNotSupported;
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
    return zero_upper(X, m, s);
}


// ---------------------------------------------------------------------------------
// Float-float forms of the solves and the Cholesky factorization (mixed form). The
// structure is the float64 kernels' above; every value is a float-float pair, stored in
// global memory as float2 (hi, lo). The preconditioner is invariant to errors in R^{-*}
// (any invertible N in place of R^{-*} Pi gives N^* (N A A^* N^*)^{-1} N = (A A^*)^{-1});
// what the factors' 2^-48 rounding moves is kappa(X) times that in the preconditioned
// system, which the refinement removes.
// ---------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ double pow2i(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

__device__ __forceinline__ ff ld_ff(const float2* p) {
    const float2 v = __ldcg(p);
    return {v.x, v.y};
}

__device__ __forceinline__ void st_ff(float2* p, ff v) { *p = make_float2(v.hi, v.lo); }

__device__ __forceinline__ ff ff_shfl_xor(ff v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ ff ff_shfl(ff v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

constexpr int FR_THREADS = 1024;

// One CTA: ctl[1] = the largest exponent of the diagonal T[i * dstride] (i < m), made even
// when `positive` (so that the square roots of the Cholesky scale exactly), and ctl[0] = 1
// when an entry is zero, subnormal or non-finite, negative with `positive`, or the
// exponents span more than 60 (the float-float solve then leaves it to the float64 one).
__global__ void __launch_bounds__(FR_THREADS) ff_range_kernel(const double* T, int64_t dstride, int m, int positive,
                                                              int* ctl) {
    __shared__ int smax[FR_THREADS / 32], smin[FR_THREADS / 32], sbad[FR_THREADS / 32];
    int emax = -4096, emin = 4096, bad = 0;
    for (int i = threadIdx.x; i < m; i += FR_THREADS) {
        const long long bits = __double_as_longlong(T[(int64_t)i * dstride]);
        const int ex = (int)((bits >> 52) & 0x7FF);
        if (ex == 0 || ex == 0x7FF || (positive && bits < 0)) {
            bad = 1;
            continue;
        }
        emax = max(emax, ex - 1023);
        emin = min(emin, ex - 1023);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = emax;
        smin[threadIdx.x >> 5] = emin;
        sbad[threadIdx.x >> 5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < FR_THREADS / 32; ++w) {
            emax = max(emax, smax[w]);
            emin = min(emin, smin[w]);
            bad |= sbad[w];
        }
        if (emax - emin > 60) bad = 1;
        if (bad) emax = 0;
        ctl[1] = positive ? (emax & ~1) : emax;   // rounds down to even (two's complement)
        ctl[0] = bad;
    }
}

// Tf (column-major, m x m, lower triangle) = T 2^-ctl[1] as float-float; an entry at or
// above 2^100 after scaling raises ctl[0].
__global__ void tri_to_ff_kernel(const double* T, int64_t t_rs, int64_t t_cs, int m, float2* Tf, int* ctl) {
    if (*(volatile int*)ctl) return;
    const double sc = pow2i(-ctl[1]);
    const int64_t total = (int64_t)m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / m), i = (int)(e - (int64_t)k * m);
        if (k > i) continue;
        const double v = T[(int64_t)i * t_rs + (int64_t)k * t_cs] * sc;
        if (!(fabs(v) < 0x1p100)) {
            *(volatile int*)ctl = 1;
            continue;
        }
        st_ff(Tf + e, ff_from_double(v));
    }
}

// The float-float inverse of each 32 x 32 diagonal block of the lower Tf, as
// tri_diag_inv_kernel: two 16 x 16 inverses by substitution on one warp, then the
// off-diagonal block -C^{-1} B A^{-1} as two small products.
__global__ void __launch_bounds__(TDI_THREADS) tri_diag_inv_ff_kernel(const float2* Tf, int m, float2* Dinv,
                                                                      const int* ctl) {
    if (*(volatile const int*)ctl) return;
    constexpr int H = TRSM_BS / 2;
    __shared__ ff a[TRSM_BS][TRSM_BS + 1];
    __shared__ ff inv[TRSM_BS][TRSM_BS + 1];
    __shared__ ff f[H][H + 1];
    __shared__ ff rd[TRSM_BS];
    const int b = blockIdx.x, t = threadIdx.x;
    const int r0 = b * TRSM_BS;
    const int bs = min(TRSM_BS, m - r0);
    for (int e = t; e < TRSM_BS * TRSM_BS; e += TDI_THREADS) {
        const int i = e / TRSM_BS, k = e % TRSM_BS;
        ff v = {i == k ? 1.f : 0.f, 0.f};
        if (i < bs && k <= i) v = ld_ff(Tf + (int64_t)(r0 + k) * m + r0 + i);
        a[i][k] = v;
    }
    __syncthreads();
    if (t < TRSM_BS) rd[t] = ff_recip(a[t][t]);   // the range check keeps every pivot normal
    __syncthreads();
    if (t < TRSM_BS) {
        const int off = (t / H) * H, jj = t % H;
        ff col[H];
#pragma unroll
        for (int i = 0; i < H; ++i) col[i] = {i == jj ? 1.f : 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < H; ++i) {
            col[i] = i >= jj ? ff_mul(col[i], rd[off + i]) : ff{0.f, 0.f};
#pragma unroll
            for (int r = i + 1; r < H; ++r) col[r] = ff_add(col[r], ff_neg(ff_mul(a[off + r][off + i], col[i])));
        }
#pragma unroll
        for (int i = 0; i < H; ++i) inv[off + i][off + jj] = col[i];
    }
    __syncthreads();
    for (int e = t; e < H * H; e += TDI_THREADS) {   // F = B A^{-1}
        const int i = e / H, j = e % H;
        ff s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < H; k += 2) {
            ff_dot_acc(s0, a[H + i][k], inv[k][j]);
            ff_dot_acc(s1, a[H + i][k + 1], inv[k + 1][j]);
        }
        f[i][j] = ff_add(ff_renorm(s0), ff_renorm(s1));
    }
    __syncthreads();
    for (int e = t; e < H * H; e += TDI_THREADS) {   // lower-left block -C^{-1} F
        const int i = e / H, j = e % H;
        ff s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < H; k += 2) {
            ff_dot_acc(s0, inv[H + i][H + k], f[k][j]);
            ff_dot_acc(s1, inv[H + i][H + k + 1], f[k + 1][j]);
        }
        inv[H + i][j] = ff_neg(ff_add(ff_renorm(s0), ff_renorm(s1)));
    }
    __syncthreads();
    float2* out = Dinv + (size_t)b * TRSM_BS * TRSM_BS;
    for (int e = t; e < TRSM_BS * TRSM_BS; e += TDI_THREADS) {
        const int i = e / TRSM_BS, j = e % TRSM_BS;
        st_ff(out + e, (i < bs && j < bs && j <= i) ? inv[i][j] : ff{0.f, 0.f});
    }
}

// The lower solve of trsm_kernel in float-float, one column of B at a time from a shared
// counter. A column is scaled by 2^-f (f its largest exponent) on the way in, and the
// solution by 2^(f - ctl[1]) on the way out, so that neither leaves the float range.
__global__ void __launch_bounds__(TRSM_THREADS, 1) trsm_ff_kernel(const float2* __restrict__ Tf, int m, double* B,
                                                                  int64_t b_rs, int ncols,
                                                                  const float2* __restrict__ Dinv, int rhs_lower,
                                                                  unsigned int* next_col, const int* ctl, int* status) {
    if (*(volatile const int*)ctl) return;
    extern __shared__ float2 xs2[];   // m: the column being solved
    ff* xs = reinterpret_cast<ff*>(xs2);
    __shared__ int col_s;
    __shared__ int wmax[TRSM_THREADS / 32];
    const int t = threadIdx.x;
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    const int eT = ctl[1];
    for (;;) {
        if (t == 0) col_s = (int)atomicAdd(next_col, 1u);
        __syncthreads();
        const int j = col_s;
        if (j >= ncols) break;
        const int bi0 = rhs_lower ? min(j, m) / TRSM_BS : 0;
        const int row0 = bi0 * TRSM_BS;
        int emax = -4096;
        for (int i = row0 + t; i < m; i += TRSM_THREADS) {
            const long long bits = __double_as_longlong(B[(int64_t)i * b_rs + j]);
            const int ex = (int)((bits >> 52) & 0x7FF);
            if (ex != 0) emax = max(emax, ex - 1023);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if ((t & 31) == 0) wmax[t >> 5] = emax;
        __syncthreads();
        emax = wmax[0];
        for (int w = 1; w < TRSM_THREADS / 32; ++w) emax = max(emax, wmax[w]);
        const int f = (emax == -4096 || emax > 1000) ? 0 : emax;   // a zero column; a non-finite one stays so
        const double sc = pow2i(-f);
        for (int i = row0 + t; i < m; i += TRSM_THREADS) xs[i] = ff_from_double(B[(int64_t)i * b_rs + j] * sc);
        __syncthreads();
        for (int blk = bi0; blk < nblk; ++blk) {
            const int r0 = blk * TRSM_BS;
            const int bs = min(TRSM_BS, m - r0);
            const int di = t / TRSM_DPARTS, part = t % TRSM_DPARTS;
            ff y = {0.f, 0.f};
            if (t < TRSM_BS * TRSM_DPARTS) {
                const float2* drow = Dinv + ((size_t)blk * TRSM_BS + di) * TRSM_BS;
                ff y0 = {0.f, 0.f}, y1 = {0.f, 0.f};
#pragma unroll
                for (int k0 = 0; k0 < TRSM_BS; k0 += 2 * TRSM_DPARTS) {
                    const int k = k0 + part;
                    if (k < bs) ff_dot_acc(y0, ld_ff(drow + k), xs[r0 + k]);
                    if (k + TRSM_DPARTS < bs) ff_dot_acc(y1, ld_ff(drow + k + TRSM_DPARTS), xs[r0 + k + TRSM_DPARTS]);
                }
                y = ff_add(ff_renorm(y0), ff_renorm(y1));
                y = ff_add(y, ff_shfl_xor(y, 1));
                y = ff_add(y, ff_shfl_xor(y, 2));
            }
            __syncthreads();
            if (t < TRSM_BS * TRSM_DPARTS && part == 0 && di < bs) xs[r0 + di] = y;
            __syncthreads();
            for (int r = r0 + bs + t; r < m; r += TRSM_THREADS) {
                ff a0 = {0.f, 0.f}, a1 = {0.f, 0.f};
                if (bs == TRSM_BS) {
                    ff tv[TRSM_BS];
#pragma unroll
                    for (int k = 0; k < TRSM_BS; ++k) tv[k] = ld_ff(Tf + (int64_t)(r0 + k) * m + r);
#pragma unroll
                    for (int k = 0; k < TRSM_BS; k += 2) {
                        ff_dot_acc(a0, tv[k], xs[r0 + k]);
                        ff_dot_acc(a1, tv[k + 1], xs[r0 + k + 1]);
                    }
                } else {
                    for (int k = 0; k < bs; ++k) ff_dot_acc(a0, ld_ff(Tf + (int64_t)(r0 + k) * m + r), xs[r0 + k]);
                }
                xs[r] = ff_add(xs[r], ff_neg(ff_add(ff_renorm(a0), ff_renorm(a1))));
            }
            __syncthreads();
        }
        const double out_sc = pow2i(f - eT);
        for (int i = row0 + t; i < m; i += TRSM_THREADS) {
            const double v = ff_to_double(xs[i]) * out_sc;
            if (!isfinite(v)) set_status(status, RTPROJ_ENONFINITE);
            B[(int64_t)i * b_rs + j] = v;
        }
        __syncthreads();   // xs and col_s are reused by the next column
    }
}

struct CholFfDev {
    CholPDev sync;           // counter, abort flag, status and spin limit of the grid barrier
    double* X;               // in: the lower triangle of X; out: L (strict upper part zero)
    float2* Xf;              // m x m float-float working copy (row-major, lower triangle)
    float2* zbuf;            // CHP_NB x CHP_NB: Z of the current panel
    int* ctl;                // ctl[0]: 1 = left to the float64 kernel; ctl[1]: the scale exponent
    int m;
};

// Grid barrier, then the float64 fallback flag: false when either says to stop (the flag
// goes through its own shared word, so that every thread takes the same branch).
__device__ bool chf_sync(const CholFfDev& q, unsigned int k, int* ok_s, int* go_s) {
    if (!chp_grid_sync(q.sync, k, ok_s)) return false;
    if (threadIdx.x == 0) *go_s = *(volatile int*)q.ctl == 0;
    __syncthreads();
    return *go_s != 0;
}

// A pivot's reciprocal (square root) in float-float; a pivot that is not positive and
// finite sends the factorization to the float64 kernel (which reports RTPROJ_ENOTSPD if
// X is not positive definite in float64 either).
__device__ __forceinline__ ff chf_pivot_rcp(ff d, int* ctl) {
    if (!(d.hi > 0.f) || !isfinite(d.hi)) {
        *(volatile int*)ctl = 1;
        return {1.f, 0.f};
    }
    return ff_recip(d);
}

__device__ __forceinline__ ff chf_pivot_rsqrt(ff d, int* ctl) {
    if (!(d.hi > 0.f) || !isfinite(d.hi)) {
        *(volatile int*)ctl = 1;
        return {1.f, 0.f};
    }
    return ff_recip(ff_sqrt(d));
}

// chp_factor_diag in float-float.
__device__ void chf_factor_diag(const CholFfDev& q, int p0, int nb, ff (*a)[CHP_NB + 1], ff (*z)[CHP_NB + 1], ff* ys,
                                bool a_loaded) {
    const int m = q.m, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int e = t; e < CHP_NB * CHP_NB; e += CHP_THREADS) {
        const int i = e / CHP_NB, j = e % CHP_NB;
        if (!a_loaded) a[i][j] = (i < nb && j <= i) ? ld_ff(q.Xf + (int64_t)(p0 + i) * m + p0 + j) : ff{0.f, 0.f};
        z[i][j] = {i == j ? 1.f : 0.f, 0.f};
    }
    __syncthreads();
    if (t == 0) ys[0] = chf_pivot_rcp(a[0][0], q.ctl);
    __syncthreads();
    for (int c = 0; c + 1 < nb; ++c) {
        const ff rc = ys[c];
        for (int r = c + 1 + warp; r < nb; r += CHP_THREADS / 32) {
            const ff mrc = ff_mul(a[r][c], rc);
            const int j = lane;
            if (j <= r) {
                ff* dst = j <= c ? &z[r][j] : &a[r][j];
                const ff src = j <= c ? z[c][j] : a[j][c];
                const ff upd = ff_add(*dst, ff_neg(ff_mul(mrc, src)));
                *dst = upd;
                if (r == c + 1 && j == r) ys[r] = chf_pivot_rcp(upd, q.ctl);
            }
        }
        __syncthreads();
    }
    const ff yc = t < nb ? chf_pivot_rsqrt(a[t][t], q.ctl) : ff{0.f, 0.f};
    __syncthreads();
    if (t < nb) ys[t] = yc;
    __syncthreads();
    for (int e = t; e < CHP_NB * CHP_NB; e += CHP_THREADS) {
        const int i = e / CHP_NB, j = e % CHP_NB;
        if (i < nb && j < nb) st_ff(q.Xf + (int64_t)(p0 + i) * m + p0 + j, j <= i ? ff_mul(a[i][j], ys[j]) : ff{0.f, 0.f});
        st_ff(q.zbuf + e, i < nb ? ff_mul(z[i][j], ys[i]) : z[i][j]);
    }
}

// chp_update_tile in float-float.
__device__ void chf_update_tile(const CholFfDev& q, int p0, int nb, int base, int tile, ff (*pr)[CHP_NB + 1],
                                ff (*pq)[CHP_NB + 1], ff (*out)[CHP_NB + 1] = nullptr) {
    const int m = q.m, t = threadIdx.x;
    int u = tile, tr = 0;
    while (u > tr) { u -= tr + 1; ++tr; }
    const int r0 = base + tr * CHP_TILE, q0 = base + u * CHP_TILE;
    for (int e = t; e < CHP_TILE * CHP_NB; e += CHP_THREADS) {
        const int i = e / CHP_NB, c = e % CHP_NB;
        pr[i][c] = (r0 + i < m && c < nb) ? ld_ff(q.Xf + (int64_t)(r0 + i) * m + p0 + c) : ff{0.f, 0.f};
        pq[i][c] = (q0 + i < m && c < nb) ? ld_ff(q.Xf + (int64_t)(q0 + i) * m + p0 + c) : ff{0.f, 0.f};
    }
    __syncthreads();
    const int i = t / CHP_TILE, j = t % CHP_TILE;
    const int r = r0 + i, c2 = q0 + j;
    if (r < m && c2 <= r) {
        float2* xp = q.Xf + (int64_t)r * m + c2;
        const ff x0 = ld_ff(xp);
        ff acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
#pragma unroll
        for (int c = 0; c < CHP_NB; c += 2) {
            ff_dot_acc(acc0, pr[i][c], pq[j][c]);
            ff_dot_acc(acc1, pr[i][c + 1], pq[j][c + 1]);
        }
        const ff xn = ff_add(x0, ff_neg(ff_add(ff_renorm(acc0), ff_renorm(acc1))));
        if (out) out[i][j] = xn;
        else st_ff(xp, xn);
    }
    __syncthreads();
}

// chol_persistent_kernel in float-float: X scaled by 2^-ctl[1] into Xf, the same panels
// and lookahead, then L = 2^(ctl[1]/2) Lf written back over X. X is left untouched when
// the factorization is sent to the float64 kernel.
__global__ void __launch_bounds__(CHP_THREADS, 1) chol_ff_kernel(CholFfDev q) {
    __shared__ ff a[CHP_NB][CHP_NB + 1];
    __shared__ ff z[CHP_NB][CHP_NB + 1];
    __shared__ ff pr[CHP_TILE][CHP_NB + 1];
    __shared__ ff pq[CHP_TILE][CHP_NB + 1];
    __shared__ ff ys[CHP_NB];
    __shared__ int ok_s, go_s;
    if (*(volatile int*)q.ctl) return;   // the range check left it to the float64 kernel
    const int m = q.m, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int G = gridDim.x;
    const int e2 = q.ctl[1];
    const int64_t total = (int64_t)m * m;
    {
        const double sc = pow2i(-e2);
        for (int64_t e = (int64_t)blockIdx.x * CHP_THREADS + t; e < total; e += (int64_t)G * CHP_THREADS) {
            const int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
            if (j > i) continue;
            const double v = q.X[e] * sc;
            if (!(fabs(v) < 0x1p100)) {
                *(volatile int*)q.ctl = 1;
                continue;
            }
            st_ff(q.Xf + e, ff_from_double(v));
        }
    }
    unsigned int nsync = 0;
    if (!chf_sync(q, ++nsync, &ok_s, &go_s)) return;
    if (blockIdx.x == 0) chf_factor_diag(q, 0, min(CHP_NB, m), a, z, ys, false);
    for (int p0 = 0; p0 < m; p0 += CHP_NB) {
        const int nb = min(CHP_NB, m - p0);
        const int base = p0 + nb, rest = m - base;
        if (rest <= 0) break;
        if (!chf_sync(q, ++nsync, &ok_s, &go_s)) return;
        // panel rows: x_c = sum_{k <= c} b_k Z[c][k], one warp per row
        for (int e = t; e < CHP_NB * CHP_NB; e += CHP_THREADS) z[e / CHP_NB][e % CHP_NB] = ld_ff(q.zbuf + e);
        __syncthreads();
        for (int r = base + blockIdx.x * (CHP_THREADS / 32) + warp; r < m; r += G * (CHP_THREADS / 32)) {
            float2* row = q.Xf + (int64_t)r * m + p0;
            const ff b = lane < nb ? ld_ff(row + lane) : ff{0.f, 0.f};
            ff x0 = {0.f, 0.f}, x1 = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < CHP_NB; k += 2) {
                const ff bk0 = ff_shfl(b, k);
                const ff bk1 = ff_shfl(b, k + 1);
                if (lane < CHP_NB && k <= lane) ff_dot_acc(x0, bk0, z[lane][k]);
                if (lane < CHP_NB && k + 1 <= lane) ff_dot_acc(x1, bk1, z[lane][k + 1]);
            }
            if (lane < nb) st_ff(row + lane, ff_add(ff_renorm(x0), ff_renorm(x1)));
        }
        if (!chf_sync(q, ++nsync, &ok_s, &go_s)) return;
        const int nt = (rest + CHP_TILE - 1) / CHP_TILE;
        const int ntiles = nt * (nt + 1) / 2;
        if (blockIdx.x == 0) {
            chf_update_tile(q, p0, nb, base, 0, pr, pq, a);
            chf_factor_diag(q, base, min(CHP_NB, rest), a, z, ys, true);
            if (G == 1)
                for (int tile = 1; tile < ntiles; ++tile) chf_update_tile(q, p0, nb, base, tile, pr, pq);
        } else {
            for (int tile = blockIdx.x; tile < ntiles; tile += G - 1) chf_update_tile(q, p0, nb, base, tile, pr, pq);
        }
    }
    if (!chf_sync(q, ++nsync, &ok_s, &go_s)) return;
    const double out_sc = pow2i(e2 / 2);
    for (int64_t e = (int64_t)blockIdx.x * CHP_THREADS + t; e < total; e += (int64_t)G * CHP_THREADS) {
        const int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
        q.X[e] = j <= i ? ff_to_double(ld_ff(q.Xf + e)) * out_sc : 0.0;
    }
}

}  // namespace

size_t ff_work_bytes(int m) { return (size_t)m * m * sizeof(float2); }

cudaError_t trsm_ff(const double* T, int64_t t_rs, int64_t t_cs, int m, double* Bm, int64_t b_rs, int ncols,
                    double* dinv_work, void* ffbuf, int* ctl, int* status, cudaStream_t s, bool rhs_lower) {
    if (m <= 0 || ncols <= 0) return cudaSuccess;
    const size_t smem = (size_t)m * sizeof(float2);
    if (smem > 200 * 1024) return trsm(T, t_rs, t_cs, true, m, Bm, b_rs, ncols, dinv_work, status, s, rhs_lower);
    const int nblk = (m + TRSM_BS - 1) / TRSM_BS;
    // the column counters after the block inverses: [0] the float64 solve, [1] this one
    unsigned int* ctr = (unsigned int*)(dinv_work + (size_t)nblk * TRSM_BS * TRSM_BS);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float2* Tf = (float2*)ffbuf;
    float2* Df = (float2*)dinv_work;
    ff_range_kernel<<<1, FR_THREADS, 0, s>>>(T, t_rs + t_cs, m, 0, ctl);
    const int64_t total = (int64_t)m * m;
    const unsigned cgrid = (unsigned)std::min<int64_t>((total + 255) / 256, 8 * std::max(sms, 1));
    tri_to_ff_kernel<<<cgrid, 256, 0, s>>>(T, t_rs, t_cs, m, Tf, ctl);
    tri_diag_inv_ff_kernel<<<nblk, TDI_THREADS, 0, s>>>(Tf, m, Df, ctl);
    cudaError_t e = cudaMemsetAsync(ctr + 1, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (smem > 48 * 1024) cudaFuncSetAttribute(trsm_ff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = (unsigned)std::min(ncols, std::max(sms, 1));
    trsm_ff_kernel<<<grid, TRSM_THREADS, smem, s>>>(Tf, m, Bm, b_rs, ncols, Df, rhs_lower ? 1 : 0, ctr + 1, ctl,
                                                     status);
    note_launch(4);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the float64 solve: runs only if the range check (or a conversion) gave up
    return trsm(T, t_rs, t_cs, true, m, Bm, b_rs, ncols, dinv_work, status, s, rhs_lower, ctl);
}

cudaError_t cholesky_ff(double* X, int m, double* part, size_t part_elems, void* ffbuf, int* ctl, int* status,
                        cudaStream_t s, long long spin_limit) {
    int dev = 0, sms = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    int per_ff = 0, per_64 = 0;
    if (coop && sms > 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_ff, chol_ff_kernel, CHP_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_64, chol_persistent_kernel, CHP_THREADS, 0);
    }
    // zbuf (CHP_NB^2 float2, one double each) and the two counter words after it
    if (per_ff < 1 || per_64 < 1 || part_elems < CHP_NB * CHP_NB + 2)
        return cholesky(X, m, part, part_elems, status, s, spin_limit);
    ff_range_kernel<<<1, FR_THREADS, 0, s>>>(X, (int64_t)m + 1, m, 1, ctl);
    note_launch();
    CholFfDev q;
    q.sync.X = X; q.sync.m = m; q.sync.zbuf = part;
    q.sync.counter = (unsigned int*)(part + CHP_NB * CHP_NB);
    q.sync.abort_flag = (int*)(q.sync.counter + 1);
    q.sync.status = status;
    q.sync.timeout = spin_limit;
    q.sync.run_if = nullptr;
    q.X = X; q.Xf = (float2*)ffbuf; q.zbuf = (float2*)part; q.ctl = ctl; q.m = m;
    cudaError_t e = cudaMemsetAsync(q.sync.counter, 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int nt = (m + CHP_TILE - 1) / CHP_TILE;
    const int G = m >= 256 ? sms : std::max(2, std::min(sms * per_ff, std::min(sms, nt * (nt + 1) / 4)));
    void* args[] = {&q};
    e = cudaLaunchCooperativeKernel((const void*)chol_ff_kernel, dim3(G), dim3(CHP_THREADS), args, 0, s);
    note_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        // not launched: the float64 kernel takes the factorization
        e = cudaMemsetAsync(ctl, 1, 1, s);   // ctl[0] is 0 or 1: its low byte set makes it 1
        if (e != cudaSuccess) return e;
    }
    return cholesky(X, m, part, part_elems, status, s, spin_limit, ctl);
}

}  // namespace rtp
