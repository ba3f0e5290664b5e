// A sparse A, optionally plus a low-rank term: A = S + U V with S m x n in compressed
// sparse row form, U m x r and V r x n dense (r small). This is the setting of the paper's
// Section 5: the sparse test matrix of Eq. 21 (five nonzeros per column) and its sum with
// a rank-10 term (Eq. 22), applied as operators at O(nnz + r(m + n)) per vector.
//
//   S_k = A G                 one CTA per (row, 32 columns of G); G generated per nonzero
//                             (the same entries as the dense forms), Eq. 12
//   X column by column as in steps a-e that follow Eq. 15, all m columns at once:
//     D = A^* P^-             (n x m) one CTA per column of A, a gather over its nonzeros
//     E = A D                 (m x m) one CTA per row of A
//     X = R^{-*} Pi E         one float64 product with the triangular R^{-*}
//   apply (the seven steps) and its refinement (Remark 4.3) with every product with A or
//   A^* summed in double-double and rounded once: c = A b, s = b - A^* h, r = A s,
//   s <- s - A^* dh. The sparse part of each of these is exact to double-double rounding,
//   so the refinement converges to the projection of the stored matrix; the low-rank
//   part (V b, U^* h and their products with U, V) is float64.
#include "rtproj_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

using namespace rtp;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

#define SP_CHECK(expr)                                  \
    do {                                                \
        if ((expr) != cudaSuccess) return RTPROJ_ECUDA; \
    } while (0)

// ---------------------------------------------------------------------------------
// Double-double building blocks: Knuth's TwoSum and the fma form of TwoProduct.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += a b to double-double accuracy
__device__ __forceinline__ void dd_fma_acc(double& hi, double& lo, double a, double b) {
    const double p = a * b;
    const double pe = fma(a, b, -p);
    double s, e;
    two_sum_d(hi, p, s, e);
    e += lo + pe;
    hi = s + e;
    lo = e - (hi - s);
}

__device__ __forceinline__ void dd_add(double& hi, double& lo, double bh, double bl) {
    double s, e;
    two_sum_d(hi, bh, s, e);
    e += lo + bl;
    hi = s + e;
    lo = e - (hi - s);
}

__device__ __forceinline__ void dd_warp_sum(double& hi, double& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const double ol = __shfl_xor_sync(0xffffffffu, lo, o);
        dd_add(hi, lo, oh, ol);
    }
}

// ---------------------------------------------------------------------------------
// The column-compressed copy: counting sort by column, then each column's entries put in
// (row, value) order, so that every sum over a column runs in one fixed order whatever the
// order in which the scatter's atomics landed.
// ---------------------------------------------------------------------------------
__global__ void count_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, int n, int64_t* cnt, int* status) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int c = col[p];
        if (c < 0 || c >= n) { set_status(status, RTPROJ_EINVAL); continue; }
        atomicAdd((unsigned long long*)&cnt[c], 1ull);
    }
}

// Exclusive scan of cnt[0..n) into ptr[0..n] in blocks of SCAN_T: per-block totals, one CTA
// scanning those totals, then each block's scan plus its offset.
constexpr int SCAN_T = 1024;

__device__ __forceinline__ int64_t block_inclusive_scan(int64_t v, int64_t* buf) {
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        const int64_t x = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += x;
        __syncthreads();
    }
    return buf[threadIdx.x];
}

__global__ void block_totals_kernel(const int64_t* cnt, int n, int64_t* tot) {
    __shared__ int64_t buf[SCAN_T];
    const int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    const int64_t incl = block_inclusive_scan(i < n ? cnt[i] : 0, buf);
    if (threadIdx.x == SCAN_T - 1) tot[blockIdx.x] = incl;
}

__global__ void scan_totals_kernel(int64_t* tot, int nb) {
    __shared__ int64_t buf[SCAN_T];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int i = b0 + threadIdx.x;
        const int64_t v = i < nb ? tot[i] : 0;
        const int64_t incl = block_inclusive_scan(v, buf);
        const int64_t base = carry;
        __syncthreads();
        if (i < nb) tot[i] = base + incl - v;
        if (threadIdx.x == SCAN_T - 1) carry = base + incl;
        __syncthreads();
    }
}

__global__ void block_scan_kernel(const int64_t* cnt, int n, const int64_t* tot, int64_t* ptr) {
    __shared__ int64_t buf[SCAN_T];
    const int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    const int64_t v = i < n ? cnt[i] : 0;
    const int64_t incl = block_inclusive_scan(v, buf);
    if (i < n) ptr[i] = tot[blockIdx.x] + incl - v;
    if (i == n - 1) ptr[n] = tot[blockIdx.x] + incl;
}

__global__ void scatter_csc_kernel(const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                                   const double* __restrict__ val, int m, int n, const int64_t* __restrict__ cptr,
                                   int64_t* cursor, int32_t* __restrict__ crow, double* __restrict__ cval) {
    for (int i = blockIdx.x; i < m; i += gridDim.x) {
        for (int64_t p = rptr[i] + threadIdx.x; p < rptr[i + 1]; p += blockDim.x) {
            const int c = col[p];
            if (c < 0 || c >= n) continue;   // counted nowhere; create fails on RTPROJ_EINVAL
            const int64_t at = cptr[c] + (int64_t)atomicAdd((unsigned long long*)&cursor[c], 1ull);
            crow[at] = i;
            cval[at] = val[p];
        }
    }
}

__device__ __forceinline__ bool entry_before(int32_t ra, double va, int32_t rb, double vb) {
    if (ra != rb) return ra < rb;
    return __double_as_longlong(va) < __double_as_longlong(vb);   // duplicates: a fixed order
}

__global__ void sort_columns_kernel(const int64_t* __restrict__ cptr, int n, int32_t* crow, double* cval) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int64_t b = cptr[c], e = cptr[c + 1];
        for (int64_t p = b + 1; p < e; ++p) {      // insertion sort
            const int32_t r = crow[p];
            const double v = cval[p];
            int64_t q = p - 1;
            while (q >= b && entry_before(r, v, crow[q], cval[q])) {
                crow[q + 1] = crow[q];
                cval[q + 1] = cval[q];
                --q;
            }
            crow[q + 1] = r;
            cval[q + 1] = v;
        }
    }
}

__global__ void check_values_kernel(const double* __restrict__ val, int64_t nnz, int* status) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(val[p])) set_status(status, RTPROJ_ENONFINITE);
}

// ---------------------------------------------------------------------------------
// ||A||_F^2 = ||S||_F^2 + 2 <S, U V> + trace((U^* U)(V V^*)), each part summed in two
// deterministic levels (per-CTA partials, then one thread).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double s, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

__global__ void sumsq_vals_kernel(const double* __restrict__ val, int64_t nnz, double* part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        s = fma(val[p], val[p], s);
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// part[b] = sum over the rows i = b, b + gridDim.x, ... of sum_p val (U V)(i, col)
__global__ void cross_term_kernel(const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, int m, int n, int r, const double* __restrict__ U,
                                  const double* __restrict__ V, double* part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int i = blockIdx.x; i < m; i += gridDim.x)
        for (int64_t p = rptr[i] + threadIdx.x; p < rptr[i + 1]; p += blockDim.x) {
            double uv = 0.0;
            for (int q = 0; q < r; ++q) uv = fma(U[(int64_t)i * r + q], V[(int64_t)q * n + col[p]], uv);
            s = fma(val[p], uv, s);
        }
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void frobenius_total_kernel(const double* part_s, int np, const double* part_x, int nx, const double* GU,
                                       const double* GV, int r, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0, x = 0.0, t = 0.0;
    for (int i = 0; i < np; ++i) s += part_s[i];
    for (int i = 0; i < nx; ++i) x += part_x[i];
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) t = fma(GU[a * r + b], GV[b * r + a], t);
    *out = sqrt(fmax(s + 2.0 * x + t, 0.0));
}

// ---------------------------------------------------------------------------------
// S = A G. G(c, j) is generated where it is used, from the counter-based Philox words
// that the dense forms use: entries 16q .. 16q+15 of column j from the block at (q, j, 0, 0)
// (uniform or +-1 bytes), Gaussian entries 4q .. 4q+3 from the block at (q, j, 1, 0).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double omega_at(int c, int j, int dist, uint32_t k0, uint32_t k1) {
    if (dist == RTPROJ_OMEGA_GAUSSIAN) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(c >> 2), (uint32_t)j, 1u, 0u), k0, k1);
        int ncos, nsin;
        if (c & 2) gauss_pair(w.z, w.w, ncos, nsin);
        else gauss_pair(w.x, w.y, ncos, nsin);
        return (double)((c & 1) ? nsin : ncos) * (1.0 / 4096.0);
    }
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(c >> 4), (uint32_t)j, 0u, 0u), k0, k1);
    return (double)omega_from_byte(block_byte(w, c & 15), dist);
}

constexpr int SK_WARPS = 8;

// one CTA per (row i, 32 columns j): the 8 warps take interleaved nonzeros of the row, each
// lane one column j; the warps' partial sums are added in a fixed order. With a low-rank
// term, S(i, j) += sum_q U(i, q) (V G)(q, j).
__global__ void sparse_sketch_kernel(const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, int l, int dist, uint32_t k0, uint32_t k1,
                                     int r, const double* __restrict__ U, const double* __restrict__ VG, int64_t ldvg,
                                     double* S, int64_t lds) {
    const int i = blockIdx.y;
    const int lane = threadIdx.x & 31, wsub = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    __shared__ double part[SK_WARPS][32];
    double acc0 = 0.0, acc1 = 0.0;
    if (j < l) {
        const int64_t e = rptr[i + 1];
        int64_t p = rptr[i] + wsub;
        for (; p + SK_WARPS < e; p += 2 * SK_WARPS) {
            acc0 = fma(val[p], omega_at(col[p], j, dist, k0, k1), acc0);
            acc1 = fma(val[p + SK_WARPS], omega_at(col[p + SK_WARPS], j, dist, k0, k1), acc1);
        }
        if (p < e) acc0 = fma(val[p], omega_at(col[p], j, dist, k0, k1), acc0);
    }
    part[wsub][lane] = acc0 + acc1;
    __syncthreads();
    if (wsub == 0 && j < l) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < SK_WARPS; ++w) s += part[w][lane];
        for (int q = 0; q < r; ++q) s = fma(U[(int64_t)i * r + q], VG[(int64_t)q * ldvg + j], s);
        S[(int64_t)i * lds + j] = s;
    }
}

// ---------------------------------------------------------------------------------
// The Gram matrix, in the paper's order (steps a-e that follow Eq. 15, for all k at once).
// ---------------------------------------------------------------------------------
// P^- = Pi^* R^{-1} (Eq. 15): P^-(perm[t], k) = R^{-1}(t, k) = RinvT(k, t)
__global__ void pminus_kernel(const double* __restrict__ RinvT, const int32_t* __restrict__ perm, int m,
                              double* Pm) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int t = (int)(idx / m), k = (int)(idx % m);
    Pm[(int64_t)perm[t] * m + k] = RinvT[(int64_t)k * m + t];
}

// D(c, :) = sum over column c's nonzeros of val P^-(row, :)  [+ sum_q V(q, c) (U^* P^-)(q, :)]
__global__ void sparse_d_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                                const double* __restrict__ cval, const double* __restrict__ Pm, int m, int n, int r,
                                const double* __restrict__ V, const double* __restrict__ UtP, double* D) {
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        const int64_t b = cptr[c], e = cptr[c + 1];
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            double s = 0.0;
            for (int64_t p = b; p < e; ++p) s = fma(cval[p], Pm[(int64_t)crow[p] * m + k], s);
            for (int q = 0; q < r; ++q) s = fma(V[(int64_t)q * n + c], UtP[(int64_t)q * m + k], s);
            D[(int64_t)c * m + k] = s;
        }
    }
}

// E(i, :) = sum over row i's nonzeros of val D(col, :)  [+ sum_q U(i, q) (V D)(q, :)]
__global__ void sparse_e_kernel(const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ D, int m, int r,
                                const double* __restrict__ U, const double* __restrict__ VD, double* E) {
    const int i = blockIdx.x;
    const int64_t b = rptr[i], e = rptr[i + 1];
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double s0 = 0.0, s1 = 0.0;
        int64_t p = b;
        for (; p + 1 < e; p += 2) {
            s0 = fma(val[p], D[(int64_t)col[p] * m + k], s0);
            s1 = fma(val[p + 1], D[(int64_t)col[p + 1] * m + k], s1);
        }
        if (p < e) s0 = fma(val[p], D[(int64_t)col[p] * m + k], s0);
        double s = s0 + s1;
        for (int q = 0; q < r; ++q) s = fma(U[(int64_t)i * r + q], VD[(int64_t)q * m + k], s);
        E[(int64_t)i * m + k] = s;
    }
}

// ---------------------------------------------------------------------------------
// Products of the apply, in double-double.
// ---------------------------------------------------------------------------------
// Rows are cut into chunks of at most SP_CHUNK nonzeros (a table built at create), so that
// a few long rows still spread over many warps. part(c, j) = the double-double sum over
// chunk c of val x_j[col]: one warp per (chunk, right-hand side j).
constexpr int SP_CHUNK = 2048;

__global__ void spmv_chunk_kernel(const int32_t* __restrict__ crow_of, const int64_t* __restrict__ cbeg,
                                  const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, const double* __restrict__ X, int64_t ldx,
                                  int nchunks, int k, double2* __restrict__ part) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)nchunks * k) return;
    const int c = (int)(wid / k), j = (int)(wid % k);
    const int64_t b = cbeg[c];
    const int64_t e = min(b + (int64_t)SP_CHUNK, rptr[crow_of[c] + 1]);
    const double* x = X + (int64_t)j * ldx;
    double hi = 0.0, lo = 0.0;
    for (int64_t p = b + lane; p < e; p += 32) dd_fma_acc(hi, lo, val[p], x[col[p]]);
    dd_warp_sum(hi, lo);
    if (lane == 0) part[(int64_t)c * k + j] = make_double2(hi, lo);
}

// out(i, j) (m x k, ld k) = (A x_j)_i: the chunks of row i added in order in double-double,
// plus the low-rank part sum_q U(i, q) (V X^*)(q, j) (a float64 sum added once), rounded
// once. One thread per (i, j).
__global__ void spmv_rows_kernel(const int32_t* __restrict__ rchunk, const double2* __restrict__ part, int m, int k,
                                 int r, const double* __restrict__ U, const double* __restrict__ VX, double* out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * k) return;
    const int i = (int)(idx / k), j = (int)(idx % k);
    double hi = 0.0, lo = 0.0;
    for (int c = rchunk[i]; c < rchunk[i + 1]; ++c) {
        const double2 v = part[(int64_t)c * k + j];
        dd_add(hi, lo, v.x, v.y);
    }
    if (r > 0) {
        double t = 0.0;
        for (int q = 0; q < r; ++q) t = fma(U[(int64_t)i * r + q], VX[(int64_t)q * k + j], t);
        dd_add(hi, lo, t, 0.0);
    }
    out[idx] = hi + lo;
}

// out(j, c) = Y(j, c) - (A^* h_j)_c for h (m x k, ld k), rounded once from double-double:
// one thread per (j, c). The low-rank part adds sum_q V(q, c) (U^* h)(q, j) as one float64
// sum. out may be Y.
__global__ void spmvT_dd_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                                const double* __restrict__ cval, const double* __restrict__ H, int k, int n, int r,
                                const double* __restrict__ V, const double* __restrict__ UtH, const double* Y,
                                int64_t ldy, double* out, int64_t ldo) {
    const int j = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double hi = 0.0, lo = 0.0;
        for (int64_t p = cptr[c]; p < cptr[c + 1]; ++p) dd_fma_acc(hi, lo, cval[p], H[(int64_t)crow[p] * k + j]);
        if (r > 0) {
            double t = 0.0;
            for (int q = 0; q < r; ++q) t = fma(V[(int64_t)q * n + c], UtH[(int64_t)q * k + j], t);
            dd_add(hi, lo, t, 0.0);
        }
        double z, e;
        two_sum_d(Y[(int64_t)j * ldy + c], -hi, z, e);
        out[(int64_t)j * ldo + c] = z + (e - lo);
    }
}

__global__ void add_kernel(double* y, const double* x, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

unsigned grid_of(int64_t total, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, (int64_t)sm_count() * 32));
}

int row_threads(int m) { return std::min(256, (m + 31) / 32 * 32); }

// Low-rank helpers on the float64 GEMM: C (r x cols, ld ldc) = U^* Y for Y m x cols
// (ld ldy), and C = V Y^* for Y cols x n (ld ldy).
cudaError_t ut_times(const rtproj_ctx* h, const double* Y, int64_t ldy, int cols, double* C, int64_t ldc) {
    Gemm64 g;
    g.M = h->lr; g.N = cols; g.K = (int)h->m;
    g.A = h->lrU; g.a_rs = 1; g.a_cs = h->lr;
    g.B = Y; g.b_rs = ldy; g.b_cs = 1;
    g.C = C; g.c_rs = ldc; g.c_cs = 1;
    return gemm64(g, h->part, h->part_elems, h->stream);
}

cudaError_t v_times_t(const rtproj_ctx* h, const double* Y, int64_t ldy, int cols, double* C, int64_t ldc) {
    Narrow64 g;
    g.M = h->lr; g.N = cols; g.K = (int)h->n;
    g.A = h->lrV; g.a_rs = h->n;
    g.B = Y; g.b_rs = 1; g.b_cs = ldy;
    g.C = C; g.c_rs = ldc;
    return gemm64_narrow(g, h->part, h->part_elems, h->stream);
}

}  // namespace

namespace rtp {

int64_t sparse_max_chunks(int64_t m, int64_t nnz) { return m + nnz / SP_CHUNK + 1; }

size_t sparse_bytes(int64_t m, int64_t n, int64_t nnz, int64_t r, int64_t l_max, int64_t k_max) {
    const int64_t nb = (n + SCAN_T - 1) / SCAN_T;
    const int64_t nz = std::max<int64_t>(nnz, 1);
    const int64_t nc = sparse_max_chunks(m, nnz);
    return align_up((size_t)(n + 1) * 8) + align_up((size_t)nz * 4) + align_up((size_t)nz * 8) +
           align_up((size_t)n * 8) + align_up((size_t)nb * 8) + 2 * align_up((size_t)m * m * 8) +
           align_up((size_t)r * std::max(l_max, m) * 8) + align_up((size_t)r * k_max * 8) +
           align_up((size_t)(2 * r * r + norm_parts()) * 8) + align_up((size_t)nc * 4) + align_up((size_t)nc * 8) +
           align_up((size_t)(m + 1) * 4) + align_up((size_t)nc * k_max * 16);
}

void sparse_bind(rtproj_ctx* h, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base + off; off += align_up(bytes); return p; };
    const int64_t n = h->n, m = h->m, r = h->lr;
    const int64_t nz = std::max<int64_t>(h->nnz, 1);
    h->csc_ptr = (int64_t*)take((size_t)(n + 1) * 8);
    h->csc_row = (int32_t*)take((size_t)nz * 4);
    h->csc_val = (double*)take((size_t)nz * 8);
    h->csc_cursor = (int64_t*)take((size_t)n * 8);
    h->scan_tot = (int64_t*)take((size_t)((n + SCAN_T - 1) / SCAN_T) * 8);
    h->Pminus = (double*)take((size_t)m * m * 8);
    h->Esp = (double*)take((size_t)m * m * 8);
    h->lr_a = (double*)take((size_t)r * std::max(h->l_max, m) * 8);
    h->lr_b = (double*)take((size_t)r * h->k_max * 8);
    h->lr_small = (double*)take((size_t)(2 * r * r + norm_parts()) * 8);
    const int64_t nc = sparse_max_chunks(m, h->nnz);
    h->chunk_row = (int32_t*)take((size_t)nc * 4);
    h->chunk_beg = (int64_t*)take((size_t)nc * 8);
    h->row_chunk = (int32_t*)take((size_t)(m + 1) * 4);
    h->chunk_part = (double*)take((size_t)nc * h->k_max * 16);
}

// The chunk table from the row pointers (on the host): row i is cut into
// max(1, ceil(nnz_i / SP_CHUNK)) chunks. Copied to the device on the handle's stream.
rtproj_status sparse_chunks(rtproj_ctx* h, const int64_t* rp_host) {
    const int64_t m = h->m;
    std::vector<int32_t> crow, rch((size_t)m + 1);
    std::vector<int64_t> cbeg;
    for (int64_t i = 0; i < m; ++i) {
        rch[(size_t)i] = (int32_t)crow.size();
        const int64_t b = rp_host[i], e = rp_host[i + 1];
        int64_t p = b;
        do {
            crow.push_back((int32_t)i);
            cbeg.push_back(p);
            p += SP_CHUNK;
        } while (p < e);
    }
    rch[(size_t)m] = (int32_t)crow.size();
    h->nchunks = (int)crow.size();
    if ((int64_t)h->nchunks > sparse_max_chunks(m, h->nnz)) return RTPROJ_EINVAL;
    SP_CHECK(cudaMemcpyAsync(h->chunk_row, crow.data(), crow.size() * 4, cudaMemcpyHostToDevice, h->stream));
    SP_CHECK(cudaMemcpyAsync(h->chunk_beg, cbeg.data(), cbeg.size() * 8, cudaMemcpyHostToDevice, h->stream));
    SP_CHECK(cudaMemcpyAsync(h->row_chunk, rch.data(), rch.size() * 4, cudaMemcpyHostToDevice, h->stream));
    SP_CHECK(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
    return RTPROJ_OK;
}

// At create: the column-compressed copy, the value check and ||A||_F.
rtproj_status sparse_prepare(rtproj_ctx* h) {
    cudaStream_t s = h->stream;
    const int m = (int)h->m, n = (int)h->n, r = h->lr;
    const int64_t nnz = h->nnz;
    const int nb = (n + SCAN_T - 1) / SCAN_T;
    SP_CHECK(cudaMemsetAsync(h->csc_cursor, 0, (size_t)n * 8, s));
    if (nnz > 0) {
        count_cols_kernel<<<grid_of(nnz, 256), 256, 0, s>>>(h->csr_col, nnz, n, h->csc_cursor, h->status);
        check_values_kernel<<<grid_of(nnz, 256), 256, 0, s>>>(h->csr_val, nnz, h->status);
        note_launch(2);
    }
    block_totals_kernel<<<nb, SCAN_T, 0, s>>>(h->csc_cursor, n, h->scan_tot);
    scan_totals_kernel<<<1, SCAN_T, 0, s>>>(h->scan_tot, nb);
    block_scan_kernel<<<nb, SCAN_T, 0, s>>>(h->csc_cursor, n, h->scan_tot, h->csc_ptr);
    note_launch(3);
    SP_CHECK(cudaMemsetAsync(h->csc_cursor, 0, (size_t)n * 8, s));
    scatter_csc_kernel<<<(unsigned)std::min(m, sm_count() * 32), 256, 0, s>>>(
        h->csr_ptr, h->csr_col, h->csr_val, m, n, h->csc_ptr, h->csc_cursor, h->csc_row, h->csc_val);
    sort_columns_kernel<<<grid_of(n, 256), 256, 0, s>>>(h->csc_ptr, n, h->csc_row, h->csc_val);
    note_launch(2);
    if (r > 0) {   // the low-rank factors must be finite too
        check_values_kernel<<<grid_of((int64_t)m * r, 256), 256, 0, s>>>(h->lrU, (int64_t)m * r, h->status);
        check_values_kernel<<<grid_of((int64_t)r * n, 256), 256, 0, s>>>(h->lrV, (int64_t)r * n, h->status);
        note_launch(2);
    }
    // ||A||_F
    const unsigned np = std::min<unsigned>(grid_of(std::max<int64_t>(nnz, 1), 256), (unsigned)norm_parts());
    sumsq_vals_kernel<<<np, 256, 0, s>>>(h->csr_val, nnz, h->norm_part);
    note_launch();
    double* GU = h->lr_small;
    double* GV = GU + (size_t)r * r;
    double* px = GV + (size_t)r * r;
    unsigned nx = 0;
    if (r > 0) {
        nx = (unsigned)std::min(m, norm_parts());
        cross_term_kernel<<<nx, 256, 0, s>>>(h->csr_ptr, h->csr_col, h->csr_val, m, n, r, h->lrU, h->lrV, px);
        note_launch();
        Gemm64 u;                                 // U^* U
        u.M = r; u.N = r; u.K = m;
        u.A = h->lrU; u.a_rs = 1; u.a_cs = r;
        u.B = h->lrU; u.b_rs = r; u.b_cs = 1;
        u.C = GU; u.c_rs = r; u.c_cs = 1;
        SP_CHECK(gemm64(u, h->part, h->part_elems, s));
        Gemm64 v;                                 // V V^*
        v.M = r; v.N = r; v.K = n;
        v.A = h->lrV; v.a_rs = n; v.a_cs = 1;
        v.B = h->lrV; v.b_rs = 1; v.b_cs = n;
        v.C = GV; v.c_rs = r; v.c_cs = 1;
        SP_CHECK(gemm64(v, h->part, h->part_elems, s));
    }
    frobenius_total_kernel<<<1, 32, 0, s>>>(h->norm_part, (int)np, px, (int)nx, GU, GV, r, h->normA);
    note_launch();
    SP_CHECK(cudaGetLastError());
    return RTPROJ_OK;
}

rtproj_status sparse_sketch(rtproj_ctx* h, uint64_t seed, int64_t l, double* S, int64_t lds) {
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
    if (h->lr > 0) {   // V G (r x l), G generated where it is used
        Narrow64 g;
        g.M = h->lr; g.N = (int)l; g.K = (int)h->n;
        g.A = h->lrV; g.a_rs = h->n;
        g.omega_dist = h->opts.omega; g.seed = seed;
        g.C = h->lr_a; g.c_rs = l;
        SP_CHECK(gemm64_narrow(g, h->part, h->part_elems, h->stream));
    }
    const dim3 grid((unsigned)((l + 31) / 32), (unsigned)h->m);
    sparse_sketch_kernel<<<grid, 32 * SK_WARPS, 0, h->stream>>>(h->csr_ptr, h->csr_col, h->csr_val, (int)l,
                                                                h->opts.omega, k0, k1, h->lr, h->lrU, h->lr_a, l, S,
                                                                lds);
    note_launch();
    SP_CHECK(cudaGetLastError());
    return RTPROJ_OK;
}

// X = R^{-*} Pi A A^* P^- (lower triangle) into Lc; D = A^* P^- lives in W's region (n x m)
rtproj_status sparse_gram(rtproj_ctx* h) {
    const int m = (int)h->m, n = (int)h->n, r = h->lr;
    cudaStream_t s = h->stream;
    const int64_t mm = (int64_t)m * m;
    double* D = h->W;
    pminus_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(h->RinvT, h->perm, m, h->Pminus);
    note_launch();
    if (r > 0) SP_CHECK(ut_times(h, h->Pminus, m, m, h->lr_a, m));                    // U^* P^-
    sparse_d_kernel<<<(unsigned)std::min(n, sm_count() * 64), row_threads(m), 0, s>>>(
        h->csc_ptr, h->csc_row, h->csc_val, h->Pminus, m, n, r, h->lrV, h->lr_a, D);
    note_launch();
    if (r > 0) {                                                                        // V D
        Narrow64 g;
        g.M = r; g.N = m; g.K = n;
        g.A = h->lrV; g.a_rs = n;
        g.B = D; g.b_rs = m; g.b_cs = 1;
        g.C = h->lr_a; g.c_rs = m;
        SP_CHECK(gemm64_narrow(g, h->part, h->part_elems, s));
    }
    sparse_e_kernel<<<m, row_threads(m), 0, s>>>(h->csr_ptr, h->csr_col, h->csr_val, D, m, r, h->lrU, h->lr_a,
                                                 h->Esp);
    note_launch();
    Gemm64 x;                                                                           // R^{-*} (Pi E)
    x.M = m; x.N = m; x.K = m;
    x.A = h->RinvT; x.a_rs = m; x.a_cs = 1; x.a_tri = 1;
    x.B = h->Esp; x.b_rs = m; x.b_cs = 1; x.bk = h->perm;
    x.C = h->Lc; x.c_rs = m; x.c_cs = 1;
    x.lower_only = true;
    SP_CHECK(gemm64(x, h->part, h->part_elems, s));
    SP_CHECK(cudaGetLastError());
    return RTPROJ_OK;
}

rtproj_status sparse_project(rtproj_ctx* h, const double* B, int64_t ldb, int k, void* Z, int64_t ldz, void* ROW,
                             int64_t ldr, void* X, int64_t ldx) {
    const rtproj_opts& o = h->opts;
    const int m = (int)h->m, n = (int)h->n, r = h->lr;
    cudaStream_t s = h->stream;
    const int64_t mk = (int64_t)m * k;
    const int64_t ck = (int64_t)h->nchunks * k;
    const unsigned chunk_blocks = (unsigned)((ck * 32 + 255) / 256);
    double2* part = reinterpret_cast<double2*>(h->chunk_part);
    const dim3 tgrid((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8 / k + 1)),
                     (unsigned)k);
    SP_CHECK(row_norms(B, ldb, k, n, h->bnorm, s));
    SP_CHECK(cudaMemsetAsync(h->stats, 0, 16, s));
    auto apply_a = [&](const double* Xr, int64_t ldxr, double* out) -> rtproj_status {   // out = A x
        phase_begin(h, RTPROJ_PHASE_APPLY_A);
        if (r > 0) SP_CHECK(v_times_t(h, Xr, ldxr, k, h->lr_b, k));
        spmv_chunk_kernel<<<chunk_blocks, 256, 0, s>>>(h->chunk_row, h->chunk_beg, h->csr_ptr, h->csr_col,
                                                       h->csr_val, Xr, ldxr, h->nchunks, k, part);
        spmv_rows_kernel<<<(unsigned)((mk + 255) / 256), 256, 0, s>>>(h->row_chunk, part, m, k, r, h->lrU, h->lr_b,
                                                                      out);
        note_launch(2);
        phase_end(h, RTPROJ_PHASE_APPLY_A);
        return RTPROJ_OK;
    };
    auto apply_at = [&](const double* Hm, const double* Y, int64_t ldy) -> rtproj_status {   // sbuf = Y - A^* h
        phase_begin(h, RTPROJ_PHASE_APPLY_AT);
        if (r > 0) SP_CHECK(ut_times(h, Hm, k, k, h->lr_b, k));
        spmvT_dd_kernel<<<tgrid, 256, 0, s>>>(h->csc_ptr, h->csc_row, h->csc_val, Hm, k, n, r, h->lrV, h->lr_b, Y,
                                              ldy, h->sbuf, n);
        note_launch();
        phase_end(h, RTPROJ_PHASE_APPLY_AT);
        return RTPROJ_OK;
    };
    // c = A b; h0 = Pi^* T1^* T1 Pi c; s = b - A^* h0
    rtproj_status st = apply_a(B, ldb, h->cbuf);
    if (st != RTPROJ_OK) return st;
    phase_begin(h, RTPROJ_PHASE_APPLY_M);
    st = middle_fp64(h, h->cbuf, h->hbuf, k);
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_APPLY_M);
    st = apply_at(h->hbuf, B, ldb);
    if (st != RTPROJ_OK) return st;
    int passes = 0;
    for (int pass = 0; pass < o.refine_passes; ++pass) {
        // r = A s; dh = Pi^* T1^* T1 Pi r; h += dh; s <- s - A^* dh (Remark 4.3)
        st = apply_a(h->sbuf, n, h->cbuf);
        if (st != RTPROJ_OK) return st;
        phase_begin(h, RTPROJ_PHASE_APPLY_M);
        st = middle_fp64(h, h->cbuf, h->dhbuf, k);
        if (st != RTPROJ_OK) return st;
        add_kernel<<<(unsigned)((mk + 255) / 256), 256, 0, s>>>(h->hbuf, h->dhbuf, mk);
        note_launch();
        SP_CHECK(cudaMemsetAsync(h->stats, 0, 16, s));
        SP_CHECK(column_stats(h->cbuf, h->hbuf, h->dhbuf, m, k, h->bnorm, h->normA, h->stats, s));
        phase_end(h, RTPROJ_PHASE_APPLY_M);
        passes = pass + 1;
        bool last = passes == o.refine_passes;
        if (o.refine_tol > 0.0 && !last) {
            unsigned long long bits[2];
            SP_CHECK(cudaMemcpyAsync(bits, h->stats, 16, cudaMemcpyDeviceToHost, s));
            SP_CHECK(cudaStreamSynchronize(s));
            double v[2];
            std::memcpy(v, bits, 16);
            if (v[1] <= o.refine_tol) last = true;
        }
        st = apply_at(h->dhbuf, h->sbuf, n);   // in place: each entry reads its own s first
        if (st != RTPROJ_OK) return st;
        if (last) break;
    }
    h->last_passes = passes;
    if (ROW) SP_CHECK(store_rows(h->sbuf, n, B, ldb, ROW, ldr, k, n, 1, RTPROJ_F64, s));
    if (Z) SP_CHECK(store_rows(h->sbuf, n, nullptr, 0, Z, ldz, k, n, 0, RTPROJ_F64, s));
    if (X) SP_CHECK(store_transposed(h->hbuf, k, m, k, X, ldx, RTPROJ_F64, s));
    SP_CHECK(cudaGetLastError());
    return RTPROJ_OK;
}

}  // namespace rtp
