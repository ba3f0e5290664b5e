// Boundary kernels: element types at the C ABI (float32 A and right-hand sides are
// widened to float64 exactly; outputs are stored in the caller's element type), the
// Frobenius norm of A, and the per-right-hand-side norms behind the residual report of
// rtproj_get_info (Section 5 measures delta = ||A z||; here it is normalised by ||A||_F
// and ||b||).
#include "rtproj_internal.cuh"

#include <algorithm>

namespace rtp {
namespace {

constexpr int BT = 256;

__global__ void widen_kernel(const float* __restrict__ src, int64_t lds, int rows, int cols, double* __restrict__ dst,
                             int64_t ldd) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / cols, c = idx % cols;
        dst[r * ldd + c] = (double)src[r * lds + c];
    }
}

// dst = src diag(d) (d optional), widened to float64
template <typename T>
__global__ void form_rows_kernel(const T* __restrict__ src, int64_t lds, int rows, int cols, const double* __restrict__ d,
                                 double* __restrict__ dst, int64_t ldd) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / cols, c = idx % cols;
        const double x = (double)src[r * lds + c];
        dst[r * ldd + c] = d ? x * d[c] : x;
    }
}

template <typename T>
__global__ void store_rows_kernel(const double* __restrict__ X, int64_t ldx, const double* __restrict__ B, int64_t ldb,
                                  T* __restrict__ dst, int64_t ldd, int rows, int cols, int sub) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / cols, c = idx % cols;
        const double x = X[r * ldx + c];
        dst[r * ldd + c] = (T)(sub ? B[r * ldb + c] - x : x);
    }
}

// 32 x 32 tiles through shared memory: reads of src and writes of dst both coalesced.
template <typename T>
__global__ void store_transposed_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols,
                                        T* __restrict__ dst, int64_t ldd) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int y = ty; y < 32; y += 8) {
        const int r = r0 + y, c = c0 + tx;
        tile[y][tx] = (r < rows && c < cols) ? src[(int64_t)r * lds + c] : 0.0;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int c = c0 + y, r = r0 + tx;
        if (c < cols && r < rows) dst[(int64_t)c * ldd + r] = (T)tile[tx][y];
    }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;   // valid in thread 0
}

// Sum of squares of X in a fixed grid-stride order: part[b] for CTA b.
__global__ void sumsq_kernel(const double* __restrict__ X, int64_t ldx, int rows, int cols, double* part) {
    __shared__ double red[BT / 32];
    const int64_t total = (int64_t)rows * cols;
    double s0 = 0.0, s1 = 0.0;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; idx + stride < total; idx += 2 * stride) {
        const double a = X[(idx / cols) * ldx + idx % cols];
        const int64_t i2 = idx + stride;
        const double b = X[(i2 / cols) * ldx + i2 % cols];
        s0 = fma(a, a, s0);
        s1 = fma(b, b, s1);
    }
    if (idx < total) {
        const double a = X[(idx / cols) * ldx + idx % cols];
        s0 = fma(a, a, s0);
    }
    const double s = block_sum(s0 + s1, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sqrt_sum_kernel(const double* part, int nparts, double* out) {
    __shared__ double red[BT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = sqrt(s);
}

// One CTA per row.
__global__ void row_norms_kernel(const double* __restrict__ X, int64_t ldx, int n, double* out) {
    __shared__ double red[BT / 32];
    const double* row = X + (int64_t)blockIdx.x * ldx;
    double s0 = 0.0, s1 = 0.0;
    int c = threadIdx.x;
    for (; c + BT < n; c += 2 * BT) {
        s0 = fma(row[c], row[c], s0);
        s1 = fma(row[c + BT], row[c + BT], s1);
    }
    if (c < n) s0 = fma(row[c], row[c], s0);
    const double s = block_sum(s0 + s1, red);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

__device__ __forceinline__ void max_bits(unsigned long long* p, double v) {
    // non-negative doubles order like their bit patterns; NaN lands above every finite value
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// One CTA per right-hand side j (column j of the m x k blocks).
__global__ void column_stats_kernel(const double* r, const double* h, const double* dh, int m, int k,
                                    const double* bnorm, const double* normA, unsigned long long* stats) {
    __shared__ double red[BT / 32];
    const int j = blockIdx.x;
    double sr = 0.0, sh = 0.0, sd = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int64_t at = (int64_t)i * k + j;
        if (r) sr = fma(r[at], r[at], sr);
        if (dh) {
            sh = fma(h[at], h[at], sh);
            sd = fma(dh[at], dh[at], sd);
        }
    }
    if (r) {
        const double t = block_sum(sr, red);
        if (threadIdx.x == 0) {
            const double den = *normA * bnorm[j];
            max_bits(&stats[0], den > 0.0 ? sqrt(t) / den : sqrt(t));
        }
    }
    if (dh) {
        // relative to ||h||, or to ||b|| / ||A||_F when h is smaller than that (a b already
        // near the null space): ||A||_F ||dh|| bounds the change A^* dh makes to Zb
        const double th = block_sum(sh, red);
        const double td = block_sum(sd, red);
        if (threadIdx.x == 0) {
            const double scale = fmax(sqrt(th), *normA > 0.0 ? bnorm[j] / *normA : 0.0);
            max_bits(&stats[1], scale > 0.0 ? sqrt(td) / scale : sqrt(td));
        }
    }
}

unsigned grid_for(int64_t total) {
    const int64_t blocks = (total + BT - 1) / BT;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
}

}  // namespace

cudaError_t widen_rows(const float* src, int64_t lds, int rows, int cols, double* dst, int64_t ldd, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    widen_kernel<<<grid_for((int64_t)rows * cols), BT, 0, s>>>(src, lds, rows, cols, dst, ldd);
    note_launch();
    return cudaGetLastError();
}

cudaError_t form_rows(const void* src, int dt, int64_t lds, int rows, int cols, const double* d, double* dst, int64_t ldd,
                      cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const unsigned g = grid_for((int64_t)rows * cols);
    if (dt == RTPROJ_F32)
        form_rows_kernel<float><<<g, BT, 0, s>>>((const float*)src, lds, rows, cols, d, dst, ldd);
    else
        form_rows_kernel<double><<<g, BT, 0, s>>>((const double*)src, lds, rows, cols, d, dst, ldd);
    note_launch();
    return cudaGetLastError();
}

cudaError_t store_rows(const double* X, int64_t ldx, const double* B, int64_t ldb, void* dst, int64_t ldd, int rows,
                       int cols, int sub, int dt, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const unsigned g = grid_for((int64_t)rows * cols);
    if (dt == RTPROJ_F32)
        store_rows_kernel<float><<<g, BT, 0, s>>>(X, ldx, B, ldb, (float*)dst, ldd, rows, cols, sub);
    else
        store_rows_kernel<double><<<g, BT, 0, s>>>(X, ldx, B, ldb, (double*)dst, ldd, rows, cols, sub);
    note_launch();
    return cudaGetLastError();
}

cudaError_t store_transposed(const double* src, int64_t lds, int rows, int cols, void* dst, int64_t ldd, int dt,
                             cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    if (dt == RTPROJ_F32)
        store_transposed_kernel<float><<<grid, 256, 0, s>>>(src, lds, rows, cols, (float*)dst, ldd);
    else
        store_transposed_kernel<double><<<grid, 256, 0, s>>>(src, lds, rows, cols, (double*)dst, ldd);
    note_launch();
    return cudaGetLastError();
}

int norm_parts() { return 4096; }

cudaError_t frobenius(const double* X, int64_t ldx, int rows, int cols, double* part, double* out, cudaStream_t s) {
    const unsigned g = std::min<unsigned>(grid_for((int64_t)rows * cols), (unsigned)norm_parts());
    sumsq_kernel<<<g, BT, 0, s>>>(X, ldx, rows, cols, part);
    sqrt_sum_kernel<<<1, BT, 0, s>>>(part, (int)g, out);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t row_norms(const double* X, int64_t ldx, int k, int n, double* out, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    row_norms_kernel<<<k, BT, 0, s>>>(X, ldx, n, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t column_stats(const double* r, const double* h, const double* dh, int m, int k, const double* bnorm,
                         const double* normA, unsigned long long* stats, cudaStream_t s) {
    if (k <= 0 || (!r && !dh)) return cudaSuccess;
    column_stats_kernel<<<k, BT, 0, s>>>(r, h, dh, m, k, bnorm, normA, stats);
    note_launch();
    return cudaGetLastError();
}

}  // namespace rtp
