// float64 GEMM on the FP64 pipe (the plain float64 form) and small helpers.
//
// The plain form runs every product of the method -- the sketch S = A G (Eq. 12),
// the Gram matrix X = P^{-1} A A^* P^{-*} (Section 4, steps a-e, done as two GEMMs),
// and the apply c = A b, the m x m stage, b - A^* h (the seven steps) -- through this
// kernel. GB300's FP64 pipe is ~1.2 TFLOP/s, so a 64x64 tile with a 4x4 register
// block per thread already saturates it; no tensor cores are involved here.
#include "rtproj_internal.cuh"

#include <algorithm>

namespace rtp {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct Gemm64Dev {
    int M, N, K, k_per_split;
    const double* A; int64_t a_rs, a_cs; const int32_t* arow;
    const double* B; int64_t b_rs, b_cs; const int32_t* bk;
    int omega_dist; uint32_t key0, key1;
    double* P;                     // partial slabs (split > 1)
    int lower_only;
    int a_tri;
    // direct epilogue (one split)
    double* C; int64_t c_rs, c_cs; const int32_t* crow;
    double alpha, beta;
    const double* Cin; int64_t cin_rs, cin_cs;
};

__global__ void __launch_bounds__(NT) gemm64_kernel(Gemm64Dev p) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN, z = blockIdx.z;
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    double* out = gridDim.z > 1 ? p.P + (size_t)z * p.M * p.N : nullptr;
    if (p.lower_only && j0 > i0 + BM - 1) return;   // tile strictly above the diagonal
    const int kbeg = z * p.k_per_split;
    const int kend = min(p.K, kbeg + p.k_per_split);
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    // triangular A: only k <= i (lower) or k >= i (upper) can be nonzero for this tile's rows
    int klo = kbeg, khi = kend;
    if (p.a_tri == 1) khi = min(khi, i0 + BM);
    if (p.a_tri == 2) klo = max(klo, (i0 / BK) * BK);
    for (int k0 = klo; k0 < khi; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = t + NT * r;
            int ii, kk;
            if (p.a_cs == 1) { ii = e / BK; kk = e % BK; } else { kk = e / BM; ii = e % BM; }
            const int gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < p.M && gk < kend) {
                const int64_t row = p.arow ? (int64_t)p.arow[gi] : (int64_t)gi;
                v = p.A[row * p.a_rs + (int64_t)gk * p.a_cs];
            }
            As[kk][ii] = v;
        }
        if (p.omega_dist == RTPROJ_OMEGA_GAUSSIAN) {
            // k0 is a multiple of 16: four Philox blocks give the 16 rows of column j.
            if (t < BN) {
                const int gj = j0 + t;
#pragma unroll
                for (int qd = 0; qd < BK / 4; ++qd) {
                    int N[4] = {0, 0, 0, 0};
                    if (gj < p.N) gauss_quad((uint32_t)((k0 >> 2) + qd), (uint32_t)gj, p.key0, p.key1, N);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int kk = 4 * qd + b;
                        Bs[kk][t] = (gj < p.N && k0 + kk < kend) ? (double)N[b] * (1.0 / 4096.0) : 0.0;
                    }
                }
            }
        } else if (p.omega_dist >= 0) {
            // k0 is a multiple of 16: one Philox block covers the 16 rows of column j.
            if (t < BN) {
                const int gj = j0 + t;
                uint4 w = make_uint4(0, 0, 0, 0);
                if (gj < p.N) w = philox4x32_10(make_uint4((uint32_t)(k0 >> 4), (uint32_t)gj, 0u, 0u), p.key0, p.key1);
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    const int gk = k0 + kk;
                    Bs[kk][t] = (gj < p.N && gk < kend) ? (double)omega_from_byte(block_byte(w, kk), p.omega_dist) : 0.0;
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int e = t + NT * r;
                int jj, kk;
                if (p.b_cs == 1) { kk = e / BN; jj = e % BN; } else { jj = e / BK; kk = e % BK; }
                const int gj = j0 + jj, gk = k0 + kk;
                double v = 0.0;
                if (gj < p.N && gk < kend) {
                    const int64_t row = p.bk ? (int64_t)p.bk[gk] : (int64_t)gk;
                    v = p.B[row * p.b_rs + (int64_t)gj * p.b_cs];
                }
                Bs[kk][jj] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
    const bool direct = gridDim.z == 1;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int gi = i0 + ty * 4 + x;
        if (gi >= p.M) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gj = j0 + tx * 4 + y;
            if (gj >= p.N) continue;
            if (!direct) {
                out[(size_t)gi * p.N + gj] = acc[x][y];
            } else if (!(p.lower_only && gj > gi)) {
                double v = p.alpha * acc[x][y];
                if (p.beta != 0.0) v += p.beta * p.Cin[(int64_t)gi * p.cin_rs + (int64_t)gj * p.cin_cs];
                const int64_t row = p.crow ? (int64_t)p.crow[gi] : (int64_t)gi;
                p.C[row * p.c_rs + (int64_t)gj * p.c_cs] = v;
            }
        }
    }
}

struct ReduceDev {
    int M, N, splits;
    const double* P;
    double* C; int64_t c_rs, c_cs; const int32_t* crow;
    double alpha, beta;
    const double* Cin; int64_t cin_rs, cin_cs;
    int lower_only;
};

__global__ void reduce_kernel(ReduceDev r) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)r.M * r.N;
    if (idx >= total) return;
    const int i = (int)(idx / r.N), j = (int)(idx % r.N);
    if (r.lower_only && j > i) return;
    double s = 0.0;
    for (int z = 0; z < r.splits; ++z) s += r.P[(size_t)z * total + idx];
    double v = r.alpha * s;
    if (r.beta != 0.0) v += r.beta * r.Cin[(int64_t)i * r.cin_rs + (int64_t)j * r.cin_cs];
    const int64_t row = r.crow ? (int64_t)r.crow[i] : (int64_t)i;
    r.C[row * r.c_rs + (int64_t)j * r.c_cs] = v;
}

__global__ void set_identity_kernel(double* X, int m) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    X[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
}

__global__ void zero_upper_kernel(double* X, int m) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    if (idx % m > idx / m) X[idx] = 0.0;
}

__global__ void transpose_kernel(const double* src, int64_t s_rs, double* dst, int64_t d_rs, int rows, int cols) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = src[(int64_t)r * s_rs + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(int64_t)c * d_rs + r] = tile[threadIdx.x][y];
    }
}

__global__ void check_finite_kernel(const double* X, int64_t rs, int rows, int cols, int* status) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * cols) return;
    const double v = X[(idx / cols) * rs + idx % cols];
    if (!isfinite(v)) set_status(status, RTPROJ_ENONFINITE);
}

}  // namespace

cudaError_t gemm64(const Gemm64& g, double* part, size_t part_elems, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const int tiles_m = (g.M + BM - 1) / BM, tiles_n = (g.N + BN - 1) / BN;
    const size_t slab = (size_t)g.M * g.N;
    int splits = 1;
    if (g.K > 0) {
        const int tiles = tiles_m * tiles_n;
        const int want = std::max(1, (4 * sm_count() + tiles - 1) / tiles);
        // Few output tiles (the m x m by m x k products of the apply): splits down to one
        // 16-k step, so that the small FP64 products use every SM; otherwise at least four.
        const int maxk = tiles < 32 ? std::max(1, (g.K + BK - 1) / BK) : std::max(1, (g.K + 63) / 64);
        splits = std::min(want, maxk);
        splits = (int)std::min<size_t>((size_t)splits, std::max<size_t>(1, part_elems / slab));
    }
    if (slab > part_elems) splits = 1;
    int kps = (g.K + splits - 1) / splits;
    kps = ((kps + BK - 1) / BK) * BK;
    splits = g.K > 0 ? (g.K + kps - 1) / kps : 1;
    Gemm64Dev p;
    p.M = g.M; p.N = g.N; p.K = g.K; p.k_per_split = std::max(kps, BK);
    p.A = g.A; p.a_rs = g.a_rs; p.a_cs = g.a_cs; p.arow = g.arow;
    p.B = g.B; p.b_rs = g.b_rs; p.b_cs = g.b_cs; p.bk = g.bk;
    p.omega_dist = g.omega_dist;
    p.key0 = (uint32_t)(g.seed & 0xFFFFFFFFull); p.key1 = (uint32_t)(g.seed >> 32);
    p.P = part;
    p.lower_only = g.lower_only ? 1 : 0;
    p.a_tri = g.a_tri;
    p.C = g.C; p.c_rs = g.c_rs; p.c_cs = g.c_cs; p.crow = g.crow;
    p.alpha = g.alpha; p.beta = g.beta; p.Cin = g.Cin; p.cin_rs = g.cin_rs; p.cin_cs = g.cin_cs;
    if (g.K <= 0) return cudaErrorInvalidValue;
    {
        dim3 grid(tiles_n, tiles_m, splits);
        gemm64_kernel<<<grid, NT, 0, s>>>(p);
        note_launch();
    }
    if (splits == 1) return cudaGetLastError();
    ReduceDev r;
    r.M = g.M; r.N = g.N; r.splits = splits; r.P = part;
    r.C = g.C; r.c_rs = g.c_rs; r.c_cs = g.c_cs; r.crow = g.crow;
    r.alpha = g.alpha; r.beta = g.beta; r.Cin = g.Cin; r.cin_rs = g.cin_rs; r.cin_cs = g.cin_cs;
    r.lower_only = g.lower_only ? 1 : 0;
    const int64_t total = (int64_t)slab;
    reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(r);
    note_launch();
    return cudaGetLastError();
}

cudaError_t set_identity(double* X, int m, cudaStream_t s) {
    const int64_t total = (int64_t)m * m;
    set_identity_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, m);
    note_launch();
    return cudaGetLastError();
}

cudaError_t zero_upper(double* X, int m, cudaStream_t s) {
    const int64_t total = (int64_t)m * m;
    zero_upper_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, m);
    note_launch();
    return cudaGetLastError();
}

cudaError_t transpose_copy(const double* src, int64_t s_rs, double* dst, int64_t d_rs, int rows, int cols, cudaStream_t s) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(src, s_rs, dst, d_rs, rows, cols);
    note_launch();
    return cudaGetLastError();
}

cudaError_t check_finite(const double* X, int64_t rs, int rows, int cols, int* status, cudaStream_t s) {
    const int64_t total = (int64_t)rows * cols;
    if (total == 0) return cudaSuccess;
    check_finite_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, rs, rows, cols, status);
    note_launch();
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------
// Narrow products C (M x N) = A (M x K) B (K x N) with M <= 64 (the rows of a low-rank
// factor) and a long K: the 64 x 64 tiles of gemm64 would waste most of their rows. The K
// range is cut into chunks; a CTA takes one chunk and a range of columns j and keeps NR
// rows' partial sums per column in registers, reading A's chunk from shared memory. B is
// read with the columns j contiguous (one thread per column), or with K contiguous (a warp
// per column, lanes over k), or generated (G of Eq. 12). The chunks' partial sums are
// added in chunk order by a second kernel (deterministic).
// ---------------------------------------------------------------------------------
namespace {

constexpr int NR_ROWS = 16;     // rows per register pass
constexpr int NR_KC = 64;       // K entries of A staged per pass
constexpr int NR_T = 256;

struct NarrowDev {
    int M, N, K, kchunk;
    const double* A; int64_t a_rs;
    const double* B; int64_t b_rs, b_cs;
    int omega_dist; uint32_t key0, key1;
    double* part;               // [chunk][M][N]
};

__device__ __forceinline__ double narrow_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// B(k, j) for k = k0 .. k0 + 3 (k0 a multiple of 4), zero at k >= ke, into b[0..3]
__device__ __forceinline__ void narrow_b4(const NarrowDev& p, int k0, int ke, int j, double (&b)[4]) {
    if (p.omega_dist == RTPROJ_OMEGA_GAUSSIAN) {
        int N4[4];
        gauss_quad((uint32_t)(k0 >> 2), (uint32_t)j, p.key0, p.key1, N4);
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = k0 + u < ke ? (double)N4[u] * (1.0 / 4096.0) : 0.0;
    } else if (p.omega_dist >= 0) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(k0 >> 4), (uint32_t)j, 0u, 0u), p.key0, p.key1);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            b[u] = k0 + u < ke ? (double)omega_from_byte(block_byte(w, (k0 & 15) + u), p.omega_dist) : 0.0;
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = k0 + u < ke ? p.B[(int64_t)(k0 + u) * p.b_rs + (int64_t)j * p.b_cs] : 0.0;
    }
}

// one thread per column j; rows [r0, r0 + NR_ROWS) of A; chunk blockIdx.y
__global__ void __launch_bounds__(NR_T) narrow_rows_kernel(NarrowDev p) {
    __shared__ double As[NR_ROWS][NR_KC];
    const int j = blockIdx.x * NR_T + threadIdx.x;
    const int kb = blockIdx.y * p.kchunk, ke = min(p.K, kb + p.kchunk);
    for (int r0 = 0; r0 < p.M; r0 += NR_ROWS) {
        double acc[NR_ROWS];
#pragma unroll
        for (int i = 0; i < NR_ROWS; ++i) acc[i] = 0.0;
        for (int k0 = kb; k0 < ke; k0 += NR_KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < NR_ROWS * NR_KC; e += NR_T) {
                const int i = e / NR_KC, k = k0 + e % NR_KC;
                As[i][e % NR_KC] = (r0 + i < p.M && k < ke) ? p.A[(int64_t)(r0 + i) * p.a_rs + k] : 0.0;
            }
            __syncthreads();
            if (j < p.N) {
                const int kn = min(NR_KC, ke - k0);
                for (int kk = 0; kk < kn; kk += 4) {
                    double b[4];
                    narrow_b4(p, k0 + kk, ke, j, b);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int i = 0; i < NR_ROWS; ++i) acc[i] = fma(As[i][kk + u], b[u], acc[i]);
                }
            }
        }
        if (j < p.N) {
#pragma unroll
            for (int i = 0; i < NR_ROWS; ++i)
                if (r0 + i < p.M) p.part[((int64_t)blockIdx.y * p.M + r0 + i) * p.N + j] = acc[i];
        }
    }
}

// one warp per column j, lanes over k (B with K contiguous: b_rs == 1)
__global__ void __launch_bounds__(NR_T) narrow_cols_kernel(NarrowDev p) {
    __shared__ double As[NR_ROWS][NR_KC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * (NR_T / 32) + warp;
    const int kb = blockIdx.y * p.kchunk, ke = min(p.K, kb + p.kchunk);
    for (int r0 = 0; r0 < p.M; r0 += NR_ROWS) {
        double acc[NR_ROWS];
#pragma unroll
        for (int i = 0; i < NR_ROWS; ++i) acc[i] = 0.0;
        for (int k0 = kb; k0 < ke; k0 += NR_KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < NR_ROWS * NR_KC; e += NR_T) {
                const int i = e / NR_KC, k = k0 + e % NR_KC;
                As[i][e % NR_KC] = (r0 + i < p.M && k < ke) ? p.A[(int64_t)(r0 + i) * p.a_rs + k] : 0.0;
            }
            __syncthreads();
            if (j < p.N)
                for (int kk = lane; kk < NR_KC && k0 + kk < ke; kk += 32) {
                    const double b = p.B[(int64_t)(k0 + kk) + (int64_t)j * p.b_cs];
#pragma unroll
                    for (int i = 0; i < NR_ROWS; ++i) acc[i] = fma(As[i][kk], b, acc[i]);
                }
        }
#pragma unroll
        for (int i = 0; i < NR_ROWS; ++i) acc[i] = narrow_warp_sum(acc[i]);
        if (j < p.N && lane == 0) {
#pragma unroll
            for (int i = 0; i < NR_ROWS; ++i)
                if (r0 + i < p.M) p.part[((int64_t)blockIdx.y * p.M + r0 + i) * p.N + j] = acc[i];
        }
    }
}

__global__ void narrow_reduce_kernel(const double* part, int chunks, int M, int N, double* C, int64_t c_rs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * N) return;
    const int i = (int)(idx / N), j = (int)(idx % N);
    double s = 0.0;
    for (int z = 0; z < chunks; ++z) s += part[((int64_t)z * M + i) * N + j];
    C[(int64_t)i * c_rs + j] = s;
}

}  // namespace

cudaError_t gemm64_narrow(const Narrow64& g, double* part, size_t part_elems, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (g.M > 64 || g.K <= 0) return cudaErrorInvalidValue;
    const bool cols = g.omega_dist < 0 && g.b_rs == 1;
    const int per_block = cols ? NR_T / 32 : NR_T;
    const int gx = (g.N + per_block - 1) / per_block;
    // chunks: about four CTAs per SM in all, each chunk a multiple of 16 (whole Philox blocks)
    const int want = std::max(1, 4 * sm_count() / gx);
    const size_t cap = std::max<size_t>(1, part_elems / ((size_t)g.M * g.N));
    int chunks = (int)std::min<size_t>((size_t)std::min(want, 65535), cap);
    int kchunk = (g.K + chunks - 1) / chunks;
    kchunk = (kchunk + 15) / 16 * 16;
    chunks = (g.K + kchunk - 1) / kchunk;
    if ((size_t)chunks * g.M * g.N > part_elems) return cudaErrorInvalidValue;
    NarrowDev p;
    p.M = g.M; p.N = g.N; p.K = g.K; p.kchunk = kchunk;
    p.A = g.A; p.a_rs = g.a_rs;
    p.B = g.B; p.b_rs = g.b_rs; p.b_cs = g.b_cs;
    p.omega_dist = g.omega_dist;
    p.key0 = (uint32_t)(g.seed & 0xFFFFFFFFull); p.key1 = (uint32_t)(g.seed >> 32);
    p.part = part;
    const dim3 grid((unsigned)gx, (unsigned)chunks);
    if (cols) narrow_cols_kernel<<<grid, NR_T, 0, s>>>(p);
    else narrow_rows_kernel<<<grid, NR_T, 0, s>>>(p);
    const int64_t total = (int64_t)g.M * g.N;
    narrow_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, chunks, g.M, g.N, g.C, g.c_rs);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace rtp
