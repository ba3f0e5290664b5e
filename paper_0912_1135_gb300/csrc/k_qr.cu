// Pivoted Householder QR of S^* (Section 4, Eq. 13) on the GPU, float64.
//
// S is m x l row-major, so column c of S^* (l x m) is row c of S: contiguous, which
// makes every reflector application a coalesced dot product + axpy over a row.
// Businger-Golub column pivoting with LAPACK-style norm downdating (vn1 the
// downdated norm, vn2 the norm at the last exact recomputation; recompute when the
// downdate loses more than half the digits). Per step j:
//   kernel 1 (one CTA): argmax of vn1 over the remaining columns (lowest index on
//     ties), swap the pivot row into place (R entries travel with it), build the
//     reflector v, beta with alpha = -sign(x_1) ||x|| for x = S[j][j..l).
//   kernel 2 (one warp per remaining column): apply I - beta v v^* and downdate.
// On exit R[i][c] = S[c][i] (i <= c) and S[:, perm] factors as in Eq. 13.
#include "rtproj_internal.cuh"

namespace rtp {
namespace {

constexpr int PIV_THREADS = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void qr_init_kernel(const double* S, int m, int l, int64_t lds, double* vn1, double* vn2, int32_t* perm) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= m) return;
    const double* row = S + (int64_t)warp * lds;
    double s = 0.0;
    for (int t = lane; t < l; t += 32) s = fma(row[t], row[t], s);
    s = warp_sum(s);
    if (lane == 0) {
        vn1[warp] = sqrt(s);
        vn2[warp] = sqrt(s);
        perm[warp] = warp;
    }
}

__global__ void __launch_bounds__(PIV_THREADS) qr_pivot_kernel(double* S, int m, int l, int64_t lds, int j,
                                                               double* vn1, double* vn2, int32_t* perm,
                                                               double* v, double* scal) {
    __shared__ double sval[PIV_THREADS / 32];
    __shared__ int sidx[PIV_THREADS / 32];
    __shared__ double snorm[PIV_THREADS / 32];
    __shared__ int piv_s;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // 1. pivot: largest vn1 over [j, m), lowest index on ties
    double best = -1.0;
    int bi = m;
    for (int c = j + t; c < m; c += PIV_THREADS) {
        const double x = vn1[c];
        if (x > best || (x == best && c < bi)) { best = x; bi = c; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { sval[wid] = best; sidx[wid] = bi; }
    __syncthreads();
    if (t == 0) {
        double b = sval[0];
        int i = sidx[0];
        for (int w = 1; w < PIV_THREADS / 32; ++w)
            if (sval[w] > b || (sval[w] == b && sidx[w] < i)) { b = sval[w]; i = sidx[w]; }
        piv_s = (i >= m) ? j : i;
    }
    __syncthreads();
    const int piv = piv_s;
    double* rj = S + (int64_t)j * lds;
    if (piv != j) {
        double* rp = S + (int64_t)piv * lds;
        for (int c = t; c < l; c += PIV_THREADS) {
            const double a = rj[c];
            rj[c] = rp[c];
            rp[c] = a;
        }
        if (t == 0) {
            double a = vn1[j]; vn1[j] = vn1[piv]; vn1[piv] = a;
            a = vn2[j]; vn2[j] = vn2[piv]; vn2[piv] = a;
            const int32_t q = perm[j]; perm[j] = perm[piv]; perm[piv] = q;
        }
    }
    __syncthreads();
    // 2. reflector for x = S[j][j..l)
    double s = 0.0;
    for (int c = j + t; c < l; c += PIV_THREADS) s = fma(rj[c], rj[c], s);
    s = warp_sum(s);
    if (lane == 0) snorm[wid] = s;
    __syncthreads();
    if (t == 0) {
        double nx2 = 0.0;
        for (int w = 0; w < PIV_THREADS / 32; ++w) nx2 += snorm[w];
        const double nx = sqrt(nx2);
        const double x0 = rj[j];
        double alpha = 0.0, beta = 0.0;
        if (nx > 0.0) {
            alpha = x0 >= 0.0 ? -nx : nx;
            beta = 1.0 / (nx * (nx + fabs(x0)));
        }
        scal[0] = alpha;
        scal[1] = beta;
        v[0] = x0 - alpha;
        vn1[j] = fabs(alpha);
    }
    for (int c = j + 1 + t; c < l; c += PIV_THREADS) v[c - j] = rj[c];
    __syncthreads();
    if (t == 0) rj[j] = scal[0];
    for (int c = j + 1 + t; c < l; c += PIV_THREADS) rj[c] = 0.0;
}

__global__ void qr_apply_kernel(double* S, int m, int l, int64_t lds, int j, double* vn1, double* vn2,
                                const double* v, const double* scal) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int c = j + 1 + warp;
    if (c >= m) return;
    const double beta = scal[1];
    double* row = S + (int64_t)c * lds;
    const int len = l - j;
    double w = 0.0;
    for (int t = lane; t < len; t += 32) w = fma(v[t], row[j + t], w);
    w = warp_sum(w) * beta;
    for (int t = lane; t < len; t += 32) row[j + t] = fma(-w, v[t], row[j + t]);
    __syncwarp();
    const double r = row[j];
    double n1 = vn1[c];
    if (n1 != 0.0) {
        double tmp = fabs(r) / n1;
        tmp = fmax(0.0, (1.0 + tmp) * (1.0 - tmp));
        const double ratio = n1 / vn2[c];
        const double tmp2 = tmp * ratio * ratio;
        if (tmp2 <= 1.4901161193847656e-08) {        // sqrt(2^-52): recompute exactly
            double s = 0.0;
            for (int t = j + 1 + lane; t < l; t += 32) s = fma(row[t], row[t], s);
            s = warp_sum(s);
            if (lane == 0) { vn1[c] = sqrt(s); vn2[c] = sqrt(s); }
        } else if (lane == 0) {
            vn1[c] = n1 * sqrt(tmp);
        }
    }
}

__global__ void qr_extract_r_kernel(const double* S, int m, int64_t lds, double* R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int i = (int)(idx / m), c = (int)(idx % m);
    R[idx] = (i <= c) ? S[(int64_t)c * lds + i] : 0.0;
}

}  // namespace

cudaError_t pivoted_qr(double* S, int m, int l, int64_t lds, double* R, int32_t* perm,
                       double* work, int* status, cudaStream_t s) {
    (void)status;
    double* vn1 = work;
    double* vn2 = work + m;
    double* scal = work + 2 * m;
    double* v = work + 2 * m + 2;
    qr_init_kernel<<<(m * 32 + 255) / 256, 256, 0, s>>>(S, m, l, lds, vn1, vn2, perm);
    note_launch();
    for (int j = 0; j < m; ++j) {
        qr_pivot_kernel<<<1, PIV_THREADS, 0, s>>>(S, m, l, lds, j, vn1, vn2, perm, v, scal);
        note_launch();
        const int cols = m - j - 1;
        if (cols > 0) {
            const int warps_per_block = 8;
            qr_apply_kernel<<<(cols + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(
                S, m, l, lds, j, vn1, vn2, v, scal);
            note_launch();
        }
    }
    const int64_t total = (int64_t)m * m;
    qr_extract_r_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(S, m, lds, R);
    note_launch();
    return cudaGetLastError();
}

}  // namespace rtp
