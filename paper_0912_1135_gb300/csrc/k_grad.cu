// Gradient of the null-space projection with respect to A (the adjoint of Eq. 1).
//
// For L = sum_j <g_j, Z b_j> with Z = I - A^*(AA^*)^{-1}A, differentiating Eq. 1 gives
// dZ = -(Z dA^* P^* + P dA Z) with P = A^*(AA^*)^{-1} (so that P^* b = h, the least-squares
// solution of Remark 4.1), hence
//     dL/db_j = Z g_j,        dL/dA = -sum_j (h_j (Z g_j)^* + w_j (Z b_j)^*),  w_j = P^* g_j.
// With H, W (k x m) holding h_j, w_j as rows and Y, Zb (k x n) holding Z g_j and Z b_j:
//     dL/dA = -(H^* Y + W^* Zb),
// one product of the m x 2k matrix [H^* | W^*] with the 2k x n matrix [Y; Zb] -- a rank-2k
// update, a dense contraction over 2k. Both operands are gathered transposed (and widened
// from float32) into rows that reduce over 2k, then multiplied on the tensor cores through
// exact digit slicing (mixed form) or on the FP64 pipe (float64 form).
#include "rtproj_internal.cuh"

#include <algorithm>

using namespace rtp;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }

// dst[c][col_off + r] = src[r][c] for the rows x cols block src (element type Tin, ld lds);
// 32 x 32 tiles through shared memory so that both sides are coalesced.
template <typename Tin>
__global__ void gather_transposed_kernel(const Tin* __restrict__ src, int64_t lds, int rows, int cols,
                                         double* __restrict__ dst, int64_t ldd, int col_off) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int y = ty; y < 32; y += 8) {
        const int r = r0 + y, c = c0 + tx;
        tile[y][tx] = (r < rows && c < cols) ? (double)src[(int64_t)r * lds + c] : 0.0;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int c = c0 + y, r = r0 + tx;
        if (c < cols && r < rows) dst[(int64_t)c * ldd + col_off + r] = tile[tx][y];
    }
}

cudaError_t gather(const void* src, int64_t lds, int rows, int cols, int dt, double* dst, int64_t ldd, int col_off,
                   cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    if (dt == RTPROJ_F32)
        gather_transposed_kernel<float><<<grid, 256, 0, s>>>((const float*)src, lds, rows, cols, dst, ldd, col_off);
    else
        gather_transposed_kernel<double><<<grid, 256, 0, s>>>((const double*)src, lds, rows, cols, dst, ldd, col_off);
    note_launch();
    return cudaGetLastError();
}

struct GradLayout {
    size_t TA, TB, SA, eA, SB, eB, out, scratch, total;
};

GradLayout grad_layout(const rtproj_ctx* h, int64_t k) {
    GradLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = align_up(off + bytes); return at; };
    const int64_t m = h->m, n = h->n, K2 = 2 * k, ldk = pad64(K2);
    const bool mixed = h->opts.mode == RTPROJ_MIXED_REFINED;
    const int s = h->opts.apply_slices;
    L.TA = take((size_t)m * K2 * 8);
    L.TB = take((size_t)n * K2 * 8);
    L.SA = take(mixed ? (size_t)s * m * ldk * 2 : 0);
    L.eA = take(mixed ? (size_t)m * 4 : 0);
    L.SB = take(mixed ? (size_t)s * n * ldk * 2 : 0);
    L.eB = take(mixed ? (size_t)n * 4 : 0);
    L.out = take(h->dtype == RTPROJ_F32 ? (size_t)m * n * 8 : 0);
    L.scratch = take(mixed ? sliced_gemm_scratch_bytes((int)m, (int)n, (int)K2) : 0);
    L.total = off;
    return L;
}

SliceStack make_stack(char* base, size_t d, size_t e, int rows, int cols, int s) {
    SliceStack st;
    st.d = (__nv_bfloat16*)(base + d);
    st.e = (int32_t*)(base + e);
    st.rows = rows;
    st.cols = cols;
    st.s = s;
    st.ld = pad64(cols);
    st.plane_stride = (int64_t)rows * st.ld;
    return st;
}

}  // namespace

extern "C" {

size_t rtproj_grad_workspace_bytes(rtproj_t h, int64_t k) {
    if (!h || k < 1 || k > ((int64_t)1 << 24)) return 0;
    return grad_layout(h, k).total;
}

rtproj_status rtproj_grad_A(rtproj_t h, int64_t k, const void* H, int64_t ldh, const void* Y, int64_t ldy,
                            const void* W, int64_t ldw, const void* Zb, int64_t ldz, void* dA, int64_t ldda,
                            void* workspace, size_t ws_bytes) {
    if (!h || !H || !Y || !W || !Zb || !dA || !workspace || k < 1 || k > ((int64_t)1 << 24)) return RTPROJ_EINVAL;
    if (ldh < h->m || ldw < h->m || ldy < h->n || ldz < h->n || ldda < h->n) return RTPROJ_EINVAL;
    if (((uintptr_t)workspace) % kAlign) return RTPROJ_EINVAL;
    const GradLayout L = grad_layout(h, k);
    if (ws_bytes < L.total) return RTPROJ_ENOMEM;
    const int m = (int)h->m, n = (int)h->n, K2 = (int)(2 * k);
    cudaStream_t s = h->stream;
    char* b = (char*)workspace;
    double* TA = (double*)(b + L.TA);   // m x 2k: [H^* | W^*]
    double* TB = (double*)(b + L.TB);   // n x 2k: [Y^* | Zb^*]
#define GR_CHECK(expr)                                  \
    do {                                                \
        if ((expr) != cudaSuccess) return RTPROJ_ECUDA; \
    } while (0)
    GR_CHECK(gather(H, ldh, (int)k, m, h->dtype, TA, K2, 0, s));
    GR_CHECK(gather(W, ldw, (int)k, m, h->dtype, TA, K2, (int)k, s));
    GR_CHECK(gather(Y, ldy, (int)k, n, h->dtype, TB, K2, 0, s));
    GR_CHECK(gather(Zb, ldz, (int)k, n, h->dtype, TB, K2, (int)k, s));
    const bool f32 = h->dtype == RTPROJ_F32;
    double* C = f32 ? (double*)(b + L.out) : (double*)dA;
    const int64_t ldc = f32 ? n : ldda;
    if (h->opts.mode == RTPROJ_MIXED_REFINED) {
        const int sl = h->opts.apply_slices;
        SliceStack SA = make_stack(b, L.SA, L.eA, m, K2, sl);
        SliceStack SB = make_stack(b, L.SB, L.eB, n, K2, sl);
        GR_CHECK(slice_rows(TA, K2, 1, nullptr, nullptr, SA, h->status, s));
        GR_CHECK(slice_rows(TB, K2, 1, nullptr, nullptr, SB, h->status, s));
        SlicedGemm g;
        g.a = SA;
        g.b = SB;
        g.terms = sl;
        g.C = C; g.c_rs = ldc; g.c_cs = 1;
        g.alpha = -1.0;
        GR_CHECK(sliced_gemm(g, b + L.scratch, L.total - L.scratch, h->status, s));
    } else {
        Gemm64 g;
        g.M = m; g.N = n; g.K = K2;
        g.A = TA; g.a_rs = K2; g.a_cs = 1;
        g.B = TB; g.b_rs = 1; g.b_cs = K2;
        g.C = C; g.c_rs = ldc; g.c_cs = 1;
        g.alpha = -1.0;
        GR_CHECK(gemm64(g, h->part, h->part_elems, s));
    }
    if (f32) GR_CHECK(store_rows(C, n, nullptr, 0, dA, ldda, m, n, 0, RTPROJ_F32, s));
#undef GR_CHECK
    return RTPROJ_OK;
}

}  // extern "C"
