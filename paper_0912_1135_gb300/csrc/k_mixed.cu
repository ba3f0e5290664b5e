// Mixed mode: every product with A on the tensor cores through exact digit slicing
// (k_slice.cu, k_umma.cu), the m x m stage in float64, and refinement (Remark 4.3).
//
// Preconditioner (Section 4):
//   S = A G           sketch_slices digits of A times the one-digit G plane (Eq. 12)
//   pivoted QR of S^* in float64 (Eq. 13); R^{-*} by a triangular solve
//   W = R^{-*} Pi A   = M' A^, where A^ is A with row i divided by 2^{e_i} (its slicing
//                     exponent) and M'[i][k] = R^{-*}[i][t] 2^{e_k} for k = perm[t]:
//                     gram_slices digits of M' against the transposed digits of A^
//   X = W W^*         gram2_slices digits of W (Eq. 14 as a Gram product), then Cholesky
// Apply, for right-hand sides b (rows of B):
//   c  = A b                       apply_slices digits        (step 1)
//   h0 = Pi^* T1^* T1 Pi c         float64                     (steps 2-6)
//   s  = b - A^* h0                resid_slices digits of A^ and of 2^{e} h0
//   repeat refine_passes times (Remark 4.3):
//     r  = A s                     resid_slices digits
//     dh = Pi^* T1^* T1 Pi r       float64
//     h  = h + dh;  s = s - A^* dh apply_slices digits
//   Z = s, ROW = b - s, least squares h.
// Because the digit products and their sums are exact, the residual products s and r
// are accurate to about 2^{-8 resid_slices} relative to |A||s| -- beyond float64 -- which
// is what lets refinement reach the exact projection of the stored matrix where every
// float64 method stops near eps * kappa (Remark 5.1).
#include "rtproj_internal.cuh"

#include <algorithm>
#include <cstring>

namespace rtp {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t kScratch = 48ull << 20;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }

int s_all(const rtproj_opts& o) {
    return std::max(std::max(o.sketch_slices, o.gram_slices), std::max(o.apply_slices, o.resid_slices));
}

struct MixedLayout {
    size_t A, eA, AT, eAT, G, eG, Mp, Ms, eM, W, eW, B, eB, H, eH, S, eS, T, eT, Tt, eTt, negEA, scratch, total;
};

MixedLayout mixed_layout(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts& o) {
    MixedLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = align_up(off + bytes); return at; };
    const int64_t ldn = pad64(n), ldm = pad64(m);
    const int sa = s_all(o);
    L.A = take((size_t)sa * m * ldn * 2);
    L.eA = take((size_t)m * 4);
    L.AT = take((size_t)sa * n * ldm * 2);
    L.eAT = take((size_t)n * 4);
    L.G = take((size_t)omega_planes(o.omega) * l_max * ldn * 2);
    L.eG = take((size_t)l_max * 4);
    L.Mp = take((size_t)m * m * 8);
    L.Ms = take((size_t)o.gram_slices * m * ldm * 2);
    L.eM = take((size_t)m * 4);
    L.W = take((size_t)o.gram2_slices * m * ldn * 2);
    L.eW = take((size_t)m * 4);
    L.B = take((size_t)o.apply_slices * k_max * ldn * 2);
    L.eB = take((size_t)k_max * 4);
    const int sh = std::max(o.apply_slices, o.resid_slices);
    L.H = take((size_t)sh * k_max * ldm * 2);
    L.eH = take((size_t)k_max * 4);
    L.S = take((size_t)o.resid_slices * k_max * ldn * 2);
    L.eS = take((size_t)k_max * 4);
    L.T = take((size_t)o.apply_slices * m * ldm * 2);
    L.eT = take((size_t)m * 4);
    L.Tt = take((size_t)o.apply_slices * m * ldm * 2);
    L.eTt = take((size_t)m * 4);
    L.negEA = take((size_t)m * 4);
    L.scratch = take(kScratch);
    L.total = off;
    return L;
}

SliceStack stack(char* base, size_t d_off, size_t e_off, int rows, int cols, int s, int64_t ld) {
    SliceStack st;
    st.d = (__nv_bfloat16*)(base + d_off);
    st.e = (int32_t*)(base + e_off);
    st.rows = rows;
    st.cols = cols;
    st.s = s;
    st.ld = ld;
    st.plane_stride = (int64_t)rows * ld;
    return st;
}

// The first s digit planes of a stack (digits are hierarchical, so this is the s-digit truncation).
SliceStack first(const SliceStack& st, int s) {
    SliceStack r = st;
    r.s = s;
    return r;
}

// Same storage, fewer rows in use (plane stride unchanged).
SliceStack rows_of(const SliceStack& st, int rows, int s) {
    SliceStack r = st;
    r.rows = rows;
    r.s = s;
    return r;
}

__global__ void mprime_kernel(const double* RinvT, const int32_t* perm, const int32_t* eA, int m, double* Mp) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int i = (int)(idx / m), t = (int)(idx % m);
    const int k = perm[t];
    Mp[(int64_t)i * m + k] = ldexp(RinvT[idx], eA[k]);
}

// D[i][perm[t]] = T[i][t] (m x m): T Pi^* with Pi the pivot permutation, so that
// (T Pi x) = D x for x in the original order.
__global__ void permute_columns_kernel(const double* T, const int32_t* perm, int m, double* D) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int i = (int)(idx / m), t = (int)(idx % m);
    D[(int64_t)i * m + perm[t]] = T[idx];
}

// D'[i][t] = D[i][t] 2^{e[t]} in place (exact), and ne[t] = -e[t]
__global__ void scale_columns_pow2_kernel(double* D, const int32_t* e, int m, int32_t* ne) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)m * m) return;
    const int t = (int)(idx % m);
    D[idx] = ldexp(D[idx], e[t]);
    if (idx < m) ne[idx] = -e[idx];
}

__global__ void axpy_kernel(double* y, const double* x, int64_t n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) y[idx] += x[idx];
}

#define MX_CHECK(expr)                              \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return RTPROJ_ECUDA; \
    } while (0)

rtproj_status gemm(rtproj_ctx* h, const SliceStack& a, const SliceStack& b, int terms, double* C, int64_t c_rs,
                   int64_t c_cs, double alpha = 1.0, double beta = 0.0, const double* Cin = nullptr,
                   int64_t cin_rs = 0, int64_t cin_cs = 0, bool lower = false, int32_t* row_exp = nullptr) {
    SlicedGemm g;
    g.a = a;
    g.b = b;
    g.terms = std::min(terms, a.s + b.s - 1);
    g.C = C; g.c_rs = c_rs; g.c_cs = c_cs;
    g.alpha = alpha; g.beta = beta; g.Cin = Cin; g.cin_rs = cin_rs; g.cin_cs = cin_cs;
    g.lower_only = lower;
    g.row_exp = row_exp;
    MX_CHECK(sliced_gemm(g, h->sg_scratch, h->sg_scratch_bytes, h->status, h->stream));
    return RTPROJ_OK;
}

}  // namespace

size_t mixed_bytes(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts& o) {
    return mixed_layout(m, n, l_max, k_max, o).total;
}

rtproj_status mixed_bind(rtproj_ctx* h, char* base, size_t bytes) {
    const rtproj_opts& o = h->opts;
    const MixedLayout L = mixed_layout(h->m, h->n, h->l_max, h->k_max, o);
    if (bytes < L.total) return RTPROJ_ENOMEM;
    const int m = (int)h->m, n = (int)h->n;
    const int64_t ldn = pad64(n), ldm = pad64(m);
    const int sa = s_all(o);
    h->As = stack(base, L.A, L.eA, m, n, sa, ldn);
    h->Ats = stack(base, L.AT, L.eAT, n, m, sa, ldm);
    h->Gs = stack(base, L.G, L.eG, (int)h->l_max, n, omega_planes(o.omega), ldn);
    h->Mprime = (double*)(base + L.Mp);
    h->Ms = stack(base, L.Ms, L.eM, m, m, o.gram_slices, ldm);
    h->Ws = stack(base, L.W, L.eW, m, n, o.gram2_slices, ldn);
    h->Bs = stack(base, L.B, L.eB, (int)h->k_max, n, o.apply_slices, ldn);
    h->Hs = stack(base, L.H, L.eH, (int)h->k_max, m, std::max(o.apply_slices, o.resid_slices), ldm);
    h->Ss = stack(base, L.S, L.eS, (int)h->k_max, n, o.resid_slices, ldn);
    h->Ts = stack(base, L.T, L.eT, m, m, o.apply_slices, ldm);
    h->Tts = stack(base, L.Tt, L.eTt, m, m, o.apply_slices, ldm);
    h->neg_eA = (int32_t*)(base + L.negEA);
    h->sg_scratch = base + L.scratch;
    h->sg_scratch_bytes = kScratch;
    return RTPROJ_OK;
}

rtproj_status mixed_prepare_a(rtproj_ctx* h) {
    phase_begin(h, RTPROJ_PHASE_SLICE);
    MX_CHECK(slice_rows_dual(h->A, h->lda, h->As, h->Ats, h->status, h->stream));
    MX_CHECK(fill_int(h->Ats.e, (int)h->n, 0, h->stream));
    phase_end(h, RTPROJ_PHASE_SLICE);
    // A is read only here in this form: remember whether it held non-finite entries, so
    // that precondition reports it without reading A again
    MX_CHECK(cudaMemcpyAsync(h->a_status_dev, h->status, sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    if (h->opts.async) return RTPROJ_OK;   // precondition folds a_status_dev into its status
    MX_CHECK(cudaMemcpyAsync(&h->a_status, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MX_CHECK(cudaStreamSynchronize(h->stream));
    return RTPROJ_OK;
}

rtproj_status mixed_sketch(rtproj_ctx* h, uint64_t seed, int64_t l, double* S, int64_t lds) {
    const int w = h->opts.omega;
    SliceStack G = rows_of(h->Gs, (int)l, omega_planes(w));
    G.max_digit = w == RTPROJ_OMEGA_RADEMACHER ? 1 : w == RTPROJ_OMEGA_GAUSSIAN ? 128 : 255;
    MX_CHECK(omega_plane(seed, h->opts.omega, (int)h->n, (int)l, G, h->stream));
    return gemm(h, first(h->As, h->opts.sketch_slices), G, h->opts.sketch_slices, S, lds, 1);
}

rtproj_status mixed_gram(rtproj_ctx* h) {
    const int m = (int)h->m, n = (int)h->n;
    const int64_t total = (int64_t)m * m;
    mprime_kernel<<<(unsigned)((total + 255) / 256), 256, 0, h->stream>>>(h->RinvT, h->perm, h->As.e, m, h->Mprime);
    note_launch();
    MX_CHECK(cudaGetLastError());
    MX_CHECK(slice_rows(h->Mprime, m, 1, nullptr, nullptr, h->Ms, h->status, h->stream));
    // W's row exponents are gathered by the product's output stage, so slicing W reads it once
    MX_CHECK(fill_int(h->Ws.e, m, kZeroRowExp, h->stream));
    rtproj_status st = gemm(h, h->Ms, first(h->Ats, h->opts.gram_slices), h->opts.gram_slices, h->W, n, 1, 1.0, 0.0,
                            nullptr, 0, 0, false, h->Ws.e);
    if (st != RTPROJ_OK) return st;
    MX_CHECK(slice_rows_given_exp(h->W, n, h->Ws, h->status, h->stream));
    return gemm(h, h->Ws, h->Ws, h->opts.gram2_slices, h->Lc, m, 1, 1.0, 0.0, nullptr, 0, 0, true);
}

// Steps 2-6 of the apply (Section 4) fold into h = Pi^* T1^* T1 Pi c with T1 = L^{-1} R^{-*}
// (L L^* = X). With D = T1 Pi (columns permuted to the original order) this is D^* (D c):
// two products of m x m digit stacks, sliced here once per preconditioner, against the
// k right-hand sides. Every digit product is exact, so each product is accurate to
// 2^{-8 apply_slices} relative to |D||c| -- tighter than float64 rounding of the same
// products, and the refinement pass corrects what remains.
// Entry t of c = A b carries the scale of row t of A (2^{e_A[t]}), and column t of D its
// inverse, so the first product runs as D' c' with D' = D diag(2^{e_A}) and c' = c
// diag(2^{-e_A}): digits sliced per right-hand side then keep every row's digits whatever
// the spread of A's row scales (rows scaled apart leave the projection unchanged).
rtproj_status mixed_prepare_middle(rtproj_ctx* h) {
    const int m = (int)h->m;
    const int64_t total = (int64_t)m * m;
    phase_begin(h, RTPROJ_PHASE_SLICE);
    permute_columns_kernel<<<(unsigned)((total + 255) / 256), 256, 0, h->stream>>>(h->T1, h->perm, m, h->Mprime);
    note_launch();
    MX_CHECK(cudaGetLastError());
    MX_CHECK(slice_rows(h->Mprime, 1, m, nullptr, nullptr, h->Tts, h->status, h->stream));      // D^*
    scale_columns_pow2_kernel<<<(unsigned)((total + 255) / 256), 256, 0, h->stream>>>(h->Mprime, h->As.e, m,
                                                                                        h->neg_eA);
    note_launch();
    MX_CHECK(cudaGetLastError());
    MX_CHECK(slice_rows(h->Mprime, m, 1, nullptr, nullptr, h->Ts, h->status, h->stream));      // D'
    phase_end(h, RTPROJ_PHASE_SLICE);
    return RTPROJ_OK;
}

namespace {

// out = D^* (D c) for the m x k block c (row-major, leading dimension k).
rtproj_status middle_mixed(rtproj_ctx* h, const double* c, double* out, int k) {
    const int ap = h->opts.apply_slices;
    const SliceStack Hk = rows_of(h->Hs, k, ap);
    MX_CHECK(slice_rows(c, 1, k, nullptr, h->neg_eA, Hk, h->status, h->stream));           // c'^*: k x m
    rtproj_status st = gemm(h, h->Ts, Hk, ap, h->ebuf, k, 1);                              // u = D' c' = D c
    if (st != RTPROJ_OK) return st;
    MX_CHECK(slice_rows(h->ebuf, 1, k, nullptr, nullptr, Hk, h->status, h->stream));        // u^*: k x m
    return gemm(h, h->Tts, Hk, ap, out, k, 1);                                             // D^* u
}

}  // namespace

rtproj_status mixed_project(rtproj_ctx* h, const double* B, int64_t ldb, int k, void* Z, int64_t ldz, void* ROW,
                            int64_t ldr, void* X, int64_t ldx) {
    const rtproj_opts& o = h->opts;
    const int m = (int)h->m, n = (int)h->n;
    cudaStream_t s = h->stream;
    rtproj_status st;
    // residual report: ||b_j|| once per apply, the maxima cleared
    MX_CHECK(row_norms(B, ldb, k, n, h->bnorm, s));
    MX_CHECK(cudaMemsetAsync(h->stats, 0, 16, s));
    // c = A b
    phase_begin(h, RTPROJ_PHASE_SLICE);
    const SliceStack Bk = rows_of(h->Bs, k, o.apply_slices);
    MX_CHECK(slice_rows(B, ldb, 1, nullptr, nullptr, Bk, h->status, s));
    phase_end(h, RTPROJ_PHASE_SLICE);
    phase_begin(h, RTPROJ_PHASE_APPLY_A);
    st = gemm(h, first(h->As, o.apply_slices), Bk, o.apply_slices, h->cbuf, k, 1);
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_APPLY_A);
    // h0 = Pi^* T1^* T1 Pi c
    phase_begin(h, RTPROJ_PHASE_APPLY_M);
    st = middle_mixed(h, h->cbuf, h->hbuf, k);
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_APPLY_M);
    // s = b - A^* h0
    phase_begin(h, RTPROJ_PHASE_SLICE);
    const SliceStack Hr = rows_of(h->Hs, k, o.resid_slices);
    MX_CHECK(slice_rows(h->hbuf, 1, k, nullptr, h->As.e, Hr, h->status, s));
    phase_end(h, RTPROJ_PHASE_SLICE);
    phase_begin(h, RTPROJ_PHASE_APPLY_AT);
    st = gemm(h, first(h->Ats, o.resid_slices), Hr, o.resid_slices, h->sbuf, 1, n, -1.0, 1.0, B, 1, ldb);
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_APPLY_AT);
    // the last pass may write Z directly when it is the only output and float64
    const bool direct_z = Z && !ROW && h->dtype == RTPROJ_F64;
    bool z_written = false;
    int passes = 0;
    for (int pass = 0; pass < o.refine_passes; ++pass) {
        // r = A s
        phase_begin(h, RTPROJ_PHASE_SLICE);
        const SliceStack Sk = rows_of(h->Ss, k, o.resid_slices);
        MX_CHECK(slice_rows(h->sbuf, n, 1, nullptr, nullptr, Sk, h->status, s));
        phase_end(h, RTPROJ_PHASE_SLICE);
        phase_begin(h, RTPROJ_PHASE_APPLY_A);
        st = gemm(h, first(h->As, o.resid_slices), Sk, o.resid_slices, h->cbuf, k, 1);
        if (st != RTPROJ_OK) return st;
        phase_end(h, RTPROJ_PHASE_APPLY_A);
        // dh, h += dh
        phase_begin(h, RTPROJ_PHASE_APPLY_M);
        st = middle_mixed(h, h->cbuf, h->dhbuf, k);
        if (st != RTPROJ_OK) return st;
        const int64_t mk = (int64_t)m * k;
        axpy_kernel<<<(unsigned)((mk + 255) / 256), 256, 0, s>>>(h->hbuf, h->dhbuf, mk);
        note_launch();
        // the pass's report: ||r_j|| = ||A s_j|| and ||dh_j|| / ||h_j||
        MX_CHECK(cudaMemsetAsync(h->stats, 0, 16, s));
        MX_CHECK(column_stats(h->cbuf, h->hbuf, h->dhbuf, m, k, h->bnorm, h->normA, h->stats, s));
        phase_end(h, RTPROJ_PHASE_APPLY_M);
        passes = pass + 1;
        bool last = passes == o.refine_passes;
        if (o.refine_tol > 0.0 && !last) {
            // Remark 4.3, to convergence: stop once every correction is below the tolerance
            unsigned long long bits[2];
            MX_CHECK(cudaMemcpyAsync(bits, h->stats, 16, cudaMemcpyDeviceToHost, s));
            MX_CHECK(cudaStreamSynchronize(s));
            double v[2];
            memcpy(v, bits, 16);
            if (v[1] <= o.refine_tol) last = true;
        }
        // s = s - A^* dh
        phase_begin(h, RTPROJ_PHASE_SLICE);
        const SliceStack Hd = rows_of(h->Hs, k, o.apply_slices);
        MX_CHECK(slice_rows(h->dhbuf, 1, k, nullptr, h->As.e, Hd, h->status, s));
        phase_end(h, RTPROJ_PHASE_SLICE);
        phase_begin(h, RTPROJ_PHASE_APPLY_AT);
        if (last && direct_z) {
            st = gemm(h, first(h->Ats, o.apply_slices), Hd, o.apply_slices, (double*)Z, 1, ldz, -1.0, 1.0, h->sbuf, 1,
                      n);
            z_written = true;
        } else {
            st = gemm(h, first(h->Ats, o.apply_slices), Hd, o.apply_slices, h->sbuf, 1, n, -1.0, 1.0, h->sbuf, 1, n);
        }
        if (st != RTPROJ_OK) return st;
        phase_end(h, RTPROJ_PHASE_APPLY_AT);
        if (last) break;
    }
    h->last_passes = passes;
    // outputs in the caller's element type; ROW before Z, since Z may alias B
    if (ROW) MX_CHECK(store_rows(h->sbuf, n, B, ldb, ROW, ldr, k, n, 1, h->dtype, s));
    if (Z && !z_written) MX_CHECK(store_rows(h->sbuf, n, nullptr, 0, Z, ldz, k, n, 0, h->dtype, s));
    if (X) MX_CHECK(store_transposed(h->hbuf, k, m, k, X, ldx, h->dtype, s));
    MX_CHECK(cudaGetLastError());
    return RTPROJ_OK;
}

}  // namespace rtp
