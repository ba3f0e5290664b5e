// Internal declarations shared by the CUDA translation units of librtproj.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "rtproj.h"

namespace rtp {

// Counts kernels enqueued by this library (reported by rtproj_launch_count).
void note_launch(int n = 1);

// Streaming multiprocessors of the current device (queried once per device; 152 on
// GB300). Grid sizes and split-K factors are derived from it.
int sm_count();

// Per-phase CUDA-event timing (opts.timing).
struct PhaseTimer {
    static constexpr int kMax = 64;
    cudaEvent_t b[kMax] = {};
    cudaEvent_t e[kMax] = {};
    int phase[kMax] = {};
    int n = 0;
    int open = -1;
    double ms[RTPROJ_NUM_PHASES] = {};
    int64_t cnt[RTPROJ_NUM_PHASES] = {};
    bool enabled = false;
};

// ---------------------------------------------------------------------------
// Device status word: the first error code written wins (never trap/assert).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* st, int code) {
    if (st) atomicCAS(st, 0, code);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and the entries of G.
// Entry (i, j) of the n x l test matrix uses byte (i & 3) of word ((i & 15) >> 2)
// of the block at counter (i >> 4, j, 0, 0), key (seed lo, seed hi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Byte b (0..15) of a Philox block -> entry of G.
__device__ __forceinline__ float omega_from_byte(uint32_t u, int dist) {
    return dist == RTPROJ_OMEGA_RADEMACHER ? (u >= 128u ? 1.0f : -1.0f)
                                           : (float)(2 * (int)u - 255) * (1.0f / 256.0f);
}

__device__ __forceinline__ uint32_t block_byte(const uint4& w, int b) {
    const uint32_t word = (b >> 2) == 0 ? w.x : (b >> 2) == 1 ? w.y : (b >> 2) == 2 ? w.z : w.w;
    return (word >> (8 * (b & 3))) & 0xFFu;
}

// Gaussian entries of G: the Box-Muller transform (Box & Muller, 1958) of two Philox
// words a, b in float32 -- u1 = ((a >> 9) + 1/2) 2^-23 in (0, 1) and u2 = (b >> 9) 2^-23
// in [0, 1), both exact; r = sqrt(-2 ln u1) <= sqrt(48 ln 2) < 5.77; the pair
// (r cos 2 pi u2, r sin 2 pi u2) -- each rounded to the nearest multiple of 2^-12 (ties to
// even). Returned as the integers N = 4096 G, |N| <= 23637.
__device__ __forceinline__ void gauss_pair(uint32_t a, uint32_t b, int& n_cos, int& n_sin) {
    const float u1 = ((float)(a >> 9) + 0.5f) * 1.1920928955078125e-07f;   // 2^-23
    const float u2 = (float)(b >> 9) * 1.1920928955078125e-07f;
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    n_cos = __float2int_rn((r * cs) * 4096.0f);
    n_sin = __float2int_rn((r * sn) * 4096.0f);
}

// The four Gaussian entries 4q .. 4q+3 of column j of G (as N = 4096 G) from the Philox
// block at counter (q, j, 1, 0).
__device__ __forceinline__ void gauss_quad(uint32_t q, uint32_t j, uint32_t k0, uint32_t k1, int (&N)[4]) {
    const uint4 w = philox4x32_10(make_uint4(q, j, 1u, 0u), k0, k1);
    gauss_pair(w.x, w.y, N[0], N[1]);
    gauss_pair(w.z, w.w, N[2], N[3]);
}

// ---------------------------------------------------------------------------
// float64 tiled GEMM on the FP64 pipe, split over K into partial slabs.
//   P[z][i][j] = sum_{k in split z} A(i,k) * B(k,j)
//   A(i,k) = A[(arow ? arow[i] : i) * a_rs + k * a_cs]
//   B(k,j) = B[(bk ? bk[k] : k) * b_rs + j * b_cs], or G(k, j) when omega_dist >= 0
// then a reduce kernel writes C[(crow ? crow[i] : i) * c_rs + j * c_cs]
//   = alpha * sum_z P[z][i][j] + beta * Cin[i * cin_rs + j * cin_cs].
// ---------------------------------------------------------------------------
struct Gemm64 {
    int M = 0, N = 0, K = 0;
    const double* A = nullptr; int64_t a_rs = 0, a_cs = 0; const int32_t* arow = nullptr;
    const double* B = nullptr; int64_t b_rs = 0, b_cs = 0; const int32_t* bk = nullptr;
    int omega_dist = -1; uint64_t seed = 0;
    double* C = nullptr; int64_t c_rs = 0, c_cs = 0; const int32_t* crow = nullptr;
    double alpha = 1.0, beta = 0.0;
    const double* Cin = nullptr; int64_t cin_rs = 0, cin_cs = 0;
    bool lower_only = false;   // compute/write only entries with i >= j (tiles above skipped)
    int a_tri = 0;             // 1: A(i,k) = 0 for k > i (lower); 2: A(i,k) = 0 for k < i (upper)
};

// Enqueues the GEMM + reduce. part/part_elems: scratch for the partial slabs.
cudaError_t gemm64(const Gemm64& g, double* part, size_t part_elems, cudaStream_t s);

// C (M x N, M <= 64, ld c_rs) = A (M x K, ld a_rs) B (K x N) for a long K, where
// B(k, j) = B[k b_rs + j b_cs] or, with omega_dist >= 0, G(k, j) of Eq. 12 (k_fp64.cu).
// part: chunks x M x N doubles of scratch.
struct Narrow64 {
    int M = 0, N = 0, K = 0;
    const double* A = nullptr; int64_t a_rs = 0;
    const double* B = nullptr; int64_t b_rs = 0, b_cs = 0;
    int omega_dist = -1; uint64_t seed = 0;
    double* C = nullptr; int64_t c_rs = 0;
};
cudaError_t gemm64_narrow(const Narrow64& g, double* part, size_t part_elems, cudaStream_t s);

// Small helpers (k_fp64.cu)
cudaError_t set_identity(double* X, int m, cudaStream_t s);
cudaError_t transpose_copy(const double* src, int64_t s_rs, double* dst, int64_t d_rs, int rows, int cols, cudaStream_t s);
cudaError_t check_finite(const double* X, int64_t rs, int rows, int cols, int* status, cudaStream_t s);
cudaError_t zero_upper(double* X, int m, cudaStream_t s);

// Pivoted QR of S^* (k_qr.cu). S is m x l row-major (row i of S = column i of S^*),
// overwritten. On exit R (m x m, upper) and perm (m) hold the factorization
// S^*[:, perm] = Q R. work: pivoted_qr_work_doubles(m, l) doubles. pivoted_qr uses the
// persistent cooperative kernel when the columns fit in shared memory, else one pivot
// kernel and one update kernel per step (pivoted_qr_steps). spin_limit bounds each
// grid-exchange wait in clock cycles (RTPROJ_ETIMEOUT when it expires).
// run_if (optional): the persistent kernel returns at once unless *run_if != 0 (the
// cluster form's fallback flag); only meaningful when pivoted_qr_persistent_ok(m, l).
size_t pivoted_qr_work_doubles(int m, int l);
cudaError_t pivoted_qr(double* S, int m, int l, int64_t lds, double* R, int32_t* perm,
                       double* work, int* status, cudaStream_t s, long long spin_limit,
                       const int* run_if = nullptr);
bool pivoted_qr_persistent_ok(int m, int l);
// The mixed form's QR in float-float on the whole grid (k_qr.cu): sets *launched when the
// kernel was enqueued; the kernel writes *fallback = 1 when the entries' range needs the
// float64 kernel, which must follow with run_if = fallback.
cudaError_t pivoted_qr_ff(double* S, int m, int l, int64_t lds, double* R, int32_t* perm, double* work, int* status,
                          cudaStream_t s, long long spin_limit, int* fallback, bool* launched);
// The mixed form's QR on one 16-CTA cluster in float-float arithmetic (k_qr_cluster.cu).
// Sets *launched when the kernel was enqueued; the kernel then writes *fallback = 1 if the
// entries' range needs the float64 kernel (which must follow with run_if = fallback).
bool qr_cluster_fits(int m, int l);
cudaError_t pivoted_qr_cluster(const double* S, int m, int l, int64_t lds, double* R, int32_t* perm, int* fallback,
                               cudaStream_t s, bool* launched);
// After the QR: checks that perm is a permutation of 0..m-1 (replacing it by the identity
// and latching RTPROJ_ETIMEOUT when a QR that gave up left it incomplete, so that no later
// kernel indexes through it out of range) and that |R_mm| > tol |R_11| (RTPROJ_ERANK).
cudaError_t qr_check(const double* R, int32_t* perm, int m, double tol, int* status, cudaStream_t s);
cudaError_t pivoted_qr_steps(double* S, int m, int l, int64_t lds, double* R, int32_t* perm,
                             double* work, int* status, cudaStream_t s);

// Triangular solves and Cholesky (k_tri.cu).
// Solves op(T) X = Bm in place; T (m x m) element (i,j) at T[i*t_rs + j*t_cs];
// lower selects forward substitution. Bm element (i, j) at Bm[i*b_rs + j], j < ncols.
// dinv_work: trsm_work_doubles(m) doubles (inverses of the 32 x 32 diagonal blocks and a
// column counter). T is read row by row across a warp's threads: t_rs = 1 coalesces.
// rhs_lower (lower solves only): Bm is zero above its diagonal, so the solution is too and
// the rows above each column are skipped.
// run_if (optional): the kernels return at once unless *run_if != 0 (a fallback enqueued
// behind the float-float solve below).
cudaError_t trsm(const double* T, int64_t t_rs, int64_t t_cs, bool lower, int m,
                 double* Bm, int64_t b_rs, int ncols, double* dinv_work, int* status, cudaStream_t s,
                 bool rhs_lower = false, const int* run_if = nullptr);
size_t trsm_work_doubles(int m);
// In-place lower Cholesky of the m x m row-major X (strict upper part zeroed). With run_if
// the cooperative kernel runs only if *run_if != 0 (cudaErrorNotSupported if it cannot be
// launched).
cudaError_t cholesky(double* X, int m, double* part, size_t part_elems, int* status, cudaStream_t s,
                     long long spin_limit, const int* run_if = nullptr);
// Float-float forms of the two for the mixed form (GB300's FP32 pipe runs 64 times the
// FP64 pipe's rate; the preconditioner needs about 2^-48 of the factors, and the refinement
// corrects the rest). Lower solves only, with the semantics of trsm(lower = true). Each
// first checks the range of the diagonal on the device; beyond what float-float holds
// (a span over 2^90, a zero, non-finite or non-positive pivot) it raises ctl[0] and the
// float64 kernels, always enqueued behind, run instead. ffbuf: ff_work_bytes(m) bytes;
// ctl: 4 ints of device memory.
size_t ff_work_bytes(int m);
cudaError_t trsm_ff(const double* T, int64_t t_rs, int64_t t_cs, int m, double* Bm, int64_t b_rs, int ncols,
                    double* dinv_work, void* ffbuf, int* ctl, int* status, cudaStream_t s, bool rhs_lower);
cudaError_t cholesky_ff(double* X, int m, double* part, size_t part_elems, void* ffbuf, int* ctl, int* status,
                        cudaStream_t s, long long spin_limit);

// ---------------------------------------------------------------------------
// Mixed mode: fixed-point bfloat16 slicing and the sliced tensor-core GEMM.
// ---------------------------------------------------------------------------
// A "slice stack" of a rows x cols matrix X (reduction over cols): for each row r an
// exponent e_r with |X[r][c]| < 2^{e_r}, and s planes D_p (p = 0..s-1) of bfloat16
// integers in [-128, 128] such that
//     X[r][c] ~= 2^{e_r} * sum_p D_p[r][c] * 2^{-7-8p}
// with truncation error below 2^{e_r - 8s}. Plane p is stored row-major with leading
// dimension ld (a multiple of 8 elements), plane stride plane_stride elements.
struct SliceStack {
    __nv_bfloat16* d = nullptr;
    int32_t* e = nullptr;
    int rows = 0, cols = 0, s = 0;
    int64_t ld = 0;
    int64_t plane_stride = 0;
    int max_digit = 128;     // bound on |digit| (255 for the G plane)
};

// Row exponent of an all-zero row while row maxima are being gathered (atomic maxima over
// parts of a row start from it); slicing reads it as exponent 0.
constexpr int kZeroRowExp = -(1 << 30);

// Slices X (element (r, c) at X[r*x_rs + c*x_cs], multiplied by 2^cexp[c] when cexp is
// given) into the stack; optional row gather. Columns cols..ld-1 are written as zeros.
cudaError_t slice_rows(const double* X, int64_t x_rs, int64_t x_cs, const int32_t* rowidx, const int32_t* cexp,
                       const SliceStack& st, int* status, cudaStream_t s);
// Digit planes of src transposed into dst (dst.rows = src.cols, dst.ld >= src.rows).
// Row exponents of X (rows x cols, contiguous rows): e[r] <- max(e[r], the frexp exponent
// of max_c |X[r][c]|), e pre-filled with kZeroRowExp; non-finite entries raise
// RTPROJ_ENONFINITE in status.
cudaError_t row_exponents(const double* X, int64_t x_rs, int rows, int cols, int32_t* e, int* status, cudaStream_t s);
// Slices X (contiguous rows) into st with the row exponents already in st.e (gathered as
// by row_exponents, kZeroRowExp for an all-zero row): one read of X, spread over spans of
// every row. Falls back to slice_rows when the fast layout conditions do not hold.
cudaError_t slice_rows_given_exp(const double* X, int64_t x_rs, const SliceStack& st, int* status, cudaStream_t s);
// Row-major digits of X (rows x cols, contiguous rows) into st and the same digits
// transposed into tst (tst.rows = st.cols, tst.cols = st.rows, same s), in one pass over
// the digits: the row exponents first, then 64 x 64 tiles that write both layouts.
cudaError_t slice_rows_dual(const double* X, int64_t x_rs, const SliceStack& st, const SliceStack& tst, int* status,
                            cudaStream_t s);
cudaError_t transpose_planes(const SliceStack& src, const SliceStack& dst, cudaStream_t s);
// Writes G^* (l x n, reduction over n) as digit planes plus row exponents (exact): one
// plane for the uniform and Rademacher entries, two for the Gaussian ones (st.s >= 2).
cudaError_t omega_plane(uint64_t seed, int dist, int n, int l, const SliceStack& st, cudaStream_t s);
// G itself as float64 (n x l, row-major), for checking step a1 on its own.
cudaError_t omega_dense(uint64_t seed, int dist, int n, int l, double* G, int64_t ldg, cudaStream_t s);
// Digit planes G^* needs for a distribution.
inline int omega_planes(int dist) { return dist == RTPROJ_OMEGA_GAUSSIAN ? 2 : 1; }
cudaError_t fill_int(int32_t* e, int n, int v, cudaStream_t s);

// C[(crow?crow[i]:i)*c_rs + j*c_cs] = alpha * (A_stack x B_stack^T)[i][j] + beta * Cin[...]
// where the product keeps slice pairs p + q <= max(sa, sb) - 1 (0-based) -- the
// Ozaki-scheme truncation -- and is exact up to that truncation.
struct SlicedGemm {
    SliceStack a, b;     // a: M x K, b: N x K (both reduce over K)
    int terms = 0;       // keep pairs with p + q < terms (terms <= sa + sb - 1)
    double* C = nullptr; int64_t c_rs = 0, c_cs = 0; const int32_t* crow = nullptr;
    double alpha = 1.0, beta = 0.0;
    const double* Cin = nullptr; int64_t cin_rs = 0, cin_cs = 0;
    bool lower_only = false;
    // Optional: row exponents of the output gathered as by row_exponents (e pre-filled with
    // kZeroRowExp), from the values as they are stored, so that slicing C needs no pass of
    // its own over C for them. Needs contiguous output rows (c_cs = 1) and !lower_only.
    int32_t* row_exp = nullptr;
};
size_t sliced_gemm_scratch_bytes(int M, int N, int K);
cudaError_t sliced_gemm(const SlicedGemm& g, void* scratch, size_t scratch_bytes, int* status, cudaStream_t s);

}  // namespace rtp

struct rtproj_ctx;
namespace rtp {
// Sparse A (k_sparse.cu): workspace bytes beyond the float64 form's layout, binding,
// the column-compressed copy and ||A||_F at create, and the sparse forms of the sketch,
// the Gram matrix and the apply.
size_t sparse_bytes(int64_t m, int64_t n, int64_t nnz, int64_t r, int64_t l_max, int64_t k_max);
void sparse_bind(rtproj_ctx* h, char* base);
rtproj_status sparse_chunks(rtproj_ctx* h, const int64_t* rp_host);
rtproj_status sparse_prepare(rtproj_ctx* h);
rtproj_status sparse_sketch(rtproj_ctx* h, uint64_t seed, int64_t l, double* S, int64_t lds);
rtproj_status sparse_gram(rtproj_ctx* h);
rtproj_status sparse_project(rtproj_ctx* h, const double* B, int64_t ldb, int k, void* Z, int64_t ldz, void* ROW,
                             int64_t ldr, void* X, int64_t ldx);
void phase_begin(rtproj_ctx* h, int phase);
void phase_end(rtproj_ctx* h, int phase);
// Steps 2-6 of the apply in float64: out = Pi^* T1^* T1 Pi c (c, out: m x k, ld k).
rtproj_status middle_fp64(rtproj_ctx* h, const double* c, double* out, int k);
}  // namespace rtp

// ---------------------------------------------------------------------------
// Boundary helpers (k_boundary.cu): element types at the ABI, norms for the reports.
// ---------------------------------------------------------------------------
namespace rtp {
// dst (rows x cols, ld ldd, float64) = src (float32, ld lds), exactly.
cudaError_t widen_rows(const float* src, int64_t lds, int rows, int cols, double* dst, int64_t ldd, cudaStream_t s);
// dst (rows x cols float64, ld ldd) = src diag(d) (d optional, n entries), src of element
// type dt (ld lds): the matrix the products read, widened and scaled exactly... up to the
// one rounding of each product x d_c.
cudaError_t form_rows(const void* src, int dt, int64_t lds, int rows, int cols, const double* d, double* dst, int64_t ldd,
                      cudaStream_t s);
// dst (rows x cols, element type dt, ld ldd) = B - X (sub) or X; X and B float64.
cudaError_t store_rows(const double* X, int64_t ldx, const double* B, int64_t ldb, void* dst, int64_t ldd, int rows,
                       int cols, int sub, int dt, cudaStream_t s);
// dst (cols x rows of element type dt, ld ldd) = transpose of src (rows x cols float64, ld lds).
cudaError_t store_transposed(const double* src, int64_t lds, int rows, int cols, void* dst, int64_t ldd, int dt,
                             cudaStream_t s);
// *out = ||X||_F for X (rows x cols float64, ld ldx); deterministic two-level sum. part: at
// least norm_parts() doubles.
int norm_parts();
cudaError_t frobenius(const double* X, int64_t ldx, int rows, int cols, double* part, double* out, cudaStream_t s);
// out[j] = ||row j of X|| for the k rows of X (k x n float64, ld ldx).
cudaError_t row_norms(const double* X, int64_t ldx, int k, int n, double* out, cudaStream_t s);
// For the m x k blocks r, h, dh (row-major, ld k; right-hand side j is column j):
// stats[0] <- max(stats[0], max_j ||r_j|| / (normA ||b_j||)) and
// stats[1] <- max(stats[1], max_j ||dh_j|| / max(||h_j||, ||b_j|| / normA)), as bit patterns of non-negative
// doubles (r or dh may be null to skip that maximum).
cudaError_t column_stats(const double* r, const double* h, const double* dh, int m, int k, const double* bnorm,
                         const double* normA, unsigned long long* stats, cudaStream_t s);
}  // namespace rtp

// ---------------------------------------------------------------------------
// Host-side handle.
// ---------------------------------------------------------------------------
struct rtproj_ctx {
    int64_t m = 0, n = 0, lda = 0, l_max = 0, k_max = 0;
    const double* A = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    rtproj_opts opts{};

    int* status = nullptr;       // device status word
    double* S = nullptr;         // m x l_max sketch, destroyed by the QR
    double* qr_work = nullptr;   // 3m + l_max
    int32_t* perm = nullptr;     // m
    double* R = nullptr;         // m x m
    double* RinvT = nullptr;     // m x m, R^{-*}
    double* Lc = nullptr;        // m x m, chol(X)
    double* Lt = nullptr;        // m x m, chol(X)^* (read by the second triangular solve)
    double* T1 = nullptr;        // m x m, Lc^{-1} R^{-*}
    double* dinv = nullptr;      // inverses of the 32 x 32 diagonal blocks (trsm)
    char* ffbuf = nullptr;       // mixed form: the float-float copy of a factor (ff_work_bytes)
    double* W = nullptr;         // m x n, P^{-1} A (float64 mode)
    double* part = nullptr;      // split-K partial slabs
    size_t part_elems = 0;
    double* cbuf = nullptr;      // m x k_max
    double* ebuf = nullptr;      // m x k_max
    double* hbuf = nullptr;      // m x k_max  (h, row-major m x k)
    double* dhbuf = nullptr;     // m x k_max
    double* sbuf = nullptr;      // k_max x n  (refinement residual)
    // mixed mode (k_mixed.cu)
    rtp::SliceStack As;          // A with rows normalised: m x n, reduction over n
    rtp::SliceStack Ats;         // the same digits transposed: n x m, reduction over m
    rtp::SliceStack Gs;          // G^*: l x n, one plane
    rtp::SliceStack Ms;          // M' = R^{-*} Pi with columns scaled by 2^{e_A}: m x m
    rtp::SliceStack Ws;          // W = P^{-1} A: m x n
    rtp::SliceStack Bs;          // right-hand sides: k x n
    rtp::SliceStack Hs;          // h or dh with rows scaled by 2^{e_A}, transposed: k x m
    rtp::SliceStack Ss;          // refinement residual s: k x n
    rtp::SliceStack Ts;          // T1 Pi (columns permuted): m x m, reduction over m
    rtp::SliceStack Tts;         // (T1 Pi)^*: m x m, reduction over m
    double* Mprime = nullptr;    // m x m
    int32_t* neg_eA = nullptr;   // m: minus A's row exponents (the m x m stage's digit scales)
    void* sg_scratch = nullptr;  // int64 split-K partials
    size_t sg_scratch_bytes = 0;

    // boundary (k_boundary.cu)
    int dtype = RTPROJ_F64;      // element type of A, B and the outputs at the ABI
    const void* A_user = nullptr;
    int64_t lda_user = 0;
    bool scaled = false;         // the products read A diag(d) (rtproj_set_scaling)
    double* A64 = nullptr;       // float32 A widened (float64 form; the mixed form widens into W)
    double* B64 = nullptr;       // k_max x n: float32 right-hand sides widened
    double* normA = nullptr;     // ||A||_F (device scalar)
    double* norm_part = nullptr; // partial sums of the Frobenius norm
    double* bnorm = nullptr;     // k_max: ||b_j|| of the current apply
    unsigned long long* stats = nullptr;   // [0] resid_rel, [1] dh_rel (bit patterns)
    long long spin_limit = 4000000000ll;
    int last_passes = 0;
    double norm_A_host = 0.0;

    // sparse A = S + U V (k_sparse.cu): S borrowed in compressed sparse row form, its
    // column-compressed copy built at create
    bool sparse = false;
    int64_t nnz = 0;
    const int64_t* csr_ptr = nullptr;
    const int32_t* csr_col = nullptr;
    const double* csr_val = nullptr;
    int64_t* csc_ptr = nullptr;       // n + 1
    int32_t* csc_row = nullptr;       // nnz, ordered by row within each column
    double* csc_val = nullptr;        // nnz
    int64_t* csc_cursor = nullptr;    // n (column counts, then scatter cursors)
    int64_t* scan_tot = nullptr;      // per-block totals of the column scan
    double* Pminus = nullptr;         // m x m, P^- = Pi^* R^{-1}
    double* Esp = nullptr;            // m x m, A A^* P^-
    int lr = 0;                       // rank r of the low-rank term (0: none)
    const double* lrU = nullptr;      // m x r, borrowed
    const double* lrV = nullptr;      // r x n, borrowed
    double* lr_a = nullptr;           // r x max(l_max, m): V G, U^* P^-, V D
    double* lr_b = nullptr;           // r x k_max: V b or U^* h
    double* lr_small = nullptr;       // U^* U, V V^* and partial sums (||A||_F)
    int nchunks = 0;                  // rows cut into chunks of nonzeros for A x
    int32_t* chunk_row = nullptr;     // row of each chunk
    int64_t* chunk_beg = nullptr;     // first nonzero of each chunk
    int32_t* row_chunk = nullptr;     // m + 1: first chunk of each row
    double* chunk_part = nullptr;     // chunks x k_max double-double partial sums

    rtp::PhaseTimer timer;
    int64_t l = 0;
    int preconditioned = 0;
    int a_status = 0;            // mixed form: status of slicing A at create (non-finite entries)
    int* a_status_dev = nullptr; // the same, kept on the device (asynchronous mode)
    float ms_pre = 0.f;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};
