// C ABI of librtproj: argument checks, workspace layout and the orchestration of the
// kernels for the preconditioner (Section 4, Eqs. 12-16) and the apply (the seven steps
// of Section 4 and the refinement of Remark 4.3).
#include "rtproj_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace rtp;

namespace {
std::atomic<uint64_t> g_launches{0};
}  // namespace

void rtp::note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int rtp::sm_count() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < kMaxDev) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    if (dev < kMaxDev) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

namespace {

void timer_flush(PhaseTimer& t) {
    if (t.n == 0) return;
    cudaEventSynchronize(t.e[t.n - 1]);
    for (int i = 0; i < t.n; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.b[i], t.e[i]) == cudaSuccess) {
            t.ms[t.phase[i]] += ms;
            t.cnt[t.phase[i]] += 1;
        }
    }
    t.n = 0;
}

}  // namespace

void rtp::phase_begin(rtproj_ctx* h, int p) {
    PhaseTimer& t = h->timer;
    if (!t.enabled) return;
    if (t.n == PhaseTimer::kMax) timer_flush(t);
    cudaEventRecord(t.b[t.n], h->stream);
    t.open = p;
}

void rtp::phase_end(rtproj_ctx* h, int p) {
    PhaseTimer& t = h->timer;
    if (!t.enabled || t.open != p) return;
    cudaEventRecord(t.e[t.n], h->stream);
    t.phase[t.n] = p;
    t.n++;
    t.open = -1;
}

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kPartElems = 1216ull * 4096ull;   // bounds every split-K slab set (see gemm64)

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t status, S, qr_work, perm, R, RinvT, Lc, Lt, T1, dinv, ffbuf, W, part, cbuf, ebuf, hbuf, dhbuf, sbuf;
    size_t A64, B64, normA, norm_part, bnorm, stats;
    size_t mixed_base, mixed_bytes;
    size_t total;
};

size_t mixed_workspace(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts& o);

bool valid_omega(int w) {
    return w == RTPROJ_OMEGA_UNIFORM || w == RTPROJ_OMEGA_RADEMACHER || w == RTPROJ_OMEGA_GAUSSIAN;
}

bool valid_opts(const rtproj_opts& o) {
    if (o.mode != RTPROJ_PLAIN_FP64 && o.mode != RTPROJ_MIXED_REFINED) return false;
    if (!valid_omega(o.omega)) return false;
    auto ok = [](int s) { return s >= 1 && s <= 10; };
    if (!ok(o.sketch_slices) || !ok(o.gram_slices) || !ok(o.gram2_slices) || !ok(o.apply_slices) ||
        !ok(o.resid_slices))
        return false;
    if (o.refine_passes < 0 || o.refine_passes > 8) return false;
    if (o.async != 0 && o.async != 1) return false;
    if (o.scalable != 0 && o.scalable != 1) return false;
    if (o.qr_form < 0 || o.qr_form > 2) return false;
    if (o.dtype != RTPROJ_F64 && o.dtype != RTPROJ_F32) return false;
    if (o.spin_limit_cycles < 1) return false;
    if (!(o.refine_tol >= 0.0)) return false;
    return true;
}

Layout make_layout(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts& o) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = align_up(off + bytes); return at; };
    L.status = take(64);
    L.S = take((size_t)m * l_max * 8);
    L.qr_work = take(pivoted_qr_work_doubles((int)m, (int)l_max) * 8);
    L.perm = take((size_t)m * 4);
    L.R = take((size_t)m * m * 8);
    L.RinvT = take((size_t)m * m * 8);
    L.Lc = take((size_t)m * m * 8);
    L.Lt = take((size_t)m * m * 8);
    L.T1 = take((size_t)m * m * 8);
    L.dinv = take(trsm_work_doubles((int)m) * 8);
    L.ffbuf = take(o.mode == RTPROJ_MIXED_REFINED ? ff_work_bytes((int)m) : 0);
    L.W = take((size_t)m * n * 8);
    L.part = take(kPartElems * 8);
    L.cbuf = take((size_t)m * k_max * 8);
    L.ebuf = take((size_t)m * k_max * 8);
    L.hbuf = take((size_t)m * k_max * 8);
    L.dhbuf = take((size_t)m * k_max * 8);
    L.sbuf = take((size_t)k_max * n * 8);
    // float32 at the ABI: A widened for the float64 form (the mixed form widens into W,
    // which it needs only after A has been sliced), right-hand sides widened per apply
    const bool f32 = o.dtype == RTPROJ_F32;
    L.A64 = take((f32 || o.scalable) && o.mode == RTPROJ_PLAIN_FP64 ? (size_t)m * n * 8 : 0);
    L.B64 = take(f32 ? (size_t)k_max * n * 8 : 0);
    L.normA = take(8);
    L.norm_part = take((size_t)norm_parts() * 8);
    L.bnorm = take((size_t)k_max * 8);
    L.stats = take(16);
    L.mixed_bytes = o.mode == RTPROJ_MIXED_REFINED ? mixed_workspace(m, n, l_max, k_max, o) : 0;
    L.mixed_base = take(L.mixed_bytes);
    L.total = off;
    return L;
}

rtproj_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RTPROJ_OK : RTPROJ_ECUDA; }

// The matrix every product reads, as float64: the caller's float64 A itself, or -- for a
// float32 A or a column scaling d -- A (diag(d)) formed once into W's region (the mixed
// form needs A only while slicing it, before any Gram product) or into A64 (the float64
// form reads it at every product). Then ||A||_F.
rtproj_status form_a(rtproj_ctx* h, const double* d) {
    const int m = (int)h->m, n = (int)h->n;
    h->scaled = d != nullptr;
    if (h->dtype == RTPROJ_F32 || d) {
        double* wide = h->opts.mode == RTPROJ_MIXED_REFINED ? h->W : h->A64;
        if (form_rows(h->A_user, h->dtype, h->lda_user, m, n, d, wide, n, h->stream) != cudaSuccess) return RTPROJ_ECUDA;
        h->A = wide;
        h->lda = n;
    } else {
        h->A = (const double*)h->A_user;
        h->lda = h->lda_user;
    }
    if (frobenius(h->A, h->lda, m, n, h->norm_part, h->normA, h->stream) != cudaSuccess) return RTPROJ_ECUDA;
    return RTPROJ_OK;
}

#define RT_CHECK(expr)                                  \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return RTPROJ_ECUDA;     \
    } while (0)

// ---------------------------------------------------------------------------------
// Plain float64 form.
// ---------------------------------------------------------------------------------
rtproj_status sketch_fp64(rtproj_ctx* h, uint64_t seed, int64_t l, double* S, int64_t lds) {
    Gemm64 g;
    g.M = (int)h->m; g.N = (int)l; g.K = (int)h->n;
    g.A = h->A; g.a_rs = h->lda; g.a_cs = 1;
    g.omega_dist = h->opts.omega; g.seed = seed;
    g.C = S; g.c_rs = lds; g.c_cs = 1;
    RT_CHECK(gemm64(g, h->part, h->part_elems, h->stream));
    return RTPROJ_OK;
}

// W = R^{-*} Pi A (P^{-1} A, m x n) and X = W W^* (lower triangle) into Lc.
rtproj_status gram_fp64(rtproj_ctx* h) {
    const int m = (int)h->m, n = (int)h->n;
    Gemm64 g;
    g.M = m; g.N = n; g.K = m;
    g.A = h->RinvT; g.a_rs = m; g.a_cs = 1;
    g.B = h->A; g.b_rs = h->lda; g.b_cs = 1; g.bk = h->perm;
    g.C = h->W; g.c_rs = n; g.c_cs = 1;
    RT_CHECK(gemm64(g, h->part, h->part_elems, h->stream));
    Gemm64 x;
    x.M = m; x.N = m; x.K = n;
    x.A = h->W; x.a_rs = n; x.a_cs = 1;
    x.B = h->W; x.b_rs = 1; x.b_cs = n;
    x.C = h->Lc; x.c_rs = m; x.c_cs = 1;
    x.lower_only = true;
    RT_CHECK(gemm64(x, h->part, h->part_elems, h->stream));
    return RTPROJ_OK;
}

}  // namespace

// h = Pi^* T1^* T1 Pi c for the m x k block c (row-major, leading dimension k): steps 2-6.
rtproj_status rtp::middle_fp64(rtproj_ctx* h, const double* c, double* out, int k) {
    const int m = (int)h->m;
    Gemm64 g;
    g.M = m; g.N = k; g.K = m;
    g.A = h->T1; g.a_rs = m; g.a_cs = 1; g.a_tri = 1;      // T1 is lower triangular
    g.B = c; g.b_rs = k; g.b_cs = 1; g.bk = h->perm;
    g.C = h->ebuf; g.c_rs = k; g.c_cs = 1;
    RT_CHECK(gemm64(g, h->part, h->part_elems, h->stream));
    Gemm64 t;
    t.M = m; t.N = k; t.K = m;
    t.A = h->T1; t.a_rs = 1; t.a_cs = m; t.a_tri = 2;      // T1^* is upper triangular
    t.B = h->ebuf; t.b_rs = k; t.b_cs = 1;
    t.C = out; t.c_rs = k; t.c_cs = 1; t.crow = h->perm;
    RT_CHECK(gemm64(t, h->part, h->part_elems, h->stream));
    return RTPROJ_OK;
}

namespace {

rtproj_status project_fp64(rtproj_ctx* h, const double* B, int64_t ldb, int k, void* Zv, int64_t ldz,
                           void* ROWv, int64_t ldr, void* Xv, int64_t ldx) {
    // float32 outputs: the row-space projection is formed in float64 (sbuf) and both
    // outputs are stored from it; float64 outputs are written by the products directly
    const bool f32 = h->dtype == RTPROJ_F32;
    const int m = (int)h->m, n = (int)h->n;
    double* Z = f32 ? nullptr : (double*)Zv;
    double* ROW = f32 ? ((Zv || ROWv) ? h->sbuf : nullptr) : (double*)ROWv;
    const int64_t ld_row = f32 ? (int64_t)n : ldr;
    Gemm64 c;                                            // step 1: c = A b
    c.M = m; c.N = k; c.K = n;
    c.A = h->A; c.a_rs = h->lda; c.a_cs = 1;
    c.B = B; c.b_rs = 1; c.b_cs = ldb;
    c.C = h->cbuf; c.c_rs = k; c.c_cs = 1;
    phase_begin(h, RTPROJ_PHASE_APPLY_A);
    RT_CHECK(gemm64(c, h->part, h->part_elems, h->stream));
    phase_end(h, RTPROJ_PHASE_APPLY_A);
    phase_begin(h, RTPROJ_PHASE_APPLY_M);
    rtproj_status st = middle_fp64(h, h->cbuf, h->hbuf, k);   // steps 2-6
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_APPLY_M);
    phase_begin(h, RTPROJ_PHASE_APPLY_AT);
    if (Z) {                                             // step 7 and b - b~
        Gemm64 z;
        z.M = k; z.N = n; z.K = m;
        z.A = h->hbuf; z.a_rs = 1; z.a_cs = k;
        z.B = h->A; z.b_rs = h->lda; z.b_cs = 1;
        z.C = Z; z.c_rs = ldz; z.c_cs = 1;
        z.alpha = -1.0; z.beta = 1.0; z.Cin = B; z.cin_rs = ldb; z.cin_cs = 1;
        RT_CHECK(gemm64(z, h->part, h->part_elems, h->stream));
    }
    if (ROW) {
        Gemm64 r;
        r.M = k; r.N = n; r.K = m;
        r.A = h->hbuf; r.a_rs = 1; r.a_cs = k;
        r.B = h->A; r.b_rs = h->lda; r.b_cs = 1;
        r.C = ROW; r.c_rs = ld_row; r.c_cs = 1;
        RT_CHECK(gemm64(r, h->part, h->part_elems, h->stream));
    }
    phase_end(h, RTPROJ_PHASE_APPLY_AT);
    if (f32) {
        if (Zv) RT_CHECK(store_rows(h->sbuf, n, B, ldb, Zv, ldz, k, n, 1, RTPROJ_F32, h->stream));
        if (ROWv) RT_CHECK(store_rows(h->sbuf, n, nullptr, 0, ROWv, ldr, k, n, 0, RTPROJ_F32, h->stream));
    }
    if (Xv) RT_CHECK(store_transposed(h->hbuf, k, m, k, Xv, ldx, h->dtype, h->stream));
    h->last_passes = 0;
    return RTPROJ_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------
// Mixed mode hooks (k_mixed.cu).
// ---------------------------------------------------------------------------------
namespace rtp {
size_t mixed_bytes(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts& o);
rtproj_status mixed_bind(rtproj_ctx* h, char* base, size_t bytes);
rtproj_status mixed_prepare_a(rtproj_ctx* h);
rtproj_status mixed_sketch(rtproj_ctx* h, uint64_t seed, int64_t l, double* S, int64_t lds);
rtproj_status mixed_gram(rtproj_ctx* h);
rtproj_status mixed_prepare_middle(rtproj_ctx* h);
rtproj_status mixed_project(rtproj_ctx* h, const double* B, int64_t ldb, int k, void* Z, int64_t ldz,
                            void* ROW, int64_t ldr, void* X, int64_t ldx);
}  // namespace rtp

namespace {
size_t mixed_workspace(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts& o) {
    return rtp::mixed_bytes(m, n, l_max, k_max, o);
}

constexpr int64_t kMaxLowRank = 64;
constexpr int64_t kMaxNnz = (int64_t)1 << 40;

// A new handle over the caller's workspace with the float64 form's layout L bound.
rtproj_ctx* bind_handle(int64_t m, int64_t n, int64_t l_max, int64_t k_max, void* workspace, size_t ws_bytes,
                        void* stream, const rtproj_opts& o, const Layout& L) {
    rtproj_ctx* h = new (std::nothrow) rtproj_ctx();
    if (!h) return nullptr;
    h->m = m; h->n = n; h->l_max = l_max; h->k_max = k_max;
    h->ws = (char*)workspace; h->ws_bytes = ws_bytes;
    h->stream = (cudaStream_t)stream;
    h->opts = o;
    h->dtype = o.dtype;
    h->spin_limit = o.spin_limit_cycles;
    char* b = h->ws;
    h->status = (int*)(b + L.status);
    h->a_status_dev = h->status + 8;
    h->S = (double*)(b + L.S);
    h->qr_work = (double*)(b + L.qr_work);
    h->perm = (int32_t*)(b + L.perm);
    h->R = (double*)(b + L.R);
    h->RinvT = (double*)(b + L.RinvT);
    h->Lc = (double*)(b + L.Lc);
    h->Lt = (double*)(b + L.Lt);
    h->T1 = (double*)(b + L.T1);
    h->dinv = (double*)(b + L.dinv);
    h->ffbuf = b + L.ffbuf;
    h->W = (double*)(b + L.W);
    h->part = (double*)(b + L.part);
    h->part_elems = kPartElems;
    h->cbuf = (double*)(b + L.cbuf);
    h->ebuf = (double*)(b + L.ebuf);
    h->hbuf = (double*)(b + L.hbuf);
    h->dhbuf = (double*)(b + L.dhbuf);
    h->sbuf = (double*)(b + L.sbuf);
    h->A64 = (double*)(b + L.A64);
    h->B64 = (double*)(b + L.B64);
    h->normA = (double*)(b + L.normA);
    h->norm_part = (double*)(b + L.norm_part);
    h->bnorm = (double*)(b + L.bnorm);
    h->stats = (unsigned long long*)(b + L.stats);
    return h;
}

// The handle's events (and phase timers), the cleared report maxima and status word.
rtproj_status finish_handle(rtproj_ctx* h) {
    if (cudaMemsetAsync(h->stats, 0, 16, h->stream) != cudaSuccess) return RTPROJ_ECUDA;
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) return RTPROJ_ECUDA;
    if (h->opts.timing) {
        h->timer.enabled = true;
        for (int i = 0; i < PhaseTimer::kMax; ++i)
            if (cudaEventCreate(&h->timer.b[i]) != cudaSuccess || cudaEventCreate(&h->timer.e[i]) != cudaSuccess)
                return RTPROJ_ECUDA;
    }
    if (cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) != cudaSuccess) return RTPROJ_ECUDA;
    return RTPROJ_OK;
}
}  // namespace

extern "C" {

void rtproj_default_opts(rtproj_opts* o) {
    if (!o) return;
    o->mode = RTPROJ_MIXED_REFINED;
    o->omega = RTPROJ_OMEGA_GAUSSIAN;
    o->sketch_slices = 5;
    o->gram_slices = 7;
    o->gram2_slices = 4;
    o->apply_slices = 7;
    o->resid_slices = 9;
    o->refine_passes = 1;
    o->timing = 0;
    o->rank_tol = 0.0;
    o->dtype = RTPROJ_F64;
    o->spin_limit_cycles = 4000000000ll;
    o->refine_tol = 0.0;
    o->async = 0;
    o->scalable = 0;
    o->qr_form = 0;
}

size_t rtproj_workspace_bytes(int64_t m, int64_t n, int64_t l_max, int64_t k_max, const rtproj_opts* opts) {
    rtproj_opts o;
    rtproj_default_opts(&o);
    if (opts) o = *opts;
    if (m < 1 || n < m || l_max < m || l_max > n || k_max < 1 || !valid_opts(o)) return 0;
    if (m > 4096 || n > (int64_t)1 << 30) return 0;
    return make_layout(m, n, l_max, k_max, o).total;
}

rtproj_status rtproj_create(rtproj_t* out, int64_t m, int64_t n, const void* A, int64_t lda, int64_t l_max,
                            int64_t k_max, void* workspace, size_t ws_bytes, void* stream, const rtproj_opts* opts) {
    if (!out) return RTPROJ_EINVAL;
    *out = nullptr;
    rtproj_opts o;
    rtproj_default_opts(&o);
    if (opts) o = *opts;
    if (!valid_opts(o)) return RTPROJ_EINVAL;
    if (!A || !workspace || m < 1 || n < m || lda < n || l_max < m || l_max > n || k_max < 1) return RTPROJ_EINVAL;
    if (m > 4096 || n > (int64_t)1 << 30) return RTPROJ_EUNSUPPORTED;
    if (((uintptr_t)workspace) % kAlign) return RTPROJ_EINVAL;
    const Layout L = make_layout(m, n, l_max, k_max, o);
    if (ws_bytes < L.total) return RTPROJ_ENOMEM;
    rtproj_ctx* h = bind_handle(m, n, l_max, k_max, workspace, ws_bytes, stream, o, L);
    if (!h) return RTPROJ_ENOMEM;
    h->A_user = A; h->lda_user = lda; h->lda = lda;
    if (form_a(h, nullptr) != RTPROJ_OK) {
        rtproj_destroy(h);
        return RTPROJ_ECUDA;
    }
    rtproj_status st = finish_handle(h);
    if (st == RTPROJ_OK && o.mode == RTPROJ_MIXED_REFINED) {
        st = mixed_bind(h, h->ws + L.mixed_base, L.mixed_bytes);
        if (st == RTPROJ_OK) st = mixed_prepare_a(h);
    }
    if (st != RTPROJ_OK) {
        rtproj_destroy(h);
        return st;
    }
    *out = h;
    return RTPROJ_OK;
}

size_t rtproj_sparse_workspace_bytes(int64_t m, int64_t n, int64_t nnz, int64_t r, int64_t l_max, int64_t k_max,
                                     const rtproj_opts* opts) {
    rtproj_opts o;
    rtproj_default_opts(&o);
    if (opts) o = *opts;
    if (m < 1 || n < m || nnz < 0 || r < 0 || l_max < m || l_max > n || k_max < 1 || !valid_opts(o)) return 0;
    if (m > 4096 || n > (int64_t)1 << 30 || r > kMaxLowRank || r > m || nnz > kMaxNnz || k_max > 65535) return 0;
    o.mode = RTPROJ_PLAIN_FP64;
    return make_layout(m, n, l_max, k_max, o).total + sparse_bytes(m, n, nnz, r, l_max, k_max);
}

rtproj_status rtproj_create_sparse(rtproj_t* out, int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                   const int32_t* col_idx, const double* val, int64_t r, const double* U,
                                   const double* V, int64_t l_max, int64_t k_max, void* workspace, size_t ws_bytes,
                                   void* stream, const rtproj_opts* opts) {
    if (!out) return RTPROJ_EINVAL;
    *out = nullptr;
    rtproj_opts o;
    rtproj_default_opts(&o);
    if (opts) o = *opts;
    if (!valid_opts(o)) return RTPROJ_EINVAL;
    if (!row_ptr || (nnz > 0 && (!col_idx || !val)) || (r > 0 && (!U || !V)) || !workspace) return RTPROJ_EINVAL;
    if (m < 1 || n < m || nnz < 0 || r < 0 || l_max < m || l_max > n || k_max < 1) return RTPROJ_EINVAL;
    if (m > 4096 || n > (int64_t)1 << 30 || r > kMaxLowRank || r > m || nnz > kMaxNnz || k_max > 65535)
        return RTPROJ_EUNSUPPORTED;
    if (o.dtype != RTPROJ_F64 || o.scalable) return RTPROJ_EUNSUPPORTED;
    if (((uintptr_t)workspace) % kAlign) return RTPROJ_EINVAL;
    o.mode = RTPROJ_PLAIN_FP64;   // the sparse form: float64 products, double-double residuals
    const Layout L = make_layout(m, n, l_max, k_max, o);
    if (ws_bytes < L.total + sparse_bytes(m, n, nnz, r, l_max, k_max)) return RTPROJ_ENOMEM;
    // the row pointers bound every later read of col_idx and val: checked here, on the host
    std::vector<int64_t> rp((size_t)m + 1);
    if (cudaMemcpyAsync(rp.data(), row_ptr, rp.size() * 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return RTPROJ_ECUDA;
    if (rp[0] != 0 || rp[m] != nnz) return RTPROJ_EINVAL;
    for (int64_t i = 0; i < m; ++i)
        if (rp[i + 1] < rp[i]) return RTPROJ_EINVAL;
    rtproj_ctx* h = bind_handle(m, n, l_max, k_max, workspace, ws_bytes, stream, o, L);
    if (!h) return RTPROJ_ENOMEM;
    h->sparse = true;
    h->nnz = nnz;
    h->csr_ptr = row_ptr; h->csr_col = col_idx; h->csr_val = val;
    h->lr = (int)r; h->lrU = U; h->lrV = V;
    sparse_bind(h, h->ws + L.total);
    rtproj_status st = finish_handle(h);
    if (st == RTPROJ_OK) st = sparse_chunks(h, rp.data());
    if (st == RTPROJ_OK) st = sparse_prepare(h);
    if (st == RTPROJ_OK) {
        // column indices in range and values finite, or the handle is refused
        int dev_status = 0;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess ||
            cudaMemcpy(&dev_status, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = RTPROJ_ECUDA;
        else
            st = (rtproj_status)dev_status;
    }
    if (st != RTPROJ_OK) {
        rtproj_destroy(h);
        return st;
    }
    *out = h;
    return RTPROJ_OK;
}

rtproj_status rtproj_set_scaling(rtproj_t h, const double* d) {
    if (!h) return RTPROJ_EINVAL;
    if (!h->opts.scalable) return RTPROJ_EUNSUPPORTED;
    h->preconditioned = 0;
    RT_CHECK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    rtproj_status st = form_a(h, d);
    if (st == RTPROJ_OK && h->opts.mode == RTPROJ_MIXED_REFINED) {
        h->a_status = RTPROJ_OK;
        st = mixed_prepare_a(h);
    }
    return st;
}

rtproj_status rtproj_sketch(rtproj_t h, uint64_t seed, int64_t l, double* S, int64_t lds) {
    if (!h || !S || l < h->m || l > h->l_max || lds < l) return RTPROJ_EINVAL;
    rtproj_status st = h->sparse ? sparse_sketch(h, seed, l, S, lds)
                       : h->opts.mode == RTPROJ_MIXED_REFINED ? mixed_sketch(h, seed, l, S, lds)
                                                              : sketch_fp64(h, seed, l, S, lds);
    if (st != RTPROJ_OK) return st;
    return cuda_status(cudaStreamSynchronize(h->stream));
}

rtproj_status rtproj_precondition(rtproj_t h, uint64_t seed, int64_t l) {
    if (!h) return RTPROJ_EINVAL;
    if (l < h->m || l > h->l_max || l > h->n) return RTPROJ_EINVAL;
    const int m = (int)h->m;
    cudaStream_t s = h->stream;
    h->preconditioned = 0;
    h->l = l;
    RT_CHECK(cudaEventRecord(h->ev0, s));
    if (h->opts.mode == RTPROJ_MIXED_REFINED) {
        if (h->a_status != RTPROJ_OK) return (rtproj_status)h->a_status;   // found when A was sliced
        // the status word starts from what slicing A found (non-finite entries), so that the
        // asynchronous mode still reports it
        RT_CHECK(cudaMemcpyAsync(h->status, h->a_status_dev, sizeof(int), cudaMemcpyDeviceToDevice, s));
    } else {
        RT_CHECK(cudaMemsetAsync(h->status, 0, sizeof(int), s));
        // a sparse A's values were checked at create
        if (!h->sparse) RT_CHECK(check_finite(h->A, h->lda, m, (int)h->n, h->status, s));
    }
    // 1. S = A G (Eq. 12)
    phase_begin(h, RTPROJ_PHASE_SKETCH);
    rtproj_status st = h->sparse ? sparse_sketch(h, seed, l, h->S, l)
                       : h->opts.mode == RTPROJ_MIXED_REFINED ? mixed_sketch(h, seed, l, h->S, l)
                                                              : sketch_fp64(h, seed, l, h->S, l);
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_SKETCH);
    // 2. S^* = Q R Pi (Eq. 13)
    phase_begin(h, RTPROJ_PHASE_QR);
    // mixed form: a float-float QR first -- on the whole grid (opts.qr_form = 0) or on one
    // cluster when S^* fits its shared memory (qr_form = 1) -- with the float64 persistent
    // kernel after it, which runs only if the float-float kernel's range check sent the
    // factorization back; the float64 QR alone for qr_form = 2 and the other forms
    bool ff_first = false;
    int* qr_flag = h->status + 4;
    if (h->opts.mode == RTPROJ_MIXED_REFINED && !h->sparse) {
        if (h->opts.qr_form == 1 && pivoted_qr_persistent_ok(m, (int)l))
            RT_CHECK(pivoted_qr_cluster(h->S, m, (int)l, l, h->R, h->perm, qr_flag, s, &ff_first));
        else if (h->opts.qr_form == 0)
            RT_CHECK(pivoted_qr_ff(h->S, m, (int)l, l, h->R, h->perm, h->qr_work, h->status, s, h->spin_limit,
                                   qr_flag, &ff_first));
    }
    RT_CHECK(pivoted_qr(h->S, m, (int)l, l, h->R, h->perm, h->qr_work, h->status, s, h->spin_limit,
                        ff_first ? qr_flag : nullptr));
    // default threshold: 8 times the sketch's relative precision -- 2^-52 in float64, 2^(-8 s)
    // for the s digits of A that the mixed form's sketch reads
    const double u_sketch = h->opts.mode == RTPROJ_MIXED_REFINED && !h->sparse
                                ? std::max(std::ldexp(1.0, -8 * h->opts.sketch_slices), std::ldexp(1.0, -52))
                                : std::ldexp(1.0, -52);
    const double tol = h->opts.rank_tol > 0 ? h->opts.rank_tol : 8.0 * u_sketch;
    RT_CHECK(qr_check(h->R, h->perm, m, tol, h->status, s));
    phase_end(h, RTPROJ_PHASE_QR);
    // R^{-*} (the transpose of P^- of Eq. 15, up to Pi)
    phase_begin(h, RTPROJ_PHASE_FACTOR);
    RT_CHECK(set_identity(h->RinvT, m, s));
    // The mixed form takes R^{-*} and the Cholesky factor in float-float (the float64
    // kernels enqueued behind them take over when the range check gives up): errors in
    // R^{-*} cancel (any invertible N in place of R^{-*} Pi gives the same preconditioner,
    // N^* (N A A^* N^*)^{-1} N), and the Cholesky's move kappa(X) 2^-48, as the float64
    // pivot reciprocals' already do. T1 = L^{-1} R^{-*} stays in float64: in float-float its
    // rounding raised ||dh|| / ||h|| of the first pass from 2e-6 to 1.3e-5 at 512 x 65536,
    // kappa 1e10. The float64 and sparse forms keep every factor in float64.
    const bool ff_factors = h->opts.mode == RTPROJ_MIXED_REFINED && !h->sparse;
    int* ff_ctl = h->status + 10;
    if (ff_factors)
        RT_CHECK(trsm_ff(h->R, 1, m, m, h->RinvT, m, m, h->dinv, h->ffbuf, ff_ctl, h->status, s, true));
    else
        RT_CHECK(trsm(h->R, 1, m, true, m, h->RinvT, m, m, h->dinv, h->status, s, true));   // R^* X = I
    phase_end(h, RTPROJ_PHASE_FACTOR);
    // 3. X = P^{-1} A A^* P^{-*} (Eq. 14 via steps a-e, as W W^*)
    phase_begin(h, RTPROJ_PHASE_GRAM);
    st = h->sparse ? sparse_gram(h) : h->opts.mode == RTPROJ_MIXED_REFINED ? mixed_gram(h) : gram_fp64(h);
    if (st != RTPROJ_OK) return st;
    phase_end(h, RTPROJ_PHASE_GRAM);
    // 4. X = L L^* (in place of Y = X^{-1}, Eq. 16), T1 = L^{-1} R^{-*}
    phase_begin(h, RTPROJ_PHASE_FACTOR);
    if (ff_factors)
        RT_CHECK(cholesky_ff(h->Lc, m, h->part, h->part_elems, h->ffbuf, ff_ctl, h->status, s, h->spin_limit));
    else
        RT_CHECK(cholesky(h->Lc, m, h->part, h->part_elems, h->status, s, h->spin_limit));
    // the solve reads L through its transpose, so that a warp's loads of T are coalesced
    RT_CHECK(transpose_copy(h->Lc, m, h->Lt, m, m, m, s));
    RT_CHECK(cudaMemcpyAsync(h->T1, h->RinvT, (size_t)m * m * 8, cudaMemcpyDeviceToDevice, s));
    RT_CHECK(trsm(h->Lt, 1, m, true, m, h->T1, m, m, h->dinv, h->status, s, true));     // R^{-*} is lower
    phase_end(h, RTPROJ_PHASE_FACTOR);
    if (h->opts.mode == RTPROJ_MIXED_REFINED) {
        st = mixed_prepare_middle(h);
        if (st != RTPROJ_OK) return st;
    }
    RT_CHECK(cudaEventRecord(h->ev1, s));
    if (h->opts.async) {
        h->preconditioned = 1;   // conditions found on the device stay latched for rtproj_get_info
        return RTPROJ_OK;
    }
    RT_CHECK(cudaStreamSynchronize(s));
    int dev_status = 0;
    RT_CHECK(cudaMemcpy(&dev_status, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    cudaEventElapsedTime(&h->ms_pre, h->ev0, h->ev1);
    if (dev_status != RTPROJ_OK) return (rtproj_status)dev_status;
    h->preconditioned = 1;
    return RTPROJ_OK;
}

rtproj_status rtproj_project(rtproj_t h, const void* B, int64_t ldb, int64_t k, void* Z, int64_t ldz,
                             void* ROW, int64_t ldr, void* X, int64_t ldx) {
    if (!h || !B || k < 1 || k > h->k_max || ldb < h->n) return RTPROJ_EINVAL;
    if (!Z && !ROW && !X) return RTPROJ_EINVAL;
    if ((Z && ldz < h->n) || (ROW && ldr < h->n) || (X && ldx < h->m)) return RTPROJ_EINVAL;
    if (!h->preconditioned) return RTPROJ_ESTATE;
    const double* Bd = (const double*)B;
    int64_t ldbd = ldb;
    if (h->dtype == RTPROJ_F32) {   // right-hand sides widened exactly; outputs stored as float32
        RT_CHECK(widen_rows((const float*)B, ldb, (int)k, (int)h->n, h->B64, h->n, h->stream));
        Bd = h->B64;
        ldbd = h->n;
    }
    if (h->sparse) return sparse_project(h, Bd, ldbd, (int)k, Z, ldz, ROW, ldr, X, ldx);
    if (h->opts.mode == RTPROJ_MIXED_REFINED) return mixed_project(h, Bd, ldbd, (int)k, Z, ldz, ROW, ldr, X, ldx);
    return project_fp64(h, Bd, ldbd, (int)k, Z, ldz, ROW, ldr, X, ldx);
}

rtproj_status rtproj_null_project(rtproj_t h, const void* B, int64_t ldb, int64_t k, void* Z, int64_t ldz) {
    if (!Z) return RTPROJ_EINVAL;
    return rtproj_project(h, B, ldb, k, Z, ldz, nullptr, 0, nullptr, 0);
}

rtproj_status rtproj_row_project(rtproj_t h, const void* B, int64_t ldb, int64_t k, void* ROW, int64_t ldr) {
    if (!ROW) return RTPROJ_EINVAL;
    return rtproj_project(h, B, ldb, k, nullptr, 0, ROW, ldr, nullptr, 0);
}

rtproj_status rtproj_lstsq(rtproj_t h, const void* B, int64_t ldb, int64_t k, void* X, int64_t ldx) {
    if (!X) return RTPROJ_EINVAL;
    return rtproj_project(h, B, ldb, k, nullptr, 0, nullptr, 0, X, ldx);
}

rtproj_status rtproj_generate_omega(uint64_t seed, int64_t n, int64_t l, int omega, double* G, int64_t ldg, void* stream) {
    if (!G || n < 1 || l < 1 || ldg < l || n > ((int64_t)1 << 30) || l > ((int64_t)1 << 30)) return RTPROJ_EINVAL;
    if (!valid_omega(omega)) return RTPROJ_EINVAL;
    RT_CHECK(omega_dense(seed, omega, (int)n, (int)l, G, ldg, (cudaStream_t)stream));
    return RTPROJ_OK;
}

rtproj_status rtproj_set_spin_limit(rtproj_t h, long long cycles) {
    if (!h || cycles < 1) return RTPROJ_EINVAL;
    h->spin_limit = cycles;
    h->opts.spin_limit_cycles = cycles;
    return RTPROJ_OK;
}

rtproj_status rtproj_export_state(rtproj_t h, double* R, int32_t* perm, double* Lc) {
    if (!h) return RTPROJ_EINVAL;
    if (!h->preconditioned) return RTPROJ_ESTATE;
    RT_CHECK(cudaStreamSynchronize(h->stream));
    const size_t mm = (size_t)h->m * h->m;
    if (R) RT_CHECK(cudaMemcpy(R, h->R, mm * 8, cudaMemcpyDeviceToHost));
    if (perm) RT_CHECK(cudaMemcpy(perm, h->perm, (size_t)h->m * 4, cudaMemcpyDeviceToHost));
    if (Lc) RT_CHECK(cudaMemcpy(Lc, h->Lc, mm * 8, cudaMemcpyDeviceToHost));
    return RTPROJ_OK;
}

rtproj_status rtproj_get_info(rtproj_t h, rtproj_info* info) {
    if (!h || !info) return RTPROJ_EINVAL;
    RT_CHECK(cudaStreamSynchronize(h->stream));
    std::memset(info, 0, sizeof(*info));
    int st = 0;
    RT_CHECK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    info->status = st;
    info->preconditioned = h->preconditioned;
    info->m = h->m; info->n = h->n; info->l = h->l;
    if (h->opts.async && h->preconditioned) {
        // the asynchronous precondition did not wait for its events; they are complete now
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) h->ms_pre = ms;
        else cudaGetLastError();
    }
    info->ms_precondition = h->ms_pre;
    if (h->l > 0) {
        const int m = (int)h->m;
        double* d = (double*)std::malloc((size_t)m * 8 * 2);
        if (!d) return RTPROJ_ENOMEM;
        RT_CHECK(cudaMemcpy2D(d, 8, h->R, (size_t)(m + 1) * 8, 8, m, cudaMemcpyDeviceToHost));
        RT_CHECK(cudaMemcpy2D(d + m, 8, h->Lc, (size_t)(m + 1) * 8, 8, m, cudaMemcpyDeviceToHost));
        info->r11 = std::fabs(d[0]);
        info->rmm = std::fabs(d[m - 1]);
        double lmax = 0, lmin = INFINITY;
        for (int i = 0; i < m; ++i) { lmax = std::max(lmax, std::fabs(d[m + i])); lmin = std::min(lmin, std::fabs(d[m + i])); }
        info->l11 = lmax;
        info->lmm = lmin;
        info->kappa_R = info->rmm > 0 ? info->r11 / info->rmm : INFINITY;
        info->kappa_pre = lmin > 0 ? lmax / lmin : INFINITY;
        std::free(d);
    }
    double nA = 0.0;
    unsigned long long st2[2] = {0, 0};
    RT_CHECK(cudaMemcpy(&nA, h->normA, 8, cudaMemcpyDeviceToHost));
    RT_CHECK(cudaMemcpy(st2, h->stats, 16, cudaMemcpyDeviceToHost));
    info->norm_A = nA;
    double v[2];
    std::memcpy(v, st2, 16);
    info->resid_rel = v[0];
    info->dh_rel = v[1];
    info->passes = h->last_passes;
    return RTPROJ_OK;
}

rtproj_status rtproj_clear_status(rtproj_t h) {
    if (!h) return RTPROJ_EINVAL;
    RT_CHECK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    return RTPROJ_OK;
}

rtproj_status rtproj_get_timings(rtproj_t h, double* ms, int64_t* count) {
    if (!h) return RTPROJ_EINVAL;
    if (!h->timer.enabled) return RTPROJ_EUNSUPPORTED;
    RT_CHECK(cudaStreamSynchronize(h->stream));
    timer_flush(h->timer);
    for (int p = 0; p < RTPROJ_NUM_PHASES; ++p) {
        if (ms) ms[p] = h->timer.ms[p];
        if (count) count[p] = h->timer.cnt[p];
        h->timer.ms[p] = 0.0;
        h->timer.cnt[p] = 0;
    }
    return RTPROJ_OK;
}

uint64_t rtproj_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

rtproj_status rtproj_destroy(rtproj_t h) {
    if (!h) return RTPROJ_EINVAL;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (int i = 0; i < PhaseTimer::kMax; ++i) {
        if (h->timer.b[i]) cudaEventDestroy(h->timer.b[i]);
        if (h->timer.e[i]) cudaEventDestroy(h->timer.e[i]);
    }
    delete h;
    return RTPROJ_OK;
}

const char* rtproj_status_string(rtproj_status s) {
    switch (s) {
        case RTPROJ_OK: return "ok";
        case RTPROJ_EINVAL: return "invalid argument";
        case RTPROJ_ESTATE: return "apply before a successful precondition";
        case RTPROJ_ERANK: return "sketch numerically rank deficient (|R_mm| <= rank_tol |R_11|)";
        case RTPROJ_ENOTSPD: return "Cholesky of the preconditioned Gram matrix broke down";
        case RTPROJ_ENONFINITE: return "non-finite value in the input or a factorization";
        case RTPROJ_ETIMEOUT: return "bounded device wait expired";
        case RTPROJ_ENOMEM: return "workspace too small";
        case RTPROJ_ECUDA: return "CUDA runtime error";
        case RTPROJ_EUNSUPPORTED: return "unsupported option or size";
    }
    return "unknown status";
}

}  // extern "C"
