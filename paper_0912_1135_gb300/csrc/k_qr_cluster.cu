// Pivoted Householder QR of S^* (Section 4, Eq. 13) on one 16-CTA thread-block cluster,
// in float-float arithmetic on the FP32 pipe: the preconditioner of the mixed form.
//
// Why: the QR's m steps are strictly sequential, and on the whole grid each step costs a
// grid-wide exchange through L2 (publish, poll, read the candidates, read the pivot
// column): several microseconds, far more than the step's arithmetic. Here S^* (l x m)
// lives in the distributed shared memory of one cluster (CTA r holds columns
// [r cpc, r cpc + cpc), 2.1 MB at 516 x 512), so a step's exchange is one hardware
// cluster barrier plus two shared-memory reads through the cluster (the sixteen
// candidates, then the pivot column). Sixteen SMs have 1/9 of the grid's FP64 pipe, so
// the reflector updates run in float-float (a value is an unevaluated sum hi + lo of two
// floats; Dekker's TwoProduct through fmaf and Knuth's TwoSum): about 2^-48 relative
// accuracy, on the FP32 pipe, which has 64 times the FP64 pipe's rate.
//
// Accuracy: the computed R is the exact factor of S^* + E with ||E|| of order
// l 2^-48 ||S||, so P^{-1}A = R^{-*} Pi A keeps kappa(P^{-1}A) near that of the sketch as
// long as 2^-48 kappa(A) << 1 (3.6e-5 at kappa = 1e10). The preconditioner only needs
// that: the refinement pass (Remark 4.3) makes the result exact whatever the
// preconditioner's own rounding. The plain float64 form keeps the float64 QR.
//
// The pivot rule is Businger-Golub (largest remaining squared norm, lowest index on ties)
// on float-float norms that are downdated from step to step and recomputed exactly when
// the downdate has cancelled (as LAPACK does); the float64 kernel recomputes every norm
// every step instead, so near-ties can resolve differently. As in LAPACK, the downdated
// norms only choose each CTA's candidate: the candidate is published with its column's
// norm summed afresh, so that the reflector stays orthogonal to float-float accuracy and
// the choice between CTAs is made on exact norms. Candidates are pushed into every CTA's
// shared memory by remote stores before the step's barrier, so that after it every read
// of them is local.
// S^* is scaled by a power of two (exact) so that its largest entry lies in [1/2, 1);
// if a column's squared norm then falls below 2^-90 (float-float would lose the digits
// of a trailing norm near float's underflow), the kernel leaves R and perm untouched and
// sets *fallback, and the float64 persistent kernel that follows it runs instead.
#include "rtproj_internal.cuh"
#include "ff.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace rtp {
namespace {

constexpr int CQ_CTAS = 16;
constexpr int CQ_THREADS = 512;
constexpr int CQ_WARPS = CQ_THREADS / 32;
constexpr int CQ_MAXC = 64;

// Warp-wide maximum of (value, index): largest value, lowest index on ties; an index of m
// marks an empty entry. Every lane receives the result.
__device__ __forceinline__ void cand_reduce(ff& best, int& bi, int m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff ob;
        ob.hi = __shfl_xor_sync(0xffffffffu, best.hi, o);
        ob.lo = __shfl_xor_sync(0xffffffffu, best.lo, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi < m && (bi == m || ff_gt(ob, best) || (ob.hi == best.hi && ob.lo == best.lo && oi < bi))) {
            best = ob;
            bi = oi;
        }
    }
}

// After the update of step j, column c (rows j .. l-1 at c[0 .. len)) loses row j from its
// trailing norm: nsq <- nsq - c_j^2, or the exact sum over rows j+1 .. l-1 when the
// downdate has cancelled below 2^-20 of the last exact value nsq_ref (then nsq_ref moves).
__device__ __forceinline__ void downdate_norm(const float2* c, int len, int q, int lane, float2* nsq, float2* nsq_ref) {
    const ff y = {c[0].x, c[0].y};
    ff ns = ff_add({nsq[q].x, nsq[q].y}, ff_neg(ff_mul(y, y)));
    const bool exact = !(ns.hi > nsq_ref[q].x * 0x1p-20f);
    if (exact) {
        ff s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
        int i = 1 + lane;
        for (; i + 32 < len; i += 64) {
            const ff x0 = {c[i].x, c[i].y}, x1 = {c[i + 32].x, c[i + 32].y};
            s0 = ff_add(s0, ff_mul(x0, x0));
            s1 = ff_add(s1, ff_mul(x1, x1));
        }
        if (i < len) {
            const ff x0 = {c[i].x, c[i].y};
            s0 = ff_add(s0, ff_mul(x0, x0));
        }
        ns = ff_warp_sum(ff_add(s0, s1));
    }
    __syncwarp();
    if (lane == 0) {
        nsq[q] = make_float2(ns.hi, ns.lo);
        if (exact) nsq_ref[q] = make_float2(ns.hi, ns.lo);
    }
    __syncwarp();
}

struct CqrDev {
    const double* S;
    int m, l;
    int64_t lds;
    double* R;
    int32_t* perm;
    int cpc;
    int* fallback;      // set to 1 when the float-float range check fails (R, perm untouched)
};

__global__ void __launch_bounds__(CQ_THREADS, 1) qr_cluster_kernel(CqrDev p) {
    extern __shared__ float2 csm[];
    const int l = p.l, m = p.m, cpc = p.cpc;
    float2* cols = csm;                          // cpc x l
    float2* v = csm + (size_t)cpc * l;           // l (rows j .. l-1 of the reflector at offset 0)
    __shared__ float2 cand_val[2][CQ_CTAS];  // by step parity: every CTA's candidate (pushed to all)
    __shared__ int cand_idx[2][CQ_CTAS];
    __shared__ float2 nsq[CQ_MAXC];          // squared norm of rows j .. l-1 before step j
    __shared__ float2 nsq_ref[CQ_MAXC];      // its value at the last exact computation
    __shared__ float2 alphaq[CQ_MAXC];
    __shared__ int posq[CQ_MAXC];
    __shared__ unsigned long long max_bits_s;
    __shared__ int bad_s;
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int c0 = b * cpc;
    const int nc = max(0, min(cpc, m - c0));

    // 1. largest |entry| of S over the cluster, from the bit patterns (no float64 arithmetic)
    if (t == 0) { max_bits_s = 0ull; bad_s = 0; }
    __syncthreads();
    {
        unsigned long long mx = 0ull;
        for (int q = 0; q < nc; ++q)
            for (int i = t; i < l; i += CQ_THREADS) {
                const unsigned long long u =
                    (unsigned long long)__double_as_longlong(p.S[(int64_t)(c0 + q) * p.lds + i]) & 0x7FFFFFFFFFFFFFFFull;
                mx = u > mx ? u : mx;
            }
        atomicMax(&max_bits_s, mx);
    }
    cluster.sync();
    unsigned long long gmax = 0ull;
    for (int r = 0; r < CQ_CTAS; ++r) {
        const unsigned long long x = *cluster.map_shared_rank(&max_bits_s, r);
        gmax = x > gmax ? x : gmax;
    }
    // scale 2^-e with the largest entry in [1/2, 1); a non-finite S cannot reach here (the
    // caller's status already holds it), but its exponent field would be clamped anyway
    int e = (int)(gmax >> 52) - 1022;
    e = max(-1000, min(1000, e));
    const double scale = ldexp(1.0, -e);

    // 2. columns into shared memory as float-float, and their squared norms
    for (int q = 0; q < nc; ++q)
        for (int i = t; i < l; i += CQ_THREADS) {
            const double x = p.S[(int64_t)(c0 + q) * p.lds + i] * scale;
            const float hi = __double2float_rn(x);
            const float lo = __double2float_rn(x - (double)hi);
            cols[(size_t)q * l + i] = make_float2(hi, lo);
        }
    __syncthreads();
    for (int q = warp; q < nc; q += CQ_WARPS) {
        const float2* c = cols + (size_t)q * l;
        ff s = {0.f, 0.f};
        for (int i = lane; i < l; i += 32) {
            const ff x = {c[i].x, c[i].y};
            s = ff_add(s, ff_mul(x, x));
        }
        s = ff_warp_sum(s);
        if (lane == 0) {
            nsq[q] = make_float2(s.hi, s.lo);
            nsq_ref[q] = make_float2(s.hi, s.lo);
            posq[q] = -1;
            if (!(s.hi >= 0x1p-90f)) atomicOr(&bad_s, 1);
        }
    }
    __syncthreads();
    if (warp == 0) {
        ff cv = {-1.f, 0.f};
        int ci = m;
        for (int q = lane; q < nc; q += 32) {
            const ff x = {nsq[q].x, nsq[q].y};
            if (ci == m || ff_gt(x, cv)) { cv = x; ci = c0 + q; }
        }
        cand_reduce(cv, ci, m);
        if (lane < CQ_CTAS) {     // the step-0 norms are exact
            *cluster.map_shared_rank(&cand_val[0][b], lane) = make_float2(cv.hi, cv.lo);
            *cluster.map_shared_rank(&cand_idx[0][b], lane) = ci;
        }
    }
    cluster.sync();
    int bad = 0;
    for (int r = 0; r < CQ_CTAS; ++r) bad |= *cluster.map_shared_rank(&bad_s, r);
    if (bad) {
        if (b == 0 && t == 0) *p.fallback = 1;
        cluster.sync();   // no CTA leaves while another may still read its shared memory
        return;
    }
    if (b == 0 && t == 0) *p.fallback = 0;

    // 3. the m steps
    for (int j = 0; j < m; ++j) {
        const int par = j & 1;
        if (j > 0) cluster.sync();   // step j's candidates are published (step 0's by the sync above)
        // the pivot: largest squared norm over the sixteen candidates (pushed here by every
        // CTA), lowest index on ties; each candidate carries its column's exact squared norm
        ff best = {-1.f, 0.f};
        int bi = m;
        if (lane < CQ_CTAS) {
            const float2 cv = cand_val[par][lane];
            const int ci = cand_idx[par][lane];
            if (ci < m) { best = {cv.x, cv.y}; bi = ci; }
        }
        cand_reduce(best, bi, m);
        const int piv = bi < m ? bi : 0;   // some CTA holds an active column while j < m
        const int owner = piv / cpc, qo = piv - owner * cpc;
        const float2* src = cluster.map_shared_rank(cols + (size_t)qo * l, owner);
        // the reflector from the pivot column's rows j .. l-1 (read through the cluster) and
        // its exact squared norm
        const float2 x0f = src[j];
        const ff x0 = {x0f.x, x0f.y};
        const ff nx = ff_sqrt(best);
        const ff alpha = x0.hi >= 0.f ? ff_neg(nx) : nx;
        const ff ax0 = x0.hi >= 0.f ? x0 : ff_neg(x0);
        const ff den = ff_mul(nx, ff_add(nx, ax0));
        const ff beta = den.hi > 0.f ? ff_recip(den) : ff{0.f, 0.f};
        for (int i = j + 1 + t; i < l; i += CQ_THREADS) v[i - j] = src[i];
        if (t == 0) {
            const ff v0 = ff_add(x0, ff_neg(alpha));
            v[0] = make_float2(v0.hi, v0.lo);
            if (b == owner) {
                posq[qo] = j;
                alphaq[qo] = make_float2(alpha.hi, alpha.lo);
                p.perm[j] = piv;
            }
        }
        __syncthreads();
        const int len = l - j;
        // each active column c: w = beta v^* c, c <- c - w v. A warp takes two columns at a
        // time with two partial sums each (four independent float-float chains), then
        // downdates the squared norm: ||c[j+1..]||^2 = ||c[j..]||^2 - c_j^2, recomputed
        // exactly when it falls below 2^-20 of its last exact value (the downdate would
        // have lost more than 20 of its 48 bits).
        for (int q0 = warp * 2; q0 < nc; q0 += 2 * CQ_WARPS) {
            const int qa = q0, qb = q0 + 1;
            const bool da = posq[qa] < 0;
            const bool db = qb < nc && posq[qb] < 0;
            if (!da && !db) continue;
            float2* ca = cols + (size_t)qa * l + j;
            float2* cb = cols + (size_t)(db ? qb : qa) * l + j;
            ff sa0 = {0.f, 0.f}, sa1 = {0.f, 0.f}, sb0 = {0.f, 0.f}, sb1 = {0.f, 0.f};
            int i = lane;
            for (; i + 32 < len; i += 64) {
                const float2 a0 = v[i], a1 = v[i + 32];
                const float2 x0a = ca[i], x1a = ca[i + 32], x0b = cb[i], x1b = cb[i + 32];
                sa0 = ff_add(sa0, ff_mul({a0.x, a0.y}, {x0a.x, x0a.y}));
                sa1 = ff_add(sa1, ff_mul({a1.x, a1.y}, {x1a.x, x1a.y}));
                sb0 = ff_add(sb0, ff_mul({a0.x, a0.y}, {x0b.x, x0b.y}));
                sb1 = ff_add(sb1, ff_mul({a1.x, a1.y}, {x1b.x, x1b.y}));
            }
            if (i < len) {
                const float2 a0 = v[i], x0a = ca[i], x0b = cb[i];
                sa0 = ff_add(sa0, ff_mul({a0.x, a0.y}, {x0a.x, x0a.y}));
                sb0 = ff_add(sb0, ff_mul({a0.x, a0.y}, {x0b.x, x0b.y}));
            }
            const ff wa = ff_mul(ff_warp_sum(ff_add(sa0, sa1)), beta);
            const ff wb = ff_mul(ff_warp_sum(ff_add(sb0, sb1)), beta);
            for (i = lane; i < len; i += 32) {
                const float2 a = v[i];
                const ff af = {a.x, a.y};
                if (da) {
                    const float2 x = ca[i];
                    const ff y = ff_add({x.x, x.y}, ff_neg(ff_mul(wa, af)));
                    ca[i] = make_float2(y.hi, y.lo);
                }
                if (db) {
                    const float2 x = cb[i];
                    const ff y = ff_add({x.x, x.y}, ff_neg(ff_mul(wb, af)));
                    cb[i] = make_float2(y.hi, y.lo);
                }
            }
            __syncwarp();
            if (da) downdate_norm(ca, len, qa, lane, nsq, nsq_ref);
            if (db) downdate_norm(cb, len, qb, lane, nsq, nsq_ref);
        }
        __syncthreads();
        // this CTA's candidate for step j+1 (warp 0): the active column with the largest
        // downdated norm, published with its exact squared norm over rows j+1 .. l-1 (which
        // the reflector of step j+1 needs) into every CTA's shared memory
        if (warp == 0) {
            ff cv = {-1.f, 0.f};
            int ci = m;
            for (int q = lane; q < nc; q += 32)
                if (posq[q] < 0) {
                    const ff x = {nsq[q].x, nsq[q].y};
                    if (ci == m || ff_gt(x, cv)) { cv = x; ci = c0 + q; }
                }
            cand_reduce(cv, ci, m);
            if (ci < m) {
                const float2* c = cols + (size_t)(ci - c0) * l;
                ff s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
                int i = j + 1 + lane;
                for (; i + 32 < l; i += 64) {
                    const ff a = {c[i].x, c[i].y}, d = {c[i + 32].x, c[i + 32].y};
                    s0 = ff_add(s0, ff_mul(a, a));
                    s1 = ff_add(s1, ff_mul(d, d));
                }
                if (i < l) {
                    const ff a = {c[i].x, c[i].y};
                    s0 = ff_add(s0, ff_mul(a, a));
                }
                cv = ff_warp_sum(ff_add(s0, s1));
            }
            if (lane < CQ_CTAS) {
                *cluster.map_shared_rank(&cand_val[par ^ 1][b], lane) = make_float2(cv.hi, cv.lo);
                *cluster.map_shared_rank(&cand_idx[par ^ 1][b], lane) = ci;
            }
        }
    }
    // R[:, pos] = rows 0 .. pos-1 of the retired column, alpha on the diagonal (scaled back)
    const double unscale = ldexp(1.0, e);
    for (int q = 0; q < nc; ++q) {
        const int pos = posq[q];
        if (pos < 0) continue;             // every column is retired by step m - 1
        const float2* c = cols + (size_t)q * l;
        for (int i = t; i < m; i += CQ_THREADS) {
            double r = 0.0;
            if (i < pos) r = ((double)c[i].x + (double)c[i].y) * unscale;
            else if (i == pos) r = ((double)alphaq[q].x + (double)alphaq[q].y) * unscale;
            p.R[(int64_t)i * m + pos] = r;
        }
    }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace

bool qr_cluster_fits(int m, int l) {
    const int cpc = (m + CQ_CTAS - 1) / CQ_CTAS;
    const size_t smem = ((size_t)cpc * l + l) * sizeof(float2);
    return cpc <= CQ_MAXC && smem <= 200 * 1024;
}

cudaError_t pivoted_qr_cluster(const double* S, int m, int l, int64_t lds, double* R, int32_t* perm, int* fallback,
                               cudaStream_t s, bool* launched) {
    *launched = false;
    if (!qr_cluster_fits(m, l)) return cudaSuccess;
    const int cpc = (m + CQ_CTAS - 1) / CQ_CTAS;
    const size_t smem = ((size_t)cpc * l + l) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(qr_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(qr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;   // the caller uses the float64 kernel
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CQ_CTAS);
    cfg.blockDim = dim3(CQ_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CQ_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, qr_cluster_kernel, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return cudaSuccess;
    }
    CqrDev p;
    p.S = S; p.m = m; p.l = l; p.lds = lds; p.R = R; p.perm = perm; p.cpc = cpc; p.fallback = fallback;
    e = cudaLaunchKernelEx(&cfg, qr_cluster_kernel, p);
    note_launch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    *launched = true;
    return cudaSuccess;
}

}  // namespace rtp
