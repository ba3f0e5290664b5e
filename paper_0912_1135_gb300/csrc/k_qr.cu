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
#include "ff.cuh"

#include <climits>
#include <cstdlib>
#include <algorithm>

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


// ---------------------------------------------------------------------------------
// Persistent form: one cooperative launch for all m steps. CTA b keeps columns
// [b*cpc, b*cpc + cpc) of S^* (rows of S) in shared memory for the whole factorization,
// one warp per column, and consecutive steps are separated by one grid-wide exchange.
// The pivot rule is the textbook one (Businger-Golub with the norms recomputed every
// step): the pivot of step j is the remaining column whose trailing rows j .. l-1 have
// the largest squared norm, lowest index on ties. Step j in CTA b:
//  1. wait until every CTA has arrived for step j, read the G candidates (one per CTA:
//     its best remaining column's index and exact squared norm) and pick the pivot;
//  2. read the pivot column (rows j .. l-1) from its staging slot; every CTA derives the
//     same alpha = -sign(x_j) ||x|| and beta = 1 / (||x|| (||x|| + |x_j|)) from the
//     published squared norm and forms v = x - alpha e_j;
//  3. every warp applies I - beta v v^* to its column (row j becomes the R entry), and
//     in the same pass recomputes the column's squared norm over rows j+1 .. l-1 and
//     copies those rows to the column's staging slot for step j+1;
//  4. thread 0 publishes the CTA's best remaining column (index and squared norm) and
//     arrives.
// So the candidate's update, norm and copy run in parallel with the other columns' (one
// warp each) instead of after them. Columns never move: the pivot column is retired and
// R[:, j] is the retired column's first j+1 entries. Staging slots and candidates
// alternate between two buffers by step parity (a retired column's slot is never
// rewritten, so late readers of a pivot column are safe). Every wait has a clock
// deadline; on expiry the kernel raises RTPROJ_ETIMEOUT and all CTAs leave their loops.
// (GB300's FP64 pipe takes 64 cycles per warp instruction, active lanes or not, so long
// float64 chains are split into independent partial sums.)
constexpr int PQ_THREADS = 128;
constexpr int PQ_MAXC = 32;
constexpr int PQ_MAX_G = 256;
constexpr int PQ_VLOAD = 5;             // slot entries per thread held in registers (l <= 640)

struct PqrDev {
    double* S; int m, l; int64_t lds;
    double* R; int32_t* perm;
    int cpc;
    double* slots;           // 2 x G x cpc x l: staging copies of the columns by step parity
    double* bval;            // 2 x G: candidate squared tail norms
    int* bidx;               // 2 x G: candidate column indices (m = none)
    unsigned int* counter;   // arrivals (monotonic)
    int* abort_flag;
    int* status;
    long long timeout;
    const int* run_if;       // when set, the kernel runs only if *run_if != 0
    int* fallback;           // float-float form: set to 1 when the float64 kernel must run instead
    int* emax;               // float-float form: G exponents of the CTAs' largest entries
    unsigned long long* best;   // float-float form: m + 1 packed winners, one word per step (zeroed)
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *p >= target (or the abort flag is raised). Returns false on abort.
// The counter is polled back to back with the deadline checked after every failed poll;
// the abort flag every 64 polls.
__device__ bool wait_geq(const unsigned int* p, unsigned int target, int* abort_flag, int* status, long long timeout) {
    const long long t0 = clock64();
    for (unsigned int it = 1;; ++it) {
        if (ld_acquire(p) >= target) return true;
        if (clock64() - t0 > timeout) {
            atomicExch(abort_flag, 1);
            set_status(status, RTPROJ_ETIMEOUT);
            return false;
        }
        if ((it & 63) == 0 && *(volatile int*)abort_flag) return false;
    }
}

// Squared norms are compared through their bit patterns: for non-negative doubles the
// integer order is the numeric order, and integer compares stay off the FP64 pipe.
__device__ __forceinline__ unsigned long long sq_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Thread 0, after the CTA barrier that follows the columns' updates: publishes the best
// remaining local column for step s (largest squared norm, lowest index on ties) and
// arrives. The barrier orders every thread's staging-slot writes before the release-add
// (release is cumulative), which publishes them at GPU scope.
__device__ __forceinline__ void publish_best(const PqrDev& p, int b, int G, int s, int nc, const int* posq,
                                             const double* nsq) {
    unsigned long long best = 0;
    int bq = -1;
    for (int q = 0; q < nc; ++q)
        if (posq[q] < 0 && (bq < 0 || sq_bits(nsq[q]) > best)) { best = sq_bits(nsq[q]); bq = q; }
    const int par = s & 1;
    p.bval[par * G + b] = bq >= 0 ? nsq[bq] : 0.0;
    p.bidx[par * G + b] = bq >= 0 ? b * p.cpc + bq : p.m;
    red_release_add(p.counter, 1u);
}

// GLOBAL_COLS: the columns stay in S in global memory (they do not fit in shared memory,
// e.g. 2048 x 4128): each CTA updates its own columns in place, readers take the pivot
// column straight from S through L2 (no staging copies), and the retired column's diagonal
// entry is kept in shared memory so that no reader sees a half-written pivot column.
// Threads per CTA: 4 warps when the columns sit in shared memory (one warp per column at
// cpc <= 4); 16 when they stay in global memory, so that a CTA's columns (cpc up to 27 at
// m = 4096) are updated by many warps at once and their L2 loads overlap.
template <bool GLOBAL_COLS>
struct PqrShape {
    static constexpr int NT = GLOBAL_COLS ? 512 : PQ_THREADS;
    static constexpr int NW = NT / 32;
};

template <bool GLOBAL_COLS>
__global__ void __launch_bounds__(PqrShape<GLOBAL_COLS>::NT, 1) qr_persistent_kernel(PqrDev p) {
    constexpr int NT = PqrShape<GLOBAL_COLS>::NT, NW = PqrShape<GLOBAL_COLS>::NW;
    extern __shared__ double smem_d[];
    const int l = p.l, m = p.m, cpc = p.cpc;
    const int64_t cs = GLOBAL_COLS ? p.lds : (int64_t)l;                        // column stride
    double* cols = GLOBAL_COLS ? p.S + (int64_t)blockIdx.x * cpc * p.lds : smem_d;  // cpc x l
    double* v = GLOBAL_COLS ? smem_d : cols + (size_t)cpc * l;               // l
    __shared__ double nsq[PQ_MAXC];        // squared norm of rows j+1 .. l-1 (exact, this step)
    __shared__ double alphaq[PQ_MAXC];     // GLOBAL_COLS: the retired column's diagonal entry
    __shared__ int posq[PQ_MAXC];          // step at which the column was retired, -1 while active
    __shared__ unsigned long long redb[2 * NW];
    __shared__ int redi[2 * NW];
    __shared__ int ok_s;
    const int b = blockIdx.x, G = gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (p.run_if && *(volatile const int*)p.run_if == 0) return;   // the same value for every CTA
    const int c0 = b * cpc;
    const int nc = max(0, min(cpc, m - c0));
    const size_t slot_par = (size_t)G * cpc * l;   // doubles per parity buffer

    if (!GLOBAL_COLS)
        for (int q = 0; q < nc; ++q)
            for (int i = t; i < l; i += NT) {
                const double x = p.S[(int64_t)(c0 + q) * p.lds + i];
                cols[(size_t)q * l + i] = x;
                p.slots[((size_t)b * cpc + q) * l + i] = x;           // step 0's staging copy
            }
    __syncthreads();
    for (int q = warp; q < nc; q += NW) {
        const double* c = cols + (size_t)q * cs;
        double s0 = 0.0, s1 = 0.0;
        int i = lane;
        for (; i + 32 < l; i += 64) {
            s0 = fma(c[i], c[i], s0);
            s1 = fma(c[i + 32], c[i + 32], s1);
        }
        if (i < l) s0 = fma(c[i], c[i], s0);
        const double s = warp_sum(s0 + s1);
        if (lane == 0) { nsq[q] = s; posq[q] = -1; }
    }
    __syncthreads();
    if (t == 0) publish_best(p, b, G, 0, nc, posq, nsq);

    bool alive = true;
    for (int j = 0; j < m && alive; ++j) {
        const int par = j & 1;
        // 1. wait for every candidate of step j
        if (t == 0) ok_s = wait_geq(p.counter, (unsigned int)(j + 1) * (unsigned int)G, p.abort_flag, p.status,
                                     p.timeout);
        __syncthreads();
        if (!ok_s) { alive = false; break; }
        // global pivot: largest squared norm, lowest column index on ties
        unsigned long long best = 0;
        int bi = m;
        for (int g = t; g < G; g += NT) {
            const unsigned long long x = sq_bits(__ldcg(p.bval + par * G + g));
            const int i = __ldcg(p.bidx + par * G + g);
            if (i < m && (bi == m || x > best || (x == best && i < bi))) { best = x; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oi < m && (bi == m || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
        }
        if (lane == 0) { redb[par * NW + warp] = best; redi[par * NW + warp] = bi; }
        __syncthreads();
        // every thread combines the warps' results (double-buffered by step parity, so no
        // second barrier is needed before they are overwritten)
        unsigned long long bb = redb[par * NW];
        int ii = redi[par * NW];
        for (int w = 1; w < NW; ++w) {
            const unsigned long long xb = redb[par * NW + w];
            const int xi = redi[par * NW + w];
            if (xi < m && (ii == m || xb > bb || (xb == bb && xi < ii))) { bb = xb; ii = xi; }
        }
        if (ii >= m) { alive = false; break; }             // cannot happen while columns remain
        const int piv = ii;
        const double nsq_piv = __longlong_as_double((long long)bb);
        // 2. the reflector from the pivot column's staging slot (rows j .. l-1), or from the
        //    pivot column itself when the columns stay in global memory
        const double* slot = GLOBAL_COLS ? p.S + (int64_t)piv * p.lds : p.slots + (size_t)par * slot_par + (size_t)piv * l;
        // the slot's loads are issued before the scalar chain so that their latency and the
        // square root and division overlap (PQ_VLOAD entries per thread in registers)
        double vr[PQ_VLOAD];
#pragma unroll
        for (int k = 0; k < PQ_VLOAD; ++k) {
            const int i = j + t + k * NT;
            vr[k] = i < l ? __ldcg(slot + i) : 0.0;
        }
        const double x0 = __ldcg(slot + j);
        const double nx = sqrt(nsq_piv);
        double alpha = 0.0, beta = 0.0;
        if (nx > 0.0) {
            alpha = x0 >= 0.0 ? -nx : nx;
            beta = 1.0 / (nx * (nx + fabs(x0)));
        }
#pragma unroll
        for (int k = 0; k < PQ_VLOAD; ++k) {
            const int i = j + t + k * NT;
            if (i < l) v[i - j] = i == j ? x0 - alpha : vr[k];
        }
        for (int i = j + t + PQ_VLOAD * NT; i < l; i += NT) v[i - j] = __ldcg(slot + i);
        if (t == 0 && piv >= c0 && piv < c0 + nc) {
            const int q = piv - c0;
            if (GLOBAL_COLS) alphaq[q] = alpha;
            else cols[(size_t)q * l + j] = alpha;
            posq[q] = j;
            p.perm[j] = piv;
        }
        __syncthreads();
        const int len = l - j;
        // 3. each active column: w = beta v^* c, c <- c - w v (row j is the R entry), the
        //    squared norm of rows j+1 .. l-1 and their copy to the staging slot of step j+1
        double* next = p.slots + (size_t)(par ^ 1) * slot_par;
        for (int q = warp; q < nc; q += NW) {
            if (posq[q] >= 0) continue;
            double* c = cols + (size_t)q * cs + j;
            // four independent loads and partial sums per lane and pass (latency overlap)
            double wa0 = 0.0, wa1 = 0.0, wa2 = 0.0, wa3 = 0.0;
            int i = lane;
            for (; i + 96 < len; i += 128) {
                const double c0 = c[i], c1 = c[i + 32], c2 = c[i + 64], c3 = c[i + 96];
                wa0 = fma(v[i], c0, wa0);
                wa1 = fma(v[i + 32], c1, wa1);
                wa2 = fma(v[i + 64], c2, wa2);
                wa3 = fma(v[i + 96], c3, wa3);
            }
            for (; i < len; i += 32) wa0 = fma(v[i], c[i], wa0);
            const double w = warp_sum((wa0 + wa1) + (wa2 + wa3)) * beta;
            double* dst = next + ((size_t)b * cpc + q) * l + j;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (i = 1 + lane; i + 96 < len; i += 128) {
                const double c0 = c[i], c1 = c[i + 32], c2 = c[i + 64], c3 = c[i + 96];
                const double x0 = fma(-w, v[i], c0), x1 = fma(-w, v[i + 32], c1);
                const double x2 = fma(-w, v[i + 64], c2), x3 = fma(-w, v[i + 96], c3);
                c[i] = x0;
                c[i + 32] = x1;
                c[i + 64] = x2;
                c[i + 96] = x3;
                if (!GLOBAL_COLS) {
                    dst[i] = x0;
                    dst[i + 32] = x1;
                    dst[i + 64] = x2;
                    dst[i + 96] = x3;
                }
                s0 = fma(x0, x0, s0);
                s1 = fma(x1, x1, s1);
                s2 = fma(x2, x2, s2);
                s3 = fma(x3, x3, s3);
            }
            for (; i < len; i += 32) {
                const double x = fma(-w, v[i], c[i]);
                c[i] = x;
                if (!GLOBAL_COLS) dst[i] = x;
                s0 = fma(x, x, s0);
            }
            const double ssq = warp_sum((s0 + s1) + (s2 + s3));
            if (lane == 0) {
                c[0] = fma(-w, v[0], c[0]);
                nsq[q] = ssq;
            }
        }
        __syncthreads();
        // 4. the CTA's candidate for step j+1
        if (t == 0) publish_best(p, b, G, j + 1, nc, posq, nsq);
    }
    if (!alive) return;
    // R[:, pos] = first pos+1 entries of the retired column
    for (int q = 0; q < nc; ++q) {
        const int pos = posq[q];
        if (pos < 0) continue;
        const double* c = cols + (size_t)q * cs;
        for (int i = t; i < m; i += NT)
            p.R[(int64_t)i * m + pos] = i < pos ? c[i] : i == pos ? (GLOBAL_COLS ? alphaq[q] : c[i]) : 0.0;
    }
}


// ---------------------------------------------------------------------------------
// Float-float form of the persistent kernel (the mixed form's QR). The same exchange,
// pivot rule (squared norms summed afresh every step, largest first, lowest index on ties)
// and column layout, with every column held as float-float pairs on the FP32 pipe (GB300's
// FP64 pipe takes 64 cycles per warp instruction, which bounds the float64 kernel's column
// updates). Before step 0 the CTAs exchange the exponents of their largest entries once,
// and S^* is scaled by 2^-E (exact) so that its largest entry lies below 1; R is scaled
// back on output. A pivot whose squared norm falls below 2^-100 (float-float would lose
// the digits of a trailing norm near float's underflow) makes every CTA return before
// writing R or perm and sets *fallback, so that the float64 kernel, enqueued after this
// one, runs instead; S itself is not modified (the global form keeps its float-float
// columns in the work area). Accuracy: R is the exact factor of S^* + E with ||E|| of
// order l 2^-48 ||S||, which the preconditioner tolerates while 2^-48 kappa(A) << 1; the
// refinement makes the projection exact whatever the preconditioner's rounding.
// The CTA's best remaining column for step s: its exact squared norm in bval, and a packed
// key in the step's word best[s] by one 64-bit atomic maximum -- the norm's bit pattern
// without its 12 lowest mantissa bits (the order of non-negative doubles), then 4095 minus
// the column index -- so that after the exchange every CTA reads the winner with one load
// instead of every CTA's candidate. Columns whose norms agree to 40 mantissa bits count as
// tied (lowest index first).
template <bool GLOBAL_COLS>
__device__ __forceinline__ void publish_best_ff(const PqrDev& p, int b, int G, int s, int nc, const int* posq,
                                                const ff* nsq) {
    int bq = -1;
    for (int q = 0; q < nc; ++q)
        if (posq[q] < 0 && (bq < 0 || ff_gt(nsq[q], nsq[bq]))) bq = q;
    const int par = s & 1;
    if (bq >= 0) {
        const double v = ff_to_double(nsq[bq]);
        p.bval[par * G + b] = v;
        const unsigned long long key =
            ((sq_bits(v) >> 12) << 12) | (unsigned long long)(4095 - (b * p.cpc + bq));
        atomicMax(p.best + s, key);
    }
    red_release_add(p.counter, 1u);
}

template <bool GLOBAL_COLS, int NT>
__global__ void __launch_bounds__(NT, 1) qr_persistent_ff_kernel(PqrDev p) {
    constexpr int NW = NT / 32;
    extern __shared__ float2 smem_f[];
    const int l = p.l, m = p.m, cpc = p.cpc;
    const int b = blockIdx.x, G = gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float2* slots = reinterpret_cast<float2*>(p.slots);
    const size_t slot_par = (size_t)G * cpc * l;                     // float2 per parity buffer
    float2* cols = GLOBAL_COLS ? slots + (size_t)b * cpc * l : smem_f;     // cpc x l
    float2* v = GLOBAL_COLS ? smem_f : cols + (size_t)cpc * l;             // l
    __shared__ ff nsq[PQ_MAXC];
    __shared__ ff alphaq[PQ_MAXC];
    __shared__ int posq[PQ_MAXC];
    __shared__ int ok_s, e_s, range_s;
    const int c0 = b * cpc;
    const int nc = max(0, min(cpc, m - c0));

    // 0. the scale: exponents of the CTAs' largest entries, and of their columns' smallest
    //    largest entry, exchanged once. Columns whose largest entries span more than 2^40
    //    (a graded S^*, e.g. rows of A scaled far apart) would take float-float's products
    //    toward float's underflow as the factorization reaches them: the float64 kernel
    //    takes the whole factorization instead.
    __shared__ double col_mx[PQ_MAXC];
    for (int q = warp; q < nc; q += NW) {
        double cm = 0.0;
        for (int i = lane; i < l; i += 32) cm = fmax(cm, fabs(p.S[(int64_t)(c0 + q) * p.lds + i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        if (lane == 0) col_mx[q] = cm;
    }
    __syncthreads();
    if (t == 0) {
        int e_hi = INT_MIN / 2, e_lo = INT_MAX / 2;
        for (int q = 0; q < nc; ++q) {
            int e = INT_MIN / 2;
            if (col_mx[q] > 0.0) frexp(col_mx[q], &e);   // col_mx < 2^e
            e_hi = max(e_hi, e);
            e_lo = min(e_lo, e);
        }
        p.emax[b] = e_hi;
        p.emax[G + b] = e_lo;
        red_release_add(p.counter, 1u);
        ok_s = wait_geq(p.counter, (unsigned int)G, p.abort_flag, p.status, p.timeout);
        int E = INT_MIN / 2, Elo = INT_MAX / 2;
        if (ok_s)
            for (int g = 0; g < G; ++g) {
                E = max(E, __ldcg(p.emax + g));
                Elo = min(Elo, __ldcg(p.emax + G + g));
            }
        e_s = E == INT_MIN / 2 ? 0 : E;
        range_s = E - Elo;
    }
    __syncthreads();
    if (!ok_s) return;
    if (range_s > 40) {                                     // the same decision in every CTA
        if (b == 0 && t == 0) *p.fallback = 1;
        return;
    }
    const int E = e_s;
    const double sc = ldexp(1.0, -E);
    for (int q = 0; q < nc; ++q)
        for (int i = t; i < l; i += NT) {
            const ff x = ff_from_double(p.S[(int64_t)(c0 + q) * p.lds + i] * sc);
            cols[(size_t)q * l + i] = make_float2(x.hi, x.lo);
            if (!GLOBAL_COLS) slots[((size_t)b * cpc + q) * l + i] = make_float2(x.hi, x.lo);
        }
    __syncthreads();
    for (int q = warp; q < nc; q += NW) {
        const float2* c = cols + (size_t)q * l;
        ff a0 = {0.f, 0.f}, a1 = {0.f, 0.f};
        int i = lane;
        for (; i + 32 < l; i += 64) {
            const ff x = {c[i].x, c[i].y}, y = {c[i + 32].x, c[i + 32].y};
            ff_dot_acc(a0, x, x);
            ff_dot_acc(a1, y, y);
        }
        if (i < l) { const ff x = {c[i].x, c[i].y}; ff_dot_acc(a0, x, x); }
        const ff s2 = ff_warp_sum(ff_add(ff_renorm(a0), ff_renorm(a1)));
        if (lane == 0) { nsq[q] = s2; posq[q] = -1; }
    }
    __syncthreads();
    if (t == 0) publish_best_ff<GLOBAL_COLS>(p, b, G, 0, nc, posq, nsq);

    for (int j = 0; j < m; ++j) {
        const int par = j & 1;
        // 1. wait for every candidate of step j (after the scale exchange: G more arrivals)
        if (t == 0) ok_s = wait_geq(p.counter, (unsigned int)(j + 2) * (unsigned int)G, p.abort_flag, p.status,
                                     p.timeout);
        __syncthreads();
        if (!ok_s) return;
        const unsigned long long key = __ldcg(p.best + j);
        if (key == 0ull) return;                               // cannot happen while columns remain
        const int piv = 4095 - (int)(key & 4095ull);
        if (piv < 0 || piv >= m) return;
        // 2. the reflector from the pivot column (rows j .. l-1): the column's loads, its norm
        //    and its first entry are all issued before any of them is used
        const float2* slot = GLOBAL_COLS ? slots + (size_t)piv * l : slots + (size_t)par * slot_par + (size_t)piv * l;
        float2 vr[PQ_VLOAD];
#pragma unroll
        for (int k = 0; k < PQ_VLOAD; ++k) {
            const int i = j + t + k * NT;
            vr[k] = i < l ? __ldcg(slot + i) : make_float2(0.f, 0.f);
        }
        const double nsq_piv = __ldcg(p.bval + par * G + piv / cpc);
        const float2 x0f = __ldcg(slot + j);
        const ff npiv = ff_from_double(nsq_piv);
        if (npiv.hi < 7.888609052210118e-31f) {                // 2^-100: the float64 kernel takes over
            if (b == 0 && t == 0) *p.fallback = 1;
            return;
        }
        const ff x0 = {x0f.x, x0f.y};
        const ff nx = ff_sqrt(npiv);
        const ff ax = x0.hi >= 0.f ? x0 : ff_neg(x0);
        const ff alpha = x0.hi >= 0.f ? ff_neg(nx) : nx;
        const ff beta = ff_recip(ff_mul(nx, ff_add(nx, ax)));
#pragma unroll
        for (int k = 0; k < PQ_VLOAD; ++k) {
            const int i = j + t + k * NT;
            if (i < l) v[i - j] = vr[k];
        }
        for (int i = j + t + PQ_VLOAD * NT; i < l; i += NT) v[i - j] = __ldcg(slot + i);
        if (t == 0) {
            const ff v0 = ff_add(x0, ff_neg(alpha));
            v[0] = make_float2(v0.hi, v0.lo);
        }
        if (t == 0 && piv >= c0 && piv < c0 + nc) {
            const int q = piv - c0;
            alphaq[q] = alpha;
            posq[q] = j;
            p.perm[j] = piv;
        }
        __syncthreads();
        const int len = l - j;
        // 3. each active column: w = beta v^* c, c <- c - w v, the squared norm of rows
        //    j+1 .. l-1 and their copy to the staging slot of step j+1
        float2* next = slots + (size_t)(par ^ 1) * slot_par;
        for (int q = warp; q < nc; q += NW) {
            if (posq[q] >= 0) continue;
            float2* c = cols + (size_t)q * l + j;
            ff a0 = {0.f, 0.f}, a1 = {0.f, 0.f}, a2 = {0.f, 0.f}, a3 = {0.f, 0.f};
            int i = lane;
            for (; i + 96 < len; i += 128) {
                const float2 c0f = c[i], c1f = c[i + 32], c2f = c[i + 64], c3f = c[i + 96];
                const float2 v0 = v[i], v1 = v[i + 32], v2 = v[i + 64], v3 = v[i + 96];
                ff_dot_acc(a0, {v0.x, v0.y}, {c0f.x, c0f.y});
                ff_dot_acc(a1, {v1.x, v1.y}, {c1f.x, c1f.y});
                ff_dot_acc(a2, {v2.x, v2.y}, {c2f.x, c2f.y});
                ff_dot_acc(a3, {v3.x, v3.y}, {c3f.x, c3f.y});
            }
            for (; i < len; i += 32) ff_dot_acc(a0, {v[i].x, v[i].y}, {c[i].x, c[i].y});
            const ff dot = ff_warp_sum(ff_add(ff_add(ff_renorm(a0), ff_renorm(a1)), ff_add(ff_renorm(a2), ff_renorm(a3))));
            const ff nw = ff_neg(ff_mul(dot, beta));
            float2* dst = next + ((size_t)b * cpc + q) * l + j;
            ff s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
            for (i = 1 + lane; i + 32 < len; i += 64) {
                const float2 ca = c[i], cb = c[i + 32];
                const float2 va = v[i], vb = v[i + 32];
                const ff xa = ff_add({ca.x, ca.y}, ff_mul(nw, {va.x, va.y}));
                const ff xb = ff_add({cb.x, cb.y}, ff_mul(nw, {vb.x, vb.y}));
                c[i] = make_float2(xa.hi, xa.lo);
                c[i + 32] = make_float2(xb.hi, xb.lo);
                if (!GLOBAL_COLS) {
                    dst[i] = make_float2(xa.hi, xa.lo);
                    dst[i + 32] = make_float2(xb.hi, xb.lo);
                }
                ff_dot_acc(s0, xa, xa);
                ff_dot_acc(s1, xb, xb);
            }
            for (; i < len; i += 32) {
                const ff x = ff_add({c[i].x, c[i].y}, ff_mul(nw, {v[i].x, v[i].y}));
                c[i] = make_float2(x.hi, x.lo);
                if (!GLOBAL_COLS) dst[i] = make_float2(x.hi, x.lo);
                ff_dot_acc(s0, x, x);
            }
            const ff ssq = ff_warp_sum(ff_add(ff_renorm(s0), ff_renorm(s1)));
            if (lane == 0) {
                const ff r0 = ff_add({c[0].x, c[0].y}, ff_mul(nw, {v[0].x, v[0].y}));
                c[0] = make_float2(r0.hi, r0.lo);
                nsq[q] = ssq;
            }
        }
        __syncthreads();
        // 4. the CTA's candidate for step j+1
        if (t == 0) publish_best_ff<GLOBAL_COLS>(p, b, G, j + 1, nc, posq, nsq);
    }
    // R[:, pos] = first pos+1 entries of the retired column, scaled back by 2^E
    for (int q = 0; q < nc; ++q) {
        const int pos = posq[q];
        if (pos < 0) continue;
        const float2* c = cols + (size_t)q * l;
        for (int i = t; i < m; i += NT) {
            const double r = i < pos ? ff_to_double({c[i].x, c[i].y}) : i == pos ? ff_to_double(alphaq[q]) : 0.0;
            p.R[(int64_t)i * m + pos] = ldexp(r, E);
        }
    }
}

}  // namespace

cudaError_t pivoted_qr_steps(double* S, int m, int l, int64_t lds, double* R, int32_t* perm,
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

size_t pivoted_qr_work_doubles(int m, int l) {
    const size_t steps = (size_t)3 * m + 3 * (size_t)l + 2048;                       // per-step form
    // staging slots (G * cpc < m + cpc columns per parity), candidates, counter and flag
    const size_t persistent = (size_t)2 * ((size_t)m + PQ_MAXC) * l + 5 * (size_t)PQ_MAX_G + (size_t)m + 65;
    return steps > persistent ? steps : persistent;
}

// One CTA: perm must hold every index 0..m-1 once (m <= 4096: a bitmap in shared
// memory); otherwise the identity replaces it. Then the rank test on |R_mm| / |R_11|.
__global__ void __launch_bounds__(1024) qr_check_kernel(const double* R, int32_t* perm, int m, double tol, int* status) {
    __shared__ unsigned int seen[128];
    __shared__ int bad;
    const int t = threadIdx.x;
    if (t < 128) seen[t] = 0u;
    if (t == 0) bad = 0;
    __syncthreads();
    for (int j = t; j < m; j += blockDim.x) {
        const int v = perm[j];
        if (v < 0 || v >= m) bad = 1;
        else if (atomicOr(&seen[v >> 5], 1u << (v & 31)) & (1u << (v & 31))) bad = 1;
    }
    __syncthreads();
    if (bad) {
        for (int j = t; j < m; j += blockDim.x) perm[j] = j;
        if (t == 0) set_status(status, RTPROJ_ETIMEOUT);   // only a QR that gave up leaves perm incomplete
        return;
    }
    if (t == 0) {
        const double r11 = fabs(R[0]);
        const double rmm = fabs(R[(int64_t)(m - 1) * m + (m - 1)]);
        if (!isfinite(r11) || !isfinite(rmm)) set_status(status, RTPROJ_ENONFINITE);
        else if (!(rmm > tol * r11)) set_status(status, RTPROJ_ERANK);
    }
}

cudaError_t qr_check(const double* R, int32_t* perm, int m, double tol, int* status, cudaStream_t s) {
    if (m > 4096) return cudaErrorInvalidValue;
    qr_check_kernel<<<1, 1024, 0, s>>>(R, perm, m, tol, status);
    note_launch();
    return cudaGetLastError();
}

// Columns per CTA of the float-float kernel's shared-memory form. Measured at 512 x 516:
// 4 (128 CTAs) 2.40 ms per factorization, 8 (64 CTAs) 2.57 ms, 16 (32 CTAs) 3.26 ms; with
// four steps in flight the smaller grids left more SMs to the other steps (17,886, 18,463
// and 18,508 projections/s), a smaller gain than the latency they cost one step.
constexpr int ff_cols_per_cta() { return 4; }

cudaError_t pivoted_qr_ff(double* S, int m, int l, int64_t lds, double* R, int32_t* perm, double* work, int* status,
                          cudaStream_t s, long long spin_limit, int* fallback, bool* launched) {
    *launched = false;
    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop || sms <= 0) return cudaSuccess;
    // columns in shared memory: about ff_cols_per_cta() columns per CTA, one warp each, so
    // that fewer CTAs take part in each step's exchange (and the rest of the GPU stays free
    // for other work); one CTA per SM with 16 warps when the columns stay in global memory
    const int cpc_min = (m + sms - 1) / sms;
    const int cpc_s = std::min(PQ_MAXC, std::max(cpc_min, ff_cols_per_cta()));
    const size_t smem_shared = ((size_t)cpc_s * l + l) * sizeof(float2);
    const bool in_smem = smem_shared + 4096 <= (size_t)smem_optin;
    const int cpc = in_smem ? cpc_s : cpc_min;
    const int G = (m + cpc - 1) / cpc;
    const size_t smem_global = (size_t)l * sizeof(float2);
    const size_t smem = in_smem ? smem_shared : smem_global;
    const int warps_s = std::min(32, std::max(4, cpc));
    const void* kern = !in_smem        ? (const void*)qr_persistent_ff_kernel<true, 512>
                       : warps_s <= 4  ? (const void*)qr_persistent_ff_kernel<false, 128>
                       : warps_s <= 8  ? (const void*)qr_persistent_ff_kernel<false, 256>
                       : warps_s <= 16 ? (const void*)qr_persistent_ff_kernel<false, 512>
                                       : (const void*)qr_persistent_ff_kernel<false, 1024>;
    const int nt = !in_smem ? 512 : warps_s <= 4 ? 128 : warps_s <= 8 ? 256 : warps_s <= 16 ? 512 : 1024;
    if (cpc > PQ_MAXC || G > PQ_MAX_G || smem + 4096 > (size_t)smem_optin) return cudaSuccess;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
    if (per_sm < 1 || G > per_sm * sms) return cudaSuccess;
    PqrDev p;
    p.S = S; p.m = m; p.l = l; p.lds = lds; p.R = R; p.perm = perm; p.cpc = cpc;
    double* w = work;
    // float-float columns: the staging slots (two parities) in shared-memory form, the
    // columns themselves in the global form; both fit the float64 form's slot area
    p.slots = w;                    w += in_smem ? (size_t)2 * G * cpc * l : (size_t)G * cpc * l;
    p.bval = w;                     w += 2 * (size_t)G;
    p.bidx = (int*)w;               w += G;          // 2G ints
    p.emax = (int*)w;               w += G;          // 2G ints: largest and smallest exponents
    p.best = (unsigned long long*)w; w += m + 1;     // one word per step
    unsigned int* ctr = (unsigned int*)w;            // counter, abort
    p.counter = ctr;
    p.abort_flag = (int*)(ctr + 1);
    p.status = status;
    p.timeout = spin_limit;
    p.run_if = nullptr;
    p.fallback = fallback;
    cudaError_t e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.best, 0, (size_t)(m + 1) * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(fallback, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&p};
    e = cudaLaunchCooperativeKernel(kern, dim3(G), dim3(nt), args, smem, s);
    note_launch();
    if (e == cudaSuccess) {
        *launched = true;
        return cudaSuccess;
    }
    cudaGetLastError();   // clear; the float64 kernel runs unconditionally
    return cudaSuccess;
}

bool pivoted_qr_persistent_ok(int m, int l) {
    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop || sms <= 0) return false;
    const int cpc = (m + sms - 1) / sms;
    const size_t smem = ((size_t)cpc * l + l) * sizeof(double);
    const int G = (m + cpc - 1) / cpc;
    return cpc <= PQ_MAXC && G <= PQ_MAX_G && smem + 4096 <= (size_t)smem_optin;
}

cudaError_t pivoted_qr(double* S, int m, int l, int64_t lds, double* R, int32_t* perm,
                       double* work, int* status, cudaStream_t s, long long spin_limit, const int* run_if) {
    // Persistent cooperative form: columns in shared memory when they fit, else in place in
    // S (global memory); per-step kernels when neither can launch.
    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (coop && sms > 0) {
        const int cpc = (m + sms - 1) / sms;
        const int G = (m + cpc - 1) / cpc;
        const size_t smem_shared = ((size_t)cpc * l + l) * sizeof(double);
        const size_t smem_global = (size_t)l * sizeof(double);
        const bool in_smem = smem_shared + 4096 <= (size_t)smem_optin;
        const size_t smem = in_smem ? smem_shared : smem_global;
        const void* kern = in_smem ? (const void*)qr_persistent_kernel<false> : (const void*)qr_persistent_kernel<true>;
        const int nt = in_smem ? PqrShape<false>::NT : PqrShape<true>::NT;
        if (cpc <= PQ_MAXC && G <= PQ_MAX_G && smem + 4096 <= (size_t)smem_optin) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
            if (per_sm >= 1 && G <= per_sm * sms) {
                PqrDev p;
                p.S = S; p.m = m; p.l = l; p.lds = lds; p.R = R; p.perm = perm; p.cpc = cpc;
                double* w = work;
                p.slots = w;                    w += in_smem ? (size_t)2 * G * cpc * l : 0;
                p.bval = w;                     w += 2 * (size_t)G;
                p.bidx = (int*)w;               w += G;          // 2G ints
                unsigned int* ctr = (unsigned int*)w;            // counter, abort
                p.counter = ctr;
                p.abort_flag = (int*)(ctr + 1);
                p.status = status;
                p.timeout = spin_limit;
                p.run_if = run_if;
                p.fallback = nullptr;
                p.emax = nullptr;
                p.best = nullptr;
                cudaError_t e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned int), s);
                if (e != cudaSuccess) return e;
                void* args[] = {&p};
                e = cudaLaunchCooperativeKernel(kern, dim3(G), dim3(nt), args, smem, s);
                note_launch();
                if (e == cudaSuccess) return cudaGetLastError();
                cudaGetLastError();   // clear and fall back
            }
        }
    }
    return pivoted_qr_steps(S, m, l, lds, R, perm, work, status, s);
}

}  // namespace rtp
