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


// ---------------------------------------------------------------------------------
// Persistent form: one cooperative launch for all m steps. CTA b keeps columns
// [b*cpc, b*cpc + cpc) of S^* (rows of S) in shared memory for the whole factorization,
// one warp per column. A step costs one grid-wide exchange. Before arriving for step j,
// each CTA publishes its candidate: its remaining column with the largest downdated
// squared norm (lowest index on ties), fully updated through step j-1 by all its warps,
// copied to the CTA's slot in global memory together with its exactly recomputed squared
// tail norm. After everyone has arrived, each CTA picks the global pivot among the
// candidates (largest squared norm, lowest column index on ties), reads that column from
// its owner's slot, forms the reflector itself (all CTAs compute bitwise the same alpha,
// beta and v) and applies it: first the row-j entry of each active column, so that the
// squared norms are downdated (LAPACK's rule, in squares: no division, no square root)
// and the next candidate is known early; the candidate's full update, slot copy and
// arrival follow, and the other columns' updates overlap the wait. Columns never move:
// the pivot column is retired and R[:, j] is the retired column's first j+1 entries.
// Slots and candidates alternate between two buffers by step parity. Every wait has a
// clock deadline; on expiry the kernel raises RTPROJ_ETIMEOUT and all CTAs leave their
// loops. (GB300's FP64 pipe takes 64 cycles per warp instruction, active lanes or not,
// so the step is arranged to keep float64 instructions off its critical path.)
constexpr int PQ_THREADS = 128;
constexpr int PQ_WARPS = PQ_THREADS / 32;
constexpr int PQ_MAXC = 32;
constexpr int PQ_MAX_G = 256;
constexpr int PQ_VLOAD = 5;             // slot entries per thread held in registers (l <= 640)

struct PqrDev {
    double* S; int m, l; int64_t lds;
    double* R; int32_t* perm;
    int cpc;
    double* slots;           // 2 x G x l: candidate columns by step parity
    double* bval;            // 2 x G: candidate squared tail norms
    int* bidx;               // 2 x G: candidate column indices (m = none)
    unsigned int* counter;   // arrivals (monotonic)
    int* abort_flag;
    int* status;
    long long timeout;
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
// The counter is polled back to back; the abort flag and the deadline every 64 polls.
__device__ bool wait_geq(const unsigned int* p, unsigned int target, int* abort_flag, int* status, long long timeout) {
    const long long t0 = clock64();
    for (unsigned int it = 1;; ++it) {
        if (ld_acquire(p) >= target) return true;
        if ((it & 63) == 0) {
            if (*(volatile int*)abort_flag) return false;
            if (clock64() - t0 > timeout) {
                atomicExch(abort_flag, 1);
                set_status(status, RTPROJ_ETIMEOUT);
                return false;
            }
        }
    }
}

// Squared norms are compared through their bit patterns: for non-negative doubles the
// integer order is the numeric order, and integer compares stay off the FP64 pipe.
__device__ __forceinline__ unsigned long long sq_bits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Candidate of this CTA for step j + 1 (parity par1): local column q (or none when q < 0),
// finishing its update with w (unless `done`) and copying rows j+1 .. l-1 to the slot;
// all warps share the rows. Its squared tail norm is recomputed exactly and published.
// Called by every thread of the CTA.
__device__ __forceinline__ void publish_candidate(const PqrDev& p, int b, int G, int par1, int j, int q, double* col,
                                                  const double* v, double w, bool done, double* s1, double* s2,
                                                  double* redv) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double ssq = 0.0;
    if (q >= 0) {
        double* slot = p.slots + ((int64_t)par1 * G + b) * p.l;
        const int first = j + 1, len1 = p.l - first;
        const int per = (len1 + PQ_WARPS - 1) / PQ_WARPS;
        const int lo = first + warp * per, hi = min(p.l, lo + per);
        double ssq1 = 0.0;
        for (int i = lo + lane; i < hi; i += 64) {
            double x = col[i];
            if (!done) {
                x = fma(-w, v[i - j], x);
                col[i] = x;
            }
            slot[i] = x;
            ssq = fma(x, x, ssq);
            const int i2 = i + 32;
            if (i2 < hi) {
                double y = col[i2];
                if (!done) {
                    y = fma(-w, v[i2 - j], y);
                    col[i2] = y;
                }
                slot[i2] = y;
                ssq1 = fma(y, y, ssq1);
            }
        }
        ssq = warp_sum(ssq + ssq1);
    }
    if (lane == 0) redv[warp] = ssq;
    // The CTA barrier orders every thread's slot writes before thread 0's release-add
    // (release is cumulative), which publishes them at GPU scope.
    __syncthreads();
    if (t == 0) {
        static_assert(PQ_WARPS == 4, "pairwise sum written for four warps");
        const double nsq = (redv[0] + redv[1]) + (redv[2] + redv[3]);
        if (q >= 0) { s1[q] = nsq; s2[q] = nsq; }
        p.bval[par1 * G + b] = q >= 0 ? nsq : 0.0;
        p.bidx[par1 * G + b] = q >= 0 ? b * p.cpc + q : p.m;
        red_release_add(p.counter, 1u);
    }
}

__global__ void __launch_bounds__(PQ_THREADS, 1) qr_persistent_kernel(PqrDev p) {
    extern __shared__ double smem_d[];
    const int l = p.l, m = p.m, cpc = p.cpc;
    double* cols = smem_d;                 // cpc x l
    double* v = cols + (size_t)cpc * l;    // l
    __shared__ double s1[PQ_MAXC], s2[PQ_MAXC], wq[PQ_MAXC];   // squared norms: downdated, at last recompute
    __shared__ int posq[PQ_MAXC];
    __shared__ unsigned char doneq[PQ_MAXC];
    __shared__ unsigned long long redb[2 * PQ_WARPS];
    __shared__ double redv[PQ_WARPS];
    __shared__ int redi[2 * PQ_WARPS];
    __shared__ int ok_s, cand_s;
    const int b = blockIdx.x, G = gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int c0 = b * cpc;
    const int nc = max(0, min(cpc, m - c0));
    const double tol3z = 1.4901161193847656e-08;   // sqrt(eps): LAPACK's recompute threshold

    for (int q = 0; q < nc; ++q)
        for (int i = t; i < l; i += PQ_THREADS) cols[(size_t)q * l + i] = p.S[(int64_t)(c0 + q) * p.lds + i];
    __syncthreads();
    for (int q = warp; q < nc; q += PQ_WARPS) {
        const double* c = cols + (size_t)q * l;
        double s = 0.0;
        for (int i = lane; i < l; i += 32) s = fma(c[i], c[i], s);
        s = warp_sum(s);
        if (lane == 0) { s1[q] = s; s2[q] = s; posq[q] = -1; }
    }
    __syncthreads();
    if (t == 0) {
        unsigned long long best = 0;
        int bq = -1;
        for (int q = 0; q < nc; ++q)
            if (bq < 0 || sq_bits(s1[q]) > best) { best = sq_bits(s1[q]); bq = q; }
        cand_s = bq;
    }
    __syncthreads();
    {
        const int q = cand_s;
        publish_candidate(p, b, G, 0, -1, q, q >= 0 ? cols + (size_t)q * l : nullptr, v, 0.0, true, s1, s2, redv);
    }

    bool alive = true;
    for (int j = 0; j < m && alive; ++j) {
        const int par = j & 1;
        // 1. wait for every candidate of step j
        if (t == 0) ok_s = wait_geq(p.counter, (unsigned int)(j + 1) * (unsigned int)G, p.abort_flag, p.status,
                                     p.timeout);
        __syncthreads();
        if (!ok_s) { alive = false; break; }
        // 2. global pivot: largest squared norm, lowest column index on ties
        unsigned long long best = 0;
        int bi = m;
        for (int g = t; g < G; g += PQ_THREADS) {
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
        if (lane == 0) { redb[par * PQ_WARPS + warp] = best; redi[par * PQ_WARPS + warp] = bi; }
        __syncthreads();
        // every thread combines the warps' results (double-buffered by step parity, so no
        // second barrier is needed before they are overwritten)
        unsigned long long bb = redb[par * PQ_WARPS];
        int ii = redi[par * PQ_WARPS];
        for (int w = 1; w < PQ_WARPS; ++w) {
            const unsigned long long xb = redb[par * PQ_WARPS + w];
            const int xi = redi[par * PQ_WARPS + w];
            if (xi < m && (ii == m || xb > bb || (xb == bb && xi < ii))) { bb = xb; ii = xi; }
        }
        if (ii >= m) { alive = false; break; }             // cannot happen while columns remain
        const int piv = ii;
        const int owner = ii / cpc;
        const double nsq = __longlong_as_double((long long)bb);
        // 3. the reflector from the owner's slot (rows j .. l-1); every thread derives alpha
        //    and beta from the published squared norm and the slot's first entry
        const double* slot = p.slots + ((int64_t)par * G + owner) * l;
        // the slot's loads are issued before the scalar chain so that their latency and the
        // square root and division overlap (PQ_VLOAD entries per thread in registers)
        double vr[PQ_VLOAD];
#pragma unroll
        for (int k = 0; k < PQ_VLOAD; ++k) {
            const int i = j + t + k * PQ_THREADS;
            vr[k] = i < l ? __ldcg(slot + i) : 0.0;
        }
        const double x0 = __ldcg(slot + j);
        const double nx = sqrt(nsq);
        double alpha = 0.0, beta = 0.0;
        if (nx > 0.0) {
            alpha = x0 >= 0.0 ? -nx : nx;
            beta = 1.0 / (nx * (nx + fabs(x0)));
        }
#pragma unroll
        for (int k = 0; k < PQ_VLOAD; ++k) {
            const int i = j + t + k * PQ_THREADS;
            if (i < l) v[i - j] = i == j ? x0 - alpha : vr[k];
        }
        for (int i = j + t + PQ_VLOAD * PQ_THREADS; i < l; i += PQ_THREADS) v[i - j] = __ldcg(slot + i);
        if (t == 0 && owner == b) {
            const int q = piv - c0;
            cols[(size_t)q * l + j] = alpha;
            posq[q] = j;
            p.perm[j] = piv;
        }
        __syncthreads();
        const int len = l - j;
        // 4a. row j of each active column and its downdated squared norm s1 - r^2; when the
        //     downdate falls to tol3z times the norm at the last recompute (LAPACK's test on
        //     the ratio), the column is updated in full here and its norm recomputed
        for (int q = warp; q < nc; q += PQ_WARPS) {
            if (posq[q] >= 0) continue;
            double* c = cols + (size_t)q * l + j;
            const double cj = c[0];
            // two independent partial sums: a dependent float64 chain costs more than the
            // pipe's issue interval per step
            double wa = 0.0, wb = 0.0;
            int i = lane;
            for (; i + 32 < len; i += 64) {
                wa = fma(v[i], c[i], wa);
                wb = fma(v[i + 32], c[i + 32], wb);
            }
            if (i < len) wa = fma(v[i], c[i], wa);
            const double w = warp_sum(wa + wb) * beta;
            const double r = fma(-w, v[0], cj);
            const double sq = s1[q];
            const double sq_new = fma(-r, r, sq);
            const bool recompute = sq != 0.0 && sq_new <= tol3z * s2[q];
            if (recompute) {
                double ss = 0.0;
                for (int i = 1 + lane; i < len; i += 32) {
                    const double x = fma(-w, v[i], c[i]);
                    c[i] = x;
                    ss = fma(x, x, ss);
                }
                ss = warp_sum(ss);
                if (lane == 0) { s1[q] = ss; s2[q] = ss; }
            } else if (lane == 0 && sq != 0.0) {
                s1[q] = sq_new;
            }
            if (lane == 0) { c[0] = r; wq[q] = w; doneq[q] = recompute ? 1 : 0; }
        }
        __syncthreads();
        // 4b. the next candidate (largest downdated squared norm, lowest index on ties): all
        //     warps finish its update, copy it to the slot and the CTA arrives
        // (every thread evaluates the same choice over the nc <= cpc columns: no barrier)
        int cand = -1;
        {
            unsigned long long bestn = 0;
            for (int q = 0; q < nc; ++q)
                if (posq[q] < 0 && (cand < 0 || sq_bits(s1[q]) > bestn)) { bestn = sq_bits(s1[q]); cand = q; }
        }
        publish_candidate(p, b, G, par ^ 1, j, cand, cand >= 0 ? cols + (size_t)cand * l : nullptr, v,
                          cand >= 0 ? wq[cand] : 0.0, cand >= 0 && doneq[cand], s1, s2, redv);
        // 4c. the remaining columns (overlapping the other CTAs' arrivals)
        for (int q = warp; q < nc; q += PQ_WARPS) {
            if (posq[q] >= 0 || q == cand || doneq[q]) continue;
            double* c = cols + (size_t)q * l + j;
            const double w = wq[q];
            for (int i = 1 + lane; i < len; i += 32) c[i] = fma(-w, v[i], c[i]);
        }
        __syncthreads();
    }
    if (!alive) return;
    // R[:, pos] = first pos+1 entries of the retired column
    for (int q = 0; q < nc; ++q) {
        const int pos = posq[q];
        const double* c = cols + (size_t)q * l;
        for (int i = t; i < m; i += PQ_THREADS) p.R[(int64_t)i * m + pos] = i <= pos ? c[i] : 0.0;
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
    const size_t persistent = (size_t)2 * PQ_MAX_G * l + 4 * (size_t)PQ_MAX_G + 64;   // slots, candidates
    return steps > persistent ? steps : persistent;
}

cudaError_t pivoted_qr(double* S, int m, int l, int64_t lds, double* R, int32_t* perm,
                       double* work, int* status, cudaStream_t s) {
    // Persistent cooperative form when the columns fit in shared memory.
    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (coop && sms > 0) {
        int cpc = (m + sms - 1) / sms;
        const size_t smem = ((size_t)cpc * l + l) * sizeof(double);
        const int G = (m + cpc - 1) / cpc;
        if (cpc <= PQ_MAXC && G <= PQ_MAX_G && smem + 4096 <= (size_t)smem_optin) {
            cudaFuncSetAttribute(qr_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_persistent_kernel, PQ_THREADS, smem);
            if (per_sm >= 1 && G <= per_sm * sms) {
                PqrDev p;
                p.S = S; p.m = m; p.l = l; p.lds = lds; p.R = R; p.perm = perm; p.cpc = cpc;
                double* w = work;
                p.slots = w;                    w += (size_t)2 * G * l;
                p.bval = w;                     w += 2 * (size_t)G;
                p.bidx = (int*)w;               w += G;          // 2G ints
                unsigned int* ctr = (unsigned int*)w;            // counter, abort
                p.counter = ctr;
                p.abort_flag = (int*)(ctr + 1);
                p.status = status;
                p.timeout = 4000000000ll;
                cudaError_t e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned int), s);
                if (e != cudaSuccess) return e;
                void* args[] = {&p};
                e = cudaLaunchCooperativeKernel((const void*)qr_persistent_kernel, dim3(G), dim3(PQ_THREADS), args,
                                                smem, s);
                note_launch();
                if (e == cudaSuccess) return cudaGetLastError();
                cudaGetLastError();   // clear and fall back
            }
        }
    }
    return pivoted_qr_steps(S, m, l, lds, R, perm, work, status, s);
}

}  // namespace rtp
