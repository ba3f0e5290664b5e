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
// [b*cpc, b*cpc + cpc) of S^* (rows of S) in shared memory for the whole
// factorization. Per step j: every CTA publishes the best remaining column norm it
// owns and arrives on a grid-wide counter; after all have arrived each CTA picks the
// global pivot (largest norm, lowest index on ties), reads the pivot column from global
// memory (every CTA writes its updated columns back after each step), forms the
// reflector itself and applies it to its active columns, downdating the norms. Columns never move: the
// pivot column is retired and R[:, j] is the retired column's first j+1 entries.
// Every wait has a clock deadline; on expiry the kernel raises RTPROJ_ETIMEOUT and all
// CTAs leave their loops.
// ---------------------------------------------------------------------------------
constexpr int PQ_THREADS = 256;
constexpr int PQ_WARPS = PQ_THREADS / 32;
constexpr int PQ_MAXC = 32;

struct PqrDev {
    double* S; int m, l; int64_t lds;
    double* R; int32_t* perm;
    int cpc;
    double* vbuf;            // 2 x l
    double* scal;            // 2 x 2
    double* bval;            // 2 x G
    int* bidx;               // 2 x G
    unsigned int* counter;   // arrivals (monotonic)
    unsigned int* flags;     // m: reflector j published
    int* abort_flag;
    int* status;
    long long timeout;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *p >= target (or the abort flag is raised). Returns false on abort.
__device__ bool wait_geq(const unsigned int* p, unsigned int target, int* abort_flag, int* status, long long timeout) {
    const long long t0 = clock64();
    while (ld_acquire(p) < target) {
        if (*(volatile int*)abort_flag) return false;
        if (clock64() - t0 > timeout) {
            atomicExch(abort_flag, 1);
            set_status(status, RTPROJ_ETIMEOUT);
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(PQ_THREADS, 1) qr_persistent_kernel(PqrDev p) {
    extern __shared__ double smem_d[];
    const int l = p.l, m = p.m, cpc = p.cpc;
    double* cols = smem_d;                 // cpc x l
    double* v = cols + (size_t)cpc * l;    // l
    __shared__ double vn1[PQ_MAXC], vn2[PQ_MAXC];
    __shared__ int posq[PQ_MAXC];
    __shared__ double redv[PQ_WARPS];
    __shared__ int redi[PQ_WARPS];
    __shared__ int piv_s, ok_s;
    __shared__ double beta_s;
    const int b = blockIdx.x, G = gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int c0 = b * cpc;
    const int nc = max(0, min(cpc, m - c0));

    for (int q = 0; q < nc; ++q)
        for (int i = t; i < l; i += PQ_THREADS) cols[(size_t)q * l + i] = p.S[(int64_t)(c0 + q) * p.lds + i];
    __syncthreads();
    for (int q = warp; q < nc; q += PQ_WARPS) {
        const double* c = cols + (size_t)q * l;
        double s = 0.0;
        for (int i = lane; i < l; i += 32) s = fma(c[i], c[i], s);
        s = warp_sum(s);
        if (lane == 0) { vn1[q] = sqrt(s); vn2[q] = sqrt(s); posq[q] = -1; }
    }
    __syncthreads();

    bool alive = true;
    for (int j = 0; j < m && alive; ++j) {
        const int par = j & 1;
        // 1. publish the local best, arrive, wait for everyone
        if (t == 0) {
            double best = -1.0;
            int bi = m;
            for (int q = 0; q < nc; ++q)
                if (posq[q] < 0 && (vn1[q] > best)) { best = vn1[q]; bi = c0 + q; }
            p.bval[par * G + b] = best;
            p.bidx[par * G + b] = bi;
            __threadfence();
            atomicAdd(p.counter, 1u);
            ok_s = wait_geq(p.counter, (unsigned int)(j + 1) * (unsigned int)G, p.abort_flag, p.status, p.timeout);
        }
        __syncthreads();
        if (!ok_s) { alive = false; break; }
        // 2. global pivot: largest norm, lowest column index on ties
        double best = -1.0;
        int bi = m;
        for (int g = t; g < G; g += PQ_THREADS) {
            const double x = __ldcg(p.bval + par * G + g);
            const int i = __ldcg(p.bidx + par * G + g);
            if (x > best || (x == best && i < bi)) { best = x; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
        __syncthreads();
        if (t == 0) {
            double bb = redv[0];
            int ii = redi[0];
            for (int w = 1; w < PQ_WARPS; ++w)
                if (redv[w] > bb || (redv[w] == bb && redi[w] < ii)) { bb = redv[w]; ii = redi[w]; }
            piv_s = ii < m ? ii : -1;
        }
        __syncthreads();
        const int piv = piv_s;
        if (piv < 0) { alive = false; break; }     // cannot happen while columns remain
        // 3. every CTA forms the reflector itself from the pivot column, read from global
        //    memory (each CTA writes its active columns back after every update), so the
        //    reflector needs no second broadcast. All CTAs sum in the same order and get
        //    bitwise the same alpha, beta and v.
        const int owner = piv / cpc;
        {
            const double* pc = p.S + (int64_t)piv * p.lds;
            double s = 0.0;
            for (int i = j + t; i < l; i += PQ_THREADS) {
                const double x = __ldcg(pc + i);
                v[i - j] = x;
                s = fma(x, x, s);
            }
            s = warp_sum(s);
            if (lane == 0) redv[warp] = s;
            __syncthreads();
            if (t == 0) {
                double nx2 = 0.0;
                for (int w = 0; w < PQ_WARPS; ++w) nx2 += redv[w];
                const double nx = sqrt(nx2);
                const double x0 = v[0];
                double alpha = 0.0, beta = 0.0;
                if (nx > 0.0) {
                    alpha = x0 >= 0.0 ? -nx : nx;
                    beta = 1.0 / (nx * (nx + fabs(x0)));
                }
                v[0] = x0 - alpha;
                beta_s = beta;
                if (owner == b) {
                    const int q = piv - c0;
                    cols[(size_t)q * l + j] = alpha;
                    posq[q] = j;
                    p.perm[j] = piv;
                }
            }
            __syncthreads();
        }
        // 4. apply I - beta v v^* to the active columns, downdate their norms
        const double beta = beta_s;
        for (int q = warp; q < nc; q += PQ_WARPS) {
            if (posq[q] >= 0) continue;
            double* c = cols + (size_t)q * l + j;
            const int len = l - j;
            double w = 0.0;
            for (int i = lane; i < len; i += 32) w = fma(v[i], c[i], w);
            w = warp_sum(w) * beta;
            for (int i = lane; i < len; i += 32) c[i] = fma(-w, v[i], c[i]);
            __syncwarp();
            const double r = c[0];
            const double n1 = vn1[q];
            if (n1 != 0.0) {
                double tmp = fabs(r) / n1;
                tmp = fmax(0.0, (1.0 + tmp) * (1.0 - tmp));
                const double ratio = n1 / vn2[q];
                if (tmp * ratio * ratio <= 1.4901161193847656e-08) {
                    double s2 = 0.0;
                    for (int i = 1 + lane; i < len; i += 32) s2 = fma(c[i], c[i], s2);
                    s2 = warp_sum(s2);
                    if (lane == 0) { vn1[q] = sqrt(s2); vn2[q] = sqrt(s2); }
                } else if (lane == 0) {
                    vn1[q] = n1 * sqrt(tmp);
                }
            }
            __syncwarp();
            // write the updated tail back for the next pivot search
            double* gcol = p.S + (int64_t)(c0 + q) * p.lds;
            for (int i = lane; i < len; i += 32) gcol[j + i] = c[i];
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

size_t pivoted_qr_work_doubles(int m, int l) { return (size_t)3 * m + 3 * (size_t)l + 2048; }

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
        if (cpc <= PQ_MAXC && smem + 4096 <= (size_t)smem_optin) {
            const int G = (m + cpc - 1) / cpc;
            cudaFuncSetAttribute(qr_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_persistent_kernel, PQ_THREADS, smem);
            if (per_sm >= 1 && G <= per_sm * sms) {
                PqrDev p;
                p.S = S; p.m = m; p.l = l; p.lds = lds; p.R = R; p.perm = perm; p.cpc = cpc;
                double* w = work;
                p.vbuf = w;                     w += 2 * (size_t)l;
                p.scal = w;                     w += 4;
                p.bval = w;                     w += 2 * (size_t)G;
                p.bidx = (int*)w;               w += G;          // 2G ints
                unsigned int* ctr = (unsigned int*)w;            // counter, abort, flags[m]
                p.counter = ctr;
                p.abort_flag = (int*)(ctr + 1);
                p.flags = ctr + 2;
                p.status = status;
                p.timeout = 4000000000ll;
                cudaError_t e = cudaMemsetAsync(ctr, 0, (size_t)(m + 2) * sizeof(unsigned int), s);
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
