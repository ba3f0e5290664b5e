// Exact fixed-point slicing of float64 operands into bfloat16 digit planes (mixed mode).
//
// For a row x of an operand (the products reduce along the row), with e the smallest
// integer such that max |x_c| < 2^e, every entry is written as
//     x_c ~= 2^e * sum_{p < s} d_p * 2^{-7-8p},     d_p integers in [-128, 128] (s <= 10),
// the balanced base-256 digits of F = round(|x_c| 2^{7+8(s-1)-e}), signed like x_c.
// Each d_p is exact in bfloat16, so the tensor cores multiply digits exactly and the
// float32 accumulator sums them exactly as long as a partial sum stays below 2^24.
// Truncation error per entry: at most 2^{e-8s} (half a unit of the last digit).
// The digits come from integer operations on the float64 bit pattern (no FP64 pipe).
#include "rtproj_internal.cuh"

#include <type_traits>

namespace rtp {
namespace {

constexpr int SL_THREADS = 256;

__device__ __forceinline__ void fixed_digits(double v, int shift_base, int s, int* dig) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const bool neg = (bits >> 63) != 0;
    int E = (int)((bits >> 52) & 0x7FFull);
    unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
    if (E == 0) {
        if (M == 0) {
            for (int p = 0; p < s; ++p) dig[p] = 0;
            return;
        }
        E = 1;
    } else {
        M |= 1ull << 52;
    }
    // F = round(M * 2^sh) < 2^(7+8(s-1)) <= 2^79 by the choice of e: 128-bit integer.
    const int sh = E - 1075 + shift_base;
    unsigned __int128 F;
    if (sh >= 0) {
        F = sh < 76 ? ((unsigned __int128)M << sh) : (unsigned __int128)0;
    } else if (sh > -64) {
        const int rs = -sh;
        unsigned long long f = M >> rs;
        if ((M >> (rs - 1)) & 1ull) f += 1ull;
        F = f;
    } else {
        F = 0;
    }
    int carry = 0;
    for (int p = s - 1; p >= 1; --p) {
        int b = (int)(unsigned)(F & 0xFFu) + carry;
        F >>= 8;
        if (b >= 128) { b -= 256; carry = 1; } else { carry = 0; }
        dig[p] = neg ? -b : b;
    }
    const int b0 = (int)(unsigned)F + carry;   // <= 128
    dig[0] = neg ? -b0 : b0;
}

struct SliceDev {
    const double* X; int64_t x_rs, x_cs; const int32_t* rowidx; const int32_t* cexp;
    int rows, cols, s;
    __nv_bfloat16* d; int64_t ld, ps;
    int32_t* e;
    int* status;
};

// One CTA per row: row maximum -> exponent, then the digits of every entry.
__global__ void __launch_bounds__(SL_THREADS) slice_rows_kernel(SliceDev a) {
    __shared__ double smax[SL_THREADS / 32];
    __shared__ int sbad[SL_THREADS / 32];
    __shared__ int e_s;
    const int r = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t roff = (a.rowidx ? (int64_t)a.rowidx[r] : (int64_t)r) * a.x_rs;
    double mx = 0.0;
    int bad = 0;
    for (int c = t; c < a.cols; c += SL_THREADS) {
        double v = a.X[roff + (int64_t)c * a.x_cs];
        if (!isfinite(v)) bad = 1;
        if (a.cexp) v = ldexp(v, a.cexp[c]);
        mx = fmax(mx, fabs(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((t & 31) == 0) { smax[t >> 5] = mx; sbad[t >> 5] = bad; }
    __syncthreads();
    if (t == 0) {
        double m2 = 0.0;
        int b2 = 0;
        for (int w = 0; w < SL_THREADS / 32; ++w) { m2 = fmax(m2, smax[w]); b2 |= sbad[w]; }
        int ex = 0;
        if (m2 > 0.0 && isfinite(m2)) frexp(m2, &ex);
        e_s = ex;
        a.e[r] = ex;
        if (b2) set_status(a.status, RTPROJ_ENONFINITE);
    }
    __syncthreads();
    const int e = e_s;
    const int base = 7 + 8 * (a.s - 1) - e;
    __nv_bfloat16* drow = a.d + (int64_t)r * a.ld;
    for (int c = t; c < a.ld; c += SL_THREADS) {
        int dig[10];
        if (c < a.cols) {
            double v = a.X[roff + (int64_t)c * a.x_cs];
            if (!isfinite(v)) v = 0.0;
            fixed_digits(v, base + (a.cexp ? a.cexp[c] : 0), a.s, dig);
        } else {
            for (int p = 0; p < 10; ++p) dig[p] = 0;
        }
        for (int p = 0; p < a.s; ++p) drow[(int64_t)p * a.ps + c] = __int2bfloat16_rn(dig[p]);
    }
}

// Transposes each digit plane: src [p][r][c] (ld_src) -> dst [p][c][r] (ld_dst), zero padded.
// Digit planes transposed through a 64 x 64 shared-memory tile: every warp reads and
// writes 32 pairs of adjacent bfloat16 (128 bytes per row), so both sides move whole
// sectors. dst row c (< dst_rows) holds column c of src; dst columns r >= rows are zero.
// Requires even ld_src and ld_dst (both are multiples of 8 elements).
__global__ void __launch_bounds__(256) transpose_planes_kernel(const __nv_bfloat16* src, int64_t ld_src,
                                                               int64_t ps_src, int rows, int cols,
                                                               __nv_bfloat16* dst, int64_t ld_dst, int64_t ps_dst,
                                                               int dst_rows) {
    __shared__ __nv_bfloat16 tile[64][66];
    const int p = blockIdx.z;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const __nv_bfloat16 zero = __int2bfloat16_rn(0);
    const __nv_bfloat16* sp = src + (int64_t)p * ps_src;
    for (int y = ty; y < 64; y += 8) {
        const int r = r0 + y, c = c0 + 2 * tx;
        __nv_bfloat162 v;
        v.x = zero;
        v.y = zero;
        if (r < rows) {
            if (c + 1 < cols) {
                v = *reinterpret_cast<const __nv_bfloat162*>(sp + (int64_t)r * ld_src + c);
            } else if (c < cols) {
                v.x = sp[(int64_t)r * ld_src + c];
            }
        }
        tile[y][2 * tx] = v.x;
        tile[y][2 * tx + 1] = v.y;
    }
    __syncthreads();
    __nv_bfloat16* dp = dst + (int64_t)p * ps_dst;
    for (int y = ty; y < 64; y += 8) {
        const int c = c0 + y, r = r0 + 2 * tx;   // dst row c, dst cols r, r + 1
        if (c >= dst_rows || r >= ld_dst) continue;
        __nv_bfloat162 v;
        v.x = tile[2 * tx][y];
        v.y = tile[2 * tx + 1][y];
        *reinterpret_cast<__nv_bfloat162*>(dp + (int64_t)c * ld_dst + r) = v;
    }
}

// G^* (l x n) as one digit plane: row j, column i holds the digit of G(i, j).
// uniform: d = 2u - 255 (exponent -1, value d / 256); rademacher: d = +-1 (exponent 7).
__global__ void omega_plane_kernel(uint32_t key0, uint32_t key1, int dist, int n, int l, __nv_bfloat16* d,
                                   int64_t ld, int64_t ps) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t blocks_per_row = ld / 16;
    if (gid >= blocks_per_row * l) return;
    const int j = (int)(gid / blocks_per_row);
    const int i0 = (int)(gid % blocks_per_row) * 16;
    alignas(16) __nv_bfloat16 out[16];
    if (dist == RTPROJ_OMEGA_GAUSSIAN) {
        // N = 4096 G = 256 d0 + d1 with d1 in [-128, 127]: two exact digit planes
        // (exponent 3: G = 2^3 (d0 2^-7 + d1 2^-15))
        alignas(16) __nv_bfloat16 lo[16];
#pragma unroll
        for (int qd = 0; qd < 4; ++qd) {
            int N[4];
            gauss_quad((uint32_t)((i0 >> 2) + qd), (uint32_t)j, key0, key1, N);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int v = (i0 + 4 * qd + b < n) ? N[b] : 0;
                const int d0 = (v + 128) >> 8;          // floor((v + 128) / 256)
                out[4 * qd + b] = __int2bfloat16_rn(d0);
                lo[4 * qd + b] = __int2bfloat16_rn(v - 256 * d0);
            }
        }
        uint4* dst1 = reinterpret_cast<uint4*>(d + ps + (int64_t)j * ld + i0);
        dst1[0] = reinterpret_cast<const uint4*>(lo)[0];
        dst1[1] = reinterpret_cast<const uint4*>(lo)[1];
    } else {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(i0 >> 4), (uint32_t)j, 0u, 0u), key0, key1);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const uint32_t u = block_byte(w, b);
            int dv = dist == RTPROJ_OMEGA_RADEMACHER ? (u >= 128u ? 1 : -1) : (2 * (int)u - 255);
            if (i0 + b >= n) dv = 0;
            out[b] = __int2bfloat16_rn(dv);
        }
    }
    uint4* dst = reinterpret_cast<uint4*>(d + (int64_t)j * ld + i0);
    dst[0] = reinterpret_cast<const uint4*>(out)[0];
    dst[1] = reinterpret_cast<const uint4*>(out)[1];
}

// G itself (n x l, float64, row-major): one thread per 16 rows of one column.
__global__ void omega_dense_kernel(uint32_t key0, uint32_t key1, int dist, int n, int l, double* G, int64_t ldg) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t blocks_per_col = (n + 15) / 16;
    if (gid >= blocks_per_col * l) return;
    const int j = (int)(gid % l);
    const int i0 = (int)(gid / l) * 16;
    double v[16];
    if (dist == RTPROJ_OMEGA_GAUSSIAN) {
#pragma unroll
        for (int qd = 0; qd < 4; ++qd) {
            int N[4];
            gauss_quad((uint32_t)((i0 >> 2) + qd), (uint32_t)j, key0, key1, N);
#pragma unroll
            for (int b = 0; b < 4; ++b) v[4 * qd + b] = (double)N[b] * (1.0 / 4096.0);
        }
    } else {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(i0 >> 4), (uint32_t)j, 0u, 0u), key0, key1);
#pragma unroll
        for (int b = 0; b < 16; ++b) v[b] = (double)omega_from_byte(block_byte(w, b), dist);
    }
#pragma unroll
    for (int b = 0; b < 16; ++b)
        if (i0 + b < n) G[(int64_t)(i0 + b) * ldg + j] = v[b];
}

__global__ void fill_int_kernel(int32_t* e, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] = v;
}

// ---------------------------------------------------------------------------------
// Contiguous rows (x_cs = 1, no row index, no column exponents): the same digits, from
// integer operations only. One CTA of SLF_THREADS per row: the row maximum of |x| is the
// maximum of the bit patterns with the sign cleared (their order is that of the values),
// non-finite entries are those with an all-ones exponent field; then every thread turns
// eight consecutive entries into eight digits per plane and stores them as one 16-byte
// vector per plane. S is a template parameter so the digits stay in registers; F fits
// 64 bits for S <= 8.
constexpr int SLF_THREADS = 512;

__device__ __forceinline__ unsigned long long u64_max(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Bits of the bfloat16 holding the integer d, |d| <= 256: d is exact in float32 (one add
// of 1.5 * 2^23 and one subtract), and the float's upper half is the bfloat16.
__device__ __forceinline__ uint32_t bf16_bits_of_int(int d) {
    const float f = __fsub_rn(__int_as_float(0x4B400000 + d), 12582912.0f);
    return __float_as_uint(f) >> 16;
}

// Digits of one entry (bit pattern `bits`) for the shift base of its row.
template <int S>
__device__ __forceinline__ void entry_digits(unsigned long long bits, int shift_base, int (&dig)[S]) {
    using U = typename std::conditional<(S <= 8), unsigned long long, unsigned __int128>::type;
    constexpr int kMaxShift = S <= 8 ? 63 : 127;
    const bool neg = (bits >> 63) != 0;
    int E = (int)((bits >> 52) & 0x7FFull);
    unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
    if (E == 0) E = 1; else M |= 1ull << 52;
    if (E == 0x7FF) M = 0;                        // non-finite: flagged by the caller, digits 0
    const int sh = E - 1075 + shift_base;
    U F = 0;
    if (M != 0) {
        if (sh >= 0) {
            F = sh < kMaxShift - 52 ? ((U)M << sh) : (U)0;
        } else if (sh > -64) {
            const int rs = -sh;
            unsigned long long f = M >> rs;
            if ((M >> (rs - 1)) & 1ull) f += 1ull;
            F = (U)f;
        }
    }
    int carry = 0;
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
        int b = (int)(unsigned)(F & 0xFFu) + carry;
        F >>= 8;
        carry = b >= 128 ? 1 : 0;
        b -= carry * 256;
        dig[p] = neg ? -b : b;
    }
    const int b0 = (int)(unsigned)F + carry;
    dig[0] = neg ? -b0 : b0;
}

// frexp exponent e of a maximum given as sign-cleared bits (max < 2^e <= 2 max): E - 1022
// for a normal value, from the leading mantissa bit for a subnormal one; `zero` when 0.
__device__ __forceinline__ int max_exponent(unsigned long long m2, int zero) {
    const int E = (int)(m2 >> 52);
    if (E > 0) return E - 1022;
    if (m2 != 0) return (64 - __clzll((long long)m2)) - 1074;
    return zero;
}

// Largest sign-cleared bit pattern and non-finite flag over columns [c0, c1) of a row,
// reduced over the CTA; thread 0 receives the result.
__device__ __forceinline__ void row_span_max(const unsigned long long* row, int c0, int c1, unsigned long long* smax,
                                             int* sbad, unsigned long long* m_out, int* bad_out) {
    const int t = threadIdx.x;
    unsigned long long mx = 0;
    int bad = 0;
    for (int c = c0 + t; c < c1; c += SLF_THREADS) {
        const unsigned long long u = __ldg(row + c) & 0x7FFFFFFFFFFFFFFFull;
        if (u >= 0x7FF0000000000000ull) bad = 1;
        else mx = u64_max(mx, u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = u64_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((t & 31) == 0) { smax[t >> 5] = mx; sbad[t >> 5] = bad; }
    __syncthreads();
    if (t == 0) {
        unsigned long long m2 = 0;
        int b2 = 0;
        for (int w = 0; w < SLF_THREADS / 32; ++w) { m2 = u64_max(m2, smax[w]); b2 |= sbad[w]; }
        *m_out = m2;
        *bad_out = b2;
    }
}

// Digits of columns [c_begin, c_end) of a row (c_begin a multiple of 8), eight per thread,
// one 16-byte store per plane.
template <int S>
__device__ __forceinline__ void row_span_digits(const SliceDev& a, const unsigned long long* row, int r, int base,
                                                int c_begin, int c_end) {
    __nv_bfloat16* drow = a.d + (int64_t)r * a.ld;
    for (int c0 = c_begin + 8 * threadIdx.x; c0 < c_end; c0 += 8 * SLF_THREADS) {
        uint32_t w[S][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            int d0[S], d1[S];
            const int c = c0 + 2 * h;
            entry_digits<S>(c < a.cols ? __ldg(row + c) : 0ull, base, d0);
            entry_digits<S>(c + 1 < a.cols ? __ldg(row + c + 1) : 0ull, base, d1);
#pragma unroll
            for (int p = 0; p < S; ++p) w[p][h] = bf16_bits_of_int(d0[p]) | (bf16_bits_of_int(d1[p]) << 16);
        }
#pragma unroll
        for (int p = 0; p < S; ++p)
            *reinterpret_cast<uint4*>(drow + (int64_t)p * a.ps + c0) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
}

// One CTA per row (many rows).
template <int S>
__global__ void __launch_bounds__(SLF_THREADS) slice_rows_fast_kernel(SliceDev a) {
    __shared__ unsigned long long smax[SLF_THREADS / 32];
    __shared__ int sbad[SLF_THREADS / 32];
    __shared__ unsigned long long m_s;
    __shared__ int bad_s;
    const int r = blockIdx.x;
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(a.X + (int64_t)r * a.x_rs);
    row_span_max(row, 0, a.cols, smax, sbad, &m_s, &bad_s);
    __syncthreads();
    const int ex = max_exponent(m_s, 0);
    if (threadIdx.x == 0) {
        a.e[r] = ex;
        if (bad_s) set_status(a.status, RTPROJ_ENONFINITE);
    }
    row_span_digits<S>(a, row, r, 7 + 8 * (S - 1) - ex, 0, (int)a.ld);
}

// Few rows: each row split over SLF_SPAN-column spans, one CTA per (span, row), in two
// launches. The first takes each span's maximum exponent into e[r] (atomicMax over spans,
// e pre-filled with SLF_ZERO_ROW), the second writes the digits of its span.
constexpr int SLF_SPAN = 8 * SLF_THREADS;
constexpr int SLF_ZERO_ROW = kZeroRowExp;

__global__ void __launch_bounds__(SLF_THREADS) slice_rows_exp_kernel(SliceDev a) {
    __shared__ unsigned long long smax[SLF_THREADS / 32];
    __shared__ int sbad[SLF_THREADS / 32];
    __shared__ unsigned long long m_s;
    __shared__ int bad_s;
    const int r = blockIdx.y, c0 = blockIdx.x * SLF_SPAN;
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(a.X + (int64_t)r * a.x_rs);
    row_span_max(row, c0, min(a.cols, c0 + SLF_SPAN), smax, sbad, &m_s, &bad_s);
    if (threadIdx.x == 0) {
        const int ex = max_exponent(m_s, SLF_ZERO_ROW);
        if (ex != SLF_ZERO_ROW) atomicMax(a.e + r, ex);
        if (bad_s) set_status(a.status, RTPROJ_ENONFINITE);
    }
}

template <int S>
__global__ void __launch_bounds__(SLF_THREADS) slice_rows_span_kernel(SliceDev a) {
    const int r = blockIdx.y, c0 = blockIdx.x * SLF_SPAN;
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(a.X + (int64_t)r * a.x_rs);
    int ex = a.e[r];
    if (ex == SLF_ZERO_ROW) ex = 0;                        // an all-zero row: exponent 0
    __syncthreads();                                       // every thread has read e[r]
    if (blockIdx.x == 0 && threadIdx.x == 0) a.e[r] = ex;
    row_span_digits<S>(a, row, r, 7 + 8 * (S - 1) - ex, c0, (int)min(a.ld, (int64_t)(c0 + SLF_SPAN)));
}

// Both digit layouts of a long-row operand in one pass over it: with the row exponents
// already in e (slice_rows_exp_kernel), CTA (bx, by) takes rows [64 by, 64 by + 64) and
// columns [64 bx, 64 bx + 64) of X, writes their digits to the row-major planes (a.d,
// rows < a.rows) and, through a shared-memory tile per plane, to the transposed planes
// t_d (row c holds column c of X, leading dimension t_ld, rows < t_rows). Tile rows at or
// past a.rows and columns at or past a.cols give zero digits (the padding of both
// layouts). Each thread turns two groups of eight consecutive entries of a row (one group
// per pass, the two in different rows) into digits: one 16-byte store per plane to the
// row-major planes; the transposed planes are written from shared memory as 16-byte
// stores of eight consecutive rows of X.
constexpr int SLD_TILE = 64;
constexpr int SLD_THREADS = 256;
constexpr int SLD_PAD = SLD_TILE + 2;   // bfloat16 per shared row: odd word stride, no bank conflicts on reads

template <int S>
__global__ void __launch_bounds__(SLD_THREADS) slice_dual_kernel(SliceDev a, __nv_bfloat16* t_d, int64_t t_ld,
                                                                 int64_t t_ps, int t_rows) {
    extern __shared__ __align__(16) unsigned char sld_raw[];
    auto tile = reinterpret_cast<__nv_bfloat16(*)[SLD_TILE][SLD_PAD]>(sld_raw);   // [S][column][row]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r0 = blockIdx.y * SLD_TILE, c0 = blockIdx.x * SLD_TILE;
    const int g = lane & 7;                                  // group of eight columns
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
        const int rr = (warp * 2 + it) * 4 + (lane >> 3);    // tile row, 0 .. 63
        const int r = r0 + rr, cb = c0 + 8 * g;
        const bool live = r < a.rows;
        int ex = live ? a.e[r] : 0;
        if (ex == SLF_ZERO_ROW) ex = 0;                      // an all-zero row: exponent 0
        const int base = 7 + 8 * (S - 1) - ex;
        const unsigned long long* row = reinterpret_cast<const unsigned long long*>(a.X + (int64_t)r * a.x_rs);
        unsigned long long bits[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) bits[k] = (live && cb + k < a.cols) ? __ldg(row + cb + k) : 0ull;
        uint32_t w[S][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            int d0[S], d1[S];
            entry_digits<S>(bits[2 * h], base, d0);
            entry_digits<S>(bits[2 * h + 1], base, d1);
#pragma unroll
            for (int p = 0; p < S; ++p) {
                const uint32_t b0 = bf16_bits_of_int(d0[p]), b1 = bf16_bits_of_int(d1[p]);
                w[p][h] = b0 | (b1 << 16);
                tile[p][8 * g + 2 * h][rr] = __ushort_as_bfloat16((unsigned short)b0);
                tile[p][8 * g + 2 * h + 1][rr] = __ushort_as_bfloat16((unsigned short)b1);
            }
        }
        if (live) {
            __nv_bfloat16* drow = a.d + (int64_t)r * a.ld + cb;
#pragma unroll
            for (int p = 0; p < S; ++p)
                *reinterpret_cast<uint4*>(drow + (int64_t)p * a.ps) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        }
    }
    __syncthreads();   // the tile is complete, and every thread has read its rows' exponents
    if (blockIdx.x == 0 && t < SLD_TILE && r0 + t < a.rows && a.e[r0 + t] == SLF_ZERO_ROW) a.e[r0 + t] = 0;
    // transposed planes: row c0 + cc, columns r0 + 8 q .. r0 + 8 q + 7 (eight lanes per row)
    for (int v = t; v < S * SLD_TILE * (SLD_TILE / 8); v += SLD_THREADS) {
        const int q = v & 7, cc = (v >> 3) & (SLD_TILE - 1), p = v / (SLD_TILE * (SLD_TILE / 8));
        const int c = c0 + cc;
        if (c >= t_rows) continue;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&tile[p][cc][8 * q]);
        *reinterpret_cast<uint4*>(t_d + (int64_t)p * t_ps + (int64_t)c * t_ld + r0 + 8 * q) =
            make_uint4(src[0], src[1], src[2], src[3]);
    }
}

}  // namespace

cudaError_t slice_rows(const double* X, int64_t x_rs, int64_t x_cs, const int32_t* rowidx, const int32_t* cexp,
                       const SliceStack& st, int* status, cudaStream_t s) {
    if (st.rows <= 0) return cudaSuccess;
    if (st.s < 1 || st.s > 10 || st.ld < st.cols || st.ld % 64) return cudaErrorInvalidValue;
    SliceDev a;
    a.X = X; a.x_rs = x_rs; a.x_cs = x_cs; a.rowidx = rowidx; a.cexp = cexp;
    a.rows = st.rows; a.cols = st.cols; a.s = st.s;
    a.d = st.d; a.ld = st.ld; a.ps = st.plane_stride; a.e = st.e; a.status = status;
    // 16-byte vector stores need 8-entry aligned planes and rows
    const bool fast = x_cs == 1 && !rowidx && !cexp && st.ld % 8 == 0 && st.plane_stride % 8 == 0 &&
                      ((uintptr_t)st.d & 15) == 0 && ((uintptr_t)X & 7) == 0;
    if (fast && st.rows < 2 * sm_count()) {
        // few rows: spread every row over several CTAs
        const cudaError_t fe = fill_int(st.e, st.rows, SLF_ZERO_ROW, s);
        if (fe != cudaSuccess) return fe;
        const dim3 grid((unsigned)((st.ld + SLF_SPAN - 1) / SLF_SPAN), (unsigned)st.rows);
        slice_rows_exp_kernel<<<grid, SLF_THREADS, 0, s>>>(a);
        note_launch();
        switch (st.s) {
            case 1: slice_rows_span_kernel<1><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 2: slice_rows_span_kernel<2><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 3: slice_rows_span_kernel<3><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 4: slice_rows_span_kernel<4><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 5: slice_rows_span_kernel<5><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 6: slice_rows_span_kernel<6><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 7: slice_rows_span_kernel<7><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 8: slice_rows_span_kernel<8><<<grid, SLF_THREADS, 0, s>>>(a); break;
            case 9: slice_rows_span_kernel<9><<<grid, SLF_THREADS, 0, s>>>(a); break;
            default: slice_rows_span_kernel<10><<<grid, SLF_THREADS, 0, s>>>(a); break;
        }
    } else if (fast) {
        switch (st.s) {
            case 1: slice_rows_fast_kernel<1><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 2: slice_rows_fast_kernel<2><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 3: slice_rows_fast_kernel<3><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 4: slice_rows_fast_kernel<4><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 5: slice_rows_fast_kernel<5><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 6: slice_rows_fast_kernel<6><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 7: slice_rows_fast_kernel<7><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 8: slice_rows_fast_kernel<8><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            case 9: slice_rows_fast_kernel<9><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
            default: slice_rows_fast_kernel<10><<<st.rows, SLF_THREADS, 0, s>>>(a); break;
        }
    } else {
        slice_rows_kernel<<<st.rows, SL_THREADS, 0, s>>>(a);
    }
    note_launch();
    return cudaGetLastError();
}

namespace {
bool fast_rows_ok(const double* X, const SliceStack& st) {
    return st.s >= 1 && st.s <= 10 && st.ld >= st.cols && st.ld % 64 == 0 && st.plane_stride % 8 == 0 &&
           ((uintptr_t)st.d & 15) == 0 && ((uintptr_t)X & 7) == 0;
}
SliceDev rows_dev(const double* X, int64_t x_rs, const SliceStack& st, int* status) {
    SliceDev a;
    a.X = X; a.x_rs = x_rs; a.x_cs = 1; a.rowidx = nullptr; a.cexp = nullptr;
    a.rows = st.rows; a.cols = st.cols; a.s = st.s;
    a.d = st.d; a.ld = st.ld; a.ps = st.plane_stride; a.e = st.e; a.status = status;
    return a;
}
}  // namespace

cudaError_t row_exponents(const double* X, int64_t x_rs, int rows, int cols, int32_t* e, int* status, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (((uintptr_t)X & 7) != 0) return cudaErrorInvalidValue;
    SliceDev a{};
    a.X = X; a.x_rs = x_rs; a.x_cs = 1; a.rows = rows; a.cols = cols; a.e = e; a.status = status;
    const dim3 grid((unsigned)((cols + SLF_SPAN - 1) / SLF_SPAN), (unsigned)rows);
    slice_rows_exp_kernel<<<grid, SLF_THREADS, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t slice_rows_given_exp(const double* X, int64_t x_rs, const SliceStack& st, int* status, cudaStream_t s) {
    if (st.rows <= 0) return cudaSuccess;
    if (!fast_rows_ok(X, st)) return slice_rows(X, x_rs, 1, nullptr, nullptr, st, status, s);
    const SliceDev a = rows_dev(X, x_rs, st, status);
    const dim3 grid((unsigned)((st.ld + SLF_SPAN - 1) / SLF_SPAN), (unsigned)st.rows);
    switch (st.s) {
        case 1: slice_rows_span_kernel<1><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 2: slice_rows_span_kernel<2><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 3: slice_rows_span_kernel<3><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 4: slice_rows_span_kernel<4><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 5: slice_rows_span_kernel<5><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 6: slice_rows_span_kernel<6><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 7: slice_rows_span_kernel<7><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 8: slice_rows_span_kernel<8><<<grid, SLF_THREADS, 0, s>>>(a); break;
        case 9: slice_rows_span_kernel<9><<<grid, SLF_THREADS, 0, s>>>(a); break;
        default: slice_rows_span_kernel<10><<<grid, SLF_THREADS, 0, s>>>(a); break;
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t slice_rows_dual(const double* X, int64_t x_rs, const SliceStack& st, const SliceStack& tst, int* status,
                            cudaStream_t s) {
    if (st.rows <= 0) return cudaSuccess;
    const bool ok = st.s >= 1 && st.s <= 10 && tst.s == st.s && st.ld % SLD_TILE == 0 && tst.ld % SLD_TILE == 0 &&
                    st.ld >= st.cols && tst.ld >= st.rows && tst.rows == st.cols && tst.cols == st.rows &&
                    st.plane_stride % 8 == 0 && tst.plane_stride % 8 == 0 && ((uintptr_t)st.d & 15) == 0 &&
                    ((uintptr_t)tst.d & 15) == 0 && ((uintptr_t)X & 7) == 0;
    if (!ok) {
        const cudaError_t e = slice_rows(X, x_rs, 1, nullptr, nullptr, st, status, s);
        return e != cudaSuccess ? e : transpose_planes(st, tst, s);
    }
    SliceDev a;
    a.X = X; a.x_rs = x_rs; a.x_cs = 1; a.rowidx = nullptr; a.cexp = nullptr;
    a.rows = st.rows; a.cols = st.cols; a.s = st.s;
    a.d = st.d; a.ld = st.ld; a.ps = st.plane_stride; a.e = st.e; a.status = status;
    cudaError_t e = fill_int(st.e, st.rows, SLF_ZERO_ROW, s);
    if (e != cudaSuccess) return e;
    const dim3 egrid((unsigned)((st.cols + SLF_SPAN - 1) / SLF_SPAN), (unsigned)st.rows);
    slice_rows_exp_kernel<<<egrid, SLF_THREADS, 0, s>>>(a);
    note_launch();
    const dim3 grid((unsigned)(st.ld / SLD_TILE), (unsigned)(tst.ld / SLD_TILE));
    const size_t smem = (size_t)st.s * SLD_TILE * SLD_PAD * sizeof(__nv_bfloat16);
    auto launch = [&](auto kern) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, SLD_THREADS, smem, s>>>(a, tst.d, tst.ld, tst.plane_stride, tst.rows);
    };
    switch (st.s) {
        case 1: launch(slice_dual_kernel<1>); break;
        case 2: launch(slice_dual_kernel<2>); break;
        case 3: launch(slice_dual_kernel<3>); break;
        case 4: launch(slice_dual_kernel<4>); break;
        case 5: launch(slice_dual_kernel<5>); break;
        case 6: launch(slice_dual_kernel<6>); break;
        case 7: launch(slice_dual_kernel<7>); break;
        case 8: launch(slice_dual_kernel<8>); break;
        case 9: launch(slice_dual_kernel<9>); break;
        default: launch(slice_dual_kernel<10>); break;
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t transpose_planes(const SliceStack& src, const SliceStack& dst, cudaStream_t s) {
    // dst row c (< dst.rows) holds column c of src; columns r >= src.rows are zero padding.
    if (src.ld % 2 || dst.ld % 2) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((dst.rows + 63) / 64), (unsigned)((dst.ld + 63) / 64), (unsigned)src.s);
    transpose_planes_kernel<<<grid, dim3(32, 8), 0, s>>>(src.d, src.ld, src.plane_stride, src.rows, src.cols, dst.d,
                                                          dst.ld, dst.plane_stride, dst.rows);
    note_launch();
    return cudaGetLastError();
}

cudaError_t omega_plane(uint64_t seed, int dist, int n, int l, const SliceStack& st, cudaStream_t s) {
    if (st.ld % 16 || st.ld < n || st.s < omega_planes(dist)) return cudaErrorInvalidValue;
    const int64_t total = (st.ld / 16) * (int64_t)l;
    omega_plane_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((uint32_t)(seed & 0xFFFFFFFFull),
                                                                       (uint32_t)(seed >> 32), dist, n, l, st.d, st.ld,
                                                                       st.plane_stride);
    note_launch();
    const int e = dist == RTPROJ_OMEGA_RADEMACHER ? 7 : dist == RTPROJ_OMEGA_GAUSSIAN ? 3 : -1;
    fill_int_kernel<<<(l + 255) / 256, 256, 0, s>>>(st.e, l, e);
    note_launch();
    return cudaGetLastError();
}

cudaError_t omega_dense(uint64_t seed, int dist, int n, int l, double* G, int64_t ldg, cudaStream_t s) {
    const int64_t total = (int64_t)((n + 15) / 16) * l;
    if (total <= 0) return cudaSuccess;
    omega_dense_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((uint32_t)(seed & 0xFFFFFFFFull),
                                                                       (uint32_t)(seed >> 32), dist, n, l, G, ldg);
    note_launch();
    return cudaGetLastError();
}

cudaError_t fill_int(int32_t* e, int n, int v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    fill_int_kernel<<<(n + 255) / 256, 256, 0, s>>>(e, n, v);
    note_launch();
    return cudaGetLastError();
}

}  // namespace rtp
