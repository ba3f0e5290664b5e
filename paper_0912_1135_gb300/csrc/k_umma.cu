// Sliced (Ozaki-scheme) GEMM on the 5th-generation tensor cores: tcgen05.mma with
// bfloat16 digit planes in shared memory and float32 accumulators in tensor memory.
//
//   C[i][j] = alpha * sum_k A(i,k) B(j,k) + beta * Cin[i][j],
//   A(i,k) = 2^{ea_i} sum_p dA_p(i,k) 2^{-7-8p},  B(j,k) = 2^{eb_j} sum_q dB_q(j,k) 2^{-7-8q}
// Only digit pairs with level g = p + q < terms (<= 10) are multiplied (the truncation
// of the Ozaki scheme). Each level has its own TMEM accumulator. Level g holds at most
// min(g+1, 10) digit pairs per k, every digit product is at most 2^15 in magnitude
// (<= 2^14 unless one operand is the one-digit G plane), and a TMEM readout happens
// every 128 k: for every level up to 7 each float32 partial sum stays below 2^24, so
// those level sums are exact; levels 8 and 9 (relative weight 2^-64 and below) may
// round by a unit of their own scale. The readout folds the level sums into two int64
// words per entry. Level g sits at position P = g + 1 of a ten-position fixed point (level
// 9, used only with terms = 10 and already inexact, is floored to the unit 2^8 of P = 10):
//   hi = sum_{P<=4} L_g 2^{8(4-P)},  lo = sum_{5<=P<=9} L_g 2^{8(9-P)} (+ floor(L_9 / 2^8))
// with lo kept below 2^40, so that sum_k A B = 2^{ea+eb-78} (hi 2^40 + lo) exactly up to the
// digit truncation. Every k adds at most 2^78 to |hi 2^40 + lo| < 2^103, so hi cannot
// overflow while a split's K stays below 2^25; choose_splits keeps every split within that
// bound where the scratch allows. (Position offset 1 rather than 0 buys the factor 2^8.)
// Split-K partials are summed in 128-bit integers by the reduce kernel and converted to
// float64 from all 128 bits.
//
// CTA: 128 threads; tile 128 (A rows, MMA M) x 32 (B rows, MMA N); K block 64 (one
// 128-byte swizzle row per operand row). Thread 0 issues the MMAs; all threads stage
// operands with cp.async into the SWIZZLE_128B K-major layout and read TMEM back.
#include "rtproj_internal.cuh"

#include <utility>

#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

namespace rtp {
namespace {

constexpr int TM = 128;
constexpr int TN = 32;
constexpr int KB = 64;
constexpr int NTHREADS = 128;
constexpr int MAXS = 10;
constexpr int A_PLANE_BYTES = TM * KB * 2;   // 16 KiB
constexpr int B_PLANE_BYTES = TN * KB * 2;   // 4 KiB

struct SgDev {
    const __nv_bfloat16* a; int64_t a_ld, a_ps; const int32_t* ea; int sa; int M;
    const __nv_bfloat16* b; int64_t b_ld, b_ps; const int32_t* eb; int sb; int N;
    int Kp;             // K rounded up to 64 (planes are zero padded to it)
    int terms;
    int k_per_split;    // multiple of kchunk
    int kchunk;         // K between TMEM readouts (128, 256 or 512: see chunk_for)
    long long* part;    // [split][M][N][2] when gridDim.z > 1
    double* C; int64_t c_rs, c_cs; const int32_t* crow;
    double alpha, beta;
    int amode, bmode;
    const double* Cin; int64_t cin_rs, cin_cs;
    int lower_only;
    int* status;
    long long timeout_cycles;
    uint32_t tmem_cols;  // power of two >= 32 * terms
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, bfloat16 inputs, float32 accumulation.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: register j of lane t = TMEM[lane base + t][col + j].
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Exact int32 value of an integer-valued float32 with |x| < 2^30, on the FMA/ALU pipes
// (64-bit float-to-integer conversion would run on GB300's small FP64 pipe). x is split
// into hi, a multiple of 256 (rounded by adding 1.5 * 2^31, whose ulp is 256), and the
// exact remainder lo, |lo| <= 128; both are read off the bits of a float offset by
// 1.5 * 2^23, which holds integers below 2^22 exactly in its mantissa.
__device__ __forceinline__ int exact_f2i(float x) {
    const float big = 3221225472.0f;               // 1.5 * 2^31
    const float hi = __fsub_rn(__fadd_rn(x, big), big);
    const float lo = __fsub_rn(x, hi);
    const int ih = __float_as_int(__fadd_rn(__fmul_rn(hi, 0.00390625f), 12582912.0f)) - 0x4B400000;
    const int il = __float_as_int(__fadd_rn(lo, 12582912.0f)) - 0x4B400000;
    return ih * 256 + il;
}

// Adds the level-g sums of one 128-row x 32-column readout (r) into the int64 words.
// When every value of the warp's readout is below 2^22 in magnitude (the usual case) one
// magic-offset add converts each; otherwise the two-part exact_f2i is used.
// The position offset of the fixed point (see the top); the same for every product.
__host__ __device__ constexpr int level_offset(int /*terms*/) { return 1; }
constexpr long long kSplitKCap = 1ll << 25;   // largest K of one split (see the top)

__device__ __forceinline__ void fold_level(int g, int D, const uint32_t (&r)[32], long long (&hi)[32],
                                           long long (&lo)[32]) {
    bool small = true;
#pragma unroll
    for (int j = 0; j < 32; ++j) small &= fabsf(__uint_as_float(r[j])) < 4194304.0f;
    const bool fast = __all_sync(0xffffffffu, small);
    const int P = g + D;
    const int sh = P <= 4 ? 8 * (4 - P) : P <= 9 ? 8 * (9 - P) : 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        int v = fast ? __float_as_int(__fadd_rn(__uint_as_float(r[j]), 12582912.0f)) - 0x4B400000
                     : exact_f2i(__uint_as_float(r[j]));
        if (P > 9) v >>= 8;                           // floor to the unit 2^8 of position 10
        if (P <= 4) hi[j] += (long long)v << sh; else lo[j] += (long long)v << sh;
    }
}

// (hi * 2^40 + lo) * 2^e rounded to nearest (ties to even), from integer operations: the
// two words form a 128-bit two's-complement integer, whose magnitude is normalised by its
// leading-zero count and cut to 53 bits with a round bit and a sticky bit. Integer
// instructions keep the conversion off GB300's FP64 pipe (64 cycles per warp instruction),
// and it is branch-free (selects and masks) because the lanes of a warp hold values of
// every sign and magnitude: the earlier form with a branch per shift range took about
// 1000 cycles per element in the epilogue. A result outside the normal range is delegated
// to ldexp.
__device__ __forceinline__ double u128_to_double(unsigned long long H, unsigned long long L, int e);

__device__ __forceinline__ double words_to_double(long long hi, long long lo, int e) {
    // V = hi * 2^40 + lo as a 128-bit two's complement value (H:L)
    const unsigned long long L = ((unsigned long long)hi << 40) + (unsigned long long)lo;
    const unsigned long long carry = L < ((unsigned long long)hi << 40) ? 1ull : 0ull;
    const unsigned long long H = (unsigned long long)(hi >> 24) + (unsigned long long)(lo >> 63) + carry;
    return u128_to_double(H, L, e);
}

// V * 2^e for the 128-bit two's-complement integer V = (H:L), rounded to nearest even.
__device__ __forceinline__ double u128_to_double(unsigned long long H, unsigned long long L, int e) {
    // |V| by a masked negation (no branch: the lanes of a warp hold values of either sign)
    const unsigned long long sg = (unsigned long long)((long long)H >> 63);
    L ^= sg;
    H ^= sg;
    const unsigned long long one = sg & 1ull;
    const unsigned long long L1 = L + one;
    H += one & (L1 == 0 ? 1ull : 0ull);
    L = L1;
    if ((H | L) == 0) return 0.0;
    // normalise: shift left by the leading zeros so that the leading one is bit 127
    const int s = H != 0 ? __clzll((long long)H) : 64 + __clzll((long long)L);
    const int s1 = s & 63;
    const unsigned long long hl = s1 ? (H << s1) | (L >> (64 - s1)) : H;
    const unsigned long long Hn = s < 64 ? hl : (L << s1);
    const unsigned long long Ln = s < 64 ? (L << s1) : 0ull;
    // 53 bits, round to nearest even on the round bit and the sticky bits below it
    unsigned long long m = Hn >> 11;
    const unsigned long long rb = (Hn >> 10) & 1ull;
    const unsigned long long st = ((Hn & 0x3FFull) | Ln) != 0 ? 1ull : 0ull;
    m += rb & (st | (m & 1ull));
    const unsigned long long ovf = m >> 53;       // rounding carried into bit 53
    m >>= ovf;
    const int ex = 127 - s + (int)ovf;             // position of the leading bit of |V|
    const int biased = ex + e + 1023;
    if (biased <= 0 || biased >= 2047) {
        const double mag = ldexp((double)m, ex - 52 + e);
        return sg ? -mag : mag;
    }
    const unsigned long long bits =
        ((unsigned long long)biased << 52) | (m & 0xFFFFFFFFFFFFFull) | (sg & 0x8000000000000000ull);
    return __longlong_as_double((long long)bits);
}

// alpha * v + beta * cin with the common cases decided on the host: amode 0 (alpha = 1),
// 1 (alpha = -1: a sign flip), 2 (general); bmode 0 (beta = 0), 1 (beta = 1), 2 (general).
// The cases cost no float64 comparisons on the device.
__device__ __forceinline__ double epilogue_value(double v, int amode, double alpha, int bmode, double beta,
                                                 const double* cin) {
    double out = amode == 0 ? v
               : amode == 1 ? __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull)
                            : alpha * v;
    if (bmode == 1) out += *cin;
    else if (bmode == 2) out = fma(beta, *cin, out);
    return out;
}
// The same with the Cin entry already loaded.
__device__ __forceinline__ double epilogue_value_v(double v, int amode, double alpha, int bmode, double beta,
                                                   double cin) {
    double out = amode == 0 ? v
               : amode == 1 ? __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull)
                            : alpha * v;
    if (bmode == 1) out += cin;
    else if (bmode == 2) out = fma(beta, cin, out);
    return out;
}
__host__ inline int alpha_mode(double a) { return a == 1.0 ? 0 : (a == -1.0 ? 1 : 2); }
__host__ inline int beta_mode(double b) { return b == 0.0 ? 0 : (b == 1.0 ? 1 : 2); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Position P of the fixed point goes to word hi (P <= 4) or lo (P >= 5), scaled by
// 2^level_shift(P); position 10 enters lo floored by 2^8 (shift 0 of v >> 8).
__host__ __device__ constexpr int level_shift(int P) { return P <= 4 ? 8 * (4 - P) : P <= 9 ? 8 * (9 - P) : 0; }

// acc += v * 2^SH modulo 2^64: one wide multiply-add (SH < 32) or one add to the upper word.
template <int SH>
__device__ __forceinline__ void add_shifted(unsigned long long& acc, int v) {
    if constexpr (SH == 32) {
        acc += (unsigned long long)(unsigned)v << 32;
    } else {
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(v), "r"(1 << SH));
    }
}

// Sum over levels [G0, G1) (positions g + D) that land in word `hi_word` of
// 0x4B400000 * 2^level_shift, modulo 2^64: the offset that the magic-number conversion
// adds to every value (0x4B400000 / 2^8 at position 10, exactly).
__host__ __device__ constexpr unsigned long long magic_bias(int G0, int G1, bool hi_word, int D) {
    unsigned long long b = 0;
    for (int g = G0; g < G1; ++g) {
        const int P = g + D;
        if ((P <= 4) != hi_word) continue;
        b += P > 9 ? (0x4B400000ull >> 8) : (0x4B400000ull << level_shift(P));
    }
    return b;
}

// Adds level L of one 16-column unit (columns CB*16 .. CB*16+15 of the warp's NCOL) into
// its word. Every value enters with the same offset 0x4B400000: the raw bits of
// x + 1.5 * 2^23 (FAST, exact when |x| < 2^22) or the exact integer plus that offset; the
// sum of the offsets is removed once per chunk.
template <int P, bool FAST, int CB, int NCOL>
__device__ __forceinline__ void fold_one(const uint32_t (&r)[16], unsigned long long (&hi)[NCOL],
                                         unsigned long long (&lo)[NCOL]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int v = FAST ? __float_as_int(__fadd_rn(__uint_as_float(r[j]), 12582912.0f))
                           : exact_f2i(__uint_as_float(r[j])) + 0x4B400000;
        if constexpr (P <= 4) add_shifted<level_shift(P)>(hi[CB * 16 + j], v);
        else if constexpr (P <= 9) add_shifted<level_shift(P)>(lo[CB * 16 + j], v);
        else add_shifted<0>(lo[CB * 16 + j], v >> 8);   // v > 0: the offset keeps it positive
    }
}
template <int P0, bool FAST, int CB, int NCOL, int... I>
__device__ __forceinline__ void fold_levels(const uint32_t (&r)[sizeof...(I)][16], unsigned long long (&hi)[NCOL],
                                            unsigned long long (&lo)[NCOL], std::integer_sequence<int, I...>) {
    (fold_one<P0 + I, FAST, CB, NCOL>(r[I], hi, lo), ...);
}

// Loads levels L0 .. L0+NG-1 of one 16-column unit (TMEM address `addr` + level * tn),
// checks them, and folds them in; with `release` the TMEM buffer is handed back to the
// MMA warp as soon as the values are in registers.
template <int L0, int NG, int CB, int NCOL, int D>
__device__ __forceinline__ void fold_group(uint32_t addr, uint32_t tn, unsigned long long (&hi)[NCOL],
                                           unsigned long long (&lo)[NCOL], bool release, uint64_t* empty_bar) {
    uint32_t r[NG][16];
#pragma unroll
    for (int g = 0; g < NG; ++g) tmem_ld16(addr + (uint32_t)(L0 + g) * tn, r[g]);
    tmem_ld_wait();
    if (release) {
        tc_fence_before();
        mbar_arrive(empty_bar);
    }
    float mx = 0.0f;
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int j = 0; j < 16; ++j) mx = fmaxf(mx, fabsf(__uint_as_float(r[g][j])));
    if (__all_sync(0xffffffffu, mx < 4194304.0f))
        fold_levels<L0 + D, true, CB, NCOL>(r, hi, lo, std::make_integer_sequence<int, NG>{});
    else
        fold_levels<L0 + D, false, CB, NCOL>(r, hi, lo, std::make_integer_sequence<int, NG>{});
}

// Level groups of one chunk readout: 16-column units in order, levels in groups of GS.
template <int TERMS, int NCOL, int CB, int L0>
__device__ __forceinline__ void readout_rec(uint32_t addr0, uint32_t tn, unsigned long long (&hi)[NCOL],
                                            unsigned long long (&lo)[NCOL], uint64_t* empty_bar) {
    constexpr int GS = NCOL == 16 ? 5 : 1;
    constexpr int NG = (TERMS - L0) < GS ? (TERMS - L0) : GS;
    constexpr bool last = (CB == NCOL / 16 - 1) && (L0 + NG >= TERMS);
    fold_group<L0, NG, CB, NCOL, level_offset(TERMS)>(addr0 + CB * 16, tn, hi, lo, last, empty_bar);
    if constexpr (L0 + NG < TERMS) readout_rec<TERMS, NCOL, CB, L0 + NG>(addr0, tn, hi, lo, empty_bar);
    else if constexpr (CB + 1 < NCOL / 16) readout_rec<TERMS, NCOL, CB + 1, 0>(addr0, tn, hi, lo, empty_bar);
}

// One chunk readout of TERMS levels for the warp's NCOL columns, then the offsets are
// removed and the carry of lo moved into hi (afterwards |lo| < 2^40).
template <int TERMS, int NCOL>
__device__ __forceinline__ void readout(uint32_t addr0, uint32_t tn, unsigned long long (&hi)[NCOL],
                                        unsigned long long (&lo)[NCOL], uint64_t* empty_bar) {
    readout_rec<TERMS, NCOL, 0, 0>(addr0, tn, hi, lo, empty_bar);
    constexpr int D = level_offset(TERMS);
    constexpr unsigned long long bh = magic_bias(0, TERMS, true, D), bl = magic_bias(0, TERMS, false, D);
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
        hi[j] -= bh;
        lo[j] -= bl;
        const long long carry = (long long)lo[j] >> 40;
        hi[j] += (unsigned long long)carry;
        lo[j] -= (unsigned long long)carry << 40;
    }
}

template <int NCOL>
__device__ __forceinline__ void readout_terms(int terms, uint32_t addr0, uint32_t tn, unsigned long long (&hi)[NCOL],
                                              unsigned long long (&lo)[NCOL], uint64_t* empty_bar) {
    switch (terms) {
        case 1: readout<1, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 2: readout<2, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 3: readout<3, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 4: readout<4, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 5: readout<5, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 6: readout<6, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 7: readout<7, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 8: readout<8, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        case 9: readout<9, NCOL>(addr0, tn, hi, lo, empty_bar); break;
        default: readout<10, NCOL>(addr0, tn, hi, lo, empty_bar); break;
    }
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B (8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Descriptor from its two 32-bit words.
__device__ __forceinline__ uint64_t make_desc(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; }

// Instruction descriptor, kind::f16: F32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(NTHREADS, 1) sliced_gemm_kernel(SgDev p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + (size_t)p.sa * A_PLANE_BYTES;
    uint64_t* bar = (uint64_t*)(sB + (size_t)p.sb * B_PLANE_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN, z = blockIdx.z;
    if (p.lower_only && j0 > i0 + TM - 1) return;     // tile strictly above the diagonal
    const int kbeg = z * p.k_per_split;
    const int kend = min(p.Kp, kbeg + p.k_per_split);

    if (t == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, p.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    long long hi[TN], lo[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) { hi[j] = 0; lo[j] = 0; }

    const uint32_t idesc = idesc_bf16(TM, TN);
    const uint32_t sA_addr = smem_addr(sA), sB_addr = smem_addr(sB);
    uint32_t phase = 0;
    bool timed_out = false;
    int kin_chunk = 0;          // K elements accumulated in TMEM since the last readout
    uint32_t started = 0;       // levels written since the last readout (bit g)

    for (int k0 = kbeg; k0 < kend && !timed_out; k0 += KB) {
        // ---- stage digit planes (cp.async, 16-byte chunks into the swizzled layout)
        for (int pl = 0; pl < p.sa; ++pl) {
            const __nv_bfloat16* src = p.a + (int64_t)pl * p.a_ps + k0;
            const uint32_t dst0 = sA_addr + pl * A_PLANE_BYTES;
            for (int idx = t; idx < TM * 8; idx += NTHREADS) {
                const int r = idx >> 3, c = idx & 7;
                const int gi = i0 + r;
                const bool ok = gi < p.M;
                const __nv_bfloat16* g = src + (int64_t)(ok ? gi : 0) * p.a_ld + c * 8;
                cp_async16(dst0 + r * 128 + ((c ^ (r & 7)) << 4), g, ok);
            }
        }
        for (int pl = 0; pl < p.sb; ++pl) {
            const __nv_bfloat16* src = p.b + (int64_t)pl * p.b_ps + k0;
            const uint32_t dst0 = sB_addr + pl * B_PLANE_BYTES;
            for (int idx = t; idx < TN * 8; idx += NTHREADS) {
                const int r = idx >> 3, c = idx & 7;
                const int gj = j0 + r;
                const bool ok = gj < p.N;
                const __nv_bfloat16* g = src + (int64_t)(ok ? gj : 0) * p.b_ld + c * 8;
                cp_async16(dst0 + r * 128 + ((c ^ (r & 7)) << 4), g, ok);
            }
        }
        cp_async_wait_all();
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- MMAs: every digit pair (pa, pb) with pa + pb < terms, 4 K-steps of 16
        if (t == 0) {
#pragma unroll 1
            for (int kk = 0; kk < KB / 16; ++kk) {
                for (int pa = 0; pa < p.sa; ++pa) {
                    const uint64_t ad = sw128_desc(sA_addr + pa * A_PLANE_BYTES + kk * 32);
                    for (int pb = 0; pb < p.sb && pa + pb < p.terms; ++pb) {
                        const int g = pa + pb;
                        const uint64_t bd = sw128_desc(sB_addr + pb * B_PLANE_BYTES + kk * 32);
                        umma_bf16(tmem + (uint32_t)(g * TN), ad, bd, idesc, (started >> g) & 1u);
                        started |= 1u << g;
                    }
                }
            }
            umma_commit(bar);
        }
        // ---- thread 0 waits (bounded) for the MMAs, which read the staged planes; the
        //      barrier then publishes completion (and any timeout) to the whole CTA.
        int to = 0;
        if (t == 0) {
            const long long t_start = clock64();
            while (!mbar_try_wait(bar, phase)) {
                if (clock64() - t_start > p.timeout_cycles) {
                    to = 1;
                    set_status(p.status, RTPROJ_ETIMEOUT);
                    break;
                }
            }
        }
        phase ^= 1u;
        timed_out = __syncthreads_or(to) != 0;
        tc_fence_after();
        if (timed_out) break;
        kin_chunk += KB;
        // ---- fold the exact level sums into hi/lo every 128 K (and at the end)
        if (kin_chunk >= p.kchunk || k0 + KB >= kend) {
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            for (int g = 0; g < p.terms; ++g) {
                uint32_t r[32];
                tmem_ld32(lane_base + (uint32_t)(g * TN), r);
                tmem_ld_wait();
                fold_level(g, level_offset(p.terms), r, hi, lo);
            }
#pragma unroll
            for (int j = 0; j < TN; ++j) {          // keep |lo| < 2^40
                const long long carry = lo[j] >> 40;
                hi[j] += carry;
                lo[j] -= carry * (1ll << 40);
            }
            kin_chunk = 0;
            started = 0;
            tc_fence_before();
        }
        __syncthreads();   // staged planes and TMEM are free for the next block
        tc_fence_after();
    }

    // ---- output
    const int i = i0 + warp * 32 + lane;
    if (i < p.M && !timed_out) {
        if (gridDim.z > 1) {
            // split-K partials, column-major per split: entry (i, j) of split z at
            // ((z N + j) M + i) * 2, so that a warp's 32 rows store contiguously
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (j0 + j < p.N)
                    *reinterpret_cast<longlong2*>(p.part + (((int64_t)z * p.N + j0 + j) * p.M + i) * 2) =
                        make_longlong2(hi[j], lo[j]);
        } else {
            const int ea = p.ea ? p.ea[i] : 0;
            const int64_t row = p.crow ? (int64_t)p.crow[i] : (int64_t)i;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int gj = j0 + j;
                if (gj >= p.N || (p.lower_only && gj > i)) continue;
                const double v =
                    words_to_double(hi[j], lo[j], ea + (p.eb ? p.eb[gj] : 0) - 86 + 8 * level_offset(p.terms));
                p.C[row * p.c_rs + (int64_t)gj * p.c_cs] =
                    epilogue_value(v, p.amode, p.alpha, p.bmode, p.beta, p.Cin + (int64_t)i * p.cin_rs + (int64_t)gj * p.cin_cs);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, p.tmem_cols);
}

struct SgReduceDev {
    const long long* part; int splits, M, N;
    const int32_t* ea; const int32_t* eb;
    double* C; int64_t c_rs, c_cs; const int32_t* crow;
    double alpha, beta;
    int amode, bmode;
    const double* Cin; int64_t cin_rs, cin_cs;
    int lower_only;
    int eoff;            // -86 + 8 level_offset(terms) = -78
};

__global__ void sliced_reduce_kernel(SgReduceDev r) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)r.M * r.N;
    if (idx >= total) return;
    const int j = (int)(idx / r.M), i = (int)(idx % r.M);   // consecutive threads: consecutive rows
    if (r.lower_only && j > i) return;
    __int128 acc = 0;
    for (int z = 0; z < r.splits; ++z) {
        const longlong2 q = *reinterpret_cast<const longlong2*>(r.part + ((int64_t)z * total + idx) * 2);
        acc += ((__int128)q.x << 40) + (__int128)q.y;
    }
    // all 128 bits: the sum of the splits may exceed what one split's hi word can hold
    const int e = (r.ea ? r.ea[i] : 0) + (r.eb ? r.eb[j] : 0) + r.eoff;
    const double v = u128_to_double((unsigned long long)(acc >> 64), (unsigned long long)acc, e);
    const int64_t row = r.crow ? (int64_t)r.crow[i] : (int64_t)i;
    r.C[row * r.c_rs + (int64_t)j * r.c_cs] =
        epilogue_value(v, r.amode, r.alpha, r.bmode, r.beta, r.Cin + (int64_t)i * r.cin_rs + (int64_t)j * r.cin_cs);
}


// =====================================================================================
// Pipelined form (sliced_gemm2_kernel): TMA loads, warp specialisation, windowed B.
//
// The digit planes of the B operand for one K block are loaded by a single 3-D TMA box
// (64 k x 32 rows x sb planes) and lie back to back in shared memory, so that "B planes
// q = 0..w-1" is one contiguous N = 32 w operand. One MMA per (A plane p, 16-k step)
// then forms every pair (p, q), q < min(sb, terms - p), at once, writing level p + q to
// TMEM columns (p + q) * 32: the D address is offset by p * 32 columns. The first MMA of
// a 128-k chunk (p = 0) covers every level (terms <= sb is required), so it alone
// carries accumulate = 0. Warp 0 issues the TMA loads into a ring of A-plane stages and
// a ring of B-plane stages; warp 1 issues the MMAs and commits each stage back to its
// producer; warps 2-9 (two per TMEM lane quarter, 16 columns each) read the level sums of
// each chunk from TMEM (double-buffered when 2 * terms * 32 <= 512 columns), hand the
// buffer back as soon as the values are in registers, and fold them into the same int64
// words as the synchronous form. Every mbarrier wait is bounded; expiry raises RTPROJ_ETIMEOUT.
// =====================================================================================
constexpr int W_EPI_WARPS = 8;                  // two per TMEM lane quarter, 16 columns each
constexpr int W_THREADS = 64 + 32 * W_EPI_WARPS;
constexpr int W_MAX_A_STAGES = 16;
constexpr int W_MAX_B_STAGES = 8;
constexpr int A_PPS = 2;                       // A planes per pipeline slot (one TMA box, one barrier)
constexpr int A_SLOT_BYTES = A_PPS * A_PLANE_BYTES;

struct Sg2Dev {
    int M, N, Kp, sa, sb, terms, k_per_split, chunk_kb, splits;
    int eoff;                     // -86 + 8 level_offset(terms) = -78: exponent of the output words
    const int32_t* ea; const int32_t* eb;
    long long* part;
    double* C; int64_t c_rs, c_cs; const int32_t* crow;
    double alpha, beta;
    int amode, bmode;
    const double* Cin; int64_t cin_rs, cin_cs;
    int lower_only;
    int* status;
    long long timeout;
    uint32_t tmem_cols;
    int acc_bufs, a_stages, b_stages;
    int tn;                       // B rows per tile: 32 or 64
    int m_fast;                   // tile order: A-row tiles fastest
    int vec2;                     // C rows contiguous and 16-byte aligned: paired stores
    int issue_cfg;                // compile-time MMA issue path (0: the general loop)
    int32_t* row_exp;             // optional: row exponents of C gathered by atomic maxima
};


// Warp-converged forms of the single-thread operations: every lane executes the
// instruction sequence with the same (warp-uniform) operands and lane 0 alone issues it,
// through a predicate rather than a branch, so that the issuing warp never diverges.
__device__ __forceinline__ void tma_load_3d_lane0(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                                  uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 e, l, 0;\n\t"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%5], %6;\n\t"
        "@e cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n\t}\n"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar)), "r"(bytes)
        : "memory");
}
__device__ __forceinline__ void umma_bf16_lane0(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                                uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 e, l, 0;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_bf16_lane0_acc(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 e, l, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc)
        : "memory");
}
__device__ __forceinline__ void umma_commit_lane0(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 e, l, 0;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(smem_addr(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase; raises the CTA-wide abort flag on expiry.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort_s, int* status,
                                           long long timeout) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_s) return false;
        if (clock64() - t0 > timeout) {
            *abort_s = 1;
            set_status(status, RTPROJ_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// The same bounded wait for a whole converged warp: every lane polls, the exit decision is
// warp-uniform (lane 0 owns the timeout and the abort flag).
__device__ __forceinline__ bool wait_phase_warp(uint64_t* bar, uint32_t parity, volatile int* abort_s, int* status,
                                                long long timeout) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    const long long t0 = clock64();
    while (true) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        int bad = 0;
        if ((threadIdx.x & 31) == 0) {
            if (*abort_s) {
                bad = 1;
            } else if (clock64() - t0 > timeout) {
                *abort_s = 1;
                set_status(status, RTPROJ_ETIMEOUT);
                bad = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, bad, 0)) return false;
    }
}

// Position in a ring of mbarrier-guarded stages: slot index, phase parity of the current
// round, and whether a full round has passed (the producer's first round needs no wait).
// Advanced incrementally: no division by the run-time stage count on the issue path.
struct Ring {
    int idx = 0, n = 1;
    uint32_t phase = 0;
    bool wrapped = false;
    __device__ explicit Ring(int stages) : n(stages) {}
    __device__ __forceinline__ void next() {
        if (++idx == n) { idx = 0; phase ^= 1u; wrapped = true; }
    }
};

// Tile order of the persistent loop. Tiles of one K split are enumerated either B-tile
// fastest or A-tile fastest (m_fast: when there are no more A-row tiles than B-row
// tiles, so that consecutive CTAs share the larger B tile through L2), and with
// lower_only only the tiles that touch the lower triangle are enumerated at all.
struct TileCoord { int i0, j0, z; };
struct TileSched {
    int tiles_m, tiles_n, tn, lower, m_fast;
    __host__ __device__ int row_count(int i) const {           // column tiles of row tile i
        if (!lower) return tiles_n;
        const int last = (i * TM + TM - 1) / tn;
        return last + 1 < tiles_n ? last + 1 : tiles_n;
    }
    __host__ __device__ int per_split() const {
        if (!lower) return tiles_m * tiles_n;
        int s = 0;
        for (int i = 0; i < tiles_m; ++i) s += row_count(i);
        return s;
    }
    __device__ TileCoord at(int t, int per_z) const {
        TileCoord c;
        c.z = t / per_z;
        int r = t - c.z * per_z;
        if (lower) {
            int i = 0;
            while (r >= row_count(i)) { r -= row_count(i); ++i; }
            c.i0 = i * TM;
            c.j0 = r * tn;
        } else if (m_fast) {
            c.i0 = (r % tiles_m) * TM;
            c.j0 = (r / tiles_m) * tn;
        } else {
            c.i0 = (r / tiles_n) * TM;
            c.j0 = (r % tiles_n) * tn;
        }
        return c;
    }
};

// Epilogue role of one warp: NCOL = tn / 2 columns of each tile, for TMEM lanes
// 32 * quarter ... + 31 (tile rows), chunk by chunk, then the tile's partial words or its
// final values.
// The MMA issuer's work on one k block for a fixed digit configuration (SA A planes,
// TERMS levels, TN B rows per level): A slots SLOT, SLOT+1, ... are awaited in turn and
// each of their planes pa meets B levels 0 .. TERMS-pa-1 in windows of 256/TN levels, four
// K steps of 16. Plane, window and K offsets, instruction descriptors and the accumulate
// flag are compile-time constants, so between two MMAs the issuing warp only adds a
// constant to a base: with the general loop's run-time bounds the issue path, not the
// tensor pipe, set the pace for windows narrower than 256 columns. Returns false on abort.
template <int SA, int TERMS, int TN, int SLOT = 0>
__device__ __forceinline__ bool issue_kblock(Ring& ra, uint32_t a_lo0, uint32_t b_lo, uint32_t desc_hi, uint32_t dbase,
                                             uint32_t acc0, uint64_t* fullA, uint64_t* emptyA, volatile int* abort_v,
                                             const Sg2Dev& p) {
    constexpr int WMAX = 256 / TN;
    constexpr uint32_t B_WIN = (uint32_t)WMAX * (uint32_t)((TN * KB * 2) >> 4);
    const int as = ra.idx;
    if (!wait_phase_warp(fullA + as, ra.phase, abort_v, p.status, p.timeout)) return false;
    const uint32_t a_slot = a_lo0 + (uint32_t)as * (A_SLOT_BYTES >> 4);
#pragma unroll
    for (int q = 0; q < A_PPS; ++q) {
        const int pa = SLOT * A_PPS + q;
        if (pa < SA) {
            const int nwin = TERMS - pa;
#pragma unroll
            for (int w0 = 0; w0 < nwin; w0 += WMAX) {
                const int nw = (nwin - w0) < WMAX ? (nwin - w0) : WMAX;
                const uint32_t id = idesc_bf16(TM, nw * TN);
                const uint32_t d = dbase + (uint32_t)((pa + w0) * TN);
#pragma unroll
                for (int kk = 0; kk < KB / 16; ++kk) {
                    const uint64_t ad = make_desc(a_slot + (uint32_t)(q * (A_PLANE_BYTES >> 4) + 2 * kk), desc_hi);
                    const uint64_t bd = make_desc(b_lo + (uint32_t)w0 / WMAX * B_WIN + (uint32_t)(2 * kk), desc_hi);
                    if (pa == 0 && kk == 0) umma_bf16_lane0(d, ad, bd, id, acc0);
                    else umma_bf16_lane0_acc(d, ad, bd, id);
                }
            }
        }
    }
    umma_commit_lane0(emptyA + as);
    ra.next();
    constexpr int NSLOTS = (SA + A_PPS - 1) / A_PPS;
    if constexpr (SLOT + 1 < NSLOTS)
        return issue_kblock<SA, TERMS, TN, SLOT + 1>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p);
    else
        return true;
}

// Configurations with a compile-time issue path (digit planes of A, levels, B rows per
// level); issue_cfg is the position in this list plus one.
struct IssueCfg { int sa, terms, tn; };
constexpr IssueCfg kIssueCfgs[] = {{7, 7, 32}, {9, 9, 32}, {3, 3, 64}, {1, 5, 64}, {5, 5, 64}, {7, 7, 64},
                                   {2, 5, 64}};   // the last: the Gaussian sketch (two G planes, five of A)

// Running record of max |v| for the row exponent, in two integer operations per value:
// the largest sign-cleared upper word (sign, exponent field, top 20 mantissa bits) and the
// OR of the lower words. The frexp exponent of the maximum follows from the upper word's
// maximum alone unless every upper word is zero; then the leading bit of the OR is that
// of the largest lower word. A non-finite value shows as an all-ones exponent field.
__device__ __forceinline__ void track_abs_max(double v, uint32_t& mxh, uint32_t& orl) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const uint32_t h = (uint32_t)(u >> 32) & 0x7FFFFFFFu;
    mxh = h > mxh ? h : mxh;
    orl |= (uint32_t)u;
}
// frexp exponent e (m < 2^e <= 2m) of the maximum recorded by track_abs_max (not all zero).
__device__ __forceinline__ int frexp_exponent_of_words(uint32_t mxh, uint32_t orl) {
    const int E = (int)(mxh >> 20);
    if (E > 0) return E - 1022;
    if (mxh != 0) return (32 - __clz((int)mxh)) + 32 - 1074;
    return (32 - __clz((int)orl)) - 1074;
}

template <int NCOL>
__device__ __forceinline__ void epilogue_role(const Sg2Dev& p, uint32_t tmem, uint64_t* tfull, uint64_t* tempty,
                                              volatile int* abort_v, int quarter, int half, int lane) {
    const int tn = 2 * NCOL;
    const TileSched ts{(p.M + TM - 1) / TM, (p.N + tn - 1) / tn, tn, p.lower_only, p.m_fast};
    const int per_z = ts.per_split();
    const int ntiles = per_z * p.splits;
    const int cb = p.chunk_kb;
    const uint32_t buf_cols = (uint32_t)(p.terms * tn);
    Ring tr(p.acc_bufs);
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const TileCoord c = ts.at(tile, per_z);
        const int kbeg = c.z * p.k_per_split;
        const int nkb = (min(p.Kp, kbeg + p.k_per_split) - kbeg) / KB;
        const int nchunks = (nkb + cb - 1) / cb;
        unsigned long long hi[NCOL], lo[NCOL];
#pragma unroll
        for (int j = 0; j < NCOL; ++j) { hi[j] = 0; lo[j] = 0; }
        for (int cc = 0; cc < nchunks; ++cc, tr.next()) {
            const int buf = tr.idx;
            if (!wait_phase(tfull + buf, tr.phase, abort_v, p.status, p.timeout)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t base =
                tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * buf_cols + (uint32_t)(half * NCOL);
            readout_terms<NCOL>(p.terms, base, (uint32_t)tn, hi, lo, tempty + buf);
        }
        if (!ok) break;
        const int i = c.i0 + quarter * 32 + lane;
        const int jb = c.j0 + half * NCOL;
        if (*abort_v) continue;
        const bool valid = i < p.M;                 // rows past M: no output (but join the shuffles)
        if (p.splits > 1) {
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < NCOL; ++j)
                if (jb + j < p.N)
                    *reinterpret_cast<longlong2*>(p.part + (((int64_t)c.z * p.N + jb + j) * p.M + i) * 2) =
                        make_longlong2((long long)hi[j], (long long)lo[j]);
        } else {
            // column exponents: one load per lane, shared through the warp
            const int ebl = (p.eb && lane < NCOL && jb + lane < p.N) ? p.eb[jb + lane] : 0;
            const int ea = (p.ea && valid ? p.ea[i] : 0) + p.eoff;
            const int64_t row = p.crow && valid ? (int64_t)p.crow[i] : (int64_t)i;
            double* crow_p = p.C + row * p.c_rs;
            const double* cin_p = p.Cin + (int64_t)i * p.cin_rs;
            if (p.bmode == 0) {
                // no Cin: the stores follow the conversions directly
                if (p.vec2) {
                    // row-contiguous output: pairs of columns as one 16-byte store; with row_exp
                    // the stored values' maximum magnitude is recorded (track_abs_max)
                    uint32_t mxh = 0, orl = 0;
#pragma unroll
                    for (int j = 0; j < NCOL; j += 2) {
                        const int gj = jb + j;
                        const int e0 = __shfl_sync(0xffffffffu, ebl, j), e1 = __shfl_sync(0xffffffffu, ebl, j + 1);
                        if (!valid || gj >= p.N || (p.lower_only && gj > i)) continue;
                        const double v0 = epilogue_value_v(words_to_double((long long)hi[j], (long long)lo[j], ea + e0),
                                                           p.amode, p.alpha, 0, 0.0, 0.0);
                        track_abs_max(v0, mxh, orl);
                        if (gj + 1 < p.N && !(p.lower_only && gj + 1 > i)) {
                            const double v1 = epilogue_value_v(
                                words_to_double((long long)hi[j + 1], (long long)lo[j + 1], ea + e1), p.amode,
                                p.alpha, 0, 0.0, 0.0);
                            track_abs_max(v1, mxh, orl);
                            *reinterpret_cast<double2*>(crow_p + gj) = make_double2(v0, v1);
                        } else {
                            crow_p[gj] = v0;
                        }
                    }
                    if (p.row_exp && valid) {
                        if (mxh >= 0x7FF00000u) set_status(p.status, RTPROJ_ENONFINITE);
                        else if ((mxh | orl) != 0) atomicMax(p.row_exp + row, frexp_exponent_of_words(mxh, orl));
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < NCOL; ++j) {
                        const int gj = jb + j;
                        const int ej = __shfl_sync(0xffffffffu, ebl, j);
                        if (!valid || gj >= p.N || (p.lower_only && gj > i)) continue;
                        crow_p[(int64_t)gj * p.c_cs] = epilogue_value_v(
                            words_to_double((long long)hi[j], (long long)lo[j], ea + ej), p.amode, p.alpha, 0, 0.0, 0.0);
                    }
                }
            } else {
                // Cin is read eight entries ahead of the stores, in groups: C may alias Cin (an
                // update in place), so a load placed after a store would wait for the previous
                // element's whole round trip
                constexpr int CG = 8;
#pragma unroll
                for (int g0 = 0; g0 < NCOL; g0 += CG) {
                    double cv[CG];
#pragma unroll
                    for (int q = 0; q < CG; ++q) {
                        const int gj = jb + g0 + q;
                        cv[q] = (p.bmode != 0 && valid && gj < p.N && !(p.lower_only && gj > i))
                                    ? __ldcg(cin_p + (int64_t)gj * p.cin_cs) : 0.0;
                    }
                    if (p.vec2) {
                        // row-contiguous output: pairs of columns as one 16-byte store
#pragma unroll
                        for (int q = 0; q < CG; q += 2) {
                            const int j = g0 + q, gj = jb + j;
                            const int e0 = __shfl_sync(0xffffffffu, ebl, j), e1 = __shfl_sync(0xffffffffu, ebl, j + 1);
                            if (!valid || gj >= p.N || (p.lower_only && gj > i)) continue;
                            const double v0 = epilogue_value_v(words_to_double((long long)hi[j], (long long)lo[j], ea + e0),
                                                               p.amode, p.alpha, p.bmode, p.beta, cv[q]);
                            if (gj + 1 < p.N && !(p.lower_only && gj + 1 > i)) {
                                const double v1 = epilogue_value_v(
                                    words_to_double((long long)hi[j + 1], (long long)lo[j + 1], ea + e1), p.amode,
                                    p.alpha, p.bmode, p.beta, cv[q + 1]);
                                *reinterpret_cast<double2*>(crow_p + gj) = make_double2(v0, v1);
                            } else {
                                crow_p[gj] = v0;
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < CG; ++q) {
                            const int j = g0 + q, gj = jb + j;
                            const int ej = __shfl_sync(0xffffffffu, ebl, j);
                            if (!valid || gj >= p.N || (p.lower_only && gj > i)) continue;
                            crow_p[(int64_t)gj * p.c_cs] =
                                epilogue_value_v(words_to_double((long long)hi[j], (long long)lo[j], ea + ej), p.amode,
                                                 p.alpha, p.bmode, p.beta, cv[q]);
                        }
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(W_THREADS, 1)
    sliced_gemm2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Sg2Dev p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int AS = p.a_stages;
    const int BSN = p.b_stages;
    const int tn = p.tn;
    const uint32_t b_plane_bytes = (uint32_t)tn * KB * 2;
    const uint32_t b_stage_bytes = (uint32_t)p.sb * b_plane_bytes;
    unsigned char* sA = smem;
    unsigned char* sB = sA + (size_t)AS * A_SLOT_BYTES;
    uint64_t* bars = (uint64_t*)(sB + (size_t)BSN * b_stage_bytes);
    uint64_t* fullA = bars;
    uint64_t* emptyA = fullA + W_MAX_A_STAGES;
    uint64_t* fullB = emptyA + W_MAX_A_STAGES;
    uint64_t* emptyB = fullB + W_MAX_B_STAGES;
    uint64_t* tfull = emptyB + W_MAX_B_STAGES;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
    __shared__ int abort_s;

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const TileSched ts{(p.M + TM - 1) / TM, (p.N + tn - 1) / tn, tn, p.lower_only, p.m_fast};
    const int per_z = ts.per_split();
    const int ntiles = per_z * p.splits;
    const int cb = p.chunk_kb;
    const uint32_t buf_cols = (uint32_t)(p.terms * tn);

    if (t == 0) {
        abort_s = 0;
        for (int i = 0; i < AS; ++i) { mbar_init(fullA + i, 1); mbar_init(emptyA + i, 1); }
        for (int i = 0; i < BSN; ++i) { mbar_init(fullB + i, 1); mbar_init(emptyB + i, 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(tfull + i, 1); mbar_init(tempty + i, 32 * W_EPI_WARPS); }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, p.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int* abort_v = &abort_s;

    // Every role walks the same tile sequence (blockIdx.x, + gridDim.x, ...), skipping the
    // tiles strictly above the diagonal when only the lower triangle is wanted.
    if (warp == 0) {
        // ---------------- TMA producer (whole warp, lane 0 issues)
        Ring ra(AS), rb(BSN);
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const TileCoord c = ts.at(tile, per_z);
            const int kbeg = c.z * p.k_per_split;
            const int nkb = (min(p.Kp, kbeg + p.k_per_split) - kbeg) / KB;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int k0 = kbeg + kb * KB;
                const int bs = rb.idx;
                if (rb.wrapped && !wait_phase_warp(emptyB + bs, rb.phase ^ 1u, abort_v, p.status, p.timeout)) {
                    ok = false;
                    break;
                }
                tma_load_3d_lane0(smem_addr(sB + (size_t)bs * b_stage_bytes), &tmB, k0, c.j0, 0, fullB + bs,
                                  b_stage_bytes);
                rb.next();
                for (int pa = 0; pa < p.sa; pa += A_PPS) {
                    // A_PPS planes per slot; a plane past the stack reads as zeros (no MMA uses it)
                    const int as = ra.idx;
                    if (ra.wrapped && !wait_phase_warp(emptyA + as, ra.phase ^ 1u, abort_v, p.status, p.timeout)) {
                        ok = false;
                        break;
                    }
                    tma_load_3d_lane0(smem_addr(sA + (size_t)as * A_SLOT_BYTES), &tmA, k0, c.i0, pa, fullA + as,
                                      A_SLOT_BYTES);
                    ra.next();
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (whole warp, lane 0 issues)
        const uint64_t d0desc = sw128_desc(smem_addr(sA));
        const uint32_t a_lo0 = (uint32_t)d0desc, desc_hi = (uint32_t)(d0desc >> 32);
        const uint32_t b_lo0 = (uint32_t)sw128_desc(smem_addr(sB));
        const int wmax = 256 / tn;                                     // levels per MMA window
        const uint32_t b_win = (uint32_t)wmax * (b_plane_bytes >> 4);  // second window's B offset
        Ring ra(AS), rb(BSN), rt(p.acc_bufs);
        int buf = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const TileCoord c = ts.at(tile, per_z);
            const int kbeg = c.z * p.k_per_split;
            const int nkb = (min(p.Kp, kbeg + p.k_per_split) - kbeg) / KB;
            int kc = 0;                                  // k blocks into the current chunk
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const bool chunk_start = kc == 0;
                if (chunk_start) {
                    buf = rt.idx;
                    if (rt.wrapped && !wait_phase_warp(tempty + buf, rt.phase ^ 1u, abort_v, p.status, p.timeout)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                const int bs = rb.idx;
                if (!wait_phase_warp(fullB + bs, rb.phase, abort_v, p.status, p.timeout)) {
                    ok = false;
                    break;
                }
                const uint32_t b_lo = b_lo0 + (uint32_t)bs * (b_stage_bytes >> 4);
                if (p.issue_cfg > 0) {
                    const uint32_t dbase = tmem + (uint32_t)buf * buf_cols;
                    const uint32_t acc0 = chunk_start ? 0u : 1u;
                    switch (p.issue_cfg) {
                    case 1: ok = issue_kblock<7, 7, 32>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    case 2: ok = issue_kblock<9, 9, 32>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    case 3: ok = issue_kblock<3, 3, 64>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    case 4: ok = issue_kblock<1, 5, 64>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    case 5: ok = issue_kblock<5, 5, 64>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    case 6: ok = issue_kblock<7, 7, 64>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    default: ok = issue_kblock<2, 5, 64>(ra, a_lo0, b_lo, desc_hi, dbase, acc0, fullA, emptyA, abort_v, p); break;
                    }
                } else
                for (int pa0 = 0; pa0 < p.sa; pa0 += A_PPS) {
                    const int as = ra.idx;
                    if (!wait_phase_warp(fullA + as, ra.phase, abort_v, p.status, p.timeout)) {
                        ok = false;
                        break;
                    }
                    // Plane pa against B levels 0 .. nwin-1: one MMA per window of up to 256 / tn
                    // levels (N = tn per level), at most two windows. Descriptors are built from
                    // precomputed words: the K step adds 32 bytes (2 units) to the start address.
#pragma unroll
                    for (int q = 0; q < A_PPS; ++q) {
                        const int pa = pa0 + q;
                        const int nwin = pa < p.sa ? min(p.sb, p.terms - pa) : 0;
                        if (nwin > 0) {
                            const int n1 = min(wmax, nwin), n2 = nwin - n1;
                            const uint32_t a_lo = a_lo0 + (uint32_t)as * (A_SLOT_BYTES >> 4) + (uint32_t)q * (A_PLANE_BYTES >> 4);
                            const uint32_t d = tmem + (uint32_t)buf * buf_cols + (uint32_t)(pa * tn);
                            const uint32_t id1 = idesc_bf16(TM, n1 * tn), id2 = idesc_bf16(TM, (n2 > 0 ? n2 : 1) * tn);
#pragma unroll
                            for (int kk = 0; kk < KB / 16; ++kk) {
                                const uint32_t acc = (chunk_start && pa == 0 && kk == 0) ? 0u : 1u;
                                const uint64_t ad = make_desc(a_lo + 2 * kk, desc_hi);
                                umma_bf16_lane0(d, ad, make_desc(b_lo + 2 * kk, desc_hi), id1, acc);
                                if (n2 > 0)
                                    umma_bf16_lane0(d + 256, ad, make_desc(b_lo + b_win + 2 * kk, desc_hi), id2, acc);
                            }
                        }
                    }
                    umma_commit_lane0(emptyA + as);
                    ra.next();
                }
                if (!ok) break;
                umma_commit_lane0(emptyB + bs);
                rb.next();
                if (++kc == cb || kb == nkb - 1) {
                    umma_commit_lane0(tfull + buf);
                    rt.next();
                    kc = 0;
                }
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9; warp w reads TMEM lanes 32 * (w % 4) ... + 31
        // (the lane quarter it may access) and columns tn/2 * half ... of each level.
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        if (tn == 64) epilogue_role<32>(p, tmem, tfull, tempty, abort_v, quarter, half, lane);
        else epilogue_role<16>(p, tmem, tfull, tempty, abort_v, quarter, half, lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, p.tmem_cols);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    return fn;
}

// 3-D map over a digit stack: (k, row, plane), box (64, box_rows, box_planes), 128-byte swizzle.
bool make_stack_map(CUtensorMap* map, const SliceStack& st, int box_rows, int box_planes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)st.ld, (cuuint64_t)st.rows, (cuuint64_t)st.s};
    cuuint64_t strides[2] = {(cuuint64_t)st.ld * 2, (cuuint64_t)st.plane_stride * 2};
    cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)st.d, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_reduce(const SlicedGemm& g, int splits, void* scratch, cudaStream_t s) {
    SgReduceDev r;
    r.part = (const long long*)scratch; r.splits = splits; r.M = g.a.rows; r.N = g.b.rows;
    r.ea = g.a.e; r.eb = g.b.e;
    r.C = g.C; r.c_rs = g.c_rs; r.c_cs = g.c_cs; r.crow = g.crow;
    r.alpha = g.alpha; r.beta = g.beta; r.amode = alpha_mode(g.alpha); r.bmode = beta_mode(g.beta);
    r.Cin = g.Cin; r.cin_rs = g.cin_rs; r.cin_cs = g.cin_cs;
    r.lower_only = g.lower_only ? 1 : 0;
    r.eoff = -86 + 8 * level_offset(g.terms);
    const int64_t total = (int64_t)r.M * r.N;
    sliced_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(r);
    note_launch();
}

bool pipelined_disabled() {
    const char* e = std::getenv("RTPROJ_SYNC_GEMM");
    return e && e[0] == '1';
}

}  // namespace

size_t sliced_gemm_scratch_bytes(int M, int N, int K) {
    (void)K;
    const size_t tiles = (size_t)((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    const size_t target = 2 * (size_t)sm_count();
    if (tiles >= target) return 0;
    const size_t splits = (target + tiles - 1) / tiles;
    return splits * (size_t)M * N * 16;
}

static int chunk_for(const SlicedGemm& g);

static cudaError_t sliced_gemm_sync(const SlicedGemm& g, void* scratch, size_t scratch_bytes, int* status, cudaStream_t s) {
    const int M = g.a.rows, N = g.b.rows, K = g.a.cols;
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (g.a.s < 1 || g.a.s > MAXS || g.b.s < 1 || g.b.s > MAXS) return cudaErrorInvalidValue;
    if (g.terms < 1 || g.terms > 10 || g.terms > g.a.s + g.b.s - 1) return cudaErrorInvalidValue;
    if (g.b.cols != K || g.a.ld % 64 || g.b.ld % 64 || g.a.ld < K || g.b.ld < K) return cudaErrorInvalidValue;
    const int Kp = (K + KB - 1) / KB * KB;
    const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + TN - 1) / TN;
    const int tiles = tiles_m * tiles_n;
    const int kchunk = chunk_for(g);
    int splits = 1;
    const int max_splits = std::max(1, (Kp + kchunk - 1) / kchunk);
    const int sms = sm_count();
    if (tiles < 2 * sms) splits = std::min(max_splits, (2 * sms + tiles - 1) / tiles);
    // every split within the fixed point's capacity (see the top), where the scratch allows
    const long long kcap = kSplitKCap;
    splits = std::max<long long>(splits, std::min<long long>(max_splits, (Kp + kcap - 1) / kcap));
    while (splits > 1 && (size_t)splits * M * N * 16 > scratch_bytes) --splits;
    int kps = (Kp + splits - 1) / splits;
    kps = (kps + kchunk - 1) / kchunk * kchunk;
    splits = (Kp + kps - 1) / kps;

    SgDev p;
    p.a = g.a.d; p.a_ld = g.a.ld; p.a_ps = g.a.plane_stride; p.ea = g.a.e; p.sa = g.a.s; p.M = M;
    p.b = g.b.d; p.b_ld = g.b.ld; p.b_ps = g.b.plane_stride; p.eb = g.b.e; p.sb = g.b.s; p.N = N;
    p.Kp = Kp; p.terms = g.terms; p.k_per_split = kps; p.kchunk = kchunk;
    p.part = (long long*)scratch;
    p.C = g.C; p.c_rs = g.c_rs; p.c_cs = g.c_cs; p.crow = g.crow;
    p.alpha = g.alpha; p.beta = g.beta; p.amode = alpha_mode(g.alpha); p.bmode = beta_mode(g.beta);
    p.Cin = g.Cin; p.cin_rs = g.cin_rs; p.cin_cs = g.cin_cs;
    p.lower_only = g.lower_only ? 1 : 0;
    p.status = status;
    p.timeout_cycles = 4000000000ll;   // ~2 s at 2 GHz per K block: a hung MMA reports ETIMEOUT
    p.tmem_cols = 32;
    while (p.tmem_cols < (uint32_t)(TN * g.terms)) p.tmem_cols <<= 1;
    const size_t smem = 1024 + (size_t)p.sa * A_PLANE_BYTES + (size_t)p.sb * B_PLANE_BYTES + 64;
    cudaError_t e = cudaFuncSetAttribute(sliced_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(tiles_n, tiles_m, splits);
    sliced_gemm_kernel<<<grid, NTHREADS, smem, s>>>(p);
    note_launch();
    if (splits > 1) {
        SgReduceDev r;
        r.part = (const long long*)scratch; r.splits = splits; r.M = M; r.N = N;
        r.ea = g.a.e; r.eb = g.b.e;
        r.C = g.C; r.c_rs = g.c_rs; r.c_cs = g.c_cs; r.crow = g.crow;
        r.alpha = g.alpha; r.beta = g.beta; r.amode = alpha_mode(g.alpha); r.bmode = beta_mode(g.beta);
    r.Cin = g.Cin; r.cin_rs = g.cin_rs; r.cin_cs = g.cin_cs;
        r.lower_only = g.lower_only ? 1 : 0;
        r.eoff = -86 + 8 * level_offset(g.terms);
        const int64_t total = (int64_t)M * N;
        sliced_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(r);
        note_launch();
    }
    return cudaGetLastError();
}


// Largest readout interval (128, 256 or 512 k) that keeps every level g <= 7 exact: each
// level holds at most min(sa, sb, terms) digit pairs per k, each product at most
// max_digit_a * max_digit_b, and a float32 sum is exact while it stays within 2^24.
static int chunk_for(const SlicedGemm& g) {
    const long long pairs = std::max(1, std::min(std::min(g.a.s, g.b.s), std::min(g.terms, 8)));
    const long long prod = (long long)g.a.max_digit * g.b.max_digit;
    int kc = 128;
    while (kc < 512 && pairs * (2 * kc) * prod <= (1ll << 24)) kc *= 2;
    return kc;
}

// Split-K factor for a persistent grid of one CTA per SM: the number of rounds of work units
// (tiles x splits) times the K blocks of one unit, plus a fixed cost per round (pipeline
// fill and output) and per split (the partial sums written and reduced), both counted in
// K blocks of 64; the lowest cost wins, fewer splits on ties. A split count just past a
// multiple of the SM count would add a nearly empty round.
// Splits whose K exceeds the fixed point's capacity (2^25, see the top) are taken only
// when the scratch cannot hold enough partials for any split count within it.
static int choose_splits(int tiles, int M, int N, int Kp, size_t scratch_bytes, int kchunk, int terms,
                         int* kps_out) {
    const int kSMs = sm_count();
    const int max_splits = std::max(1, (Kp + kchunk - 1) / kchunk);
    const double per_split = (double)M * N * 32.0 / (7.0e12 / 1.0e6);   // partials: microseconds
    const long long kcap = kSplitKCap;
    const int min_sp = (int)std::min<long long>(max_splits, (Kp + kcap - 1) / kcap);
    const int top = std::max(std::min(max_splits, 64), min_sp);
    int best = 1, best_kps = (Kp + kchunk - 1) / kchunk * kchunk;
    double best_cost = 1e300;
    bool best_capped = false;
    for (int sp = 1; sp <= top; ++sp) {
        if (sp > 1 && (size_t)sp * M * N * 16 > scratch_bytes) break;
        int kps = (Kp + sp - 1) / sp;
        kps = (kps + kchunk - 1) / kchunk * kchunk;
        const int eff = (Kp + kps - 1) / kps;
        if (eff != sp) continue;
        const bool capped = kps <= kcap;
        if (best_capped && !capped) continue;
        const long long units = (long long)tiles * eff;
        const long long rounds = (units + kSMs - 1) / kSMs;
        // one K block of 64 is about one microsecond on one SM for these products
        const double cost = (double)rounds * ((double)kps / KB + 3.0) + (sp > 1 ? per_split * sp : 0.0);
        if ((capped && !best_capped) || cost < best_cost - 1e-9) {
            best_cost = cost; best = eff; best_kps = kps; best_capped = capped;
        }
    }
    *kps_out = best_kps;
    return best;
}

namespace {
cudaError_t sliced_gemm_impl(const SlicedGemm& g0, void* scratch, size_t scratch_bytes, int* status, cudaStream_t s,
                             bool* exp_done) {
    SlicedGemm g = g0;
    bool swapped = false;
    // The pipelined kernel needs terms <= sb (the first MMA of a chunk covers every level).
    // Put the operand with more digits on the B side: swap and write C transposed.
    if (g.b.s < g.terms && g.a.s >= g.terms && !g.crow && !g.lower_only) {
        std::swap(g.a, g.b);
        std::swap(g.c_rs, g.c_cs);
        std::swap(g.cin_rs, g.cin_cs);
        swapped = true;
    }
    const int M = g.a.rows, N = g.b.rows, K = g.a.cols;
    if (M <= 0 || N <= 0) return cudaSuccess;
    const bool shapes_ok = g.a.s >= 1 && g.a.s <= MAXS && g.b.s >= 1 && g.b.s <= MAXS && g.terms >= 1 &&
                           g.terms <= 10 && g.terms <= g.b.s && g.b.cols == K && g.a.ld % 64 == 0 &&
                           g.b.ld % 64 == 0 && g.a.ld >= K && g.b.ld >= K;
    if (!shapes_ok || pipelined_disabled()) return sliced_gemm_sync(g, scratch, scratch_bytes, status, s);
    // 64 B rows per tile when the levels of one accumulator set fit TMEM at that width
    // (terms * 64 <= 512 columns) and the output is wider than 64: half the A-plane reads
    // per flop and twice the MMA work per pipeline stage. 32 otherwise, and also when 64
    // would leave a single TMEM accumulator set on a short contraction (K <= 1024: few
    // chunks per tile, so the per-tile output must overlap the next tile's MMAs, which
    // takes two sets). Both choices were measured faster where they apply.
    const int Kp0 = (K + KB - 1) / KB * KB;
    const bool wide_ok = g.terms * 64 <= 512 && N > 64 && (2 * g.terms * 64 <= 512 || Kp0 > 1024);
    const int tn = wide_ok ? 64 : 32;
    CUtensorMap mapA, mapB;
    if (!make_stack_map(&mapA, g.a, TM, A_PPS) || !make_stack_map(&mapB, g.b, tn, g.b.s))
        return sliced_gemm_sync(g, scratch, scratch_bytes, status, s);
    const int Kp = (K + KB - 1) / KB * KB;
    const int kchunk = chunk_for(g);
    int kps = 0;
    const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + tn - 1) / tn;
    const TileSched ts{tiles_m, tiles_n, tn, g.lower_only ? 1 : 0, tiles_m <= tiles_n ? 1 : 0};
    const int splits = choose_splits(ts.per_split(), M, N, Kp, scratch_bytes, kchunk, g.terms, &kps);
    Sg2Dev p;
    p.M = M; p.N = N; p.Kp = Kp; p.sa = g.a.s; p.sb = g.b.s; p.terms = g.terms; p.k_per_split = kps;
    p.eoff = -86 + 8 * level_offset(g.terms);
    p.chunk_kb = kchunk / KB;
    p.ea = g.a.e; p.eb = g.b.e;
    p.part = (long long*)scratch;
    p.C = g.C; p.c_rs = g.c_rs; p.c_cs = g.c_cs; p.crow = g.crow;
    p.alpha = g.alpha; p.beta = g.beta; p.amode = alpha_mode(g.alpha); p.bmode = beta_mode(g.beta);
    p.Cin = g.Cin; p.cin_rs = g.cin_rs; p.cin_cs = g.cin_cs;
    p.lower_only = g.lower_only ? 1 : 0;
    p.status = status;
    p.timeout = 4000000000ll;
    p.tn = tn;
    p.m_fast = ts.m_fast;
    p.vec2 = (g.c_cs == 1 && g.c_rs % 2 == 0 && ((uintptr_t)g.C & 15) == 0) ? 1 : 0;
    p.issue_cfg = 0;
    for (int i = 0; i < (int)(sizeof(kIssueCfgs) / sizeof(kIssueCfgs[0])); ++i)
        if (kIssueCfgs[i].sa == g.a.s && kIssueCfgs[i].terms == g.terms && kIssueCfgs[i].tn == tn) p.issue_cfg = i + 1;
    p.acc_bufs = (2 * g.terms * tn <= 512) ? 2 : 1;
    p.tmem_cols = 32;
    while (p.tmem_cols < (uint32_t)(p.acc_bufs * g.terms * tn)) p.tmem_cols <<= 1;
    // Split shared memory between the A-plane ring (sa slots per K block) and the B-stage
    // ring (one stage per K block) so that the producer can run as many K blocks ahead as
    // possible: maximise min(b_stages, a_stages / sa).
    const size_t b_stage = (size_t)g.b.s * tn * KB * 2;
    const size_t fixed = 1024 + (2 * W_MAX_A_STAGES + 2 * W_MAX_B_STAGES + 4) * 8 + 16;
    // 200 KB, not the 227 KB a CTA may take: an SM then also holds one CTA of the pivoted QR
    // (about 23 KB), so that a step's products can run while the next step's latency-bound
    // QR occupies the SMs
    const size_t budget = 200 * 1024 - fixed;
    int best_bs = 0, best_as = 0;
    double best_depth = -1.0;
    const int a_slots_per_kb = (g.a.s + A_PPS - 1) / A_PPS;
    for (int bsn = 2; bsn <= W_MAX_B_STAGES; ++bsn) {
        if ((size_t)bsn * b_stage + 2 * A_SLOT_BYTES > budget) break;
        const int asn = (int)std::min<size_t>(W_MAX_A_STAGES, (budget - (size_t)bsn * b_stage) / A_SLOT_BYTES);
        const double depth = std::min<double>(bsn, (double)asn / a_slots_per_kb);
        if (depth > best_depth + 1e-9) { best_depth = depth; best_bs = bsn; best_as = asn; }
    }
    if (best_as < 2 || best_bs < 2) return sliced_gemm_sync(g, scratch, scratch_bytes, status, s);
    p.a_stages = best_as;
    p.b_stages = best_bs;
    const size_t smem = fixed + (size_t)best_bs * b_stage + (size_t)best_as * A_SLOT_BYTES;
    cudaError_t e = cudaFuncSetAttribute(sliced_gemm2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    p.splits = splits;
    p.row_exp = (g.row_exp && !swapped && splits == 1 && p.bmode == 0 && p.vec2 && !g.crow) ? g.row_exp : nullptr;
    *exp_done = p.row_exp != nullptr;
    const int ntiles = ts.per_split() * splits;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    const int grid = std::min(ntiles, sms);   // persistent: one CTA per SM walks the tiles
    sliced_gemm2_kernel<<<grid, W_THREADS, smem, s>>>(mapA, mapB, p);
    note_launch();
    if (splits > 1) launch_reduce(g, splits, scratch, s);
    return cudaGetLastError();
}
}  // namespace

cudaError_t sliced_gemm(const SlicedGemm& g, void* scratch, size_t scratch_bytes, int* status, cudaStream_t s) {
    if (g.row_exp && (g.c_cs != 1 || g.lower_only)) return cudaErrorInvalidValue;   // whole contiguous rows only
    bool exp_done = false;
    const cudaError_t e = sliced_gemm_impl(g, scratch, scratch_bytes, status, s, &exp_done);
    if (e != cudaSuccess || !g.row_exp || exp_done) return e;
    // the output path that gathers them was not taken: one pass over C
    return row_exponents(g.C, g.c_rs, g.a.rows, g.b.rows, g.row_exp, status, s);
}

}  // namespace rtp
