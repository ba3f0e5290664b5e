// Float-float arithmetic on the FP32 pipe: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2 (about 48 significant bits). TwoSum is Knuth's, the
// product's error term comes from fmaf (the FMA form of Dekker's TwoProduct). Used by the
// pivoted QR kernels of the mixed form, where GB300's FP32 pipe (64 times the FP64 pipe's
// rate) carries the reflector updates.
#pragma once

namespace rtp {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ ff ff_sqrt(ff x) {
    if (!(x.hi > 0.f)) return {0.f, 0.f};
    const float s = sqrtf(x.hi);
    const float e = (fmaf(-s, s, x.hi) + x.lo) / (2.f * s);
    return quick_two_sum(s, e);
}

__device__ __forceinline__ ff ff_recip(ff d) {
    const float q = 1.f / d.hi;
    const float r = fmaf(-d.hi, q, 1.f) - d.lo * q;     // 1 - d q, to float-float accuracy
    return quick_two_sum(q, r * q);
}

// x > y for normalised float-float values (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ bool ff_gt(ff x, ff y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }

__device__ __forceinline__ ff ff_warp_sum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

// acc += x y with one TwoSum on the high parts; the rounding errors of the product and
// the low parts accumulate in acc.lo (a dot product to float-float accuracy times its
// length, the same order as the float64 sums it replaces).
__device__ __forceinline__ void ff_dot_acc(ff& acc, ff x, ff y) {
    const float p = x.hi * y.hi;
    const float e = fmaf(x.lo, y.hi, fmaf(x.hi, y.lo, fmaf(x.hi, y.hi, -p)));
    const ff s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + e;
}

__device__ __forceinline__ ff ff_renorm(ff x) { return quick_two_sum(x.hi, x.lo); }

__device__ __forceinline__ ff ff_from_double(double d) {
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

}  // namespace rtp
