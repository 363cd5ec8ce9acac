// Float-float ("paired FP32") scalar arithmetic: a value is h + l, two FP32
// words with |l| <= ulp(h) / 2, about 48 significant bits.  The sums and
// products are Dekker's (T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971): TwoSum
// (Knuth) for the head words, the product's rounding error by FMA, the low
// words added in FP32.  Square root and quotient take the FP32 result and
// one correction from the exact residual (Dekker's sqrt2 / div2).
// On GB300 an FP64 warp instruction occupies the SM sub-partition's FP64
// pipe for 64 cycles whether one lane or 32 are active; these run on the
// FP32 pipe (4-cycle latency, full rate) and serve the per-column scalars
// of the paired-FP32 kernels.
#pragma once

namespace tlr {

struct FF {
    float h, l;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = ff_two_sum(a.h, b.h);
    return ff_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.h, -a.l}; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff_fast(p, e);
}
// a / b: q = fl(a.h / b.h), then q + (a - q b) / b.h with a - q b exact in its head
__device__ __forceinline__ FF ff_div(FF a, FF b) {
    const float q = __fdiv_rn(a.h, b.h);
    const FF qb = ff_mul(FF{q, 0.f}, b);
    const FF r = ff_add(a, ff_neg(qb));
    return ff_fast(q, __fdiv_rn(r.h, b.h));
}
// sqrt(a), a >= 0: s = fl(sqrt(a.h)), then s + (a - s^2) / (2 s)
__device__ __forceinline__ FF ff_sqrt(FF a) {
    if (!(a.h > 0.f)) return FF{a.h == 0.f ? 0.f : __fsqrt_rn(a.h), 0.f};
    const float s = __fsqrt_rn(a.h);
    const float p = __fmul_rn(s, s), pe = __fmaf_rn(s, s, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), pe), a.l);
    return ff_fast(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

}  // namespace tlr
