// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and
// the FMA product error (Dekker, "A floating-point technique for extending
// the available precision", Numer. Math. 18, 1971); division and square root
// by one Newton correction of an FP32 estimate (Karp and Markstein, "High
// precision division and square root", ACM TOMS 23, 1997).
//
// On this GPU FP64 issues at 1/64 of the FP32 rate, so a handful of FP32
// instructions per operation is much cheaper than one FP64 operation.  The
// transformations need every FP32 add and multiply rounded to nearest as
// written (no reassociation; FMA contraction of the products is harmless)
// and stay exact away from underflow.
#pragma once

namespace bz {

// Every operation below is rounded as written, also in translation units
// compiled with FMA contraction: on the device through the _rn intrinsics,
// which the compiler never fuses, so a result does not depend on the call
// site it was inlined into.
#ifdef __CUDA_ARCH__
#define FF_ADD(a, b) __fadd_rn((a), (b))
#define FF_SUB(a, b) __fsub_rn((a), (b))
#define FF_MUL(a, b) __fmul_rn((a), (b))
#define FF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define FF_ADD(a, b) ((a) + (b))
#define FF_SUB(a, b) ((a) - (b))
#define FF_MUL(a, b) ((a) * (b))
#define FF_FMA(a, b, c) fmaf((a), (b), (c))
#endif

struct ff {
    float hi, lo;
};

__host__ __device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = FF_ADD(a, b);
    const float bb = FF_SUB(s, a);
    return {s, FF_ADD(FF_SUB(a, FF_SUB(s, bb)), FF_SUB(b, bb))};
}

__host__ __device__ __forceinline__ ff ff_fast_two_sum(float a, float b)  // |a| >= |b| or a == 0
{
    const float s = FF_ADD(a, b);
    return {s, FF_SUB(b, FF_SUB(s, a))};
}

__host__ __device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    const float p = FF_MUL(a, b);
    return {p, FF_FMA(a, b, -p)};
}

__host__ __device__ __forceinline__ ff ff_from(float a) { return {a, 0.0f}; }

// nearest float-float of a double (exact to 48 bits)
__host__ __device__ __forceinline__ ff ff_from_double(double v)
{
#ifdef __CUDA_ARCH__
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(__dsub_rn(v, (double)h))};
#else
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
#endif
}

__host__ __device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__host__ __device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s.lo = FF_ADD(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = FF_ADD(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__host__ __device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = ff_two_sum(a.hi, b);
    s.lo = FF_ADD(s.lo, a.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = ff_two_prod(a.hi, b.hi);
    p.lo = FF_ADD(p.lo, FF_ADD(FF_MUL(a.hi, b.lo), FF_MUL(a.lo, b.hi)));
    return ff_fast_two_sum(p.hi, p.lo);
}

__host__ __device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    ff p = ff_two_prod(a.hi, b);
    p.lo = FF_ADD(p.lo, FF_MUL(a.lo, b));
    return ff_fast_two_sum(p.hi, p.lo);
}

__host__ __device__ __forceinline__ ff ff_sqr(ff a)
{
    ff p = ff_two_prod(a.hi, a.hi);
    p.lo = FF_ADD(p.lo, FF_MUL(FF_MUL(2.0f, a.hi), a.lo));
    return ff_fast_two_sum(p.hi, p.lo);
}

// a / b: FP32 quotient q of the leading parts, then q + (a - q b) / b
__host__ __device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q = FF_MUL(a.hi, 1.0f / b.hi);
    const ff r = ff_sub(a, ff_mul_f(b, q));
    return ff_fast_two_sum(q, FF_MUL(r.hi, 1.0f / b.hi));
}

// sqrt(a) for a > 0: y = a x with x ~ 1/sqrt(a), then y + (a - y^2) x / 2
__host__ __device__ __forceinline__ ff ff_sqrt(ff a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
#ifdef __CUDA_ARCH__
    const float x = rsqrtf(a.hi);
#else
    const float x = 1.0f / sqrtf(a.hi);
#endif
    const float y = FF_MUL(a.hi, x);
    const ff r = ff_sub(a, ff_two_prod(y, y));
    return ff_fast_two_sum(y, FF_MUL(FF_MUL(r.hi, x), 0.5f));
}

// sign tests and comparisons (hi carries the sign of a normalised value)
__host__ __device__ __forceinline__ bool ff_gt0(ff a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }
__host__ __device__ __forceinline__ bool ff_ge0(ff a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo >= 0.0f); }
__host__ __device__ __forceinline__ bool ff_lt(ff a, ff b) { return ff_gt0(ff_sub(b, a)); }
__host__ __device__ __forceinline__ bool ff_ge(ff a, ff b) { return ff_ge0(ff_sub(a, b)); }
__host__ __device__ __forceinline__ float ff_to_float(ff a) { return FF_ADD(a.hi, a.lo); }

__host__ __device__ __forceinline__ ff ff_abs(ff a) { return a.hi < 0.0f ? ff_neg(a) : a; }

// F(-|z|) of the Student-t distribution with two degrees of freedom,
// 1 / (r (r + |z|)) with r = sqrt(2 + z^2) (no cancellation in the tails)
__host__ __device__ __forceinline__ ff ff_t2_tail(ff z)
{
    const ff r = ff_sqrt(ff_add_f(ff_sqr(z), 2.0f));
    return ff_div(ff_from(1.0f), ff_mul(r, ff_add(r, ff_abs(z))));
}

// floor of a normalised float-float as an int (|a| < 2^22), without a
// conversion instruction: the integer-valued float f plus 1.5 2^23 holds f
// in its low mantissa bits
__host__ __device__ __forceinline__ int ff_floor(ff a)
{
    const float f = floorf(a.hi);
#ifdef __CUDA_ARCH__
    int j = __float_as_int(f + 12582912.0f) - 0x4B400000;
#else
    int j = (int)f;
#endif
    if (f == a.hi && a.lo < 0.0f) --j;
    return j;
}

}  // namespace bz
