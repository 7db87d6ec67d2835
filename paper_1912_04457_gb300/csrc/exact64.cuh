// IEEE binary64 multiplication and conversions with round-to-nearest-even,
// evaluated with integer instructions only.  A value is held as
// (-1)^neg m 2^e with m = 0 (zero) or 2^52 <= m < 2^53, so every result is
// the one the FP64 unit returns for the same operands (IEEE 754 binary64,
// roundTiesToEven) for finite operands whose results stay normal; the
// callers keep to that range and fall back to FP64 instructions outside it.
// On this GPU FP64 instructions, conversions included, issue at 1/64 of the
// FP32 rate, so the thermal-mass sums take this path for their products.
// The header also compiles as plain C++ (the host unit test checks it
// against the host's double arithmetic).
#pragma once
#include <cstdint>
#include <cstring>

#ifndef __CUDACC__
#define BZ_HD inline
#else
#define BZ_HD __host__ __device__ __forceinline__
#endif

namespace bz {

struct Exact64 {
    uint64_t m;  // 0, or 2^52 <= m < 2^53
    int e;       // value = m 2^e
    int neg;
};

BZ_HD int clz64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

BZ_HD uint64_t umulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Rounds m 2^-sh (1 <= sh <= 63) to the nearest integer, ties to even.
BZ_HD uint64_t shr_rne(uint64_t m, int sh)
{
    const uint64_t q = m >> sh;
    const uint64_t rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    return q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
}

// (double)n, rounded to nearest even when |n| >= 2^53.
BZ_HD Exact64 x64_from_ll(long long n)
{
    Exact64 r;
    r.neg = n < 0;
    const uint64_t a = r.neg ? 0ull - (uint64_t)n : (uint64_t)n;
    if (a == 0) {
        r.m = 0;
        r.e = 0;
        return r;
    }
    const int nb = 64 - clz64(a);  // bit length
    if (nb <= 53) {
        r.m = a << (53 - nb);
        r.e = nb - 53;
    } else {
        int sh = nb - 53;
        uint64_t m = shr_rne(a, sh);
        if (m == (1ull << 53)) {
            m >>= 1;
            ++sh;
        }
        r.m = m;
        r.e = sh;
    }
    return r;
}

// The exact value of a finite double.
BZ_HD Exact64 x64_from_double(double d)
{
    uint64_t b;
    memcpy(&b, &d, sizeof b);
    Exact64 r;
    r.neg = (int)(b >> 63);
    const int be = (int)((b >> 52) & 0x7ffu);
    const uint64_t frac = b & ((1ull << 52) - 1ull);
    if (be == 0) {  // zero (subnormals do not occur in the callers' range)
        r.m = 0;
        r.e = 0;
    } else {
        r.m = frac | (1ull << 52);
        r.e = be - 1075;
    }
    return r;
}

BZ_HD double x64_to_double(Exact64 x)
{
    uint64_t b = (uint64_t)x.neg << 63;
    if (x.m) b |= ((uint64_t)(x.e + 1075) << 52) | (x.m & ((1ull << 52) - 1ull));
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

// a * b rounded to nearest even (a zero operand gives a signed zero).
BZ_HD Exact64 x64_mul(Exact64 a, Exact64 b)
{
    Exact64 r;
    r.neg = a.neg ^ b.neg;
    if (a.m == 0 || b.m == 0) {
        r.m = 0;
        r.e = 0;
        return r;
    }
    // the 105- or 106-bit product hi 2^64 + lo, cut to 53 bits
    const uint64_t hi = umulhi64(a.m, b.m), lo = a.m * b.m;
    int sh = (hi >> 41) ? 53 : 52;
    uint64_t m = (hi << (64 - sh)) | (lo >> sh);
    const uint64_t rem = lo & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m += (rem > half || (rem == half && (m & 1ull))) ? 1ull : 0ull;
    if (m == (1ull << 53)) {
        m >>= 1;
        ++sh;
    }
    r.m = m;
    r.e = a.e + b.e + sh;
    return r;
}

// u x rounded to nearest even, for an integer 0 < u < 2^53 (exactly a
// double) and a nonzero x: the product of the two doubles.
BZ_HD Exact64 x64_mul_u(uint64_t u, Exact64 x)
{
    Exact64 r;
    r.neg = x.neg;
    const uint64_t hi = umulhi64(u, x.m), lo = u * x.m;
    const int nb = hi ? 128 - clz64(hi) : 64 - clz64(lo);  // bit length of the product (>= 53)
    const int sh = nb - 53;                                // 0 .. 53
    uint64_t m;
    if (sh == 0) {
        m = lo;
    } else {
        m = (hi << (64 - sh)) | (lo >> sh);
        const uint64_t rem = lo & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        m += (rem > half || (rem == half && (m & 1ull))) ? 1ull : 0ull;
    }
    int e = x.e + sh;
    if (m == (1ull << 53)) {
        m >>= 1;
        ++e;
    }
    r.m = m;
    r.e = e;
    return r;
}

// llrint(x 2^k), rounded to nearest even; false when |x 2^k| >= 2^62 (the
// caller then uses the FP64 conversion).
BZ_HD bool x64_rint_scaled(Exact64 x, int k, long long* out)
{
    if (x.m == 0) {
        *out = 0;
        return true;
    }
    const int s = x.e + k;
    uint64_t v;
    if (s >= 0) {
        if (s > 9) return false;  // m 2^s >= 2^62
        v = x.m << s;
    } else if (s >= -63) {
        v = shr_rne(x.m, -s);
    } else {
        v = 0;  // below 2^-10: rounds to 0
    }
    *out = x.neg ? -(long long)v : (long long)v;
    return true;
}

}  // namespace bz
