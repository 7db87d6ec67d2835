// Conversions between FP32 and int64 with integer instructions only.  On
// this GPU the hardware conversion instructions issue on the FP64 pipe (1/64
// of the FP32 rate), which made them the bottleneck of the streaming kernels.
#pragma once
#include <cstdint>

namespace bz {

// Round half even of a finite |w| < 2^62 to int64.
__device__ __forceinline__ long long rint_ll(float w)
{
    const float aw = fabsf(w);
    if (aw < 4194304.0f) {  // 2^22: the 1.5 2^23 shifter puts round(w) in the low mantissa bits
        return (long long)(__float_as_int(w + 12582912.0f) - 0x4B400000);
    }
    const unsigned b = __float_as_uint(w);
    const int e = (int)((b >> 23) & 0xffu) - 150;  // |w| >= 2^22: w is m 2^e with e >= -1
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    long long v;
    if (e >= 0) {
        v = m << e;
    } else {  // e == -1: m/2, half even
        v = (m >> 1) + ((m & 1) & ((m >> 1) & 1));
    }
    return (b >> 31) ? -v : v;
}

// int64 to the nearest float (ties to even): keep the leading 24 bits, round
// on the rest, assemble sign, exponent and mantissa.
__device__ __forceinline__ float ll2float_rn(long long v)
{
    const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    if (a == 0) return 0.0f;
    int nb = 64 - __clzll((long long)a);  // bit length
    unsigned long long m;
    if (nb <= 24) {
        m = a << (24 - nb);
    } else {
        const int sh = nb - 24;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        m += (rem > half || (rem == half && (m & 1ull))) ? 1ull : 0ull;
        if (m == (1ull << 24)) {
            m >>= 1;
            ++nb;
        }
    }
    const float f = __uint_as_float(((unsigned)(126 + nb) << 23) | ((unsigned)m & 0x7fffffu));
    return v < 0 ? -f : f;
}

}  // namespace bz
