// Host check of the integer binary64 arithmetic in exact64.cuh against the
// host's IEEE double arithmetic (round to nearest even): int64 -> double,
// products, and llrint of a product scaled by 2^-10.  Prints the number of
// cases and of mismatches; exit status 1 on any mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "exact64.cuh"

using namespace bz;

static bool same(double a, double b) { return std::memcmp(&a, &b, sizeof a) == 0; }

int main(int argc, char** argv)
{
    const long long n = argc > 1 ? std::atoll(argv[1]) : 2000000;
    std::mt19937_64 rng(12345);
    long long bad = 0, cases = 0;
    for (long long i = 0; i < n; ++i) {
        // integers of every bit length, both signs, with ties in the low bits
        const int bits = (int)(rng() % 64);
        long long v = (long long)(rng() >> (63 - bits));
        if (rng() & 1) v &= ~0xFFFll;
        if (rng() & 1) v |= 0x800ll;
        if (rng() & 1) v = -v;
        const Exact64 a = x64_from_ll(v);
        ++cases;
        if (!same(x64_to_double(a), (double)v)) ++bad;
        // a factor like 1/(2E) of the mass sums, and the small integer coefficients
        double r = 0.5 / std::sqrt(std::ldexp((double)(rng() >> 11), -50) + 1e-3);
        if (rng() % 4 == 0) r = std::ldexp(r, (int)(rng() % 40) - 20);
        const double c = (double)(1 + rng() % 9);
        const double cv = c * (double)v;
        const Exact64 acv = x64_mul(x64_from_double(c), a);
        ++cases;
        if (!same(x64_to_double(acv), cv)) ++bad;
        const double p = cv * r;
        const Exact64 ap = x64_mul(acv, x64_from_double(r));
        ++cases;
        if (!same(x64_to_double(ap), p)) ++bad;
        // an integer times a double, the integer exact (|c v| < 2^53)
        if (std::fabs(cv) < 9007199254740992.0 && v != 0) {
            const uint64_t u = (uint64_t)std::fabs(cv);
            Exact64 pu = x64_mul_u(u, x64_from_double(r));
            pu.neg ^= (int)(cv < 0);
            ++cases;
            if (!same(x64_to_double(pu), p)) ++bad;
        }
        long long q;
        if (x64_rint_scaled(ap, -10, &q)) {
            ++cases;
            if (q != std::llrint(p * (1.0 / 1024.0))) ++bad;
        } else if (std::fabs(p * (1.0 / 1024.0)) < 4611686018427387904.0) {
            ++bad;  // refused a value inside the range
        }
    }
    std::printf("%lld %lld\n", cases, bad);
    return bad ? 1 : 0;
}
