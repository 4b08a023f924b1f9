// Host check of csrc/wcns_f64int.cuh, the FP64 path's integer division and
// square root: every result must equal the host's IEEE division and square
// root (correctly rounded to nearest even by IEEE 754) bit for bit.  The
// FP32 seeds the device takes from approximate rcp / rsqrt instructions are
// modelled by the correctly rounded value moved by up to +-U ulps.
//
// usage: host_f64int_check <cases> <U>; prints the mismatch counts.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#define __device__
#define __forceinline__ inline

namespace wcns {
static int g_ulps = 0;
static uint64_t g_rng = 0x2545F4914F6CDD1Dull;
inline uint64_t next_rand()
{
    g_rng ^= g_rng << 13;
    g_rng ^= g_rng >> 7;
    g_rng ^= g_rng << 17;
    return g_rng;
}
inline float perturb(float r)
{
    uint32_t u;
    memcpy(&u, &r, 4);
    u += (uint32_t)((int)(next_rand() % (uint64_t)(2 * g_ulps + 1)) - g_ulps);
    memcpy(&r, &u, 4);
    return r;
}
inline float rcpf(float x) { return perturb(1.0f / x); }
inline float rsqrtf_a(float x) { return perturb(1.0f / std::sqrt(x)); }
inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b)
{
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
inline int __double2hiint(double d) { uint64_t b; memcpy(&b, &d, 8); return (int)(uint32_t)(b >> 32); }
inline int __double2loint(double d) { uint64_t b; memcpy(&b, &d, 8); return (int)(uint32_t)b; }
inline double __hiloint2double(int hi, int lo)
{
    const uint64_t b = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
    double d;
    memcpy(&d, &b, 8);
    return d;
}
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __dsqrt_rn(double a) { return std::sqrt(a); }
using std::max;
}  // namespace wcns

#include "wcns_f64int.cuh"

static uint64_t bits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static double dbl(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t with_exp(uint64_t b, uint64_t e) { return (b & 0x800FFFFFFFFFFFFFull) | (e << 52); }
static bool same(double x, double y) { return bits(x) == bits(y) || (std::isnan(x) && std::isnan(y)); }

int main(int argc, char** argv)
{
    const long long n = argc > 1 ? atoll(argv[1]) : 1000000;
    wcns::g_ulps = argc > 2 ? atoi(argv[2]) : 2;
    uint64_t s = 0x9E3779B97F4A7C15ull;
    auto rnd = [&s]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
    const uint64_t special[] = {0, 0x8000000000000000ull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
                                0x7FF8000000000000ull, 1, 0x000FFFFFFFFFFFFFull, 0x0010000000000000ull,
                                0x7FEFFFFFFFFFFFFFull, 0x3FF0000000000000ull, 0xBFF0000000000000ull,
                                0x3FFFFFFFFFFFFFFFull, 0x4000000000000000ull};
    const int ns = sizeof(special) / sizeof(special[0]);
    long long bad_div = 0, bad_sqrt = 0;
    for (long long i = 0; i < n; ++i) {
        uint64_t a = rnd(), b = rnd(), c = rnd();
        switch (i % 8) {
        case 0: a = with_exp(a, 1023 - 40 + rnd() % 81); b = with_exp(b, 1023 - 40 + rnd() % 81); break;
        case 1: a = with_exp(a, 1 + rnd() % 2046); b = with_exp(b, 1 + rnd() % 2046); break;
        case 2: {   // quotient exponents at the edges of the normal range
            const uint64_t eb = 1 + rnd() % 2046;
            long long ea = (long long)eb + ((rnd() & 1) ? 1022 : -1021) + (long long)(rnd() % 8) - 4;
            ea = ea < 1 ? 1 : (ea > 2046 ? 2046 : ea);
            a = with_exp(a, (uint64_t)ea);
            b = with_exp(b, eb);
            break;
        }
        case 3:     // power-of-two and short divisors
            b = with_exp(b & 0x800FFF0000000000ull, 1023 + rnd() % 8);
            if (rnd() & 1) b &= 0xFFF0000000000000ull;
            a = with_exp(a, 1023 + rnd() % 8);
            break;
        case 4: b = with_exp(b, 1023); a = with_exp(b + (rnd() % 16) - 8, 1023 + (rnd() % 3) - 1); break;
        case 5: {   // exact quotients
            const double bd = (double)(1 + rnd() % (1u << 26)), kd = (double)(1 + rnd() % (1u << 26));
            a = bits(bd * kd);
            b = bits(bd);
            break;
        }
        case 6: a = (rnd() & 1) ? 0x8000000000000000ull : 0; b = with_exp(b, 1 + rnd() % 2046); break;
        default: a = special[rnd() % ns]; b = (rnd() & 1) ? special[rnd() % ns] : with_exp(b, 1023); break;
        }
        switch (i % 4) {
        case 0: c = with_exp(c & 0x7FFFFFFFFFFFFFFFull, 1023 - 40 + rnd() % 81); break;
        case 1: { const double q = (double)(rnd() >> 11); c = bits(q * q) + (rnd() % 5) - 2; break; }
        case 2: c = with_exp(c & 0x7FFFFFFFFFFFFFFFull, 1 + rnd() % 2046); break;
        default: c = special[rnd() % ns]; break;
        }
        if (!same(wcns::ddiv_int(dbl(a), dbl(b)), dbl(a) / dbl(b))) {
            if (bad_div < 5) fprintf(stderr, "div %016llx / %016llx\n", (unsigned long long)a, (unsigned long long)b);
            ++bad_div;
        }
        if (!same(wcns::dsqrt_int(dbl(c)), std::sqrt(dbl(c)))) {
            if (bad_sqrt < 5) fprintf(stderr, "sqrt %016llx\n", (unsigned long long)c);
            ++bad_sqrt;
        }
    }
    printf("cases %lld ulps %d div_mismatches %lld sqrt_mismatches %lld\n", n, wcns::g_ulps, bad_div, bad_sqrt);
    return 0;
}
