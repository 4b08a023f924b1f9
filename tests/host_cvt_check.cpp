// Host check of csrc/wcns_cvt.cuh, the FP32 path's FP64 <-> FP32 conversions
// by integer arithmetic: float(x) must equal the host's IEEE conversion
// (round to nearest even) except that results below FLT_MIN become signed
// zeros; double(x) must be exact except that subnormal inputs become signed
// zeros; the zero test must agree with x == 0.
//
// usage: host_cvt_check <cases>; prints the mismatch counts.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#define __device__
#define __forceinline__ inline

namespace wcns {
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
}  // namespace wcns

#include "wcns_cvt.cuh"

static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static uint64_t dbits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static double dbl(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static float flt(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

int main(int argc, char** argv)
{
    const long long n = argc > 1 ? atoll(argv[1]) : 1000000;
    uint64_t s = 88172645463325252ull;
    auto rnd = [&s]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
    const uint64_t sp64[] = {0, 0x8000000000000000ull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
                             0x7FF8000000000000ull, 0x7FF0000000000001ull, 0x47EFFFFFE0000000ull,
                             0x47EFFFFFF0000000ull, 0x47EFFFFFEFFFFFFFull, 0x3810000000000000ull,
                             0x380FFFFFFFFFFFFFull, 0x380FFFFFF0000000ull, 0x3800000000000000ull, 1,
                             0x3FF0000010000000ull, 0x3FF0000030000000ull};
    const uint32_t sp32[] = {0, 0x80000000u, 0x7f800000u, 0xff800000u, 0x7fc00000u, 1, 0x00800000u, 0x7f7fffffu};
    long long bad64 = 0, bad32 = 0, badz = 0;
    for (long long i = 0; i < n; ++i) {
        uint64_t b = rnd();
        if (i % 2 == 0) {   // the float range, exact ties and exact values
            b = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(1023 - 130 + rnd() % 261) << 52);
            if (i % 8 == 0) b = (b & ~0x1FFFFFFFull) | 0x10000000ull;
            if (i % 16 == 2) b &= ~0x1FFFFFFFull;
        }
        if (i % 97 == 5) b = sp64[rnd() % (sizeof(sp64) / 8)];
        const double x = dbl(b);
        const float got = wcns::f64_to_f32_ftz(x);
        float want = (float)x;
        if (std::isnan(want)) {
            if (!std::isnan(got)) ++bad64;
        } else {
            if (std::fpclassify(want) == FP_SUBNORMAL) want = std::copysign(0.0f, want);
            if (fbits(got) != fbits(want)) {
                if (bad64 < 5) fprintf(stderr, "f64->f32 %016llx\n", (unsigned long long)b);
                ++bad64;
            }
        }
        if (wcns::f64_is_zero(x) != (x == 0.0)) ++badz;
        uint32_t u = (uint32_t)rnd();
        if (i % 53 == 7) u = sp32[rnd() % (sizeof(sp32) / 4)];
        const float y = flt(u);
        const double g = wcns::f32_to_f64_ftz(y);
        if (std::isnan(y)) {
            if (!std::isnan(g)) ++bad32;
        } else {
            const double w = std::fpclassify(y) == FP_SUBNORMAL ? std::copysign(0.0, (double)y) : (double)y;
            if (dbits(g) != dbits(w)) {
                if (bad32 < 5) fprintf(stderr, "f32->f64 %08x\n", u);
                ++bad32;
            }
        }
    }
    printf("cases %lld f64_to_f32_mismatches %lld f32_to_f64_mismatches %lld zero_mismatches %lld\n", n, bad64,
           bad32, badz);
    return 0;
}
