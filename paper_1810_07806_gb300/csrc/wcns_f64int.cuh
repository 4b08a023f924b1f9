// wcns_f64int.cuh -- correctly rounded FP64 division and square root in
// 64-bit integer fixed point (device code of the FP64 path).
//
// Self-contained apart from the primitives the includer declares in
// namespace wcns first: rcpf and rsqrtf_a (FP32 approximations), and the
// CUDA intrinsics __umul64hi, __double2hiint, __double2loint,
// __hiloint2double, __float_as_uint, __uint_as_float, __ddiv_rn, __dsqrt_rn
// and max (unsigned).
// The device build includes it from wcns_fp64.cuh after wcns_device.cuh; the
// CPU test suite compiles it for the host with host versions of those
// primitives (with perturbed seeds) and checks it against IEEE division.
#pragma once

namespace wcns {

// ------------------------------------------------------------------------
// Correctly rounded FP64 division and square root on the integer pipes.
// The FP64 unit of this GPU completes about two lanes per clock per SM, 1/64
// of the FP32 rate, and a hardware division or square root is a sequence of
// several FP64 operations, so these two dominate the FP64 face.  For normal
// operands with a normal result they are computed here in 64-bit fixed
// point: an FP32 reciprocal (reciprocal square root) seed, two Newton-Raphson
// steps, one product for the estimate, one exact remainder test that fixes
// the estimate to the truncated 54-bit result, and round-to-nearest-even
// from its last bit and the remainder, as IEEE 754 defines the rounding.
// A zero numerator or radicand gives the signed zero directly; every other
// case (zero divisor, subnormal, infinite or NaN operand, a quotient outside
// the normal range) takes the hardware operation.  Either way the
// result is the IEEE result, bit for bit.
// ------------------------------------------------------------------------
typedef unsigned long long u64;

// 1.f of a normal double as the integer 2^52 + f, in [2^52, 2^53)
__device__ __forceinline__ u64 mant53(unsigned hi, unsigned lo)
{
    return ((u64)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
}

// X ~ 2^116 / m for m in [2^52, 2^53), i.e. X / 2^64 ~ 2^52 / m in (1/2, 1].
// frac23: the top 23 fraction bits of m.
__device__ __forceinline__ u64 recip_fx(u64 m, unsigned frac23)
{
    // rcp of 1.f in [1, 2) lies in (1/2, 1] up to its 1-ulp error: clamped to
    // [1/2, 1); exponent field 126 gives X = 1.f 2^63, and rcp = 1, X = 2^64 - 1
    const unsigned rb = max(__float_as_uint(rcpf(__uint_as_float(0x3f800000u | frac23))), 0x3f000000u);
    u64 X = rb >= 0x3f800000u ? ~0ull : ((u64)(0x800000u | (rb & 0x7fffffu)) << 40);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        // x += x (1 - m x / 2^52): E = 2^64 - m X / 2^52, small and signed
        const u64 P = (__umul64hi(m, X) << 12) | ((m * X) >> 52);
        const long long E = (long long)(0ull - P);
        X = E >= 0 ? X + __umul64hi(X, (u64)E) : X - __umul64hi(X, (u64)(-E));
    }
    return X;
}

__device__ __forceinline__ double ddiv_int(double a, double b)
{
    const unsigned ha = (unsigned)__double2hiint(a), la = (unsigned)__double2loint(a);
    const unsigned hb = (unsigned)__double2hiint(b), lb = (unsigned)__double2loint(b);
    const int ea = (int)((ha >> 20) & 0x7ffu), eb = (int)((hb >> 20) & 0x7ffu);
    int e = ea - eb + 1023;   // biased exponent of the quotient for ma >= mb
    const bool b_normal = (unsigned)(eb - 1) < 2046u;
    // 0 / b = signed zero (constant data makes many zero numerators)
    if (b_normal && ((ha & 0x7fffffffu) | la) == 0u) return __hiloint2double((int)((ha ^ hb) & 0x80000000u), 0);
    if (!b_normal || (unsigned)(ea - 1) >= 2046u || (unsigned)(e - 2) >= 2044u) return __ddiv_rn(a, b);
    u64 ma = mant53(ha, la);
    const u64 mb = mant53(hb, lb);
    if (ma < mb) { ma <<= 1; --e; }   // ma in [mb, 2 mb): quotient in [1, 2)
    const u64 X = recip_fx(mb, ((hb & 0xfffffu) << 3) | (lb >> 29));
    // Q ~ ma 2^53 / mb = 2 ma X / 2^64, then exact: 0 <= ma 2^53 - Q mb < mb
    u64 Q = (__umul64hi(ma, X) << 1) | ((ma * X) >> 63);
    long long r = (long long)(((ma & 0x7ffull) << 53) - Q * mb);   // exact: |r| < 2^55
    if (r < 0) { --Q; r += (long long)mb; }
    else if (r >= (long long)mb) { ++Q; r -= (long long)mb; }
    // Q in [2^53, 2^54): 53 result bits and the round bit; r != 0: sticky
    u64 M = Q >> 1;
    if ((Q & 1ull) && (r != 0 || (M & 1ull))) ++M;
    if (M >> 53) { M >>= 1; ++e; }
    const unsigned hi = ((ha ^ hb) & 0x80000000u) | ((unsigned)e << 20) | ((unsigned)(M >> 32) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(unsigned)M);
}

__device__ __forceinline__ double dsqrt_int(double a)
{
    const unsigned ha = (unsigned)__double2hiint(a), la = (unsigned)__double2loint(a);
    const int ea = (int)(ha >> 20);   // with the sign bit: positive normal iff 1 <= ea <= 2046
    if (((ha & 0x7fffffffu) | la) == 0u) return a;   // sqrt(+-0) = +-0
    if ((unsigned)(ea - 1) >= 2046u) return __dsqrt_rn(a);
    const unsigned frac23 = ((ha & 0xfffffu) << 3) | (la >> 29);
    u64 m = mant53(ha, la);
    int E = ea - 1023;
    const bool odd = (E & 1) != 0;
    if (odd) { m <<= 1; --E; }        // a = m 2^(E - 52), m in [2^52, 2^54), E even
    // y ~ 1 / sqrt(t), t = m / 2^52 in [1, 4); Y = y 2^64
    const unsigned yb = max(__float_as_uint(rsqrtf_a(__uint_as_float(((odd ? 128u : 127u) << 23) | frac23))), 0x3f000000u);
    u64 Y = yb >= 0x3f800000u ? ~0ull : ((u64)(0x800000u | (yb & 0x7fffffu)) << 40);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        // y += y (1 - t y^2) / 2: E2 = 2^64 - m (Y^2 / 2^64) / 2^52, small and signed
        const u64 Y2 = __umul64hi(Y, Y);
        const u64 P = (__umul64hi(m, Y2) << 12) | ((m * Y2) >> 52);
        const long long E2 = (long long)(0ull - P);
        Y = E2 >= 0 ? Y + (__umul64hi(Y, (u64)E2) >> 1) : Y - (__umul64hi(Y, (u64)(-E2)) >> 1);
    }
    // Q ~ sqrt(m 2^54) = t y 2^53 = m Y / 2^63, then exact: Q^2 <= m 2^54 < (Q + 1)^2
    u64 Q = (__umul64hi(m, Y) << 1) | ((m * Y) >> 63);
    long long r = (long long)(((m & 0x3ffull) << 54) - Q * Q);   // exact: |r| < 2^57
    if (r < 0) { --Q; r += (long long)(2 * Q + 1); }
    else if (r > (long long)(2 * Q)) { r -= (long long)(2 * Q + 1); ++Q; }
    u64 M = Q >> 1;                    // Q in [2^53, 2^54)
    int eb = E / 2 + 1023;
    if ((Q & 1ull) && (r != 0 || (M & 1ull))) ++M;
    if (M >> 53) { M >>= 1; ++eb; }
    const unsigned hi = ((unsigned)eb << 20) | ((unsigned)(M >> 32) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(unsigned)M);
}

}  // namespace wcns
