// wcns_cvt.cuh -- FP64 <-> FP32 conversions by integer arithmetic (device
// code of the FP32 path).
//
// Uses only the CUDA reinterpretation intrinsics __double2hiint,
// __double2loint, __hiloint2double, __float_as_uint and __uint_as_float,
// which the includer provides (the CUDA headers on the device; the CPU test
// suite compiles this header for the host with host versions and checks it
// against the host's IEEE conversions).
#pragma once

namespace wcns {

// Conversions between FP64 and FP32 by integer arithmetic on the IEEE-754
// encodings.  The FP64 pipe of this GPU is about 64x slower than FP32, so a
// per-element cvt there costs more than the integer ops below.  Both follow
// the FP32 path's flush-to-zero rule: FP32 subnormals (inputs, or results of
// the narrowing) become signed zeros.
__device__ __forceinline__ bool f64_is_zero(double x)   // +0 or -0
{
    return ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) == 0;
}

// float(x), rounded to nearest even; overflow gives inf, NaN stays NaN,
// results below FLT_MIN are signed zeros.
__device__ __forceinline__ float f64_to_f32_ftz(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int ed = (int)((hi >> 20) & 0x7ffu);
    const int ef = ed - 1023 + 127;
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 of the 52 bits
    const unsigned rest = lo & 0x1fffffffu;                       // the 29 dropped bits
    unsigned r = sign | ((unsigned)ef << 23) | mant;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;   // may carry to inf
    // below FLT_MIN: zero, except the values that round up to FLT_MIN
    if (ef <= 0) r = (ef == 0 && mant == 0x7fffffu) ? (sign | 0x800000u) : sign;
    if (ef >= 255) r = sign | 0x7f800000u;
    if (ed == 0x7ff) r = sign | 0x7f800000u | ((hi & 0xfffffu) | lo ? 0x400000u : 0u);
    return __uint_as_float(r);
}

// double(x), exact.
__device__ __forceinline__ double f32_to_f64_ftz(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    const unsigned ed = e == 0xffu ? 0x7ffu : e + (1023u - 127u);
    unsigned hi = (u & 0x80000000u) | (ed << 20) | (m >> 3), lo = m << 29;
    if (e == 0) { hi = u & 0x80000000u; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

}  // namespace wcns
