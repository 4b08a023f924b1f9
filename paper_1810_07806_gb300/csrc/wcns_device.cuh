// wcns_device.cuh -- device building blocks of the TCNS sweep (sm_103a).
//
// Per face j+1/2 of one grid line the sweep computes (arXiv 1810.07806):
//   Roe-averaged eigen-system of the two bounding nodes (Sec. 3: the
//   interpolation runs on characteristic variables),
//   characteristic variables of the six stencil nodes j-2 .. j+3,
//   per field: smoothness indicators beta_k (Eq. 10, 11, 15), the TENO
//   scale separation gamma_k (Eq. 16), normalisation chi_k (Eq. 17) and
//   cutoff delta_k (Eq. 18) for the left-biased stencil and its mirror,
//   the interpolated value from the equivalent five-point stencil of the
//   retained set (Table 1; Eq. 12 with the weights of Eq. 19),
//   back-projection, and the Roe or van Leer midpoint flux.
// The node update is the sixth-order MD difference of Eq. 3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "wcns_cvt.cuh"

namespace wcns {

constexpr int GHOST = 5;   // node i reads nodes i-5 .. i+5

// Eq. 3 coefficients from sixth-order Taylor matching:
// sum a_m (2m-1) = 1, sum a_m (2m-1)^3 = 0, sum a_m (2m-1)^5 = 0.
constexpr double MD_A1 = 75.0 / 64.0;
constexpr double MD_A2 = -25.0 / 384.0;
constexpr double MD_A3 = 3.0 / 640.0;
// Eq. 4 (HWCNS: midpoints i+-1/2, nodes i+-1, i+-2) and Eq. 5 (MND: midpoints
// i+-1/2, nodes i+-1, midpoints i+-3/2), by the same sixth-order matching.
constexpr double HW_B1 = 64.0 / 45.0;
constexpr double HW_B2 = -2.0 / 9.0;
constexpr double HW_B3 = 1.0 / 180.0;
constexpr double MND_C1 = 3.0 / 2.0;
constexpr double MND_C2 = -3.0 / 10.0;
constexpr double MND_C3 = 1.0 / 30.0;
// Midpoint-to-node formulas (values of the C ABI's WCNS_DIFF_*).
enum { DIFF_MD = 0, DIFF_HWCNS = 1, DIFF_MND = 2 };

// Table 1: coefficients (a_{i-2} .. a_{i+2}) of the single five-point
// stencil equivalent to each retained set, indexed by the flag word
// delta_1 | delta_2 << 1 | delta_3 << 2.  Index 0 (nothing retained) cannot
// occur because the largest chi_k is at least 1/3; it maps to S_0*.
#define WCNS_TABLE1_ROWS                                                   \
    {{3.0 / 128, -5.0 / 32, 45.0 / 64, 15.0 / 32, -5.0 / 128},  /* -    */ \
     {3.0 / 8, -5.0 / 4, 15.0 / 8, 0.0, 0.0},                   /* 100  */ \
     {0.0, -1.0 / 8, 3.0 / 4, 3.0 / 8, 0.0},                    /* 010  */ \
     {3.0 / 88, -5.0 / 22, 75.0 / 88, 15.0 / 44, 0.0},          /* 110  */ \
     {0.0, 0.0, 3.0 / 8, 3.0 / 4, -1.0 / 8},                    /* 001  */ \
     {1.0 / 16, -5.0 / 24, 5.0 / 8, 5.0 / 8, -5.0 / 48},        /* 101  */ \
     {0.0, -1.0 / 12, 5.0 / 8, 1.0 / 2, -1.0 / 24},             /* 011  */ \
     {3.0 / 128, -5.0 / 32, 45.0 / 64, 15.0 / 32, -5.0 / 128}}  /* 111  */
static __constant__ double c_table1_f64[8][5] = WCNS_TABLE1_ROWS;
static __constant__ float c_table1_f32[8][5] = WCNS_TABLE1_ROWS;

// Weight functions of the node-to-midpoint interpolation (values of the
// C ABI's WCNS_W_*).
enum { W_TENO = 0, W_JS = 1, W_LINEAR = 2, W_Z = 3 };

struct SchemeConst {
    double gamma, gm1;
    double C, eps, CT;
    int q;
    int weights;         // W_TENO | W_JS | W_LINEAR | W_Z
    double eps_js;       // epsilon of Eq. 14
    int diff;            // DIFF_MD | DIFF_HWCNS | DIFF_MND
    float sqrt_eps_jsf;  // sqrt(eps of Eq. 14) in float, for the FP32 rescaled JS eps
    double keep_all_K;   // tau < K * (min beta + eps) guarantees no cut (exact test)
    double screen_lo;    // (C_T (1 - 1e-9))^(1/q) (1 - 1e-9): g_k / g_max below it cuts
    double screen_hi;    // (3 C_T (1 + 1e-9))^(1/q) (1 + 1e-9): at or above it keeps
    float Cf, CTf, Kf;
    float gammaf, gm1f;  // gamma, gamma - 1 in float
};

// The FP32 path's reference state U_r = (rho_r, 0, .., 0, E_r), p_r =
// (gamma - 1) E_r, H_r = E_r + p_r, as the face code uses it (all zero: the
// plain form).  Stage values are u = U - U_r.  Projection, selection and
// interpolation are linear in u up to the selection's rescaling, so they run
// on u directly; the fluxes need rho = u_rho + rho_r, the pressure difference
// p - p_r = (gamma - 1)(u_E - |m|^2 / (2 rho)) (m_r = 0) and
// E + p = u_E + (p - p_r) + H_r.
struct Ref32 {
    float rho, e, p, h;
};

// FP32 reciprocal: the hardware approximation (PTX rcp.approx.ftz.f32, at
// most 1 ulp from 1/x over the full range).  Every argument in the FP32 path
// is a normal number (rescaled indicators are floored at FLT_MIN, densities
// and sound speeds are positive), so flushing subnormals changes nothing.
__device__ __forceinline__ float rcpf(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32 reciprocal square root: PTX rsqrt.approx.ftz.f32 (relative error
// below 2^-22).  sqrt(x) is formed as x * rsqrtf_a(x) where both are needed.
__device__ __forceinline__ float rsqrtf_a(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Eq. 12 with the comparison weights (FP32), both biased values of one
// characteristic field from its six values s[0..5] = w_{j-2} .. w_{j+3}.
// The values are rescaled by sc = max |s| (floored at FLT_MIN) as for the
// TENO cut, so beta_k and tau are O(1) and eps becomes eps / sc^2.  With
// b_k = beta_k + eps and b_m = min b:
//   WCNS-Z  (alpha_k = d_k (1 + tau_5 / b_k)):  omega_k ~ d_k (b_m/b_k)(b_k + tau)/(b_m + tau)
//   WCNS-JS (Eq. 14, alpha_k = d_k / b_k^2):    omega_k ~ d_k (b_m / b_k)^2
// (alpha_k divided by its value at b_m: every factor is bounded, nothing
// overflows); the JS eps is clamped to [FLT_MIN, 1e30], where the weights
// are already the linear ones.  Linear: omega_k = d_k, i.e. Eq. 7.
template <int WT>
__device__ __forceinline__ void weights_pair_fp32(const float s[6], float sqrt_eps, const SchemeConst& K,
                                                  float& uL, float& uR)
{
    float sc = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) sc = fmaxf(sc, fabsf(s[m]));
    sc = fmaxf(sc, 1.17549435e-38f);
    const float inv = rcpf(sc);
    float t[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) t[m] = s[m] * inv;
    const float a2 = fmaf(-2.0f, t[1], t[0]) + t[2];
    const float b2 = fmaf(-2.0f, t[2], t[1]) + t[3];
    const float c2 = fmaf(-2.0f, t[3], t[2]) + t[4];
    const float d2 = fmaf(-2.0f, t[4], t[3]) + t[5];
    const float D1L[3] = {0.5f * fmaf(3.0f, t[2], fmaf(-4.0f, t[1], t[0])), 0.5f * (t[3] - t[1]),
                          0.5f * (fmaf(4.0f, t[3], -3.0f * t[2]) - t[4])};
    const float D2L[3] = {a2, b2, c2};
    const float D1R[3] = {0.5f * fmaf(3.0f, t[3], fmaf(-4.0f, t[4], t[5])), 0.5f * (t[2] - t[4]),
                          0.5f * (fmaf(4.0f, t[2], -3.0f * t[3]) - t[1])};
    const float D2R[3] = {d2, c2, b2};
    const float d[3] = {1.0f / 16.0f, 10.0f / 16.0f, 5.0f / 16.0f};
    float eps_s;
    if constexpr (WT == W_JS) {
        const float e = K.sqrt_eps_jsf * inv;
        eps_s = fminf(fmaxf(e * e, 1.17549435e-38f), 1e30f);
    } else {
        const float e = sqrt_eps * inv;
        eps_s = fmaxf(e * e, 1.17549435e-38f);
    }
    auto side = [&](const float* D1, const float* D2, float centre) {
        float w[3];
        if constexpr (WT == W_LINEAR) {
#pragma unroll
            for (int k = 0; k < 3; ++k) w[k] = d[k];
        } else {
            float b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) b[k] = fmaf(D1[k], D1[k], D2[k] * D2[k]) + eps_s;
            const float bm = fminf(fminf(b[0], b[1]), b[2]);
            if constexpr (WT == W_Z) {
                const float tau = fabsf(b[0] - b[2]);
                const float den = rcpf(bm + tau);
#pragma unroll
                for (int k = 0; k < 3; ++k) w[k] = d[k] * (bm * rcpf(b[k])) * ((b[k] + tau) * den);
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float r = bm * rcpf(b[k]);
                    w[k] = d[k] * r * r;
                }
            }
            const float iw = rcpf(w[0] + w[1] + w[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) w[k] *= iw;
        }
        float u = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) u = fmaf(w[k], fmaf(0.125f, D2[k], fmaf(0.5f, D1[k], centre)), u);
        return u * sc;
    };
    uL = side(D1L, D2L, t[2]);
    uR = side(D1R, D2R, t[3]);
}

// Eq. 12 with the weights of Eq. 19, as the equivalent Table-1 stencil.
// The all-retained row (Eq. 7) is inlined; reduced rows come from constant
// memory (only cut faces take that branch).
template <typename T>
__device__ __forceinline__ T interp_row(int flags, const T s[5])
{
    if (flags == 7) {
        T u = T(3.0 / 128) * s[0];
        u = fma(T(-5.0 / 32), s[1], u);
        u = fma(T(45.0 / 64), s[2], u);
        u = fma(T(15.0 / 32), s[3], u);
        return fma(T(-5.0 / 128), s[4], u);
    }
    const T* row;
    if constexpr (sizeof(T) == 8) row = c_table1_f64[flags];
    else row = c_table1_f32[flags];
    T u = row[0] * s[0];
#pragma unroll
    for (int j = 1; j < 5; ++j) u = fma(row[j], s[j], u);
    return u;
}

// ------------------------------------------------------------------------
// Paired FP32 arithmetic (Blackwell packed f32x2 instructions).  The left-
// and right-biased halves of a face, and mirrored node pairs (m, 5 - m), run
// the same operations on different data; carrying them in the two lanes of
// a float2 halves the instructions issued for that work.
// ------------------------------------------------------------------------
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.f), a); }

// FP32 cutoff (Eq. 16-18) of both biased stencils of a field at once, from
// their rescaled indicators (lane x: left, lane y: right).  chi_k is
// invariant under s -> s/sc except through eps, so the stencil values are
// rescaled (beta, tau become O(1) and cannot underflow) and eps becomes
// max(eps/sc^2, FLT_MIN).  Per lane: the exact no-cut test first (also tau ==
// 0); if either side may cut, the ratio form runs for both lanes in packed
// arithmetic.  With b_k = beta_k + eps and m = argmin b (the largest gamma),
// g_k / g_m = (b_m / b_k)(C b_k + tau)/(C b_m + tau), every factor bounded (the
// literal tau / b_k overflows FP32 when b_k sits at the eps floor), and
// chi_k < C_T is tested as s_k < C_T sum s with s_k = (g_k / g_m)^q.  A side
// that passed the no-cut test keeps its 7.
__device__ __forceinline__ void cut_x2(float2 B0, float2 B1, float2 B2, float eps_s, const SchemeConst& K,
                                       int& fL, int& fR)
{
    const float2 d02 = sub2(B0, B2);
    const float tauL = fabsf(d02.x), tauR = fabsf(d02.y);
    const float bmL = fminf(fminf(B0.x, B1.x), B2.x) + eps_s;
    const float bmR = fminf(fminf(B0.y, B1.y), B2.y) + eps_s;
    const bool cutL = tauL >= K.Kf * bmL, cutR = tauR >= K.Kf * bmR;
    fL = fR = 7;
    if (!(cutL || cutR)) return;
    const float2 tau = make_float2(tauL, tauR), bm = make_float2(bmL, bmR);
    const float2 e2 = bc2(eps_s), C2 = bc2(K.Cf);
    const float2 b[3] = {add2(B0, e2), add2(B1, e2), add2(B2, e2)};
    const float2 den = make_float2(rcpf(fmaf(K.Cf, bmL, tauL)), rcpf(fmaf(K.Cf, bmR, tauR)));
    float2 sk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 rb = make_float2(rcpf(b[k].x), rcpf(b[k].y));
        float2 r = mul2(mul2(bm, rb), mul2(fma2(C2, b[k], tau), den));
        r = make_float2(fminf(1.0f, r.x), fminf(1.0f, r.y));
        float2 pw;
        if (K.q == 6) {
            const float2 r2 = mul2(r, r);
            pw = mul2(mul2(r2, r2), r2);
        } else {
            pw = r;
            for (int e = 1; e < K.q; ++e) pw = mul2(pw, r);
        }
        sk[k] = pw;
    }
    const float2 lim = mul2(bc2(K.CTf), add2(add2(sk[0], sk[1]), sk[2]));
    int l = 0, rr = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!(sk[k].x < lim.x)) l |= 1 << k;
        if (!(sk[k].y < lim.y)) rr |= 1 << k;
    }
    if (cutL) fL = l;
    if (cutR) fR = rr;
}

// Both biased selections and interpolations of one characteristic field,
// paired: S0 = (w_{j-2}, w_{j+3}), S1 = (w_{j-1}, w_{j+2}), S2 = (w_j, w_{j+1})
// are the left stencil's s0..s2 in .x and the mirrored right stencil's in
// .y (s3, s4 are the swapped S2, S1).  The six values are rescaled once by
// 1/sc, sc = max |s| (floored at FLT_MIN so an all-zero field keeps every
// stencil without a branch), and the second differences the mirrored
// stencils share are formed once.  Returns (u_L, u_R) and the two flag words.
// FAST: only the exact no-cut test runs; a side it cannot settle sets
// `slow` (the caller then evaluates the face again with FAST off, where the
// same test sends that side to the full cutoff), and the returned value is
// Eq. 7, which is then also the full path's value whenever slow stays clear.
template <bool FAST>
__device__ __forceinline__ float2 select_interp_x2(float2 S0, float2 S1, float2 S2, float sqrt_eps,
                                                   const SchemeConst& K, int& fL, int& fR, bool& slow)
{
    float sc = fmaxf(fmaxf(fmaxf(fabsf(S0.x), fabsf(S0.y)), fmaxf(fabsf(S1.x), fabsf(S1.y))),
                     fmaxf(fabsf(S2.x), fabsf(S2.y)));
    sc = fmaxf(sc, 1.17549435e-38f);
    const float inv = rcpf(sc);
    const float e = sqrt_eps * inv;
    const float eps_s = fmaxf(e * e, 1.17549435e-38f);
    const float2 iv = bc2(inv);
    const float2 T0 = mul2(S0, iv), T1 = mul2(S1, iv), T2 = mul2(S2, iv);
    const float2 T3 = swap2(T2), T4 = swap2(T1);
    // second differences (left a2, b2, c2 / right d2, c2, b2) and first (Eq. 10-11)
    const float2 D20 = add2(fma2(bc2(-2.f), T1, T0), T2);
    const float2 D21 = add2(fma2(bc2(-2.f), T2, T1), T3);
    const float2 D22 = add2(fma2(bc2(-2.f), T3, T2), T4);
    const float2 D10 = mul2(bc2(0.5f), fma2(bc2(3.f), T2, fma2(bc2(-4.f), T1, T0)));
    const float2 D11 = mul2(bc2(0.5f), sub2(T3, T1));
    const float2 D12 = mul2(bc2(0.5f), sub2(fma2(bc2(4.f), T3, mul2(bc2(-3.f), T2)), T4));
    const float2 B0 = fma2(D10, D10, mul2(D20, D20));   // Eq. 15
    const float2 B1 = fma2(D11, D11, mul2(D21, D21));
    const float2 B2 = fma2(D12, D12, mul2(D22, D22));
    if constexpr (FAST) {
        // the no-cut test of cut_x2, the same expressions
        const float2 d02 = sub2(B0, B2);
        const float bmL = fminf(fminf(B0.x, B1.x), B2.x) + eps_s;
        const float bmR = fminf(fminf(B0.y, B1.y), B2.y) + eps_s;
        if (fabsf(d02.x) >= K.Kf * bmL || fabsf(d02.y) >= K.Kf * bmR) slow = true;
        fL = fR = 7;
    } else {
        cut_x2(B0, B1, B2, eps_s, K, fL, fR);
    }
    if (FAST || (fL & fR) == 7) {                         // Eq. 7 on both sides
        float2 u = mul2(bc2(3.0f / 128), S0);
        u = fma2(bc2(-5.0f / 32), S1, u);
        u = fma2(bc2(45.0f / 64), S2, u);
        u = fma2(bc2(15.0f / 32), swap2(S2), u);
        return fma2(bc2(-5.0f / 128), swap2(S1), u);
    }
    const float sl[5] = {S0.x, S1.x, S2.x, S2.y, S1.y};
    const float sr[5] = {S0.y, S1.y, S2.y, S2.x, S1.x};
    return make_float2(interp_row<float>(fL, sl), interp_row<float>(fR, sr));
}

// ------------------------------------------------------------------------
// Euler primitives and midpoint fluxes (FP32 path; the FP64 path has its own
// in the oracle's operation order).  Every multiply-add is written out as
// fmaf or as separate operations: the FP32 units compile without
// contraction, so all instances of this code round identically.
// ------------------------------------------------------------------------
// pressure_ir takes 1 / rho.  On a state relative to the reference
// (u_E = E - E_r, m_r = 0) it gives p - p_r.
template <int ND>
__device__ __forceinline__ float pressure_ir(const float* U, float ir, float gm1)
{
    float m2 = U[1] * U[1];
#pragma unroll
    for (int a = 1; a < ND; ++a) m2 = fmaf(U[1 + a], U[1 + a], m2);
    return gm1 * fmaf(-0.5f * m2, ir, U[ND + 1]);
}

// (rho_r: the reference density the state is measured from, 0 for a full state)
template <int ND>
__device__ __forceinline__ float pressure_of(const float* U, float gm1, float rho_r = 0.f)
{
    return pressure_ir<ND>(U, rcpf(U[0] + rho_r), gm1);
}

// Physical flux of a full state U with pressure p.
template <int ND, int D>
__device__ __forceinline__ void phys_flux(const float* U, float p, float* F)
{
    const float un = U[1 + D] * rcpf(U[0]);
    F[0] = U[1 + D];
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = U[1 + a] * un;
    F[1 + D] = fmaf(U[1 + D], un, p);
    F[ND + 1] = (U[ND + 1] + p) * un;
}

// The same flux of a state u = U - U_r with p' = p - p_r: the momentum flux
// carries p' (the constant p_r cancels in every difference of fluxes), the
// energy flux (E + p) u_n = (u_E + p' + H_r) u_n.
template <int ND, int D>
__device__ __forceinline__ void phys_flux_ref(const float* U, float pr, const Ref32& R, float* F)
{
    const float un = U[1 + D] * rcpf(U[0] + R.rho);
    F[0] = U[1 + D];
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = U[1 + a] * un;
    F[1 + D] = fmaf(U[1 + D], un, pr);
    F[ND + 1] = ((U[ND + 1] + pr) + R.h) * un;
}

// Roe (1981) flux difference splitting, F = (F_L + F_R - sum |lam_k| alpha_k r_k)/2
// with the wave strengths alpha_k of the Roe-averaged state.  UL, UR are
// states relative to the reference U_r (Ref32) and pL, pR their p - p_r;
// rL, rR are 1 / sqrt(rho) of the full densities: sqrt(rho) = rho r,
// 1 / rho = r^2, and the Roe weights sqrt(rho)/rho are r itself.  The
// momentum flux carries p - p_r (a constant offset of every face's flux,
// which the differences of Eq. 3-5 remove); differences of states and
// pressures are those of the full ones.
template <int ND, int D>
__device__ __forceinline__ void roe_flux(const float* UL, const float* UR, float pL, float pR, float rL,
                                         float rR, float gm1, const Ref32& R, float* F)
{
    constexpr int NV = ND + 2;
    const float iL = rL * rL, iR = rR * rR;
    const float unL = UL[1 + D] * iL, unR = UR[1 + D] * iR;
    float FL[NV], FR[NV];
    FL[0] = UL[1 + D];
    FR[0] = UR[1 + D];
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        FL[1 + a] = UL[1 + a] * unL;
        FR[1 + a] = UR[1 + a] * unR;
    }
    FL[1 + D] = fmaf(UL[1 + D], unL, pL);
    FR[1 + D] = fmaf(UR[1 + D], unR, pR);
    const float eL = (UL[ND + 1] + pL) + R.h, eR = (UR[ND + 1] + pR) + R.h;   // E + p
    FL[ND + 1] = eL * unL;
    FR[ND + 1] = eR * unR;
    const float sL = (UL[0] + R.rho) * rL, sR = (UR[0] + R.rho) * rR;
    const float w = rcpf(sL + sR);
    float vel[ND], dv[ND], q2 = 0.f;
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        vel[a] = fmaf(UL[1 + a], rL, UR[1 + a] * rR) * w;
        dv[a] = fmaf(UR[1 + a], iR, -UL[1 + a] * iL);
        q2 = fmaf(vel[a], vel[a], q2);
    }
    const float H = fmaf(eL, rL, eR * rR) * w;
    const float c2 = gm1 * fmaf(-0.5f, q2, H);
    const float rc = rsqrtf_a(c2);
    const float c = c2 * rc;
    const float ic2 = rc * rc;
    const float rho = sL * sR;
    const float un = vel[D];
    const float drho = UR[0] - UL[0], dp = pR - pL;
    const float rcdv = rho * c * dv[D];
    const float a0 = 0.5f * (dp - rcdv) * ic2;
    const float aN = 0.5f * (dp + rcdv) * ic2;
    const float a1 = fmaf(-dp, ic2, drho);
    const float l0 = fabsf(un - c) * a0, l1 = fabsf(un) * a1, lN = fabsf(un + c) * aN;
    const float lt = fabsf(un) * rho;
    const float dl = lN - l0;
    // sum of |lam_k| alpha_k r_k
    float Dm[NV];
    Dm[0] = (l0 + l1) + lN;
#pragma unroll
    for (int a = 0; a < ND; ++a) Dm[1 + a] = fmaf(vel[a], Dm[0], a == D ? c * dl : lt * dv[a]);
    float e = fmaf(H, l0 + lN, fmaf(un * c, dl, 0.5f * q2 * l1));
#pragma unroll
    for (int a = 0; a < ND; ++a)
        if (a != D) e = fmaf(vel[a], lt * dv[a], e);
    Dm[ND + 1] = e;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = 0.5f * ((FL[v] + FR[v]) - Dm[v]);
}

// AUSM (Liou and Steffen 1993): interface Mach number M_L^+ + M_R^- and
// pressure p_L^+ + p_R^- (second- and third-degree Mach polynomials for
// |M| <= 1, upwind values outside), each side with its own speed of sound;
// F = m (Phi_L + Phi_R)/2 - |m| (Phi_R - Phi_L)/2 + p_n e_D with
// Phi = rho c (1, u, H).
__device__ __forceinline__ void ausm_split(float M, float p, float s, float& Ms, float& ps)
{
    if (fabsf(M) <= 1.f) {
        const float Mps = M + s;
        const float a = Mps * Mps;
        Ms = s * 0.25f * a;
        ps = 0.25f * p * a * fmaf(-s, M, 2.f);
    } else {
        const float a = 0.5f * fmaf(s, fabsf(M), M);
        Ms = a;
        ps = p * a / M;
    }
}

// (full states UL, UR with their pressures)
template <int ND, int D>
__device__ __forceinline__ void ausm_flux(const float* UL, const float* UR, float pL, float pR, float gamma,
                                          float* F)
{
    constexpr int NV = ND + 2;
    const float iL = 1.f / UL[0], iR = 1.f / UR[0];
    const float cL = sqrtf(gamma * pL * iL), cR = sqrtf(gamma * pR * iR);
    const float ML = UL[1 + D] * iL / cL, MR = UR[1 + D] * iR / cR;
    float Mp, pp, Mm, pm;
    ausm_split(ML, pL, 1.f, Mp, pp);
    ausm_split(MR, pR, -1.f, Mm, pm);
    const float m = Mp + Mm;
    // per-side weights of rho c: (m + |m|)/2 on the left, (m - |m|)/2 on the right
    const float wl = 0.5f * (m + fabsf(m)) * cL, wr = 0.5f * (m - fabsf(m)) * cR;
    F[0] = fmaf(wl, UL[0], wr * UR[0]);
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = fmaf(wl, UL[1 + a], wr * UR[1 + a]);
    F[1 + D] = F[1 + D] + (pp + pm);
    F[NV - 1] = fmaf(wl, UL[NV - 1] + pL, wr * (UR[NV - 1] + pR));
}

// van Leer (1982) flux vector splitting: F = F+(U_L) + F-(U_R) (full states).
template <int ND, int D>
__device__ __forceinline__ void vanleer_half(const float* U, float p, float gamma, float gm1, float sgn, float* F)
{
    constexpr int NV = ND + 2;
    const float ir = 1.f / U[0];
    const float c = sqrtf(gamma * p * ir);
    const float un = U[1 + D] * ir;
    const float M = un / c;
    if (M >= 1.f || M <= -1.f) {
        if ((M >= 1.f) == (sgn > 0.f)) {
            phys_flux<ND, D>(U, p, F);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = 0.f;
        }
        return;
    }
    const float Ms = M + sgn;
    const float fm = sgn * 0.25f * U[0] * c * Ms * Ms;
    float t2 = 0.f;
#pragma unroll
    for (int a = 0; a < ND; ++a)
        if (a != D) t2 = fmaf(U[1 + a] * ir, U[1 + a] * ir, t2);
    const float wn = fmaf(gm1, un, sgn * 2.f * c);
    F[0] = fm;
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = fm * (U[1 + a] * ir);
    F[1 + D] = fm * wn / gamma;
    F[NV - 1] = fm * fmaf(0.5f, t2, wn * wn / (2.f * fmaf(gamma, gamma, -1.f)));
}

}  // namespace wcns
