// wcns_fp64.cuh -- the FP64 face computation in one fixed evaluation order.
//
// The FP64 path is the reference-precision path: every operation of a face
// (Roe average and eigenvectors, projection, smoothness indicators and
// cutoff, the convex combination of Eq. 12 with the weights of Eq. 19,
// back-projection, positivity check, midpoint flux), of the MD difference,
// of the SSP-RK3 stage sums and of the CFL rule is evaluated in one
// documented order with round-to-nearest and no contraction into FMA.  The
// result is a deterministic function of the input bits, so a stencil cut
// never depends on incidental rounding and runs are reproducible bit for
// bit.  Terms whose coefficient is an exact zero or one are omitted or
// folded, which leaves every rounded result unchanged.
#pragma once
#include "wcns_device.cuh"
#include "wcns_f64int.cuh"

namespace wcns {

__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dadd_rn(a, -b); }

// Division and square root of the face code: the hardware operations.  The
// integer forms of wcns_f64int.cuh have 2.5x the throughput in isolation and
// make the first steps from initial data 1.36x faster, but on developed 2D
// flow the sweep was 1.23x slower with them (cause not identified yet); they
// serve the per-node code of the scalar solver, where every lane runs the
// same operations (div_int_).  Every form gives the IEEE result.
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double div_int_(double a, double b) { return ddiv_int(a, b); }

// p = (gamma-1) (E - (0.5 * sum m_a^2) / rho), sum taken in axis order.
template <int ND>
__device__ __forceinline__ double pressure_exact(const double* U, double gm1)
{
    double ke = mul_(U[1], U[1]);
#pragma unroll
    for (int a = 1; a < ND; ++a) ke = add_(ke, mul_(U[1 + a], U[1 + a]));
    ke = div_(mul_(0.5, ke), U[0]);
    return mul_(gm1, sub_(U[ND + 1], ke));
}

// Roe-averaged left eigenvectors of dF_d/dU between nodes a and b, in the
// form needed for projection.  Field order: (u_n - c, entropy, shear waves
// of the tangential axes in axis order, u_n + c).
template <int ND>
struct ProjFP64 {
    double vel[ND];
    double q2, H, c, un;
    double l0[ND + 2];   // row of u_n - c
    double l1[ND + 2];   // entropy row
    double lN[ND + 2];   // row of u_n + c
};

template <int ND, int D>
__device__ __forceinline__ void proj_setup_fp64(const double* Ua, const double* Ub, double gm1,
                                                ProjFP64<ND>& P)
{
    const double ra = sqrt_(Ua[0]);
    const double rb = sqrt_(Ub[0]);
    const double Ha = div_(add_(Ua[ND + 1], pressure_exact<ND>(Ua, gm1)), Ua[0]);
    const double Hb = div_(add_(Ub[ND + 1], pressure_exact<ND>(Ub, gm1)), Ub[0]);
    const double den = add_(ra, rb);
    double q2 = 0.0;
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        P.vel[a] = div_(add_(mul_(ra, div_(Ua[1 + a], Ua[0])), mul_(rb, div_(Ub[1 + a], Ub[0]))), den);
        q2 = (a == 0) ? mul_(P.vel[0], P.vel[0]) : add_(q2, mul_(P.vel[a], P.vel[a]));
    }
    P.q2 = q2;
    P.H = div_(add_(mul_(ra, Ha), mul_(rb, Hb)), den);
    const double c2 = mul_(gm1, sub_(P.H, mul_(0.5, q2)));
    P.c = sqrt_(c2);
    P.un = P.vel[D];
    const double b1 = div_(gm1, c2);
    const double b2 = mul_(mul_(0.5, b1), q2);
    const double unc = div_(P.un, P.c);
    const double ic = div_(1.0, P.c);
    P.l0[0] = mul_(0.5, add_(b2, unc));
    P.lN[0] = mul_(0.5, sub_(b2, unc));
    P.l1[0] = sub_(1.0, b2);
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        const double t = mul_(-b1, P.vel[a]);
        P.l0[1 + a] = mul_(0.5, a == D ? sub_(t, ic) : t);
        P.lN[1 + a] = mul_(0.5, a == D ? add_(t, ic) : t);
        P.l1[1 + a] = mul_(b1, P.vel[a]);
    }
    P.l0[ND + 1] = mul_(0.5, b1);
    P.lN[ND + 1] = mul_(0.5, b1);
    P.l1[ND + 1] = -b1;
}

// Characteristic variables of one node, left-to-right sums.
template <int ND, int D>
__device__ __forceinline__ void project_fp64(const ProjFP64<ND>& P, const double* U, double* W)
{
    double s0 = mul_(P.l0[0], U[0]), s1 = mul_(P.l1[0], U[0]), sN = mul_(P.lN[0], U[0]);
#pragma unroll
    for (int v = 1; v < ND + 2; ++v) {
        s0 = add_(s0, mul_(P.l0[v], U[v]));
        s1 = add_(s1, mul_(P.l1[v], U[v]));
        sN = add_(sN, mul_(P.lN[v], U[v]));
    }
    W[0] = s0;
    W[1] = s1;
    int k = 2;
#pragma unroll
    for (int t = 0; t < ND; ++t) {
        if (t == D) continue;
        W[k++] = add_(mul_(-P.vel[t], U[0]), U[1 + t]);
    }
    W[ND + 1] = sN;
}

// Eq. 10, 11, 15 and 16-18 on one stencil s[0..4] = u_{i-2} .. u_{i+2},
// in one fixed order; chi_k is evaluated as s_k / sum s with
// s_k = (g_k / max g)^q, which equals Eq. 17 and cannot overflow.
__device__ __forceinline__ void derivs_fp64(const double s[5], double D1[3], double D2[3],
                                            double beta[3])
{
    D1[0] = mul_(0.5, add_(sub_(s[0], mul_(4.0, s[1])), mul_(3.0, s[2])));
    D1[1] = mul_(0.5, sub_(s[3], s[1]));
    D1[2] = mul_(0.5, sub_(add_(mul_(-3.0, s[2]), mul_(4.0, s[3])), s[4]));
    D2[0] = add_(sub_(s[0], mul_(2.0, s[1])), s[2]);
    D2[1] = add_(sub_(s[1], mul_(2.0, s[2])), s[3]);
    D2[2] = add_(sub_(s[2], mul_(2.0, s[3])), s[4]);
#pragma unroll
    for (int k = 0; k < 3; ++k) beta[k] = add_(mul_(D1[k], D1[k]), mul_(D2[k], D2[k]));
}

__device__ __forceinline__ int select_fp64(const double s[5], const SchemeConst& K, double D1[3],
                                           double D2[3])
{
    double beta[3];
    derivs_fp64(s, D1, D2, beta);
    const double tau = fabs(sub_(beta[0], beta[2]));
    // No stencil can be cut unless the largest gamma exceeds the smallest by
    // the factor (3 C_T)^(-1/q); this bound (with a 2% margin) lets smooth
    // stencils skip the divisions while deciding exactly as the full test.
    const double bmin = fmin(fmin(beta[0], beta[1]), beta[2]) + K.eps;
    if (tau < K.keep_all_K * bmin) return 7;
    // Division-free screen.  With b_k = beta_k + eps and b_m the smallest,
    // r_k = g_k / g_max = (C b_k + tau) b_m / (b_k (C b_m + tau)), and since
    // 1 <= sum_j r_j^q <= 3, r_k^q < C_T (1 - 1e-9) cuts stencil k and
    // r_k^q >= 3 C_T (1 + 1e-9) keeps it, whatever the other stencils.  The
    // 1e-9 margins dwarf the rounding of both this test and the exact form
    // below (a few ulps), so a decision taken here is the one the exact form
    // takes; a stencil inside the band, or a product out of range, goes to
    // the exact form.
    {
        const double cb = K.C * bmin + tau;
        int screened = 7;
        bool open = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double bk = beta[k] + K.eps;
            const double x = (K.C * bk + tau) * bmin, y = bk * cb;
            if (!(isfinite(x) && isfinite(y))) open = true;
            else if (x < K.screen_lo * y) screened &= ~(1 << k);
            else if (!(x >= K.screen_hi * y)) open = true;
        }
        if (!open) return screened;
    }
    double g[3], gmax = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g[k] = add_(K.C, div_(tau, add_(beta[k], K.eps)));
        if (g[k] > gmax) gmax = g[k];
    }
    double sk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double r = div_(g[k], gmax);
        double p = r;
        for (int e = 1; e < K.q; ++e) p = mul_(p, r);
        sk[k] = p;
    }
    const double ssum = add_(add_(sk[0], sk[1]), sk[2]);
    int flags = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (!(div_(sk[k], ssum) < K.CT)) flags |= 1 << k;
    return flags;
}


// Exact convex-combination weights omega_k^(T) of Eq. 19 for every flag word,
// (delta_k d_k) / sum_j delta_j d_j with the sum taken in k order; filled
// from the host (the same IEEE divisions) before the first launch.
static __constant__ double c_omega[8][3];

// Fills this translation unit's copy of c_omega (host side, before launches).
static inline cudaError_t fill_omega_table()
{
    const double d[3] = {1.0 / 16.0, 10.0 / 16.0, 5.0 / 16.0};
    double w[8][3];
    for (int f = 0; f < 8; ++f) {
        double ds = 0.0;
        for (int k = 0; k < 3; ++k) ds += ((f >> k) & 1) ? d[k] : 0.0;
        for (int k = 0; k < 3; ++k) w[f][k] = f == 0 ? d[k] : (((f >> k) & 1) ? d[k] : 0.0) / ds;
    }
    return cudaMemcpyToSymbol(c_omega, w, sizeof w);
}

// Eq. 9 and Eq. 12: u = sum_k omega_k (u_i + D1_k / 2 + D2_k / 8).
__device__ __forceinline__ double interp_fp64(int flags, const double s[5], const double D1[3],
                                              const double D2[3])
{
    double u = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double uk = add_(add_(s[2], mul_(D1[k], 0.5)), mul_(D2[k], 0.125));
        const double w = flags == 7 ? (k == 0 ? 1.0 / 16.0 : (k == 1 ? 10.0 / 16.0 : 5.0 / 16.0))
                                    : c_omega[flags][k];
        u = k == 0 ? mul_(w, uk) : add_(u, mul_(w, uk));
    }
    return u;
}

// u_L of one stencil s[0..4] = u_{i-2} .. u_{i+2} with the weights K.weights
// selects: TENO (flags of Eq. 18, weights of Eq. 19), WCNS-JS (Eq. 14),
// WCNS-Z (alpha_k = d_k (1 + tau_5 / (beta_k + eps)), Borges et al.) or the
// linear weights d_k of Eq. 13.  Eq. 12 with omega_k = alpha_k / sum alpha,
// alpha summed in k order.  flags = 7 for every choice but TENO.
__device__ __forceinline__ double interp_weights_fp64(const double s[5], const SchemeConst& K,
                                                      int& flags)
{
    double D1[3], D2[3];
    if (K.weights == W_TENO) {
        flags = select_fp64(s, K, D1, D2);
        return interp_fp64(flags, s, D1, D2);
    }
    double beta[3];
    derivs_fp64(s, D1, D2, beta);
    flags = 7;
    if (K.weights == W_LINEAR) return interp_fp64(7, s, D1, D2);
    const double d[3] = {1.0 / 16.0, 10.0 / 16.0, 5.0 / 16.0};
    double a[3];
    if (K.weights == W_Z) {
        const double tau = fabs(sub_(beta[0], beta[2]));
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = mul_(d[k], add_(1.0, div_(tau, add_(beta[k], K.eps))));
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double b = add_(beta[k], K.eps_js);
            a[k] = div_(d[k], mul_(b, b));
        }
    }
    const double asum = add_(add_(a[0], a[1]), a[2]);
    double u = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double uk = add_(add_(s[2], mul_(D1[k], 0.5)), mul_(D2[k], 0.125));
        const double w = div_(a[k], asum);
        u = k == 0 ? mul_(w, uk) : add_(u, mul_(w, uk));
    }
    return u;
}

// U = R w with the right eigenvectors (columns): acoustic u_n - c, entropy,
// shear waves, acoustic u_n + c.
template <int ND, int D>
__device__ __forceinline__ void back_project_fp64(const ProjFP64<ND>& P, const double* w, double* U)
{
    constexpr int NV = ND + 2;
    const double c = P.c, un = P.un, H = P.H;
    U[0] = add_(add_(w[0], w[1]), w[NV - 1]);
    int k = 2;
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        const double r0 = a == D ? sub_(P.vel[a], c) : P.vel[a];
        const double rN = a == D ? add_(P.vel[a], c) : P.vel[a];
        double m = add_(mul_(r0, w[0]), mul_(P.vel[a], w[1]));
        if (a != D) m = add_(m, w[k++]);
        U[1 + a] = add_(m, mul_(rN, w[NV - 1]));
    }
    double e = add_(mul_(sub_(H, mul_(un, c)), w[0]), mul_(mul_(0.5, P.q2), w[1]));
    k = 2;
#pragma unroll
    for (int t = 0; t < ND; ++t) {
        if (t == D) continue;
        e = add_(e, mul_(P.vel[t], w[k++]));
    }
    U[NV - 1] = add_(e, mul_(add_(H, mul_(un, c)), w[NV - 1]));
}

// Physical flux in direction D.
template <int ND, int D>
__device__ __forceinline__ void phys_flux_fp64(const double* U, double gm1, double* F)
{
    const double un = div_(U[1 + D], U[0]);
    const double p = pressure_exact<ND>(U, gm1);
    F[0] = U[1 + D];
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = mul_(U[1 + a], un);
    F[1 + D] = add_(F[1 + D], p);
    F[ND + 1] = mul_(add_(U[ND + 1], p), un);
}

// Roe (1981): F = (F(U_L) + F(U_R))/2 - R |Lambda| L (U_R - U_L) / 2 at the Roe
// average of U_L and U_R, with L and R in the same closed form as above.
template <int ND, int D>
__device__ __forceinline__ void roe_flux_fp64(const double* UL, const double* UR, double gm1, double* F)
{
    constexpr int NV = ND + 2;
    double FL[NV], FR[NV], dU[NV], alpha[NV];
    phys_flux_fp64<ND, D>(UL, gm1, FL);
    phys_flux_fp64<ND, D>(UR, gm1, FR);
    ProjFP64<ND> P;
    proj_setup_fp64<ND, D>(UL, UR, gm1, P);
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[v] = sub_(UR[v], UL[v]);
    project_fp64<ND, D>(P, dU, alpha);
    const double c = P.c, un = P.un;
    alpha[0] = mul_(fabs(sub_(un, c)), alpha[0]);
#pragma unroll
    for (int k = 1; k < NV - 1; ++k) alpha[k] = mul_(fabs(un), alpha[k]);
    alpha[NV - 1] = mul_(fabs(add_(un, c)), alpha[NV - 1]);
    double s[NV];
    back_project_fp64<ND, D>(P, alpha, s);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = sub_(mul_(0.5, add_(FL[v], FR[v])), mul_(0.5, s[v]));
}

// van Leer (1982) flux vector splitting, half sgn = +1 (F+) or -1 (F-).
template <int ND, int D>
__device__ __forceinline__ void vanleer_half_fp64(const double* U, double gamma, double gm1, double sgn,
                                                  double* F)
{
    constexpr int NV = ND + 2;
    const double rho = U[0];
    const double p = pressure_exact<ND>(U, gm1);
    const double c = sqrt_(div_(mul_(gamma, p), rho));
    const double un = div_(U[1 + D], rho);
    const double M = div_(un, c);
    if (M >= 1.0 || M <= -1.0) {
        if ((M >= 1.0) == (sgn > 0.0)) {
            phys_flux_fp64<ND, D>(U, gm1, F);
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = 0.0;
        }
        return;
    }
    const double ms = add_(M, sgn);
    const double fm = mul_(mul_(mul_(mul_(mul_(sgn, 0.25), rho), c), ms), ms);
    double t2 = 0.0;
    bool first = true;
#pragma unroll
    for (int a = 0; a < ND; ++a) {
        if (a == D) continue;
        const double va = div_(U[1 + a], rho);
        t2 = first ? mul_(va, va) : add_(t2, mul_(va, va));
        first = false;
    }
    const double wn = add_(mul_(gm1, un), mul_(mul_(sgn, 2.0), c));
    F[0] = fm;
#pragma unroll
    for (int a = 0; a < ND; ++a) F[1 + a] = mul_(fm, div_(U[1 + a], rho));
    F[1 + D] = div_(mul_(fm, wn), gamma);
    const double den = mul_(2.0, sub_(mul_(gamma, gamma), 1.0));
    F[NV - 1] = mul_(fm, add_(div_(mul_(wn, wn), den), mul_(0.5, t2)));
}

// AUSM (Liou and Steffen 1993), one side's split Mach number and pressure
// (s = +1: M+, p+ of the left state; s = -1: M-, p- of the right state).
__device__ __forceinline__ void ausm_split_fp64(double M, double p, double s, double& Ms, double& ps)
{
    if (fabs(M) <= 1.0) {
        const double a = add_(M, s);
        Ms = mul_(mul_(mul_(s, 0.25), a), a);
        ps = mul_(mul_(mul_(mul_(0.25, p), a), a), sub_(2.0, mul_(s, M)));
    } else {
        const double t = add_(M, mul_(s, fabs(M)));
        Ms = mul_(0.5, t);
        ps = div_(mul_(mul_(0.5, p), t), M);
    }
}

// AUSM flux: F = m (Phi_L + Phi_R)/2 - |m| (Phi_R - Phi_L)/2 + (p_L^+ + p_R^-) e_D,
// m = M_L^+ + M_R^-, Phi = rho c (1, u, H), each side with its own c.
template <int ND, int D>
__device__ __forceinline__ void ausm_flux_fp64(const double* UL, const double* UR, double gamma,
                                               double gm1, double* F)
{
    constexpr int NV = ND + 2;
    const double* W[2] = {UL, UR};
    double Phi[2][NV], M[2], p[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const double* X = W[side];
        const double rho = X[0];
        p[side] = pressure_exact<ND>(X, gm1);
        const double c = sqrt_(div_(mul_(gamma, p[side]), rho));
        M[side] = div_(div_(X[1 + D], rho), c);
        const double rc = mul_(rho, c);
        Phi[side][0] = rc;
#pragma unroll
        for (int a = 0; a < ND; ++a) Phi[side][1 + a] = mul_(rc, div_(X[1 + a], rho));
        Phi[side][NV - 1] = mul_(rc, div_(add_(X[NV - 1], p[side]), rho));
    }
    double Mp, pp, Mm, pm;
    ausm_split_fp64(M[0], p[0], 1.0, Mp, pp);
    ausm_split_fp64(M[1], p[1], -1.0, Mm, pm);
    const double m = add_(Mp, Mm);
    const double hm = mul_(0.5, m), ham = mul_(0.5, fabs(m));
#pragma unroll
    for (int v = 0; v < NV; ++v)
        F[v] = sub_(mul_(hm, add_(Phi[0][v], Phi[1][v])), mul_(ham, sub_(Phi[1][v], Phi[0][v])));
    F[1 + D] = add_(F[1 + D], add_(pp, pm));
}

// The whole face j+1/2 from the six nodes u[0..5] = U_{j-2} .. U_{j+3}.
template <int ND, int DIR, int FLUX>
__device__ __forceinline__ void face_fp64(double (&u)[6][ND + 2], const SchemeConst& K, double* F,
                                          uint8_t* fl, bool& fell_back)
{
    constexpr int NV = ND + 2;
    const double gm1 = K.gm1;
    ProjFP64<ND> P;
    proj_setup_fp64<ND, DIR>(u[2], u[3], gm1, P);
    double Uj[NV], Uj1[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { Uj[v] = u[2][v]; Uj1[v] = u[3][v]; }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        double W[NV];
        project_fp64<ND, DIR>(P, u[m], W);
#pragma unroll
        for (int v = 0; v < NV; ++v) u[m][v] = W[v];
    }
    double wL[NV], wR[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double sl[5], sr[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) { sl[m] = u[m][k]; sr[m] = u[5 - m][k]; }
        int fL, fR;
        wL[k] = interp_weights_fp64(sl, K, fL);
        wR[k] = interp_weights_fp64(sr, K, fR);
        fl[k] = (uint8_t)(fL | (fR << 3));
    }
    double UL[NV], UR[NV];
    back_project_fp64<ND, DIR>(P, wL, UL);
    back_project_fp64<ND, DIR>(P, wR, UR);
    if (!(UL[0] > 0.0) || !(UR[0] > 0.0) || !(pressure_exact<ND>(UL, gm1) > 0.0) ||
        !(pressure_exact<ND>(UR, gm1) > 0.0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { UL[v] = Uj[v]; UR[v] = Uj1[v]; }
        fell_back = true;
    }
    if (FLUX == 0) {
        roe_flux_fp64<ND, DIR>(UL, UR, gm1, F);
    } else if (FLUX == 2) {
        ausm_flux_fp64<ND, DIR>(UL, UR, K.gamma, gm1, F);
    } else {
        double Fp[NV], Fm[NV];
        vanleer_half_fp64<ND, DIR>(UL, K.gamma, gm1, 1.0, Fp);
        vanleer_half_fp64<ND, DIR>(UR, K.gamma, gm1, -1.0, Fm);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = add_(Fp[v], Fm[v]);
    }
}

// Eq. 4 or 5 for one node and variable from the midpoint fluxes
// f0..f5 = f_{i-5/2} .. f_{i+5/2} and the node-flux differences
// d1 = f_{i+1} - f_{i-1}, d2 = f_{i+2} - f_{i-2} (sums left to right);
// returns the derivative times h.
__device__ __forceinline__ double diff_alt_fp64(int diff, double f1, double f2, double f3, double f4,
                                                double d1, double d2)
{
    if (diff == DIFF_HWCNS)
        return add_(add_(mul_(HW_B1, sub_(f3, f2)), mul_(HW_B2, d1)), mul_(HW_B3, d2));
    return add_(add_(mul_(MND_C1, sub_(f3, f2)), mul_(MND_C2, d1)), mul_(MND_C3, sub_(f4, f1)));
}

// Eq. 3 for one node and variable: fp = (a1 d1 + a2 d2) + a3 d3; returns fp / h
// as fp * (1/h).
__device__ __forceinline__ double md_fp64(double f0, double f1, double f2, double f3, double f4,
                                          double f5, double ih)
{
    const double fp = add_(add_(mul_(MD_A1, sub_(f3, f2)), mul_(MD_A2, sub_(f4, f1))),
                           mul_(MD_A3, sub_(f5, f0)));
    return mul_(fp, ih);
}

}  // namespace wcns
