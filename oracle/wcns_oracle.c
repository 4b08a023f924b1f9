/*
 * wcns_oracle.c -- plain, slow FP64 CPU oracle of the TCNS scheme
 * (fifth-order WCNS with TENO-style ENO-like stencil selection) of
 * Zhang, Zhang & Xu, "Towards optimal high-order compact schemes for
 * simulating compressible flows" (arXiv 1810.07806).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that
 * the CUDA library is compared against.  Only the test suite, the package
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA
 * contraction, so every product and sum below rounds as written).
 *
 * What it computes, step by step, in the paper's order:
 *   Eq. 2    du_i/dt = -f'_i, summed over directions (dimension by dimension)
 *   Eq. 3    sixth-order explicit midpoint-to-node difference (MD)
 *   Eq. 4-5  the HWCNS and MND alternatives (midpoint and node fluxes)
 *   Eq. 6    scalar upwind midpoint flux (scalar problems)
 *   Eq. 8-11 three 3-point sub-stencils and their Taylor interpolants
 *   Eq. 12-13 convex combination, optimal weights d = (1, 10, 5)/16
 *   Eq. 14-15 Jiang-Shu weights and the WCNS smoothness indicator beta_k
 *   WCNS-Z   the comparison scheme of Sec. 3, weights of Borges et al.
 *            (cited, not printed): alpha_k = d_k (1 + tau_5 / (beta_k + eps))
 *   Eq. 16-19 TENO scale separation gamma_k, normalisation chi_k, sharp
 *            cutoff delta_k, and the final weights omega_k^(T)
 *   Sec. 3   characteristic-variable interpolation, ideal gas, van Leer,
 *            Roe or AUSM midpoint flux (Sec. 1 names all three), third-order
 *            SSP Runge-Kutta under a CFL rule.
 *
 * Readings of points the paper leaves open (each one is listed in the
 * design notes with its reason):
 *   - MD coefficients a = (75/64, -25/384, 3/640): sixth-order Taylor
 *     matching of Eq. 3 (the paper defers them to its references); by the
 *     same matching b = (64/45, -2/9, 1/180) for Eq. 4 and
 *     c = (3/2, -3/10, 1/30) for Eq. 5.  The node fluxes of Eq. 4-5 are the
 *     physical fluxes of the node states.
 *   - AUSM is the original advection upstream splitting of Liou and
 *     Steffen (1993): interface Mach number M_L^+ + M_R^- and pressure
 *     p_L^+ + p_R^- from the second- and third-degree Mach polynomials,
 *     each side with its own speed of sound, the convected vector upwinded
 *     by the sign of the interface Mach number.
 *   - The characteristic projection uses the eigenvectors of the flux
 *     Jacobian at the Roe average of the two nodes that bound the face; the
 *     same projection serves the left- and right-biased interpolations.
 *   - The right-biased value u_R at face j+1/2 is the left-biased procedure
 *     applied to the mirrored stencil (u_{j+3}, u_{j+2}, u_{j+1}, u_j, u_{j-1}).
 *   - chi_k is evaluated in a ratio form (divide every gamma by the largest
 *     before the q-th power), algebraically identical to Eq. 17 but free of
 *     overflow; the literal form is also evaluated and the two must agree
 *     where the literal form is finite.  delta_k = 0 iff chi_k < C_T.
 *   - SSP-RK3 in Shu-Osher form; dt = CFL / max_i sum_d (|u_d| + c)/h_d.
 *   - Transmissive boundaries copy the boundary node into 5 ghost nodes;
 *     periodic boundaries wrap.  Reflecting walls (Sec. 3.9, Rayleigh-Taylor)
 *     sit on the face outside the boundary node: ghost -1-k mirrors node k
 *     with the normal momentum negated.  Fixed-state boundaries fill every
 *     ghost node with the given state.
 *   - A body force g per unit mass adds (0, rho g, rho u.g) to the RHS
 *     (Sec. 3.9: g = (0, 1)), after the directions are summed.
 *   - If an interpolated midpoint state has rho <= 0 or p <= 0 the face
 *     falls back to first order (U_L = U_j, U_R = U_{j+1}) and is counted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_MAXV 5
#define ORA_GHOST 5

/* Scheme switches (the oracle's own numbering). */
enum { ORA_FLUX_ROE = 0, ORA_FLUX_VANLEER = 1, ORA_FLUX_AUSM = 2 };
enum { ORA_DIFF_MD = 0, ORA_DIFF_HWCNS = 1, ORA_DIFF_MND = 2 };
/* Boundary kinds per side; AUTO follows periodic[] (periodic or transmissive). */
enum { ORA_BC_AUTO = 0, ORA_BC_REFLECT = 2, ORA_BC_FIXED = 3 };
enum { ORA_W_TENO = 0, ORA_W_JS = 1, ORA_W_LINEAR = 2, ORA_W_Z = 3 };

typedef struct {
    int ndim;             /* 1, 2 or 3                                   */
    int n[3];             /* nodes per direction (x, y, z)               */
    double h[3];          /* node spacing per direction                  */
    int periodic[3];      /* 1 = periodic, 0 = transmissive              */
    double gamma;         /* ratio of specific heats                     */
    int flux;             /* ORA_FLUX_*                                  */
    int weights;          /* ORA_W_*                                     */
    double C, eps, CT;    /* Eq. 16, 18: 1, 1e-40, 1e-5                  */
    int q;                /* Eq. 16: 6                                   */
    double eps_js;        /* Eq. 14: 1e-6                                */
    int characteristic;   /* 1 = interpolate characteristic variables    */
    int diff;             /* ORA_DIFF_*: Eq. 3, 4 or 5                   */
    int bc_lo[3], bc_hi[3];               /* ORA_BC_* per axis side      */
    double bc_state[3][2][ORA_MAXV];      /* conserved state, FIXED sides */
    double gravity[3];                    /* body force per unit mass    */
} ora_cfg;

/* ------------------------------------------------------------------ */
/* Eq. 3: the MD coefficients from sixth-order Taylor matching.        */
/* sum a_m (2m-1) = 1, sum a_m (2m-1)^3 = 0, sum a_m (2m-1)^5 = 0.     */
/* ------------------------------------------------------------------ */
static const double MD_A1 = 75.0 / 64.0;
static const double MD_A2 = -25.0 / 384.0;
static const double MD_A3 = 3.0 / 640.0;

void ora_md_coeffs(double a[3]) { a[0] = MD_A1; a[1] = MD_A2; a[2] = MD_A3; }

/* Eq. 4 (HWCNS): f'_i h = b1 (f_{i+1/2} - f_{i-1/2}) + b2 (f_{i+1} - f_{i-1})
 * + b3 (f_{i+2} - f_{i-2}); half-widths 1/2, 1, 2.  Eq. 5 (MND): c1 (...)
 * + c2 (f_{i+1} - f_{i-1}) + c3 (f_{i+3/2} - f_{i-3/2}); half-widths 1/2, 1,
 * 3/2.  Both from sum coef_m (2 w_m) w_m^(p-1) = [p = 1], p = 1, 3, 5. */
static const double HW_B1 = 64.0 / 45.0;
static const double HW_B2 = -2.0 / 9.0;
static const double HW_B3 = 1.0 / 180.0;
static const double MND_C1 = 3.0 / 2.0;
static const double MND_C2 = -3.0 / 10.0;
static const double MND_C3 = 1.0 / 30.0;

void ora_diff_coeffs(int diff, double c[3])
{
    if (diff == ORA_DIFF_HWCNS) { c[0] = HW_B1; c[1] = HW_B2; c[2] = HW_B3; }
    else if (diff == ORA_DIFF_MND) { c[0] = MND_C1; c[1] = MND_C2; c[2] = MND_C3; }
    else { c[0] = MD_A1; c[1] = MD_A2; c[2] = MD_A3; }
}

/* f'_i h from the six midpoint fluxes fm[0..5] = f_{i-5/2} .. f_{i+5/2} and
 * the five node fluxes fn[0..4] = f_{i-2} .. f_{i+2} by Eq. 3, 4 or 5. */
static double diff_node(int diff, const double fm[6], const double fn[5])
{
    if (diff == ORA_DIFF_HWCNS)
        return HW_B1 * (fm[3] - fm[2]) + HW_B2 * (fn[3] - fn[1]) + HW_B3 * (fn[4] - fn[0]);
    if (diff == ORA_DIFF_MND)
        return MND_C1 * (fm[3] - fm[2]) + MND_C2 * (fn[3] - fn[1]) + MND_C3 * (fm[4] - fm[1]);
    return MD_A1 * (fm[3] - fm[2]) + MD_A2 * (fm[4] - fm[1]) + MD_A3 * (fm[5] - fm[0]);
}

/* ------------------------------------------------------------------ */
/* Eq. 10-11 times h and h^2 (the h-free forms), Eq. 9, Eq. 15.        */
/* s[0..4] = u_{i-2}, u_{i-1}, u_i, u_{i+1}, u_{i+2}.                  */
/* ------------------------------------------------------------------ */
static void substencil_derivatives(const double s[5], double D1[3], double D2[3])
{
    /* h u^(1)_{i,k}, Eq. 10 */
    D1[0] = 0.5 * (s[0] - 4.0 * s[1] + 3.0 * s[2]);
    D1[1] = 0.5 * (s[3] - s[1]);
    D1[2] = 0.5 * (-3.0 * s[2] + 4.0 * s[3] - s[4]);
    /* h^2 u^(2)_{i,k}, Eq. 11 */
    D2[0] = s[0] - 2.0 * s[1] + s[2];
    D2[1] = s[1] - 2.0 * s[2] + s[3];
    D2[2] = s[2] - 2.0 * s[3] + s[4];
}

/* Eq. 16-18 in ratio form: returns flags (bit k-1 = delta_k); writes chi
 * (ratio form), chi_lit (literal Eq. 16-17, may be inf/nan). */
static int teno_select(const double beta[3], double C, double eps, double CT, int q,
                       double chi[3], double chi_lit[3])
{
    double tau = fabs(beta[0] - beta[2]);             /* tau_5 */
    double g[3], gmax = 0.0;
    for (int k = 0; k < 3; ++k) {
        g[k] = C + tau / (beta[k] + eps);
        if (g[k] > gmax) gmax = g[k];
    }
    double s[3], ssum = 0.0, lit[3], litsum = 0.0;
    for (int k = 0; k < 3; ++k) {
        double r = g[k] / gmax, p = 1.0, pl = 1.0;
        for (int e = 0; e < q; ++e) { p *= r; pl *= g[k]; }
        s[k] = p; ssum += p;
        lit[k] = pl; litsum += pl;
    }
    int flags = 0;
    for (int k = 0; k < 3; ++k) {
        chi[k] = s[k] / ssum;
        chi_lit[k] = lit[k] / litsum;
        if (!(chi[k] < CT)) flags |= 1 << k;         /* Eq. 18: kept unless chi < C_T */
    }
    return flags;
}

/* Left-biased node-to-midpoint interpolation u_{L,i+1/2} from s[0..4].
 * force_flags >= 0 forces delta (for tests); otherwise the weights are
 * chosen by cfg->weights.  Returns the flags used (TENO) or 7. */
static double interp_left(const ora_cfg* cfg, const double s[5], int force_flags,
                          int* flags_out, double* margin_out, double* litdev_out)
{
    static const double d[3] = {1.0 / 16.0, 10.0 / 16.0, 5.0 / 16.0};  /* Eq. 13 */
    double D1[3], D2[3], beta[3], uk[3], w[3];
    substencil_derivatives(s, D1, D2);
    for (int k = 0; k < 3; ++k) {
        uk[k] = s[2] + D1[k] * 0.5 + D2[k] * 0.125;          /* Eq. 9, dx = h/2 */
        beta[k] = D1[k] * D1[k] + D2[k] * D2[k];             /* Eq. 15 */
    }
    int flags = 7;
    double margin = INFINITY, litdev = 0.0;
    if (force_flags >= 0) {
        flags = force_flags;
    } else if (cfg->weights == ORA_W_TENO) {
        double chi[3], chi_lit[3];
        flags = teno_select(beta, cfg->C, cfg->eps, cfg->CT, cfg->q, chi, chi_lit);
        for (int k = 0; k < 3; ++k) {
            double m = fabs(chi[k] - cfg->CT);
            if (m < margin) margin = m;
            if (isfinite(chi_lit[k])) {
                double dv = fabs(chi_lit[k] - chi[k]);
                if (dv > litdev) litdev = dv;
            }
        }
    }
    if (force_flags < 0 && cfg->weights == ORA_W_Z) {
        double tau = fabs(beta[0] - beta[2]), a[3], asum = 0.0;
        for (int k = 0; k < 3; ++k) {
            a[k] = d[k] * (1.0 + tau / (beta[k] + cfg->eps));
            asum += a[k];
        }
        for (int k = 0; k < 3; ++k) w[k] = a[k] / asum;
    } else if (force_flags < 0 && cfg->weights == ORA_W_JS) {
        double a[3], asum = 0.0;                               /* Eq. 14 */
        for (int k = 0; k < 3; ++k) {
            double b = beta[k] + cfg->eps_js;
            a[k] = d[k] / (b * b);
            asum += a[k];
        }
        for (int k = 0; k < 3; ++k) w[k] = a[k] / asum;
    } else {
        double dsum = 0.0;                                     /* Eq. 19 */
        for (int k = 0; k < 3; ++k) dsum += ((flags >> k) & 1) ? d[k] : 0.0;
        for (int k = 0; k < 3; ++k) w[k] = (((flags >> k) & 1) ? d[k] : 0.0) / dsum;
    }
    double u = 0.0;                                            /* Eq. 12 */
    for (int k = 0; k < 3; ++k) u += w[k] * uk[k];
    if (flags_out) *flags_out = flags;
    if (margin_out) *margin_out = margin;
    if (litdev_out) *litdev_out = litdev;
    return u;
}

/* Exported point kernel for tests: left-biased interpolation of one
 * 5-point stencil.  Returns u_L; writes delta flags, cutoff margin
 * min_k |chi_k - C_T| and the ratio-vs-literal chi deviation. */
double ora_interp_left(const ora_cfg* cfg, const double s[5], int force_flags,
                       int* flags, double* margin, double* litdev)
{
    return interp_left(cfg, s, force_flags, flags, margin, litdev);
}

/* Exported: the chi_k and flags of one stencil (ratio form), for tests. */
int ora_teno_chi(const ora_cfg* cfg, const double s[5], double chi[3], double chi_lit[3],
                 double beta_out[3])
{
    double D1[3], D2[3], beta[3];
    substencil_derivatives(s, D1, D2);
    for (int k = 0; k < 3; ++k) beta[k] = D1[k] * D1[k] + D2[k] * D2[k];
    if (beta_out) for (int k = 0; k < 3; ++k) beta_out[k] = beta[k];
    return teno_select(beta, cfg->C, cfg->eps, cfg->CT, cfg->q, chi, chi_lit);
}

/* ------------------------------------------------------------------ */
/* Euler equations, ideal gas (Sec. 3): U = (rho, rho u_1..u_nd, E).   */
/* ------------------------------------------------------------------ */
static double pressure(int nd, double gamma, const double* U)
{
    double ke = 0.0;
    for (int a = 0; a < nd; ++a) ke += U[1 + a] * U[1 + a];
    ke = 0.5 * ke / U[0];
    return (gamma - 1.0) * (U[nd + 1] - ke);
}

/* Physical flux in direction d. */
static void phys_flux(int nd, int d, double gamma, const double* U, double* F)
{
    double rho = U[0], un = U[1 + d] / rho, p = pressure(nd, gamma, U);
    F[0] = U[1 + d];
    for (int a = 0; a < nd; ++a) F[1 + a] = U[1 + a] * un;
    F[1 + d] += p;
    F[nd + 1] = (U[nd + 1] + p) * un;
}

void ora_phys_flux(int nd, int d, double gamma, const double* U, double* F)
{
    phys_flux(nd, d, gamma, U, F);
}

/* Eigen-system of dF_d/dU at the Roe average of states Ua and Ub.
 * R is nv x nv row-major with right eigenvectors as COLUMNS; L holds the
 * left eigenvectors as ROWS, L = R^{-1}; lam the eigenvalues.  Field order:
 * (u_n - c, u_n [entropy], tangential shear waves in axis order, u_n + c). */
static void roe_eigen(int nd, int d, double gamma, const double* Ua, const double* Ub,
                      double* R, double* L, double* lam)
{
    const int nv = nd + 2;
    double ra = sqrt(Ua[0]), rb = sqrt(Ub[0]);
    double vel[3] = {0, 0, 0}, q2 = 0.0;
    double Ha = (Ua[nd + 1] + pressure(nd, gamma, Ua)) / Ua[0];
    double Hb = (Ub[nd + 1] + pressure(nd, gamma, Ub)) / Ub[0];
    for (int a = 0; a < nd; ++a) {
        vel[a] = (ra * (Ua[1 + a] / Ua[0]) + rb * (Ub[1 + a] / Ub[0])) / (ra + rb);
        q2 += vel[a] * vel[a];
    }
    double H = (ra * Ha + rb * Hb) / (ra + rb);
    double c2 = (gamma - 1.0) * (H - 0.5 * q2);
    double c = sqrt(c2);
    double un = vel[d];
    double b1 = (gamma - 1.0) / c2, b2 = 0.5 * b1 * q2;
    memset(R, 0, sizeof(double) * nv * nv);
    memset(L, 0, sizeof(double) * nv * nv);
#define RR(i, j) R[(i) * nv + (j)]
#define LL(i, j) L[(i) * nv + (j)]
    /* column 0: acoustic u_n - c */
    RR(0, 0) = 1.0;
    for (int a = 0; a < nd; ++a) RR(1 + a, 0) = vel[a] - (a == d ? c : 0.0);
    RR(nv - 1, 0) = H - un * c;
    /* column 1: entropy */
    RR(0, 1) = 1.0;
    for (int a = 0; a < nd; ++a) RR(1 + a, 1) = vel[a];
    RR(nv - 1, 1) = 0.5 * q2;
    /* shear columns */
    int col = 2;
    for (int t = 0; t < nd; ++t) {
        if (t == d) continue;
        RR(1 + t, col) = 1.0;
        RR(nv - 1, col) = vel[t];
        ++col;
    }
    /* last column: acoustic u_n + c */
    RR(0, nv - 1) = 1.0;
    for (int a = 0; a < nd; ++a) RR(1 + a, nv - 1) = vel[a] + (a == d ? c : 0.0);
    RR(nv - 1, nv - 1) = H + un * c;

    /* rows of L */
    LL(0, 0) = 0.5 * (b2 + un / c);
    for (int a = 0; a < nd; ++a) LL(0, 1 + a) = 0.5 * (-b1 * vel[a] - (a == d ? 1.0 / c : 0.0));
    LL(0, nv - 1) = 0.5 * b1;
    LL(1, 0) = 1.0 - b2;
    for (int a = 0; a < nd; ++a) LL(1, 1 + a) = b1 * vel[a];
    LL(1, nv - 1) = -b1;
    int row = 2;
    for (int t = 0; t < nd; ++t) {
        if (t == d) continue;
        LL(row, 0) = -vel[t];
        LL(row, 1 + t) = 1.0;
        ++row;
    }
    LL(nv - 1, 0) = 0.5 * (b2 - un / c);
    for (int a = 0; a < nd; ++a) LL(nv - 1, 1 + a) = 0.5 * (-b1 * vel[a] + (a == d ? 1.0 / c : 0.0));
    LL(nv - 1, nv - 1) = 0.5 * b1;
#undef RR
#undef LL
    lam[0] = un - c;
    for (int k = 1; k < nv - 1; ++k) lam[k] = un;
    lam[nv - 1] = un + c;
}

void ora_roe_eigen(int nd, int d, double gamma, const double* Ua, const double* Ub,
                   double* R, double* L, double* lam)
{
    roe_eigen(nd, d, gamma, Ua, Ub, R, L, lam);
}

/* Roe flux-difference splitting (Roe 1981):
 * F = 1/2 (F(U_L) + F(U_R)) - 1/2 R |Lambda| L (U_R - U_L), Roe average of U_L, U_R. */
static void roe_flux(int nd, int d, double gamma, const double* UL, const double* UR, double* F)
{
    const int nv = nd + 2;
    double R[ORA_MAXV * ORA_MAXV], Lm[ORA_MAXV * ORA_MAXV], lam[ORA_MAXV];
    double FL[ORA_MAXV], FR[ORA_MAXV], dU[ORA_MAXV], alpha[ORA_MAXV];
    phys_flux(nd, d, gamma, UL, FL);
    phys_flux(nd, d, gamma, UR, FR);
    roe_eigen(nd, d, gamma, UL, UR, R, Lm, lam);
    for (int v = 0; v < nv; ++v) dU[v] = UR[v] - UL[v];
    for (int k = 0; k < nv; ++k) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) s += Lm[k * nv + v] * dU[v];
        alpha[k] = fabs(lam[k]) * s;
    }
    for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int k = 0; k < nv; ++k) s += R[v * nv + k] * alpha[k];
        F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * s;
    }
}

/* van Leer (1982) flux-vector splitting, one half.  sign = +1 gives F+,
 * sign = -1 gives F-. */
static void vanleer_half(int nd, int d, double gamma, const double* U, int sign, double* F)
{
    const int nv = nd + 2;
    double rho = U[0], p = pressure(nd, gamma, U);
    double c = sqrt(gamma * p / rho), un = U[1 + d] / rho, M = un / c;
    if (M >= 1.0) {
        if (sign > 0) phys_flux(nd, d, gamma, U, F); else for (int v = 0; v < nv; ++v) F[v] = 0.0;
        return;
    }
    if (M <= -1.0) {
        if (sign < 0) phys_flux(nd, d, gamma, U, F); else for (int v = 0; v < nv; ++v) F[v] = 0.0;
        return;
    }
    double s = (double)sign;
    double fm = s * 0.25 * rho * c * (M + s) * (M + s);        /* mass flux */
    double t2 = 0.0;
    for (int a = 0; a < nd; ++a) if (a != d) t2 += (U[1 + a] / rho) * (U[1 + a] / rho);
    double wn = (gamma - 1.0) * un + s * 2.0 * c;
    F[0] = fm;
    for (int a = 0; a < nd; ++a) F[1 + a] = fm * (U[1 + a] / rho);
    F[1 + d] = fm * wn / gamma;
    F[nv - 1] = fm * (wn * wn / (2.0 * (gamma * gamma - 1.0)) + 0.5 * t2);
}

void ora_vanleer_half(int nd, int d, double gamma, const double* U, int sign, double* F)
{
    vanleer_half(nd, d, gamma, U, sign, F);
}

/* AUSM (Liou and Steffen 1993).  Split Mach numbers and pressures of one
 * side: M+- = +-(M +- 1)^2 / 4 and p+- = p (M +- 1)^2 (2 -+ M) / 4 when
 * |M| <= 1, otherwise the upwind values (M +- |M|) / 2 and p (M +- |M|) / (2 M).
 * F = m (Phi_L + Phi_R) / 2 - |m| (Phi_R - Phi_L) / 2 + (0, p_n, 0) with
 * m = M_L^+ + M_R^-, p_n = p_L^+ + p_R^- on the normal momentum, and
 * Phi = rho c (1, u_1 .. u_nd, H). */
static void ausm_split(double M, double p, int sign, double* Ms, double* ps)
{
    const double s = (double)sign;
    if (fabs(M) <= 1.0) {
        *Ms = s * 0.25 * (M + s) * (M + s);
        *ps = 0.25 * p * (M + s) * (M + s) * (2.0 - s * M);
    } else {
        *Ms = 0.5 * (M + s * fabs(M));
        *ps = 0.5 * p * (M + s * fabs(M)) / M;
    }
}

static void ausm_flux(int nd, int d, double gamma, const double* UL, const double* UR, double* F)
{
    const int nv = nd + 2;
    const double* U[2] = {UL, UR};
    double Phi[2][ORA_MAXV], M[2], p[2];
    for (int side = 0; side < 2; ++side) {
        const double* W = U[side];
        const double rho = W[0];
        p[side] = pressure(nd, gamma, W);
        const double c = sqrt(gamma * p[side] / rho);
        M[side] = (W[1 + d] / rho) / c;
        const double rc = rho * c;
        Phi[side][0] = rc;
        for (int a = 0; a < nd; ++a) Phi[side][1 + a] = rc * (W[1 + a] / rho);
        Phi[side][nv - 1] = rc * ((W[nv - 1] + p[side]) / rho);
    }
    double Mp, pp, Mm, pm;
    ausm_split(M[0], p[0], +1, &Mp, &pp);
    ausm_split(M[1], p[1], -1, &Mm, &pm);
    const double m = Mp + Mm;
    for (int v = 0; v < nv; ++v)
        F[v] = 0.5 * m * (Phi[0][v] + Phi[1][v]) - 0.5 * fabs(m) * (Phi[1][v] - Phi[0][v]);
    F[1 + d] += pp + pm;
}

void ora_ausm_flux(int nd, int d, double gamma, const double* UL, const double* UR, double* F)
{
    ausm_flux(nd, d, gamma, UL, UR, F);
}

void ora_ausm_split(double M, double p, int sign, double* Ms, double* ps)
{
    ausm_split(M, p, sign, Ms, ps);
}

void ora_roe_flux(int nd, int d, double gamma, const double* UL, const double* UR, double* F)
{
    roe_flux(nd, d, gamma, UL, UR, F);
}

/* ------------------------------------------------------------------ */
/* One direction of the semi-discrete operator on one grid line.       */
/* ------------------------------------------------------------------ */
typedef struct {
    long nonphys;        /* faces that fell back to first order */
    double litdev;       /* max |chi_ratio - chi_literal|         */
} ora_stats;

/* A2-A6 for one face j+1/2 of a padded line P (node m at P[(m + GHOST) * nv]).
 * Writes the midpoint flux F[nv], the flags of each characteristic field
 * (bits 0-2 left-biased, 3-5 right-biased) and the cutoff margin. */
static void face_flux(const ora_cfg* cfg, int d, const double* P, int j, double* F,
                      uint8_t* flags, double* margin, ora_stats* st)
{
    const int nd = cfg->ndim, nv = nd + 2;
    const double* Uj = &P[(j + ORA_GHOST) * nv];
    const double* Uj1 = &P[(j + 1 + ORA_GHOST) * nv];
    double R[ORA_MAXV * ORA_MAXV], Lm[ORA_MAXV * ORA_MAXV], lam[ORA_MAXV];
    double W[6][ORA_MAXV];                                      /* nodes j-2..j+3 */
    if (cfg->characteristic) {
        roe_eigen(nd, d, cfg->gamma, Uj, Uj1, R, Lm, lam);      /* A2 */
        for (int m = 0; m < 6; ++m) {                           /* A3 */
            const double* Um = &P[(j - 2 + m + ORA_GHOST) * nv];
            for (int k = 0; k < nv; ++k) {
                double s = 0.0;
                for (int v = 0; v < nv; ++v) s += Lm[k * nv + v] * Um[v];
                W[m][k] = s;
            }
        }
    } else {
        for (int m = 0; m < 6; ++m)
            for (int k = 0; k < nv; ++k) W[m][k] = P[(j - 2 + m + ORA_GHOST) * nv + k];
    }
    double wL[ORA_MAXV], wR[ORA_MAXV];
    for (int k = 0; k < nv; ++k) {                              /* A4-A5 */
        double sl[5], sr[5];
        for (int m = 0; m < 5; ++m) { sl[m] = W[m][k]; sr[m] = W[5 - m][k]; }
        int fL, fR; double mL, mR, dl, dr;
        wL[k] = interp_left(cfg, sl, -1, &fL, &mL, &dl);
        wR[k] = interp_left(cfg, sr, -1, &fR, &mR, &dr);
        if (flags) flags[k] = (uint8_t)(fL | (fR << 3));
        if (margin) margin[k] = mL < mR ? mL : mR;
        if (dl > st->litdev) st->litdev = dl;
        if (dr > st->litdev) st->litdev = dr;
    }
    double UL[ORA_MAXV], UR[ORA_MAXV];
    if (cfg->characteristic) {
        for (int v = 0; v < nv; ++v) {
            double sl = 0.0, sr = 0.0;
            for (int k = 0; k < nv; ++k) { sl += R[v * nv + k] * wL[k]; sr += R[v * nv + k] * wR[k]; }
            UL[v] = sl; UR[v] = sr;
        }
    } else {
        for (int v = 0; v < nv; ++v) { UL[v] = wL[v]; UR[v] = wR[v]; }
    }
    if (!(UL[0] > 0.0) || !(UR[0] > 0.0) || !(pressure(nd, cfg->gamma, UL) > 0.0) ||
        !(pressure(nd, cfg->gamma, UR) > 0.0)) {
        for (int v = 0; v < nv; ++v) { UL[v] = Uj[v]; UR[v] = Uj1[v]; }
        st->nonphys++;
    }
    if (cfg->flux == ORA_FLUX_ROE) {                            /* A6 */
        roe_flux(nd, d, cfg->gamma, UL, UR, F);
    } else if (cfg->flux == ORA_FLUX_AUSM) {
        ausm_flux(nd, d, cfg->gamma, UL, UR, F);
    } else {
        double Fp[ORA_MAXV], Fm[ORA_MAXV];
        vanleer_half(nd, d, cfg->gamma, UL, +1, Fp);
        vanleer_half(nd, d, cfg->gamma, UR, -1, Fm);
        for (int v = 0; v < nv; ++v) F[v] = Fp[v] + Fm[v];
    }
}

/* A1: node m of a line (any integer m) under the boundary rule of d: writes
 * the node's conserved variables into out[] from the line accessor
 * (line[node * node_stride + v * var_stride]). */
static void ghost_node(const ora_cfg* cfg, int d, const double* line, long node_stride,
                       long var_stride, int m, double* out)
{
    const int n = cfg->n[d], nv = cfg->ndim + 2;
    int src = m, sign = 1;
    if (cfg->periodic[d]) {
        src = ((m % n) + n) % n;
    } else if (m < 0 || m >= n) {
        const int kind = m < 0 ? cfg->bc_lo[d] : cfg->bc_hi[d];
        if (kind == ORA_BC_FIXED) {
            for (int v = 0; v < nv; ++v) out[v] = cfg->bc_state[d][m < 0 ? 0 : 1][v];
            return;
        }
        if (kind == ORA_BC_REFLECT) {
            while (src < 0 || src >= n) {       /* mirror about the wall faces */
                src = src < 0 ? -1 - src : 2 * n - 1 - src;
                sign = -sign;
            }
        } else {
            src = m < 0 ? 0 : n - 1;            /* transmissive: zero gradient */
        }
    }
    for (int v = 0; v < nv; ++v) out[v] = line[src * node_stride + v * var_stride];
    if (sign < 0) out[1 + d] = -out[1 + d];
}

/* Body force: L += (0, rho g, rho u.g) at every node, sums in axis order. */
static int has_gravity(const ora_cfg* cfg)
{
    return cfg->gravity[0] != 0.0 || cfg->gravity[1] != 0.0 || cfg->gravity[2] != 0.0;
}

static void add_source(const ora_cfg* cfg, const double* U, double* L, long N)
{
    const int nd = cfg->ndim, nv = nd + 2;
    for (long i = 0; i < N; ++i) {
        double se = 0.0;
        for (int a = 0; a < nd; ++a) {
            L[(1 + a) * N + i] += cfg->gravity[a] * U[i];
            se += cfg->gravity[a] * U[(1 + a) * N + i];
        }
        L[(nv - 1) * N + i] += se;
    }
}

/* One direction of the semi-discrete operator on one grid line.
 * line: pointer to the n_d nodes' variables, stride between nodes, stride
 * between variables.  Adds the -f' contributions into Lout (same strides).
 * flags/margin: per face (n_d + 5 faces, j = f - 3) per characteristic
 * field, may be NULL. */
static void euler_line(const ora_cfg* cfg, int d, const double* line, long node_stride,
                       long var_stride, double* Lout, uint8_t* flags, double* margin,
                       long fl_field_stride, ora_stats* st)
{
    const int nd = cfg->ndim, nv = nd + 2, n = cfg->n[d];
    const int np = n + 2 * ORA_GHOST, nf = n + 5;
    double* P = (double*)malloc(sizeof(double) * np * nv);   /* padded nodes */
    double* Fc = (double*)malloc(sizeof(double) * nf * nv);  /* face fluxes  */
    for (int m = -ORA_GHOST; m < n + ORA_GHOST; ++m)         /* A1 */
        ghost_node(cfg, d, line, node_stride, var_stride, m, &P[(m + ORA_GHOST) * nv]);
    for (int f = 0; f < nf; ++f) {
        uint8_t fl[ORA_MAXV];
        double mg[ORA_MAXV];
        face_flux(cfg, d, P, f - 3, &Fc[f * nv], fl, mg, st);  /* face j+1/2, j = f-3 */
        for (int k = 0; k < nv; ++k) {
            if (flags) flags[k * fl_field_stride + f] = fl[k];
            if (margin) margin[k * fl_field_stride + f] = mg[k];
        }
    }
    /* A7: Eq. 3 (or 4, 5).  Node i: faces i-5/2 .. i+5/2 are f = i .. i+5;
     * the node fluxes of Eq. 4-5 are the physical fluxes of nodes i-2..i+2. */
    double* Fn = NULL;
    if (cfg->diff != ORA_DIFF_MD) {
        Fn = (double*)malloc(sizeof(double) * (n + 4) * nv);   /* nodes -2 .. n+1 */
        for (int m = -2; m < n + 2; ++m)
            phys_flux(nd, d, cfg->gamma, &P[(m + ORA_GHOST) * nv], &Fn[(m + 2) * nv]);
    }
    const double ih = 1.0 / cfg->h[d];
    for (int i = 0; i < n; ++i) {
        for (int v = 0; v < nv; ++v) {
            double fm[6], fn[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < 6; ++k) fm[k] = Fc[(i + k) * nv + v];
            if (Fn) for (int k = 0; k < 5; ++k) fn[k] = Fn[(i + k) * nv + v];
            Lout[i * node_stride + v * var_stride] -= diff_node(cfg->diff, fm, fn) * ih;  /* Eq. 2 */
        }
    }
    free(Fn);
    free(P);
    free(Fc);
}

/* Number of lines in direction d and the mapping line -> base offset. */
static long n_nodes(const ora_cfg* cfg)
{
    long N = 1;
    for (int a = 0; a < cfg->ndim; ++a) N *= cfg->n[a];
    return N;
}

static long lines_in(const ora_cfg* cfg, int d) { return n_nodes(cfg) / cfg->n[d]; }

/* Element stride of axis a in the SoA array U[var][z][y][x]. */
static long axis_stride(const ora_cfg* cfg, int a)
{
    long s = 1;
    for (int b = 0; b < a; ++b) s *= cfg->n[b];
    return s;
}

/* Base offset of line `ln` in direction d: the other axes in (z, y, x)
 * order with x fastest among them. */
static long line_base(const ora_cfg* cfg, int d, long ln)
{
    long base = 0;
    for (int a = 0; a < cfg->ndim; ++a) {
        if (a == d) continue;
        long c = ln % cfg->n[a];
        ln /= cfg->n[a];
        base += c * axis_stride(cfg, a);
    }
    return base;
}

/* Offset of direction d's block in the flags / margin arrays. */
long ora_flags_offset(const ora_cfg* cfg, int d)
{
    long off = 0;
    int nv = cfg->ndim + 2;
    for (int a = 0; a < d; ++a) off += (long)nv * lines_in(cfg, a) * (cfg->n[a] + 5);
    return off;
}

long ora_flags_size(const ora_cfg* cfg) { return ora_flags_offset(cfg, cfg->ndim); }

/* Semi-discrete RHS (Eq. 2) of the Euler equations: L = -sum_d dF_d/dx_d.
 * U, L: SoA [var][z][y][x].  flags/margin: optional, ora_flags_size bytes /
 * doubles, layout [d][field][line][face].  Returns number of fallback faces;
 * writes the max ratio-vs-literal chi deviation into *litdev if given. */
long ora_euler_rhs(const ora_cfg* cfg, const double* U, double* L, uint8_t* flags,
                   double* margin, double* litdev)
{
    const int nv = cfg->ndim + 2;
    const long N = n_nodes(cfg);
    for (long i = 0; i < (long)nv * N; ++i) L[i] = 0.0;
    long nonphys = 0;
    double ld = 0.0;
    for (int d = 0; d < cfg->ndim; ++d) {
        const long nl = lines_in(cfg, d), nf = cfg->n[d] + 5;
        const long stride = axis_stride(cfg, d);
        const long foff = ora_flags_offset(cfg, d);
        #pragma omp parallel for schedule(static) reduction(+ : nonphys) reduction(max : ld)
        for (long ln = 0; ln < nl; ++ln) {
            ora_stats st = {0, 0.0};
            long base = line_base(cfg, d, ln);
            euler_line(cfg, d, U + base, stride, N, L + base,
                       flags ? flags + foff + ln * nf : NULL,
                       margin ? margin + foff + ln * nf : NULL, nl * nf, &st);
            nonphys += st.nonphys;
            if (st.litdev > ld) ld = st.litdev;
        }
    }
    if (has_gravity(cfg)) add_source(cfg, U, L, N);
    if (litdev) *litdev = ld;
    return nonphys;
}

/* Direction-d contributions of a range of grid lines only (a bounded sample
 * of the full RHS: the full RHS is the sum over every line of every
 * direction).  Adds into L; returns fallback faces. */
long ora_euler_rhs_lines(const ora_cfg* cfg, const double* U, double* L, int d, long line_lo,
                         long line_hi)
{
    const long N = n_nodes(cfg);
    const long stride = axis_stride(cfg, d);
    long nonphys = 0;
    #pragma omp parallel for schedule(static) reduction(+ : nonphys)
    for (long ln = line_lo; ln < line_hi; ++ln) {
        ora_stats st = {0, 0.0};
        long base = line_base(cfg, d, ln);
        euler_line(cfg, d, U + base, stride, N, L + base, NULL, NULL, 0, &st);
        nonphys += st.nonphys;
    }
    return nonphys;
}

/* The RHS at selected nodes only (same arithmetic as ora_euler_rhs): for
 * each node index idx[p] (flattened x-fastest), L_out[v * npts + p]. */
long ora_euler_rhs_at(const ora_cfg* cfg, const double* U, long npts, const long* idx,
                      double* Lout)
{
    const int nd = cfg->ndim, nv = nd + 2;
    const long N = n_nodes(cfg);
    long nonphys = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(+ : nonphys)
    for (long p = 0; p < npts; ++p) {
        ora_stats st = {0, 0.0};
        long coord[3] = {0, 0, 0}, rest = idx[p];
        for (int a = 0; a < nd; ++a) { coord[a] = rest % cfg->n[a]; rest /= cfg->n[a]; }
        double acc[ORA_MAXV];
        for (int v = 0; v < nv; ++v) acc[v] = 0.0;
        for (int d = 0; d < nd; ++d) {
            double P[(2 * ORA_GHOST + 1) * ORA_MAXV];   /* nodes i-5 .. i+5 */
            long c0[3] = {coord[0], coord[1], coord[2]};
            c0[d] = 0;
            long base = 0;
            for (int a = nd - 1; a >= 0; --a) base = base * cfg->n[a] + c0[a];
            for (int m = -ORA_GHOST; m <= ORA_GHOST; ++m)
                ghost_node(cfg, d, U + base, axis_stride(cfg, d), N, (int)coord[d] + m,
                           &P[(m + ORA_GHOST) * nv]);
            /* faces i-5/2 .. i+5/2 are j = i-3 .. i+2; with the padded origin at
             * node i, j runs -3 .. 2 and the face array index is j + 3 */
            double Fc[6][ORA_MAXV], Fn[5][ORA_MAXV];
            for (int f = 0; f < 6; ++f) face_flux(cfg, d, P, f - 3, Fc[f], NULL, NULL, &st);
            for (int k = 0; k < 5; ++k) phys_flux(nd, d, cfg->gamma, &P[(k - 2 + ORA_GHOST) * nv], Fn[k]);
            const double ih = 1.0 / cfg->h[d];
            for (int v = 0; v < nv; ++v) {
                double fm[6], fn[5];
                for (int k = 0; k < 6; ++k) fm[k] = Fc[k][v];
                for (int k = 0; k < 5; ++k) fn[k] = Fn[k][v];
                acc[v] -= diff_node(cfg->diff, fm, fn) * ih;
            }
        }
        if (has_gravity(cfg)) {
            double se = 0.0;
            for (int a = 0; a < nd; ++a) {
                acc[1 + a] += cfg->gravity[a] * U[idx[p]];
                se += cfg->gravity[a] * U[(1 + a) * N + idx[p]];
            }
            acc[nv - 1] += se;
        }
        for (int v = 0; v < nv; ++v) Lout[v * npts + p] = acc[v];
        nonphys += st.nonphys;
    }
    return nonphys;
}

/* A9: dt = CFL / max_i sum_d (|u_d| + c) / h_d. */
double ora_cfl_dt(const ora_cfg* cfg, const double* U, double cfl)
{
    const int nd = cfg->ndim;
    const long N = n_nodes(cfg);
    double lmax = 0.0;
    #pragma omp parallel for schedule(static) reduction(max : lmax)
    for (long i = 0; i < N; ++i) {
        double Ui[ORA_MAXV];
        for (int v = 0; v < nd + 2; ++v) Ui[v] = U[v * N + i];
        double c = sqrt(cfg->gamma * pressure(nd, cfg->gamma, Ui) / Ui[0]);
        double s = 0.0;
        for (int a = 0; a < nd; ++a) s += (fabs(Ui[1 + a] / Ui[0]) + c) / cfg->h[a];
        if (s > lmax) lmax = s;
    }
    return cfl / lmax;
}

/* A10: one SSP-RK3 step (Shu-Osher form) of size dt, in place. */
long ora_rk3_step(const ora_cfg* cfg, double* U, double dt)
{
    const long M = (long)(cfg->ndim + 2) * n_nodes(cfg);
    double* U1 = (double*)malloc(sizeof(double) * M);
    double* Lr = (double*)malloc(sizeof(double) * M);
    long np = 0;
    np += ora_euler_rhs(cfg, U, Lr, NULL, NULL, NULL);
    for (long i = 0; i < M; ++i) U1[i] = U[i] + dt * Lr[i];
    np += ora_euler_rhs(cfg, U1, Lr, NULL, NULL, NULL);
    for (long i = 0; i < M; ++i) U1[i] = 0.75 * U[i] + 0.25 * (U1[i] + dt * Lr[i]);
    np += ora_euler_rhs(cfg, U1, Lr, NULL, NULL, NULL);
    for (long i = 0; i < M; ++i) U[i] = U[i] / 3.0 + 2.0 / 3.0 * (U1[i] + dt * Lr[i]);
    free(U1);
    free(Lr);
    return np;
}

/* Advance to t_end (or max_steps) with the CFL rule; the last step is
 * clipped to land on t_end.  Returns fallback faces; writes t and steps. */
long ora_euler_run(const ora_cfg* cfg, double* U, double cfl, double t_end, int max_steps,
                   double* t_out, int* steps_out)
{
    double t = 0.0;
    int s = 0;
    long np = 0;
    while (t < t_end && s < max_steps) {
        double dt = ora_cfl_dt(cfg, U, cfl);
        if (t + dt > t_end) dt = t_end - t;
        np += ora_rk3_step(cfg, U, dt);
        t += dt;
        ++s;
    }
    if (t_out) *t_out = t;
    if (steps_out) *steps_out = s;
    return np;
}

/* A11: sum_i U_i * prod_d h_d per variable. */
void ora_conserved(const ora_cfg* cfg, const double* U, double* out)
{
    const long N = n_nodes(cfg);
    double vol = 1.0;
    for (int a = 0; a < cfg->ndim; ++a) vol *= cfg->h[a];
    for (int v = 0; v < cfg->ndim + 2; ++v) {
        double s = 0.0;
        for (long i = 0; i < N; ++i) s += U[v * N + i];
        out[v] = s * vol;
    }
}

/* ------------------------------------------------------------------ */
/* Scalar conservation laws on a periodic grid (Sec. 3.2-3.3).         */
/* kind 0: linear advection f = u, a_hat = 1.                          */
/* kind 1: inviscid Burgers f = u^2/2, a_hat = (u_L + u_R)/2.          */
/* ------------------------------------------------------------------ */
static double scalar_f(int kind, double u) { return kind == 0 ? u : 0.5 * u * u; }

void ora_scalar_rhs(const ora_cfg* cfg, int kind, int n, double h, const double* u, double* L)
{
    const int nf = n + 5;
    double* F = (double*)malloc(sizeof(double) * nf);
    for (int f = 0; f < nf; ++f) {
        int j = f - 3;
        double sl[5], sr[5];
        for (int m = 0; m < 5; ++m) {
            int il = ((j - 2 + m) % n + n) % n;      /* u_{j-2..j+2}      */
            int ir = ((j + 3 - m) % n + n) % n;      /* u_{j+3..j-1}      */
            sl[m] = u[il];
            sr[m] = u[ir];
        }
        double uL = interp_left(cfg, sl, -1, NULL, NULL, NULL);
        double uR = interp_left(cfg, sr, -1, NULL, NULL, NULL);
        double a = kind == 0 ? 1.0 : 0.5 * (uL + uR);
        F[f] = 0.5 * ((scalar_f(kind, uR) + scalar_f(kind, uL)) - fabs(a) * (uR - uL)); /* Eq. 6 */
    }
    for (int i = 0; i < n; ++i) {
        double fn[5];
        for (int k = 0; k < 5; ++k) fn[k] = scalar_f(kind, u[((i - 2 + k) % n + n) % n]);
        L[i] = -diff_node(cfg->diff, &F[i], fn) / h;
    }
    free(F);
}

/* SSP-RK3 with a fixed number of equal steps reaching t_end. */
void ora_scalar_run(const ora_cfg* cfg, int kind, int n, double h, double t_end, int nsteps,
                    double* u)
{
    double* u1 = (double*)malloc(sizeof(double) * n);
    double* L = (double*)malloc(sizeof(double) * n);
    double dt = t_end / nsteps;
    for (int s = 0; s < nsteps; ++s) {
        ora_scalar_rhs(cfg, kind, n, h, u, L);
        for (int i = 0; i < n; ++i) u1[i] = u[i] + dt * L[i];
        ora_scalar_rhs(cfg, kind, n, h, u1, L);
        for (int i = 0; i < n; ++i) u1[i] = 0.75 * u[i] + 0.25 * (u1[i] + dt * L[i]);
        ora_scalar_rhs(cfg, kind, n, h, u1, L);
        for (int i = 0; i < n; ++i) u[i] = u[i] / 3.0 + 2.0 / 3.0 * (u1[i] + dt * L[i]);
    }
    free(u1);
    free(L);
}

/* One RK3 step for the scalar operator (for the Taylor-polynomial pin). */
void ora_scalar_rk3_step(const ora_cfg* cfg, int kind, int n, double h, double dt, double* u)
{
    ora_scalar_run(cfg, kind, n, h, dt, 1, u);
}
