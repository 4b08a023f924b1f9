// wcns_sweep.cuh -- the fused per-direction sweep kernel.
//
// One CTA owns a tile of TL grid lines x TS nodes along direction DIR.  It
//  (1) stages the TS + 10 nodes of each line (5 ghost nodes per side: node i
//      reads faces i +- 1/2, 3/2, 5/2 and face j + 1/2 reads nodes
//      j-2 .. j+3) in shared memory, coalesced along x, applying the
//      boundary rule (transmissive = copy the boundary node, periodic = wrap);
//  (2) computes the TS + 5 midpoint fluxes of each line, one face per
//      thread: characteristic projection, TENO selection and Table-1
//      interpolation of both biased values (or the JS, Z or linear
//      weights), back-projection, Roe, van Leer or AUSM flux (Sec. 1-3 of
//      arXiv 1810.07806), into shared memory;
//  (3) forms -f'_i by the sixth-order MD difference (Eq. 3), or the HWCNS or
//      MND difference (Eq. 4, 5) with the physical fluxes of the staged
//      nodes, and writes or accumulates it into L (Eq. 2: the directions
//      are summed).
#pragma once
#include <type_traits>
#include "wcns_fp64.cuh"

namespace wcns {

enum { FLUX_ROE = 0, FLUX_VANLEER = 1, FLUX_AUSM = 2 };
enum { BC_TRANSMISSIVE = 0, BC_PERIODIC = 1, BC_REFLECTING = 2, BC_FIXED = 3 };

// Batched sweeps run over many independent grids ("instances") of one
// dimension at once: each CTA takes one tile from a table and reads its
// instance's geometry.  Instance i's state is an SoA block [var][nodes_i] at
// element offset `off` of the batch arrays.
struct BatchInst {
    long long off;            // element offset of the instance's block
    long long N;              // nodes of the instance
    int n[3];                 // nodes per axis
    int periodic[3];          // boundary rule per axis
    double h[3];              // node spacing per axis
    double inv_h[3];          // 1 / h per axis
    float inv_hf[3];
    int bc[3][2];             // boundary kind of each side (BC_*)
    double bcs[3][2][5];      // fixed states (conserved variables)
    double grav[3];           // body force per unit mass
    int has_grav;             // some component of grav is non-zero
};

struct BatchTile {
    int inst;                 // instance index
    int pos0;                 // first node along the sweep direction
    int lfirst;               // first line of the tile (x sweep: row; y/z: x column)
    int outer;                // y/z sweeps: the remaining axis index
};

// Device-resident scalars of a run: one per grid (handle), one per batch
// instance.  The sweeps read dt (and, in FP32, the reference state) through
// a pointer to the first member.
struct StepScalars {
    double dt;            // step of the current RK step (0 = finished)
    double t;             // time reached at the end of the current step
    double t_end;         // clip target (inf when unused)
    unsigned long long lam_bits;   // max wave-speed sum (non-negative double bits)
    unsigned long long steps;      // steps that advanced time since the last reset
    // FP32 path: the constant reference state U_r = (rho_r, 0, .., 0, E_r)
    // the single-precision stage values are measured from (all zero until
    // set: the plain form), with p_r = (gamma - 1) E_r and H_r = E_r + p_r
    double ref_rho, ref_E;
    float ref_rhof, ref_Ef, ref_pf, ref_hf;
    unsigned long long ref_keys[2];   // order keys of min rho and min p while they are reduced
};

struct SweepArgs {
    const void* U;            // input state, LT, SoA
    void* L;                  // output RHS, T, SoA
    long long N;              // nodes
    int n[3];                 // nodes per axis
    int periodic;             // boundary rule of this direction
    double inv_h;             // 1 / h_DIR
    int accumulate;           // 0: L = -f'   1: L -= f'
    uint8_t* flags;           // nullable debug output, block of this direction
    long long* fallback;      // count of first-order fallback faces (batched
                              // mode: one counter per instance, indexed by it)
    const double* dt;         // nullable: skip all work when *dt == 0 (finished)
    SchemeConst K;
    float sqrt_eps_f;         // sqrt(eps) in float, for the FP32 rescaled eps
    float inv_hf;             // 1 / h_DIR in float
    // FP32 steps: the last sweep of a stage also applies the SSP-RK3 stage
    // combination (stage 1..3; 0 = plain RHS).  U0 is the FP64 base state, D
    // the FP32 increment, S_out the next stage's FP32 input (batch arrays in
    // batched mode).
    int fuse_stage;
    double* U0;
    float* D;
    float* S_out;
    // boundary rule of a non-periodic direction (single grids; batched
    // sweeps read their instance's): WCNS_BC_* kinds of the low and high side
    // and the fixed states; the last sweep of an RHS adds the body-force
    // source (0, rho g, rho u.g) when source is set (batched: for the
    // instances with a body force)
    int bc_lo, bc_hi;
    double bcs[2][5];
    int source;
    double grav[3];
    // batched mode only
    const BatchInst* insts;
    const BatchTile* tiles;
    const double* inst_dt;    // dt of instance i at inst_dt[i * dt_stride]
    int dt_stride;            // in doubles
    // persistent batched launch (nullable): the tile counter this launch
    // takes work from (zero at launch) and the number of tiles
    unsigned int* work;
    long long ntiles;
    // FP32: load L after the faces into the staged nodes' space (only for a
    // plain Eq. 3 node phase without a source, and without a fused stage
    // whose arrays the tile stages in shared memory; the launch then passes
    // TileGeom::smem_bytes(true))
    int alias_L;
    // launched as a programmatic dependent of the previous sweep of the same
    // RHS: stage and compute the faces (which read only the RHS's input),
    // then wait for that sweep before the first access to L
    int pdl;
};

// Whether a sweep with these arguments may share the staged nodes' space
// with the prefetched L (see SweepArgs::alias_L); fuse_smem: the tile stages
// a fused stage's arrays in shared memory (TileGeom::FUSE_SMEM).
inline bool sweep_alias_L(const SweepArgs& a, bool fuse_smem)
{
    return a.K.diff == DIFF_MD && !a.source && (!a.fuse_stage || !fuse_smem);
}

// 4-byte asynchronous global->shared copies (cp.async): the staging loads
// and the prefetch of the RHS being accumulated proceed while the CTA
// computes, instead of stalling the issuing warps.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16-byte copy (both addresses 16-byte aligned), cached in L2 only.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NW>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NW) : "memory"); }

// Tile shapes: lines per tile (TL) x nodes per line (TS); TL * (TS + 5) faces
// is a multiple of the 256 threads.  Configuration 0 is the default; the
// autotuner (FP32, 2D/3D) may pick, per direction, 1 (x: 16 lines of 59,
// four faces per thread, a quarter of the tiles to set up; y/z: longer
// pencils, fewer recomputed halo faces) or 2 (x: 8 lines of 123, fewer
// recomputed halo faces; y/z: narrower tiles).
constexpr int tile_lines(int nd, int dir, int cfg)
{
    return nd == 1 ? 1 : (dir == 0 ? (cfg == 0 ? 4 : (cfg == 1 ? 16 : 8)) : (cfg == 0 ? 16 : 8));
}
constexpr int tile_nodes(int nd, int dir, int cfg)
{
    return nd == 1 ? (cfg == 1 ? 1019 : 251)
                   : (dir == 0 ? (cfg == 0 ? 59 : (cfg == 1 ? 59 : 123)) : (cfg == 1 ? 123 : 59));
}
// The tile configuration of batched sweeps: FP32 1D batches take tiles of
// 1019 nodes (four faces per thread, a quarter of the tiles to set up: 19%
// off the step of 4096 Shu-Osher instances of 200-4000 nodes; 507 and 2043
// measured slower), while a single 1D grid keeps 251 (a grid of a few
// hundred nodes would otherwise run each sweep in one CTA) and so do FP64
// batches (bound by the FP64 pipe, 3% slower with 507); 2D and 3D batches
// take the default.
template <typename T>
constexpr int batch_cfg(int nd) { return nd == 1 && sizeof(T) == 4 ? 1 : 0; }

template <typename T, int ND, int DIR, int CFG = 0>
struct TileGeom {
    static constexpr int TL = tile_lines(ND, DIR, CFG);   // lines per tile
    static constexpr int TS = tile_nodes(ND, DIR, CFG);   // nodes per line
    static constexpr int P = TS + 2 * GHOST;                          // staged nodes
    // pitch of a staged x line: room for the 16-byte aligned start (up to 3
    // nodes before pos0 - 5) of the vectorised staging
    static constexpr int SP = DIR == 0 ? (P + 3 + 3) / 4 * 4 : P;
    static constexpr int NF = TS + 5;                                 // faces
    static constexpr int THREADS = 256;
    // FP32: at most 64 registers so four CTAs share an SM.  FP64: at most 128,
    // two CTAs (measured a little faster than one CTA with 175 registers).
    static constexpr int MIN_CTAS = sizeof(T) == 4 ? 4 : 2;
    // FP32 sweeps that accumulate prefetch the TS nodes of L they update
    static constexpr bool PREFETCH_L = sizeof(T) == 4;
    // The FP32 x sweep (the last of a step's stage) can fuse the stage
    // combination.  The small x tiles of configuration 0 prefetch its FP64
    // base state and FP32 increment into shared memory; the larger tiles
    // (configurations 1 and 2) would then fit only 2 CTAs on an SM, so they
    // load them from global memory in the node phase and share the staged
    // nodes' space with the prefetched L.
    static constexpr bool FUSE = sizeof(T) == 4 && DIR == 0;
    static constexpr bool FUSE_SMEM = FUSE && CFG == 0;
    // Bytes of the staged nodes, faces and (unless it shares the staged
    // nodes' space, alias_L) the prefetched L, rounded up to 16 bytes, then
    // the fused stage arrays.  A launch passes the size of its own layout.
    static constexpr size_t front_bytes(bool alias_L)
    {
        return (sizeof(T) * (size_t)(ND + 2) * TL * (SP + NF + (PREFETCH_L && !alias_L ? TS : 0)) + 15) &
               ~(size_t)15;
    }
    static constexpr size_t smem_bytes(bool alias_L = false)
    {
        return front_bytes(alias_L) +
               (FUSE_SMEM ? (size_t)(ND + 2) * TL * TS * (sizeof(double) + sizeof(float)) : 0);
    }
};

// Shared-memory index: the memory-contiguous index is the fastest one.
template <int DIR, int TL, int W>
__device__ __forceinline__ int sidx(int v, int l, int s)
{
    return DIR == 0 ? (v * TL + l) * W + s : (v * W + s) * TL + l;
}

// ---------------------------------------------------------------- FP64 face
// (the FP64 face selects the weights at run time: WT is not used, and it
// has its own division-free screen: FAST is not used)
template <int ND, int DIR, int FLUX, int WT, bool FAST = false>
__device__ __forceinline__ bool face_flux(double (&u)[6][ND + 2], const SweepArgs& a, const Ref32&, double* F,
                                          uint8_t* fl, bool& fell_back)
{
    face_fp64<ND, DIR, FLUX>(u, a.K, F, fl, fell_back);
    return true;
}

// ---------------------------------------------------------------- FP32 face
// WT: the weights, fixed at compile time (W_TENO, or the comparison weights
// W_JS, W_LINEAR, W_Z in their own instances).  u holds U - U_r (Ref32);
// every operation is written out (the FP32 units compile without
// multiply-add contraction), so each instance of this code, single-grid or
// batched, rounds the same way.  FAST (TENO): the face is evaluated only if
// every side of every field passes the exact no-cut test; otherwise the
// function returns false early (F, fl not written) and the caller runs the
// face again with FAST off.  A face evaluated either way gives the same bits.
template <int ND, int DIR, int FLUX, int WT, bool FAST = false>
__device__ __forceinline__ bool face_flux(float (&u)[6][ND + 2], const SweepArgs& a, const Ref32& R, float* F,
                                          uint8_t* fl, bool& fell_back)
{
    constexpr int NV = ND + 2;
    const float gm1 = a.K.gm1f;
    // Roe average of nodes j, j+1 and the closed form of L u:
    //   P = b1 (u_E - vel.m + q2 u_rho / 2), Q = (u_n u_rho - m_n) / c,
    //   w_0 = (P + Q)/2, w_1 = u_rho - P, w_t = m_t - vel_t u_rho, w_N = (P - Q)/2.
    const float* Ua = u[2];
    const float* Ub = u[3];
    // (ra = 1 / sqrt(rho_j): sqrt(rho_j) = rho_j ra, 1 / rho_j = ra^2)
    const float rhoa = Ua[0] + R.rho, rhob = Ub[0] + R.rho;
    const float ra = rsqrtf_a(rhoa), rb = rsqrtf_a(rhob);
    const float wsum = rcpf(fmaf(rhoa, ra, rhob * rb));
    float vel[ND], q2 = 0.f;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        vel[d] = fmaf(Ua[1 + d], ra, Ub[1 + d] * rb) * wsum;
        q2 = fmaf(vel[d], vel[d], q2);
    }
    // p - p_r of both nodes; E + p = u_E + (p - p_r) + H_r
    const float pa = pressure_ir<ND>(Ua, ra * ra, gm1), pb = pressure_ir<ND>(Ub, rb * rb, gm1);
    const float H = fmaf((Ua[ND + 1] + pa) + R.h, ra, ((Ub[ND + 1] + pb) + R.h) * rb) * wsum;
    const float c2 = gm1 * fmaf(-0.5f, q2, H);
    const float ic = rsqrtf_a(c2);
    const float c = c2 * ic;
    const float hb1 = 0.5f * gm1 * (ic * ic);   // b1 / 2
    const float un = vel[DIR];
    float Uj[NV], Uj1[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { Uj[v] = Ua[v]; Uj1[v] = Ub[v]; }
    float UL[NV], UR[NV];
    if constexpr (WT == W_TENO) {
        // mirrored node pairs (m, 5 - m) in the two lanes: W2[m][k] =
        // (W_m[k], W_{5-m}[k]), i.e. the left stencil's value in .x and the
        // mirrored right stencil's in .y
        float2 W2[3][NV];
        const float2 hq = bc2(0.5f * q2), hb = bc2(hb1), qa = bc2(0.5f * ic * un), qb = bc2(-0.5f * ic);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float2 U2[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) U2[v] = make_float2(u[m][v], u[5 - m][v]);
            float2 vm = mul2(bc2(vel[0]), U2[1]);
#pragma unroll
            for (int d = 1; d < ND; ++d) vm = fma2(bc2(vel[d]), U2[1 + d], vm);
            const float2 Ph = mul2(hb, sub2(fma2(hq, U2[0], U2[ND + 1]), vm));   // P/2
            const float2 Qh = fma2(qa, U2[0], mul2(qb, U2[1 + DIR]));            // Q/2
            W2[m][0] = add2(Ph, Qh);
            W2[m][1] = fma2(bc2(-2.f), Ph, U2[0]);
            int k = 2;
#pragma unroll
            for (int t = 0; t < ND; ++t) {
                if (t == DIR) continue;
                W2[m][k++] = fma2(bc2(-vel[t]), U2[0], U2[1 + t]);
            }
            W2[m][NV - 1] = sub2(Ph, Qh);
        }
        float2 w2[NV];   // (u_L, u_R) of each characteristic field
        bool slow = false;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            int fL, fR;
            w2[k] = select_interp_x2<FAST>(W2[0][k], W2[1][k], W2[2][k], a.sqrt_eps_f, a.K, fL, fR, slow);
            fl[k] = (uint8_t)(fL | (fR << 3));
        }
        if constexpr (FAST) {
            if (slow) return false;
        }
        // U = R w for both sides at once
        const float2 r = add2(add2(w2[0], w2[1]), w2[NV - 1]);
        const float2 dw = sub2(w2[NV - 1], w2[0]);
        float2 U2[NV];
        U2[0] = r;
        float2 e = fma2(bc2(H), add2(w2[0], w2[NV - 1]), fma2(bc2(un * c), dw, mul2(hq, w2[1])));
        int k = 2;
#pragma unroll
        for (int t = 0; t < ND; ++t) {
            if (t == DIR) {
                U2[1 + t] = fma2(bc2(vel[t]), r, mul2(bc2(c), dw));
            } else {
                U2[1 + t] = fma2(bc2(vel[t]), r, w2[k]);
                e = fma2(bc2(vel[t]), w2[k], e);
                ++k;
            }
        }
        U2[NV - 1] = e;
#pragma unroll
        for (int v = 0; v < NV; ++v) { UL[v] = U2[v].x; UR[v] = U2[v].y; }
    } else {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            float* U = u[m];
            float vm = vel[0] * U[1];
#pragma unroll
            for (int d = 1; d < ND; ++d) vm = fmaf(vel[d], U[1 + d], vm);
            const float Ph = hb1 * (fmaf(0.5f * q2, U[0], U[ND + 1]) - vm);   // P/2
            const float Qh = 0.5f * ic * fmaf(un, U[0], -U[1 + DIR]);         // Q/2
            float W[NV];
            W[0] = Ph + Qh;
            W[1] = fmaf(-2.f, Ph, U[0]);
            int k = 2;
#pragma unroll
            for (int t = 0; t < ND; ++t) {
                if (t == DIR) continue;
                W[k++] = fmaf(-vel[t], U[0], U[1 + t]);
            }
            W[NV - 1] = Ph - Qh;
#pragma unroll
            for (int v = 0; v < NV; ++v) U[v] = W[v];
        }
        float wL[NV], wR[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            float s6[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) s6[m] = u[m][k];
            weights_pair_fp32<WT>(s6, a.sqrt_eps_f, a.K, wL[k], wR[k]);
            fl[k] = 0x3F;
        }
        const float rl = wL[0] + wL[1] + wL[NV - 1], rr = wR[0] + wR[1] + wR[NV - 1];
        const float dl = wL[NV - 1] - wL[0], dr = wR[NV - 1] - wR[0];
        UL[0] = rl;
        UR[0] = rr;
        float el = fmaf(H, wL[0] + wL[NV - 1], fmaf(un * c, dl, 0.5f * q2 * wL[1]));
        float er = fmaf(H, wR[0] + wR[NV - 1], fmaf(un * c, dr, 0.5f * q2 * wR[1]));
        int k = 2;
#pragma unroll
        for (int t = 0; t < ND; ++t) {
            if (t == DIR) {
                UL[1 + t] = fmaf(vel[t], rl, c * dl);
                UR[1 + t] = fmaf(vel[t], rr, c * dr);
            } else {
                UL[1 + t] = fmaf(vel[t], rl, wL[k]);
                UR[1 + t] = fmaf(vel[t], rr, wR[k]);
                el = fmaf(vel[t], wL[k], el);
                er = fmaf(vel[t], wR[k], er);
                ++k;
            }
        }
        UL[NV - 1] = el;
        UR[NV - 1] = er;
    }
    const float rhoL = UL[0] + R.rho, rhoR = UR[0] + R.rho;
    float rL = rsqrtf_a(rhoL), rR = rsqrtf_a(rhoR);
    float pL = pressure_ir<ND>(UL, rL * rL, gm1), pR = pressure_ir<ND>(UR, rR * rR, gm1);   // p - p_r
    if (!(rhoL > 0.f) || !(rhoR > 0.f) || !(pL + R.p > 0.f) || !(pR + R.p > 0.f)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { UL[v] = Uj[v]; UR[v] = Uj1[v]; }
        pL = pa;
        pR = pb;
        rL = ra;
        rR = rb;
        fell_back = true;
    }
    if (FLUX == FLUX_ROE) {
        roe_flux<ND, DIR>(UL, UR, pL, pR, rL, rR, gm1, R, F);
    } else {
        // the splittings take the full states (with R zero: the same values)
        float VL[NV], VR[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { VL[v] = UL[v]; VR[v] = UR[v]; }
        VL[0] = UL[0] + R.rho;
        VR[0] = UR[0] + R.rho;
        VL[NV - 1] = UL[NV - 1] + R.e;
        VR[NV - 1] = UR[NV - 1] + R.e;
        const float PL = pL + R.p, PR = pR + R.p;
        if (FLUX == FLUX_AUSM) {
            ausm_flux<ND, DIR>(VL, VR, PL, PR, a.K.gammaf, F);
        } else {
            float Fp[NV], Fm[NV];
            vanleer_half<ND, DIR>(VL, PL, a.K.gammaf, gm1, 1.f, Fp);
            vanleer_half<ND, DIR>(VR, PR, a.K.gammaf, gm1, -1.f, Fm);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] = Fp[v] + Fm[v];
        }
    }
    return true;
}

// f(U_{s+k}) - f(U_{s-k}) in direction DIR for the staged nodes of line l
// (physical fluxes; FP64 in the oracle's order).
template <int ND, int DIR, int TL, int P, typename T>
__device__ __forceinline__ void node_flux_diff(const T* sS, int l, int s, int k, const SchemeConst& K,
                                               const Ref32& R, T* d)
{
    constexpr int NV = ND + 2;
    T Up[NV], Um[NV], Fp[NV], Fm[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        Up[v] = sS[sidx<DIR, TL, P>(v, l, s + k)];
        Um[v] = sS[sidx<DIR, TL, P>(v, l, s - k)];
    }
    if constexpr (sizeof(T) == 8) {
        phys_flux_fp64<ND, DIR>(Up, K.gm1, Fp);
        phys_flux_fp64<ND, DIR>(Um, K.gm1, Fm);
#pragma unroll
        for (int v = 0; v < NV; ++v) d[v] = sub_(Fp[v], Fm[v]);
    } else {
        // (relative to U_r: the fluxes differ from the physical ones by a
        // constant, which the difference removes)
        phys_flux_ref<ND, DIR>(Up, pressure_of<ND>(Up, K.gm1f, R.rho), R, Fp);
        phys_flux_ref<ND, DIR>(Um, pressure_of<ND>(Um, K.gm1f, R.rho), R, Fm);
#pragma unroll
        for (int v = 0; v < NV; ++v) d[v] = Fp[v] - Fm[v];
    }
}

// ---------------------------------------------------------------- kernel
// A staged value in the sweep's type (FP64 -> FP32 by the integer rounding).
template <typename T, typename LT>
__device__ __forceinline__ T stage_cvt(LT x)
{
    if constexpr (sizeof(T) == 4 && sizeof(LT) == 8) return f64_to_f32_ftz(x);
    else return (T)x;
}

// One tile of a sweep (tile: the index into the batch's tile table; single
// grids take the tile from the launch coordinates).
template <typename T, typename LT, int ND, int DIR, int FLUX, bool BATCH, int CFG, int WT>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, long long tile)
{
    constexpr int NV = ND + 2;
    using G = TileGeom<T, ND, DIR, CFG>;
    constexpr int TL = G::TL, TS = G::TS, P = G::P, SP = G::SP, NF = G::NF;
    constexpr bool kAsyncStage = sizeof(LT) == sizeof(T) && sizeof(T) == 4;
    constexpr bool kPre = G::PREFETCH_L;
    constexpr bool kAsync = kAsyncStage || kPre;

    // The grid (one instance, or the tile's instance in batched mode).
    const LT* Ub;
    T* Lb;
    long long N;
    int nx, ny, nz, nd, periodic, pos0, lfirst;
    long long outer;
    const double* dtp;
    long long* fbp = a.fallback;
    T ih;
    double* U0b = a.U0;
    float* Db = a.D;
    float* Sob = a.S_out;
    // boundary rule of this direction's sides, fixed states, body force
    int bcl = a.bc_lo, bch = a.bc_hi;
    const double(*bcs)[5] = a.bcs;
    const double* gravp = a.grav;
    int source = a.source;
    if constexpr (BATCH) {
        const BatchTile bt = a.tiles[tile];
        const BatchInst& I = a.insts[bt.inst];
        bcl = I.bc[DIR][0];
        bch = I.bc[DIR][1];
        bcs = I.bcs[DIR];
        gravp = I.grav;
        source = a.source && I.has_grav;
        Ub = reinterpret_cast<const LT*>(a.U) + I.off;
        Lb = reinterpret_cast<T*>(a.L) + I.off;
        if (a.fuse_stage) {
            U0b += I.off;
            Db += I.off;
            if (Sob != nullptr) Sob += I.off;   // stages 1 and 2 only
        }
        N = I.N;
        nx = I.n[0];
        ny = I.n[1];
        nz = I.n[2];
        nd = I.n[DIR];
        periodic = I.periodic[DIR];
        if constexpr (sizeof(T) == 8) ih = I.inv_h[DIR];
        else ih = I.inv_hf[DIR];
        pos0 = bt.pos0;
        lfirst = bt.lfirst;
        outer = bt.outer;
        dtp = a.inst_dt + (long long)bt.inst * a.dt_stride;
        fbp = a.fallback + bt.inst;
    } else {
        Ub = reinterpret_cast<const LT*>(a.U);
        Lb = reinterpret_cast<T*>(a.L);
        N = a.N;
        nx = a.n[0];
        ny = a.n[1];
        nz = a.n[2];
        nd = a.n[DIR];
        periodic = a.periodic;
        if constexpr (sizeof(T) == 8) ih = a.inv_h;
        else ih = a.inv_hf;
        pos0 = blockIdx.y * TS;
        lfirst = blockIdx.x * TL;
        outer = blockIdx.z;
        dtp = a.dt;
    }
    // A finished run (dt == 0) skips the work.  The FP32 sweep reads the flag
    // after its staging copies are in flight, so the read costs no latency.
    if constexpr (!kAsyncStage) {
        if (dtp != nullptr && f64_is_zero(*dtp)) return;
    }
    // FP32 steps: the reference state of the run (or instance); a plain
    // right-hand side (no clock) uses none
    Ref32 R{0.f, 0.f, 0.f, 0.f};
    double ref_rho = 0.0, ref_E = 0.0;
    if constexpr (sizeof(T) == 4) {
        if (dtp != nullptr) {
            const StepScalars* scp = reinterpret_cast<const StepScalars*>(dtp);
            R = Ref32{scp->ref_rhof, scp->ref_Ef, scp->ref_pf, scp->ref_hf};
            ref_rho = scp->ref_rho;
            ref_E = scp->ref_E;
        }
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sS = reinterpret_cast<T*>(smem_raw);
    T* sF = sS + NV * TL * SP;
    // prefetched L (FP32 accumulating sweeps).  A sweep whose node phase
    // needs neither the staged nodes (plain Eq. 3, no source) nor a fused
    // stage loads L after the faces into the staged nodes' space: the tile
    // then needs less shared memory and more CTAs fit on an SM.
    const bool aliasL = kPre && a.alias_L != 0;
    T* sL = aliasL ? sS : sF + NV * TL * NF;
    // fused stage combination (FP32 x sweep): prefetched base state and increment
    double* sU0 = reinterpret_cast<double*>(smem_raw + G::front_bytes(aliasL));
    float* sD = reinterpret_cast<float*>(sU0 + (G::FUSE_SMEM ? NV * TL * TS : 0));
    float* sUf = reinterpret_cast<float*>(sU0);   // stage 2: float(U0) in the same space

    long long sd;
    int lcount;
    long long base0, lstride;   // base offset of local line l = base0 + l * lstride
    long long line0;            // global line index of local line 0 (for flags)
    if (DIR == 0) {
        // rows of x lines: the product of the other extents (a 64-bit N / nx
        // here, once per thread and tile, cost 1% of the x sweep's
        // instructions)
        const int rows = ND == 1 ? 1 : (ND == 2 ? ny : ny * nz);
        sd = 1;
        lcount = min(TL, rows - lfirst);
        base0 = (long long)lfirst * nx;
        lstride = nx;
        line0 = lfirst;
    } else {
        sd = (DIR == 1) ? (long long)nx : (long long)nx * ny;
        lcount = min(TL, nx - lfirst);
        base0 = (DIR == 1 ? outer * nx * ny : outer * nx) + lfirst;
        lstride = 1;
        line0 = outer * nx + lfirst;
    }
    const int tcount = min(TS, nd - pos0);
    const int nfaces = tcount + 5;

    // (1) stage nodes pos0-5 .. pos0+TS+4 of each line (the node of staged
    // position s is p = pos0 - 5 + s, boundary-mapped).  Positions lie in
    // [pos0 - 5, pos0 + TS + 5), so one conditional wrap suffices unless the
    // periodic axis is shorter than the staged window.  The staged x lines
    // may start up to 3 positions early (soff) so that their copies are
    // 16-byte aligned; the faces read from sSr = sS + soff.
    const LT* U = Ub;
    const bool wrap_mod = periodic && nd < P;
    // reflecting walls (ghost -1-k mirrors node k, normal momentum negated;
    // the axis has at least 5 nodes) and fixed states: synchronous copies
    const bool bc_special = bcl >= BC_REFLECTING || bch >= BC_REFLECTING;
    // node p of line l into staged position sm
    auto stage_pos = [&](int l, int sm, int p) {
        if (periodic) {
            if (wrap_mod) { p %= nd; if (p < 0) p += nd; }
            else p = p < 0 ? p + nd : (p >= nd ? p - nd : p);
        } else if (bc_special && (p < 0 || p >= nd)) {
            const int kind = p < 0 ? bcl : bch;
            if (kind == BC_FIXED) {
                const double* st = bcs[p < 0 ? 0 : 1];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const double r = v == 0 ? ref_rho : (v == NV - 1 ? ref_E : 0.0);
                    sS[sidx<DIR, TL, SP>(v, l, sm)] = stage_cvt<T>(st[v] - r);
                }
                return;
            }
            if (kind == BC_REFLECTING) {
                // (clamped: positions past the last node a face needs, in a
                // short final tile, would mirror to before the line's start)
                const int q = min(max(p < 0 ? -1 - p : 2 * nd - 1 - p, 0), nd - 1);
                const LT* src = U + base0 + l * lstride + (long long)q * sd;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const T val = stage_cvt<T>(src[v * N]);
                    sS[sidx<DIR, TL, SP>(v, l, sm)] = v == 1 + DIR ? -val : val;
                }
                return;
            }
            p = p < 0 ? 0 : nd - 1;   // the other side is transmissive
        } else {
            p = min(max(p, 0), nd - 1);
        }
        const LT* src = U + base0 + l * lstride + (long long)p * sd;
#pragma unroll
        for (int v = 0; v < NV; ++v, src += N) {
            if constexpr (kAsyncStage) cp_async4(&sS[sidx<DIR, TL, SP>(v, l, sm)], src);
            else sS[sidx<DIR, TL, SP>(v, l, sm)] = stage_cvt<T>(*src);
        }
    };
    // 16-byte copies need x extents a multiple of 4 (every line and variable
    // block then starts 16-byte aligned) and a 16-byte aligned state
    bool vec4 = false;
    if constexpr (kAsyncStage)
        vec4 = (nx & 3) == 0 && (reinterpret_cast<unsigned long long>(Ub) & 15ull) == 0;
    int soff = 0;
    bool staged = false;
    if constexpr (kAsyncStage && DIR == 0) {
        if (vec4) {
            // x lines: aligned chunks of 4 nodes from x0 = floor4(pos0 - 5); a
            // chunk inside the line is one copy per variable, one at an end of
            // the line is staged node by node
            const int x0 = (pos0 - GHOST) & ~3;
            soff = pos0 - GHOST - x0;
            constexpr int NC = SP / 4;
            for (int e = threadIdx.x; e < TL * NC; e += blockDim.x) {
                const int c = e % NC, l = e / NC;
                if (l >= lcount) continue;
                const int pc = x0 + 4 * c;
                if (pc >= 0 && pc + 4 <= nd) {
                    const LT* src = U + base0 + l * lstride + pc;
#pragma unroll
                    for (int v = 0; v < NV; ++v, src += N) cp_async16(&sS[sidx<DIR, TL, SP>(v, l, 4 * c)], src);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) stage_pos(l, 4 * c + i, pc + i);
                }
            }
            staged = true;
        }
    } else if constexpr (kAsyncStage && DIR != 0 && TL % 4 == 0) {
        if (vec4) {
            // y/z: the lines are x-adjacent, so four lines of a node position are
            // one copy per variable (lcount is a multiple of 4: lfirst is a
            // multiple of TL)
            constexpr int TLW = TL / 4;
            for (int e = threadIdx.x; e < TLW * P; e += blockDim.x) {
                const int l = (e % TLW) * 4, s = e / TLW;
                if (l >= lcount) continue;
                int p = pos0 - GHOST + s;
                if (!periodic && bc_special && (p < 0 || p >= nd)) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) stage_pos(l + i, s, p);
                    continue;
                }
                if (periodic) {
                    if (wrap_mod) { p %= nd; if (p < 0) p += nd; }
                    else p = p < 0 ? p + nd : (p >= nd ? p - nd : p);
                } else {
                    p = min(max(p, 0), nd - 1);
                }
                const LT* src = U + base0 + l + (long long)p * sd;
#pragma unroll
                for (int v = 0; v < NV; ++v, src += N) cp_async16(&sS[sidx<DIR, TL, SP>(v, l, s)], src);
            }
            staged = true;
        }
    }
    if (!staged) {
        for (int e = threadIdx.x; e < TL * P; e += blockDim.x) {
            int l, s;
            if (DIR == 0) { s = e % P; l = e / P; } else { l = e % TL; s = e / TL; }
            if (l >= lcount) continue;
            stage_pos(l, s, pos0 - GHOST + s);
        }
    }
    const T* sSr = sS + soff;
    if constexpr (kAsync) cp_async_commit();   // group: staged nodes
    if constexpr (kAsyncStage) {
        if (dtp != nullptr && f64_is_zero(*dtp)) {
            cp_async_wait<0>();
            return;
        }
    }
    // y/z sweeps with 16-byte copies and a 16-byte aligned L: four x-adjacent
    // lines of a node per copy, and four lines per thread in the Eq. 3 node
    // phase (128-bit shared and global accesses, packed arithmetic)
    bool vecL = false;
    if constexpr (sizeof(T) == 4 && DIR != 0 && TL % 4 == 0)
        vecL = vec4 && (reinterpret_cast<unsigned long long>(Lb) & 15ull) == 0;
    const bool diff_md = a.K.diff == DIFF_MD;
    // the previous sweep of this RHS has finished (and its L is visible)
    bool dep_done = a.pdl == 0;
    auto dep_wait = [&]() {
        if (!dep_done) {
            asm volatile("griddepcontrol.wait;\n" ::: "memory");
            dep_done = true;
        }
    };
    // the accumulated L: read straight from global memory by the y/z node
    // phase of four lines per thread and by a fused stage that reads its
    // operands from global memory, else copied into sL
    bool directL = vecL && diff_md && !source;
    if constexpr (G::FUSE && !G::FUSE_SMEM) directL = directL || a.fuse_stage != 0;
    // the L values this tile adds to (cp.async into sL)
    auto prefetch_L = [&]() {
        const T* Lg = Lb;
        if constexpr (sizeof(T) == 4 && DIR != 0 && TL % 4 == 0) {
            if (vecL) {
                constexpr int TLW = TL / 4;
                for (int e = threadIdx.x; e < TLW * TS; e += blockDim.x) {
                    const int l = (e % TLW) * 4, t = e / TLW;
                    if (l >= lcount || t >= tcount) continue;
                    const T* src = Lg + base0 + l + (long long)(pos0 + t) * sd;
#pragma unroll
                    for (int v = 0; v < NV; ++v, src += N) cp_async16(&sL[sidx<DIR, TL, TS>(v, l, t)], src);
                }
                return;
            }
        }
        for (int e = threadIdx.x; e < TL * TS; e += blockDim.x) {
            int l, t;
            if (DIR == 0) { t = e % TS; l = e / TS; } else { l = e % TL; t = e / TL; }
            if (l >= lcount || t >= tcount) continue;
            const T* src = Lg + base0 + l * lstride + (long long)(pos0 + t) * sd;
#pragma unroll
            for (int v = 0; v < NV; ++v, src += N) cp_async4(&sL[sidx<DIR, TL, TS>(v, l, t)], src);
        }
    };
    if constexpr (kPre) {
        if (a.accumulate && !aliasL && !directL) {
            dep_wait();
            prefetch_L();                      // group: lands while the faces are computed
        }
        if constexpr (G::FUSE_SMEM) {
            // stage 1 needs float(U0) = its own staged input; stage 2 reads
            // float(U0) from the output buffer it then overwrites; stage 3
            // accumulates into the FP64 state
            if (a.fuse_stage > 1) {
                const bool s3 = a.fuse_stage == 3;
                for (int e = threadIdx.x; e < TL * TS; e += blockDim.x) {
                    const int t = e % TS, l = e / TS;
                    if (l >= lcount || t >= tcount) continue;
                    const long long g = base0 + l * lstride + (long long)(pos0 + t) * sd;
                    const float* Dp = Db + g;
                    if (s3) {
                        const double* U0p = U0b + g;
#pragma unroll
                        for (int v = 0; v < NV; ++v, U0p += N, Dp += N) {
                            cp_async8(&sU0[sidx<DIR, TL, TS>(v, l, t)], U0p);
                            cp_async4(&sD[sidx<DIR, TL, TS>(v, l, t)], Dp);
                        }
                    } else {
                        const float* Sp = Sob + g;
#pragma unroll
                        for (int v = 0; v < NV; ++v, Sp += N, Dp += N) {
                            cp_async4(&sUf[sidx<DIR, TL, TS>(v, l, t)], Sp);
                            cp_async4(&sD[sidx<DIR, TL, TS>(v, l, t)], Dp);
                        }
                    }
                }
            }
        }
        cp_async_commit();
        cp_async_wait<1>();                    // staged nodes have landed
    } else if constexpr (kAsync) {
        cp_async_wait<0>();
    }
    // the deferred-face list of step (2), emptied before this barrier
    constexpr bool kDefer = sizeof(T) == 4 && WT == W_TENO && ND == 3;
    __shared__ int s_slow[kDefer ? TL * NF : 1];
    __shared__ int s_nslow;
    if (kDefer && threadIdx.x == 0) s_nslow = 0;
    __syncthreads();

    // (2) midpoint fluxes of faces j + 1/2, j = pos0 - 3 + f.  3D FP32 TENO
    // sweeps defer a face whose selection needs the full cutoff (Eq. 16-18)
    // to a second pass over a shared list: the first pass carries only the
    // exact no-cut test, and the few deferred faces then run the full code
    // side by side in whole warps instead of as divergent branches (5% off
    // the Taylor-Green step).  A deferred face is evaluated twice, so where
    // cuts are frequent (shocked 1D batches: 5% slower) the single pass stays.
    int fb = 0;
    auto load_face = [&](int l, int f, T (&u)[6][NV]) {
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int v = 0; v < NV; ++v) u[m][v] = sSr[sidx<DIR, TL, SP>(v, l, f + m)];
    };
    auto store_face = [&](int l, int f, const T (&F)[NV], const uint8_t (&fl)[NV], bool fell) {
        // faces shared with the next tile are owned (counted, flagged) by it
        const bool owned = f < TS || pos0 + TS >= nd;
        fb += (fell && owned) ? 1 : 0;
#pragma unroll
        for (int v = 0; v < NV; ++v) sF[sidx<DIR, TL, NF>(v, l, f)] = F[v];
        if (a.flags != nullptr && owned) {
            const long long lines = N / nd;
            const long long j3 = pos0 + f;   // j + 3
#pragma unroll
            for (int k = 0; k < NV; ++k)
                a.flags[((long long)k * lines + line0 + l) * (nd + 5) + j3] = fl[k];
        }
    };
    for (int e = threadIdx.x; e < TL * NF; e += blockDim.x) {
        int l, f;
        if (DIR == 0) { f = e % NF; l = e / NF; } else { l = e % TL; f = e / TL; }
        if (l >= lcount || f >= nfaces) continue;
        T u[6][NV];
        load_face(l, f, u);
        T F[NV];
        uint8_t fl[NV];
        bool fell = false;
        if (!face_flux<ND, DIR, FLUX, WT, kDefer>(u, a, R, F, fl, fell)) {
            s_slow[atomicAdd(&s_nslow, 1)] = e;
            continue;
        }
        store_face(l, f, F, fl, fell);
    }
    // synced: every face is stored and every staged node read, as of the
    // last barrier (a tile with no deferred face needs no other barrier
    // unless the node phase reads asynchronously copied data)
    bool synced = false;
    if constexpr (kDefer) {
        __syncthreads();
        const int nslow = s_nslow;
        synced = nslow == 0;
        for (int k = threadIdx.x; k < nslow; k += blockDim.x) {
            const int e = s_slow[k];
            int l, f;
            if (DIR == 0) { f = e % NF; l = e / NF; } else { l = e % TL; f = e / TL; }
            T u[6][NV];
            load_face(l, f, u);
            T F[NV];
            uint8_t fl[NV];
            bool fell = false;
            face_flux<ND, DIR, FLUX, WT, false>(u, a, R, F, fl, fell);
            store_face(l, f, F, fl, fell);
        }
    }
    if (fb) atomicAdd((unsigned long long*)fbp, (unsigned long long)fb);
    if constexpr (kPre) {
        bool pending = a.accumulate && !aliasL && !directL;   // prefetched before the faces
        if constexpr (G::FUSE_SMEM) pending = pending || a.fuse_stage > 1;
        if (aliasL && a.accumulate && !directL) {
            if (!synced) __syncthreads();      // every face has read the staged nodes
            dep_wait();
            prefetch_L();
            cp_async_commit();
            pending = true;
        }
        if (pending) {
            cp_async_wait<0>();                // the copies have landed
            synced = false;
        }
    }
    if (!synced) __syncthreads();

    // (3) Eq. 3 (or Eq. 4, 5) at nodes pos0 .. pos0 + tcount - 1.  The node
    // loop is instantiated per variant (ALT, fused stage, accumulate) so that
    // each carries no run-time branch per variable: the Eq. 3 loop has no
    // trace of the node fluxes Eq. 4-5 need, and a fused stage only its own
    // reads and writes.
    const int diff = a.K.diff;
    // dt of the fused stage in FP32, converted once per thread
    float dtf = 0.f;
    if constexpr (G::FUSE) {
        if (a.fuse_stage) dtf = f64_to_f32_ftz(*dtp);
    }
    // ALT: Eq. 4-5 and / or the body-force source; the plain Eq. 3 instance
    // carries neither.  STAGE: the fused SSP-RK3 stage (0: none, L written).
    // ACC: L accumulates (every direction after the first).
    auto node_phase = [&](auto alt_tag, auto stage_tag, auto acc_tag) {
        constexpr bool ALT = decltype(alt_tag)::value;
        constexpr int STAGE = decltype(stage_tag)::value;
        constexpr bool ACC = decltype(acc_tag)::value;
        if constexpr (sizeof(T) == 4 && DIR != 0 && TL % 4 == 0 && !ALT && STAGE == 0) {
            if (vecL) {
                // lanes = the four lines; every lane rounds as the scalar loop
                // (the negated coefficients give -f' exactly: rounding to
                // nearest is symmetric)
                constexpr int TLW = TL / 4;
                const float2 ih2 = bc2(ih), a1 = bc2(-T(MD_A1)), a2 = bc2(-T(MD_A2)), a3 = bc2(-T(MD_A3));
                for (int e = threadIdx.x; e < TLW * TS; e += blockDim.x) {
                    const int l = (e % TLW) * 4, t = e / TLW;
                    if (l >= lcount || t >= tcount) continue;
                    float4* Lp = reinterpret_cast<float4*>(Lb + base0 + l + (long long)(pos0 + t) * sd);
                    const long long N4 = N / 4;
                    // the L being accumulated, all variables loaded at once
                    float4 pv4[ACC ? NV : 1];
                    if constexpr (ACC) {
#pragma unroll
                        for (int v = 0; v < NV; ++v) pv4[v] = Lp[v * N4];
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v, Lp += N4) {
                        float2 f[6][2];
#pragma unroll
                        for (int m = 0; m < 6; ++m) {
                            const float4 q = *reinterpret_cast<const float4*>(&sF[sidx<DIR, TL, NF>(v, l, t + m)]);
                            f[m][0] = make_float2(q.x, q.y);
                            f[m][1] = make_float2(q.z, q.w);
                        }
                        const float4 prev = ACC ? pv4[v] : make_float4(0.f, 0.f, 0.f, 0.f);
                        float2 out[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 nfp = fma2(a1, sub2(f[3][h], f[2][h]),
                                                    fma2(a2, sub2(f[4][h], f[1][h]), mul2(a3, sub2(f[5][h], f[0][h]))));
                            if constexpr (ACC) {
                                const float2 pv = h == 0 ? make_float2(prev.x, prev.y) : make_float2(prev.z, prev.w);
                                out[h] = fma2(nfp, ih2, pv);
                            } else {
                                out[h] = mul2(nfp, ih2);
                            }
                        }
                        *Lp = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
                    }
                }
                return;
            }
        }
        for (int e = threadIdx.x; e < TL * TS; e += blockDim.x) {
            int l, t;
            if (DIR == 0) { t = e % TS; l = e / TS; } else { l = e % TL; t = e / TL; }
            if (l >= lcount || t >= tcount) continue;
            const long long g = base0 + l * lstride + (long long)(pos0 + t) * sd;
            // this node's elements of variable v: pointer + v N, advanced per variable
            T* Lp = Lb + g;
            float* Dp = Db + g;
            float* Sp = Sob + g;
            double* U0p = U0b + g;
            // a fused stage's operands when the tile does not stage them in
            // shared memory: loaded here, all variables at once, so that the
            // loads overlap one another and the Eq. 3 arithmetic below
            // (with the L being accumulated)
            constexpr bool kDirectL = ACC && STAGE != 0 && !G::FUSE_SMEM;
            // (stage 1's float(U0), its own staged input, is still in sS: a
            // fused stage's L is never copied there)
            float fa[STAGE == 2 && !G::FUSE_SMEM ? NV : 1], fd[STAGE != 0 && !G::FUSE_SMEM ? NV : 1];
            double fu[STAGE == 3 && !G::FUSE_SMEM ? NV : 1];
            T fl0[kDirectL ? NV : 1];
            if constexpr (STAGE != 0 && !G::FUSE_SMEM) {
                const float* Dq = Dp;
                const float* Sq = Sob + g;
                const double* Uq = U0b + g;
                const T* Lq = Lp;
#pragma unroll
                for (int v = 0; v < NV; ++v, Dq += N, Sq += N, Uq += N, Lq += N) {
                    if constexpr (kDirectL) fl0[v] = *Lq;
                    if constexpr (STAGE == 2) fa[v] = *Sq;          // float(U0)
                    if constexpr (STAGE >= 2) fd[v] = *Dq;
                    if constexpr (STAGE == 3) fu[v] = *Uq;
                }
            }
            // Eq. 4-5 also difference the physical fluxes of the nodes i+-1
            // (and i+-2): d1 = f_{i+1} - f_{i-1}, d2 = f_{i+2} - f_{i-2}
            T d1[NV], d2[NV], S[NV];
            if constexpr (ALT) {
#pragma unroll
                for (int v = 0; v < NV; ++v) d1[v] = d2[v] = S[v] = T(0);
                if (diff != DIFF_MD) node_flux_diff<ND, DIR, TL, SP>(sSr, l, t + GHOST, 1, a.K, R, d1);
                if (diff == DIFF_HWCNS) node_flux_diff<ND, DIR, TL, SP>(sSr, l, t + GHOST, 2, a.K, R, d2);
                if (source) {
                    // (0, rho g_a, sum_a g_a m_a), the sum from 0 in axis order
                    T rho = sSr[sidx<DIR, TL, SP>(0, l, t + GHOST)];
                    if constexpr (sizeof(T) == 4) rho = rho + R.rho;
                    T se = T(0);
#pragma unroll
                    for (int b = 0; b < ND; ++b) {
                        const T gb = T(gravp[b]), mb = sSr[sidx<DIR, TL, SP>(1 + b, l, t + GHOST)];
                        if constexpr (sizeof(T) == 8) {
                            S[1 + b] = mul_(gb, rho);
                            se = add_(se, mul_(gb, mb));
                        } else {
                            S[1 + b] = gb * rho;
                            se = fma(gb, mb, se);
                        }
                    }
                    S[NV - 1] = se;
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T f0 = sF[sidx<DIR, TL, NF>(v, l, t + 0)], f1 = sF[sidx<DIR, TL, NF>(v, l, t + 1)];
                const T f2 = sF[sidx<DIR, TL, NF>(v, l, t + 2)], f3 = sF[sidx<DIR, TL, NF>(v, l, t + 3)];
                const T f4 = sF[sidx<DIR, TL, NF>(v, l, t + 4)], f5 = sF[sidx<DIR, TL, NF>(v, l, t + 5)];
                if constexpr (sizeof(T) == 8) {
                    double q;                                      // L -= f'
                    if constexpr (ALT)
                        q = diff == DIFF_MD ? md_fp64(f0, f1, f2, f3, f4, f5, ih)
                                            : mul_(diff_alt_fp64(diff, f1, f2, f3, f4, d1[v], d2[v]), ih);
                    else q = md_fp64(f0, f1, f2, f3, f4, f5, ih);
                    double lval;
                    if constexpr (ACC) lval = sub_(*Lp, q);
                    else lval = -q;
                    if constexpr (ALT) {
                        if (source && v > 0) lval = add_(lval, S[v]);   // after every direction
                    }
                    *Lp = lval;
                } else {
                    T fp;
                    if constexpr (!ALT)
                        fp = fma(T(MD_A1), f3 - f2, fma(T(MD_A2), f4 - f1, T(MD_A3) * (f5 - f0)));
                    else if (diff == DIFF_MD)
                        fp = fma(T(MD_A1), f3 - f2, fma(T(MD_A2), f4 - f1, T(MD_A3) * (f5 - f0)));
                    else if (diff == DIFF_HWCNS)
                        fp = fma(T(HW_B1), f3 - f2, fma(T(HW_B2), d1[v], T(HW_B3) * d2[v]));
                    else
                        fp = fma(T(MND_C1), f3 - f2, fma(T(MND_C2), d1[v], T(MND_C3) * (f4 - f1)));
                    // L = -f' (first direction) or L - f'
                    T lv;
                    if constexpr (ACC) {
                        if constexpr (kDirectL) lv = fmaf(-fp, ih, fl0[kDirectL ? v : 0]);
                        else if constexpr (kPre) lv = fmaf(-fp, ih, sL[sidx<DIR, TL, TS>(v, l, t)]);
                        else lv = fmaf(-fp, ih, *Lp);
                    } else {
                        lv = -fp * ih;
                    }
                    if constexpr (ALT) {
                        if (source) lv += S[v];
                    }
                    // SSP-RK3 stage on U = U0 + D (FP64 base, FP32 increment):
                    //   D1 = dt L;  D2 = (D1 + dt L)/4;  U0 += 2/3 (D2 + dt L)
                    // The next stage's input is float(U0) + D; float(U0) is
                    // this stage's staged input in stage 1 and the prefetched
                    // output buffer in stage 2 (the step starts from float(U0)).
                    if constexpr (STAGE == 1) {
                        const float dd = dtf * lv;
                        const float u0f = sSr[sidx<DIR, TL, SP>(v, l, t + GHOST)];
                        *Dp = dd;
                        *Sp = u0f + dd;
                    } else if constexpr (STAGE == 2) {
                        const float d1 = G::FUSE_SMEM ? sD[sidx<DIR, TL, TS>(v, l, t)] : fd[G::FUSE_SMEM ? 0 : v];
                        const float u0f = G::FUSE_SMEM ? sUf[sidx<DIR, TL, TS>(v, l, t)] : fa[G::FUSE_SMEM ? 0 : v];
                        const float dd = 0.25f * fmaf(dtf, lv, d1);
                        *Dp = dd;
                        *Sp = u0f + dd;
                    } else if constexpr (STAGE == 3) {
                        // the next step's first input float(U) comes from its
                        // time-step pass, so stage 3 writes the FP64 state only
                        const double u0 = G::FUSE_SMEM ? sU0[sidx<DIR, TL, TS>(v, l, t)] : fu[G::FUSE_SMEM ? 0 : v];
                        const float d2 = G::FUSE_SMEM ? sD[sidx<DIR, TL, TS>(v, l, t)] : fd[G::FUSE_SMEM ? 0 : v];
                        const float dd = (2.0f / 3.0f) * fmaf(dtf, lv, d2);
                        *U0p = u0 + f32_to_f64_ftz(dd);
                    } else {
                        *Lp = lv;
                    }
                }
                Lp += N;
                if constexpr (STAGE != 0) {
                    Dp += N;
                    Sp += N;
                    U0p += N;
                }
            }
        }
    };
    using std::integral_constant;
    auto run_nodes = [&](auto alt_tag) {
        if constexpr (G::FUSE) {
            if (a.fuse_stage != 0) {
                const bool acc = a.accumulate != 0;
                if (a.fuse_stage == 1) {
                    if (acc) node_phase(alt_tag, integral_constant<int, 1>{}, std::true_type{});
                    else node_phase(alt_tag, integral_constant<int, 1>{}, std::false_type{});
                } else if (a.fuse_stage == 2) {
                    if (acc) node_phase(alt_tag, integral_constant<int, 2>{}, std::true_type{});
                    else node_phase(alt_tag, integral_constant<int, 2>{}, std::false_type{});
                } else {
                    if (acc) node_phase(alt_tag, integral_constant<int, 3>{}, std::true_type{});
                    else node_phase(alt_tag, integral_constant<int, 3>{}, std::false_type{});
                }
                return;
            }
        }
        if (a.accumulate) node_phase(alt_tag, integral_constant<int, 0>{}, std::true_type{});
        else node_phase(alt_tag, integral_constant<int, 0>{}, std::false_type{});
    };
    dep_wait();
    if (diff == DIFF_MD && !source) run_nodes(std::false_type{});
    else run_nodes(std::true_type{});
}

// The sweep kernel.  Single grids and tile-table batches run one tile per
// CTA.  Persistent batched launches (a.work non-null) start a fixed number of
// CTAs, each of which takes tiles from a device counter (atomicAdd) until the
// table is exhausted; no CTA waits for another, so nothing can hang.
template <typename T, typename LT, int ND, int DIR, int FLUX, bool BATCH = false, int CFG = 0, int WT = 0>
__global__ void __launch_bounds__(256, TileGeom<T, ND, DIR, CFG>::MIN_CTAS) sweep_kernel(const SweepArgs a)
{
    // a sweep launched as this one's programmatic dependent may start as
    // soon as every CTA of this grid is running (it waits for this grid's
    // completion itself before it touches L)
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    if constexpr (BATCH) {
        if (a.work != nullptr) {
            __shared__ long long s_tile;
            for (;;) {
                __syncthreads();   // the previous tile is done with shared memory
                if (threadIdx.x == 0) s_tile = (long long)atomicAdd(a.work, 1u);
                __syncthreads();
                const long long t = s_tile;
                if (t >= a.ntiles) return;
                sweep_tile<T, LT, ND, DIR, FLUX, BATCH, CFG, WT>(a, t);
            }
        }
        sweep_tile<T, LT, ND, DIR, FLUX, BATCH, CFG, WT>(a, blockIdx.x);
    } else {
        sweep_tile<T, LT, ND, DIR, FLUX, BATCH, CFG, WT>(a, 0);
    }
}

}  // namespace wcns
