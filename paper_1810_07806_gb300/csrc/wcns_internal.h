// wcns_internal.h -- launch interface between the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <math.h>
#include <stdio.h>
#include "../../include/wcns.h"
#include "wcns_sweep.cuh"

namespace wcns {

static_assert((int)DIFF_MD == (int)WCNS_DIFF_MD6 && (int)DIFF_HWCNS == (int)WCNS_DIFF_HWCNS &&
                  (int)DIFF_MND == (int)WCNS_DIFF_MND && (int)FLUX_AUSM == (int)WCNS_FLUX_AUSM &&
                  (int)FLUX_ROE == (int)WCNS_FLUX_ROE && (int)FLUX_VANLEER == (int)WCNS_FLUX_VANLEER,
              "scheme codes");
static_assert((int)BC_TRANSMISSIVE == (int)WCNS_BC_TRANSMISSIVE && (int)BC_PERIODIC == (int)WCNS_BC_PERIODIC &&
                  (int)BC_REFLECTING == (int)WCNS_BC_REFLECTING && (int)BC_FIXED == (int)WCNS_BC_FIXED,
              "boundary codes");
static_assert((int)W_TENO == (int)WCNS_W_TENO && (int)W_JS == (int)WCNS_W_JS &&
                  (int)W_LINEAR == (int)WCNS_W_LINEAR && (int)W_Z == (int)WCNS_W_Z,
              "weight codes");

// Checks the scheme options every entry point shares: nullptr when valid,
// otherwise the reason.
inline const char* scheme_params_error(const wcns_scheme_params* p)
{
    if (p->flux != WCNS_FLUX_ROE && p->flux != WCNS_FLUX_VANLEER && p->flux != WCNS_FLUX_AUSM)
        return "unsupported flux";
    if (p->diff != WCNS_DIFF_MD6 && p->diff != WCNS_DIFF_HWCNS && p->diff != WCNS_DIFF_MND)
        return "unsupported difference scheme";
    if (p->weights < WCNS_W_TENO || p->weights > WCNS_W_Z) return "unknown weights";
    if (p->precision != WCNS_FP64 && p->precision != WCNS_FP32)
        return "precision must be WCNS_FP64 or WCNS_FP32";
    if (p->characteristic != 1) return "characteristic must be 1";
    if (p->entropy_fix != 0) return "entropy_fix must be 0";
    if (!(p->C > 0.0) || !(p->eps > 0.0) || !(p->CT > 0.0) || !(p->CT < 1.0 / 3.0))
        return "need C > 0, eps > 0, 0 < C_T < 1/3";
    if (p->q < 1 || p->q > 16) return "q must be in 1..16";
    if (p->weights == WCNS_W_JS && !(p->eps_js > 0.0)) return "eps_js must be positive";
    if (!(p->cfl > 0.0)) return "cfl must be positive";
    return nullptr;
}

// A checked grid: node counts, spacings and the boundary rule of each axis.
struct GridInfo {
    int ndim = 0, nv = 0;
    int n[3] = {1, 1, 1};
    long long N = 1;
    double h[3] = {1, 1, 1}, inv_h[3] = {0, 0, 0};
    int periodic[3] = {0, 0, 0};
    int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    double bc_state[3][2][5] = {};
    double gravity[3] = {0, 0, 0};
    bool special_bc = false;   // some side reflects or holds a fixed state
    bool has_gravity = false;
};

// Checks a grid and fills G; nullptr when valid, otherwise the reason (in
// buf).  Spacing: (hi - lo)/(n - 1) when both sides of the axis are
// transmissive, (hi - lo)/n otherwise.
inline const char* grid_error(const wcns_grid* g, double gamma, GridInfo& G, char* buf, size_t bufsz)
{
    if (g->ndim < 1 || g->ndim > 3) return "ndim must be 1, 2 or 3";
    G.ndim = g->ndim;
    G.nv = g->ndim + 2;
    for (int a = 0; a < g->ndim; ++a) {
        const int lo = g->bc[a][0], hi = g->bc[a][1];
        for (int k : {lo, hi})
            if (k < WCNS_BC_TRANSMISSIVE || k > WCNS_BC_FIXED) {
                snprintf(buf, bufsz, "axis %d: unknown boundary kind", a);
                return buf;
            }
        const int per = lo == WCNS_BC_PERIODIC;
        if ((hi == WCNS_BC_PERIODIC) != per) {
            snprintf(buf, bufsz, "axis %d: periodic must be set on both sides", a);
            return buf;
        }
        const bool both_trans = lo == WCNS_BC_TRANSMISSIVE && hi == WCNS_BC_TRANSMISSIVE;
        const bool reflect = lo == WCNS_BC_REFLECTING || hi == WCNS_BC_REFLECTING;
        if (g->n[a] < (both_trans ? 2 : (reflect ? 5 : 1)) || !(g->hi[a] > g->lo[a])) {
            snprintf(buf, bufsz, "axis %d: bad node count or extent (a reflecting axis needs 5 nodes)", a);
            return buf;
        }
        for (int sd = 0; sd < 2; ++sd) {
            G.bc[a][sd] = g->bc[a][sd];
            if (g->bc[a][sd] == WCNS_BC_REFLECTING) G.special_bc = true;
            if (g->bc[a][sd] != WCNS_BC_FIXED) continue;
            G.special_bc = true;
            const double* st = g->bc_state[a][sd];
            double ke = 0.0;
            for (int b = 0; b < g->ndim; ++b) ke += st[1 + b] * st[1 + b];
            const double p = (gamma - 1.0) * (st[g->ndim + 1] - 0.5 * ke / st[0]);
            if (!(st[0] > 0.0) || !(p > 0.0) || !isfinite(p)) {
                snprintf(buf, bufsz, "axis %d side %d: the fixed state needs rho > 0 and p > 0", a, sd);
                return buf;
            }
            for (int v = 0; v < G.nv; ++v) G.bc_state[a][sd][v] = st[v];
        }
        G.n[a] = g->n[a];
        G.periodic[a] = per;
        G.h[a] = (g->hi[a] - g->lo[a]) / (both_trans ? g->n[a] - 1 : g->n[a]);
        G.inv_h[a] = 1.0 / G.h[a];
        G.N *= g->n[a];
        if (!isfinite(g->gravity[a])) return "gravity must be finite";
        G.gravity[a] = g->gravity[a];
        if (g->gravity[a] != 0.0) G.has_gravity = true;
    }
    return nullptr;
}

// Reflecting or fixed sides, or a body force (the allocation-free step does
// not take them).
inline bool grid_has_single_grid_features(const wcns_grid* g)
{
    for (int a = 0; a < g->ndim && a < 3; ++a) {
        if (g->bc[a][0] >= WCNS_BC_REFLECTING || g->bc[a][1] >= WCNS_BC_REFLECTING) return true;
        if (g->gravity[a] != 0.0) return true;
    }
    return false;
}

// Device constants of a valid parameter set.
inline SchemeConst make_scheme_const(const wcns_scheme_params* p, double gamma)
{
    SchemeConst K{};
    K.gamma = gamma;
    K.gm1 = gamma - 1.0;
    K.C = p->C;
    K.eps = p->eps;
    K.CT = p->CT;
    K.q = p->q;
    K.weights = p->weights;
    K.eps_js = p->eps_js;
    K.diff = p->diff;
    K.sqrt_eps_jsf = (float)sqrt(p->eps_js > 0.0 ? p->eps_js : 0.0);
    // A stencil can only be cut if max g / min g exceeds (3 C_T)^(-1/q); since
    // max g / min g <= 1 + tau / (C (min beta + eps)), tau below
    // 0.98 (ratio - 1) C (min beta + eps) keeps all three.
    K.keep_all_K = 0.98 * (pow(3.0 * p->CT, -1.0 / p->q) - 1.0) * p->C;
    K.screen_lo = pow(p->CT * (1.0 - 1e-9), 1.0 / p->q) * (1.0 - 1e-9);
    K.screen_hi = pow(3.0 * p->CT * (1.0 + 1e-9), 1.0 / p->q) * (1.0 + 1e-9);
    K.Cf = (float)p->C;
    K.CTf = (float)p->CT;
    K.Kf = (float)K.keep_all_K;
    K.gammaf = (float)gamma;
    K.gm1f = (float)(gamma - 1.0);
    return K;
}

// Invariants of every tile shape a sweep is compiled for: the TL x (TS + 5)
// face slots fill whole passes of the CTA's threads (the face and node loops
// stride by them), a staged x line has a 16-byte multiple pitch with room for
// its aligned start (up to 3 nodes before pos0 - 5; y/z lines are the fast
// index, so there TL a multiple of 4 gives the 16-byte alignment), and the
// 16-line x tile leaves room for 4 CTAs per SM.
template <typename T, int ND, int DIR, int CFG>
constexpr bool tile_shape_ok()
{
    using G = TileGeom<T, ND, DIR, CFG>;
    return (G::TL * G::NF) % G::THREADS == 0 &&
           (DIR == 0 ? G::SP % 4 == 0 && G::SP >= G::P + 3 : G::SP == G::P && G::TL % 4 == 0) && G::TS >= 1 &&
           G::TL >= 1;
}
template <typename T>
constexpr bool all_tile_shapes_ok()
{
    return tile_shape_ok<T, 1, 0, 0>() && tile_shape_ok<T, 1, 0, 1>() &&
           tile_shape_ok<T, 2, 0, 0>() && tile_shape_ok<T, 2, 0, 1>() && tile_shape_ok<T, 2, 0, 2>() &&
           tile_shape_ok<T, 2, 1, 0>() && tile_shape_ok<T, 2, 1, 1>() && tile_shape_ok<T, 2, 1, 2>() &&
           tile_shape_ok<T, 3, 0, 0>() && tile_shape_ok<T, 3, 0, 1>() && tile_shape_ok<T, 3, 0, 2>() &&
           tile_shape_ok<T, 3, 1, 0>() && tile_shape_ok<T, 3, 1, 1>() && tile_shape_ok<T, 3, 1, 2>() &&
           tile_shape_ok<T, 3, 2, 0>() && tile_shape_ok<T, 3, 2, 1>() && tile_shape_ok<T, 3, 2, 2>();
}
static_assert(all_tile_shapes_ok<float>() && all_tile_shapes_ok<double>(), "sweep tile shape invariants");
static_assert(TileGeom<float, 3, 0, 1>::smem_bytes(true) + 4096 <= 56 * 1024,
              "the 16-line x tile must leave room for 4 CTAs per SM");

// Launch one sweep kernel; a.pdl: as a programmatic dependent of the
// previous kernel on the stream (the sweep waits for it before its first
// access to L, see SweepArgs::pdl).
template <typename Kernel>
inline cudaError_t launch_sweep_kernel(Kernel k, dim3 grid, int threads, size_t smem, cudaStream_t s,
                                       const SweepArgs& a)
{
    if (!a.pdl) {
        k<<<grid, threads, smem, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

// Launch a batched sweep kernel k over ntiles tiles: one CTA per tile, or
// (a.work set) the persistent form with as many CTAs as are resident on the
// device (`resident`: a per-kernel cache, 0 until first computed; atomic, so
// host threads launching at once may both compute it, without a race).
template <typename Kernel>
inline cudaError_t launch_tiles(Kernel k, int threads, size_t smem, const SweepArgs& a, long long ntiles,
                                cudaStream_t s, std::atomic<int>& resident)
{
    if (ntiles <= 0) return cudaSuccess;
    long long grid = ntiles;
    if (a.work != nullptr) {
        int res = resident.load(std::memory_order_relaxed);
        if (res == 0) {
            int dev = 0, sms = 0, per = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem);
            if (e != cudaSuccess) return e;
            res = sms * (per > 0 ? per : 1);
            resident.store(res, std::memory_order_relaxed);
        }
        if (grid > res) grid = res;
    }
    return launch_sweep_kernel(k, dim3((unsigned)grid), threads, smem, s, a);
}

// Launch one sweep of direction dir, FP64 or FP32 (input and output in the
// sweep's precision).
cudaError_t launch_sweep_fp64(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32(int nd, int dir, int flux, int cfg, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32_cfg0(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32_cfg1(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32_cfg2(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t prepare_sweeps_fp32_cfg0();
cudaError_t prepare_sweeps_fp32_cfg1();
cudaError_t prepare_sweeps_fp32_cfg2();
// FP32 sweeps with the comparison weights (tile configuration 0).
cudaError_t launch_sweep_fp32_weights(int wt, int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32_w1(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32_w2(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_fp32_w3(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s);
cudaError_t prepare_sweeps_fp32_weights();
cudaError_t prepare_sweeps_fp32_w1();
cudaError_t prepare_sweeps_fp32_w2();
cudaError_t prepare_sweeps_fp32_w3();
// Batched sweeps over a tile table (wcns_batch.cu); ntiles CTAs.
cudaError_t launch_sweep_batch_fp64(int nd, int dir, int flux, const SweepArgs& a, long long ntiles,
                                    cudaStream_t s);
cudaError_t launch_sweep_batch_fp32(int nd, int dir, int flux, const SweepArgs& a, long long ntiles,
                                    cudaStream_t s);
cudaError_t prepare_sweeps_batch_fp64();
cudaError_t prepare_sweeps_batch_fp32();
// FP32 batched sweeps with the comparison weights (sweep_fp32_weights*.cu)
cudaError_t launch_sweep_batch_fp32_weights(int wt, int nd, int dir, int flux, const SweepArgs& a,
                                            long long ntiles, cudaStream_t s);
cudaError_t launch_sweep_batch_fp32_w1(int nd, int dir, int flux, const SweepArgs& a, long long ntiles,
                                       cudaStream_t s);
cudaError_t launch_sweep_batch_fp32_w2(int nd, int dir, int flux, const SweepArgs& a, long long ntiles,
                                       cudaStream_t s);
cudaError_t launch_sweep_batch_fp32_w3(int nd, int dir, int flux, const SweepArgs& a, long long ntiles,
                                       cudaStream_t s);
// Raise the dynamic shared-memory limit of every sweep instance (once per device).
cudaError_t prepare_sweeps_fp64();
cudaError_t prepare_sweeps_fp32();

// Time step, RK stages, reductions (wcns_rk.cu).  StepScalars: wcns_sweep.cuh.

cudaError_t launch_cfl(int nd, const double* U, long long N, const double* h, double gamma,
                       double cfl, int clip, StepScalars* sc, cudaStream_t s);
// FP32-path variant: per-node speeds in FP32 (rounded upward), FP64 max and
// dt; S (nullable) receives float(U - U_r), U_r the reference state in sc,
// from the same pass.
cudaError_t launch_cfl_fast(int nd, const double* U, long long N, const double* h, double gamma,
                            double cfl, int clip, StepScalars* sc, cudaStream_t s, float* S = nullptr);
cudaError_t launch_set_dt(double dt, int clip, StepScalars* sc, cudaStream_t s);
cudaError_t launch_reset_clock(double t_end, StepScalars* sc, cudaStream_t s);
// FP64 stage combinations (Shu-Osher SSP-RK3) over M = nv*N values.
cudaError_t launch_rk_fp64(int stage, double* U0, double* U1, const double* L, long long M,
                           const StepScalars* sc, cudaStream_t s);
// S = float(U - U_r) with the reference state of sc (sc nullable: U_r = 0);
// skipped when sc->dt == 0, i.e. the run has finished.
cudaError_t launch_to_fp32(int nv, const double* U, float* S, long long N, const StepScalars* sc, cudaStream_t s);
// The FP32 path's reference state of state U (N nodes) into sc: rho_r = min
// rho, p_r = min p (so 0 <= U - U_r <= U in density and energy), E_r =
// p_r / (gamma - 1), m_r = 0.  Three launches on s.
cudaError_t launch_reference(int nd, const double* U, long long N, double gamma, StepScalars* sc,
                             cudaStream_t s);
cudaError_t launch_conserved(int nv, const double* U, long long N, double vol, double* partials,
                             int nblocks, cudaStream_t s);
int conserved_blocks(long long N);

}  // namespace wcns
#include <vector>
struct wcns_batch;
namespace wcns {
// Batch helpers for the serving loop (wcns_batch.cu).
cudaError_t batch_finished_slots(wcns_batch* b, std::vector<int>& out, cudaStream_t s);
int batch_active_count(const wcns_batch* b);
bool batch_fits(const wcns_batch* b, long long nodes);
long long batch_capacity_nodes(const wcns_batch* b);

// Sets the thread-local message returned by wcns_last_error().
void set_last_error(const char* msg);

}  // namespace wcns
