// wcns_internal.h -- launch interface between the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include "../../include/wcns.h"
#include "wcns_sweep.cuh"

namespace wcns {

static_assert((int)DIFF_MD == (int)WCNS_DIFF_MD6 && (int)DIFF_HWCNS == (int)WCNS_DIFF_HWCNS &&
                  (int)DIFF_MND == (int)WCNS_DIFF_MND && (int)FLUX_AUSM == (int)WCNS_FLUX_AUSM &&
                  (int)FLUX_ROE == (int)WCNS_FLUX_ROE && (int)FLUX_VANLEER == (int)WCNS_FLUX_VANLEER,
              "scheme codes");
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
    K.Cf = (float)p->C;
    K.CTf = (float)p->CT;
    K.Kf = (float)K.keep_all_K;
    K.gammaf = (float)gamma;
    K.gm1f = (float)(gamma - 1.0);
    return K;
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
// Raise the dynamic shared-memory limit of every sweep instance (once per device).
cudaError_t prepare_sweeps_fp64();
cudaError_t prepare_sweeps_fp32();

// Time step, RK stages, reductions (wcns_rk.cu).
struct StepScalars {      // device-resident
    double dt;            // step of the current RK step (0 = finished)
    double t;             // time reached at the end of the current step
    double t_end;         // clip target (inf when unused)
    unsigned long long lam_bits;   // max wave-speed sum (non-negative double bits)
    unsigned long long steps;      // steps that advanced time since the last reset
};

cudaError_t launch_cfl(int nd, const double* U, long long N, const double* h, double gamma,
                       double cfl, int clip, StepScalars* sc, cudaStream_t s);
// FP32-path variant: per-node speeds in FP32 (rounded upward), FP64 max and dt.
cudaError_t launch_cfl_fast(int nd, const double* U, long long N, const double* h, double gamma,
                            double cfl, int clip, StepScalars* sc, cudaStream_t s);
cudaError_t launch_set_dt(double dt, int clip, StepScalars* sc, cudaStream_t s);
cudaError_t launch_reset_clock(double t_end, StepScalars* sc, cudaStream_t s);
// FP64 stage combinations (Shu-Osher SSP-RK3) over M = nv*N values.
cudaError_t launch_rk_fp64(int stage, double* U0, double* U1, const double* L, long long M,
                           const StepScalars* sc, cudaStream_t s);
// S = float(U) (skipped when *dt == 0, i.e. the run has finished).
cudaError_t launch_to_fp32(const double* U, float* S, long long M, const StepScalars* sc, cudaStream_t s);
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
