// wcns_internal.h -- launch interface between the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>
#include "wcns_sweep.cuh"

namespace wcns {

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
