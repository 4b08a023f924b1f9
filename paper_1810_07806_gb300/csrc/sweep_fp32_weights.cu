// sweep_fp32_weights.cu -- FP32 instances of the fused sweep with the
// comparison weights SWEEP_WT (W_JS in this unit; W_LINEAR and W_Z in the
// units that include it, so the three compile in parallel).  Tile
// configuration 0 only; single grids and batches.
#include "wcns_internal.h"

#ifndef SWEEP_WT
#define SWEEP_WT 1
#endif

namespace wcns {
namespace {

template <int ND, int DIR, int FLUX>
cudaError_t go(const SweepArgs& a, cudaStream_t s, bool prepare)
{
    using G = TileGeom<float, ND, DIR, 0>;
    auto k = sweep_kernel<float, float, ND, DIR, FLUX, false, 0, SWEEP_WT>;
    if (prepare)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes());
    SweepArgs b = a;
    b.alias_L = sweep_alias_L(a, G::FUSE_SMEM) ? 1 : 0;
    const size_t smem = G::smem_bytes(b.alias_L != 0);
    dim3 grid;
    const int nd = a.n[DIR];
    if (DIR == 0) {
        const long long rows = a.N / a.n[0];
        grid = dim3((unsigned)((rows + G::TL - 1) / G::TL), (nd + G::TS - 1) / G::TS, 1);
    } else {
        grid = dim3((a.n[0] + G::TL - 1) / G::TL, (nd + G::TS - 1) / G::TS,
                    DIR == 1 ? (ND == 3 ? a.n[2] : 1) : a.n[1]);
    }
    return launch_sweep_kernel(k, grid, G::THREADS, smem, s, b);
}

template <int FLUX>
cudaError_t dispatch(int nd, int dir, const SweepArgs& a, cudaStream_t s, bool prep)
{
    if (nd == 1) return go<1, 0, FLUX>(a, s, prep);
    if (nd == 2) return dir == 0 ? go<2, 0, FLUX>(a, s, prep) : go<2, 1, FLUX>(a, s, prep);
    if (dir == 0) return go<3, 0, FLUX>(a, s, prep);
    if (dir == 1) return go<3, 1, FLUX>(a, s, prep);
    return go<3, 2, FLUX>(a, s, prep);
}

cudaError_t run(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s, bool prep)
{
    return flux == FLUX_ROE    ? dispatch<FLUX_ROE>(nd, dir, a, s, prep)
           : flux == FLUX_AUSM ? dispatch<FLUX_AUSM>(nd, dir, a, s, prep)
                               : dispatch<FLUX_VANLEER>(nd, dir, a, s, prep);
}

// batched instances (tile table or persistent)
template <int ND, int DIR, int FLUX>
cudaError_t go_batch(const SweepArgs& a, long long ntiles, cudaStream_t s, bool prepare)
{
    using G = TileGeom<float, ND, DIR, batch_cfg<float>(ND)>;
    auto k = sweep_kernel<float, float, ND, DIR, FLUX, true, batch_cfg<float>(ND), SWEEP_WT>;
    if (prepare)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes());
    SweepArgs b = a;
    b.alias_L = sweep_alias_L(a, G::FUSE_SMEM) ? 1 : 0;
    static std::atomic<int> resident[2] = {0, 0};
    return launch_tiles(k, G::THREADS, G::smem_bytes(b.alias_L != 0), b, ntiles, s, resident[b.alias_L]);
}

template <int FLUX>
cudaError_t dispatch_batch(int nd, int dir, const SweepArgs& a, long long ntiles, cudaStream_t s, bool prep)
{
    if (nd == 1) return go_batch<1, 0, FLUX>(a, ntiles, s, prep);
    if (nd == 2) return dir == 0 ? go_batch<2, 0, FLUX>(a, ntiles, s, prep) : go_batch<2, 1, FLUX>(a, ntiles, s, prep);
    if (dir == 0) return go_batch<3, 0, FLUX>(a, ntiles, s, prep);
    if (dir == 1) return go_batch<3, 1, FLUX>(a, ntiles, s, prep);
    return go_batch<3, 2, FLUX>(a, ntiles, s, prep);
}

cudaError_t run_batch(int nd, int dir, int flux, const SweepArgs& a, long long ntiles, cudaStream_t s, bool prep)
{
    return flux == FLUX_ROE    ? dispatch_batch<FLUX_ROE>(nd, dir, a, ntiles, s, prep)
           : flux == FLUX_AUSM ? dispatch_batch<FLUX_AUSM>(nd, dir, a, ntiles, s, prep)
                               : dispatch_batch<FLUX_VANLEER>(nd, dir, a, ntiles, s, prep);
}

}  // namespace

#define WCNS_CAT2(a, b) a##b
#define WCNS_CAT(a, b) WCNS_CAT2(a, b)

cudaError_t WCNS_CAT(launch_sweep_fp32_w, SWEEP_WT)(int nd, int dir, int flux, const SweepArgs& a,
                                                     cudaStream_t s)
{
    return run(nd, dir, flux, a, s, false);
}

cudaError_t WCNS_CAT(launch_sweep_batch_fp32_w, SWEEP_WT)(int nd, int dir, int flux, const SweepArgs& a,
                                                           long long ntiles, cudaStream_t s)
{
    return run_batch(nd, dir, flux, a, ntiles, s, false);
}

cudaError_t WCNS_CAT(prepare_sweeps_fp32_w, SWEEP_WT)()
{
    SweepArgs a{};
    for (int nd = 1; nd <= 3; ++nd)
        for (int d = 0; d < nd; ++d)
            for (int f = 0; f < 3; ++f) {
                cudaError_t e = run(nd, d, f, a, 0, true);
                if (e == cudaSuccess) e = run_batch(nd, d, f, a, 0, 0, true);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

#if SWEEP_WT == 1
cudaError_t launch_sweep_fp32_weights(int wt, int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s)
{
    if (wt == W_JS) return launch_sweep_fp32_w1(nd, dir, flux, a, s);
    if (wt == W_LINEAR) return launch_sweep_fp32_w2(nd, dir, flux, a, s);
    if (wt == W_Z) return launch_sweep_fp32_w3(nd, dir, flux, a, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_batch_fp32_weights(int wt, int nd, int dir, int flux, const SweepArgs& a,
                                            long long ntiles, cudaStream_t s)
{
    if (wt == W_JS) return launch_sweep_batch_fp32_w1(nd, dir, flux, a, ntiles, s);
    if (wt == W_LINEAR) return launch_sweep_batch_fp32_w2(nd, dir, flux, a, ntiles, s);
    if (wt == W_Z) return launch_sweep_batch_fp32_w3(nd, dir, flux, a, ntiles, s);
    return cudaErrorInvalidValue;
}

cudaError_t prepare_sweeps_fp32_weights()
{
    cudaError_t e = prepare_sweeps_fp32_w1();
    if (e == cudaSuccess) e = prepare_sweeps_fp32_w2();
    if (e == cudaSuccess) e = prepare_sweeps_fp32_w3();
    return e;
}
#endif

}  // namespace wcns
