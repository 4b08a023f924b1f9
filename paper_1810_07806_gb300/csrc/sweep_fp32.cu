// sweep_fp32.cu -- FP32 instances of the fused sweep (rescaled smoothness
// indicators) for tile configuration SWEEP_CFG (0, 1 or 2; one translation
// unit per configuration so they compile in parallel).  The input state is
// single precision.
#include "wcns_internal.h"

#ifndef SWEEP_CFG
#define SWEEP_CFG 0
#endif

namespace wcns {

template <int ND, int DIR, int FLUX>
static cudaError_t go(const SweepArgs& a, cudaStream_t s, bool prepare)
{
    constexpr int CFG = ND == 1 ? 0 : SWEEP_CFG;
    using G = TileGeom<float, ND, DIR, CFG>;
    auto k = sweep_kernel<float, float, ND, DIR, FLUX, false, CFG>;
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
static cudaError_t dispatch(int nd, int dir, const SweepArgs& a, cudaStream_t s, bool prep)
{
    if (nd == 1) return SWEEP_CFG == 0 ? go<1, 0, FLUX>(a, s, prep) : cudaErrorInvalidValue;
    if (nd == 2) return dir == 0 ? go<2, 0, FLUX>(a, s, prep) : go<2, 1, FLUX>(a, s, prep);
    if (dir == 0) return go<3, 0, FLUX>(a, s, prep);
    if (dir == 1) return go<3, 1, FLUX>(a, s, prep);
    return go<3, 2, FLUX>(a, s, prep);
}

#define WCNS_CAT2(a, b) a##b
#define WCNS_CAT(a, b) WCNS_CAT2(a, b)

cudaError_t WCNS_CAT(launch_sweep_fp32_cfg, SWEEP_CFG)(int nd, int dir, int flux, const SweepArgs& a,
                                                        cudaStream_t s)
{
    return flux == FLUX_ROE ? dispatch<FLUX_ROE>(nd, dir, a, s, false)
                            : flux == FLUX_AUSM ? dispatch<FLUX_AUSM>(nd, dir, a, s, false)
                            : dispatch<FLUX_VANLEER>(nd, dir, a, s, false);
}

cudaError_t WCNS_CAT(prepare_sweeps_fp32_cfg, SWEEP_CFG)()
{
    SweepArgs a{};
    for (int nd = SWEEP_CFG == 0 ? 1 : 2; nd <= 3; ++nd)
        for (int d = 0; d < nd; ++d)
            for (int f = 0; f < 3; ++f) {
                cudaError_t e = f == 0 ? dispatch<FLUX_ROE>(nd, d, a, 0, true)
                                       : f == 1 ? dispatch<FLUX_VANLEER>(nd, d, a, 0, true)
                                       : dispatch<FLUX_AUSM>(nd, d, a, 0, true);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

#if SWEEP_CFG == 0
cudaError_t launch_sweep_fp32(int nd, int dir, int flux, int cfg, const SweepArgs& a, cudaStream_t s)
{
    if (a.K.weights != W_TENO) return launch_sweep_fp32_weights(a.K.weights, nd, dir, flux, a, s);
    if (nd == 1 || cfg == 0) return launch_sweep_fp32_cfg0(nd, dir, flux, a, s);
    if (cfg == 1) return launch_sweep_fp32_cfg1(nd, dir, flux, a, s);
    return launch_sweep_fp32_cfg2(nd, dir, flux, a, s);
}

cudaError_t prepare_sweeps_fp32()
{
    cudaError_t e = prepare_sweeps_fp32_cfg0();
    if (e == cudaSuccess) e = prepare_sweeps_fp32_cfg1();
    if (e == cudaSuccess) e = prepare_sweeps_fp32_cfg2();
    if (e == cudaSuccess) e = prepare_sweeps_fp32_weights();
    return e;
}
#endif

}  // namespace wcns
