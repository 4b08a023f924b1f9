// sweep_fp64.cu -- FP64 instances of the fused sweep (plain path, parity
// with the FP64 oracle: the flag-deciding arithmetic runs in fixed order).
#include "wcns_internal.h"

namespace wcns {

template <int ND, int DIR, int FLUX>
static cudaError_t go(const SweepArgs& a, cudaStream_t s, bool prepare)
{
    using G = TileGeom<double, ND, DIR>;
    auto k = sweep_kernel<double, double, ND, DIR, FLUX>;
    const size_t smem = G::smem_bytes();
    if (prepare) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid;
    const int nd = a.n[DIR];
    if (DIR == 0) {
        const long long rows = a.N / a.n[0];
        grid = dim3((unsigned)((rows + G::TL - 1) / G::TL), (nd + G::TS - 1) / G::TS, 1);
    } else {
        grid = dim3((a.n[0] + G::TL - 1) / G::TL, (nd + G::TS - 1) / G::TS,
                    DIR == 1 ? (ND == 3 ? a.n[2] : 1) : a.n[1]);
    }
    k<<<grid, G::THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int FLUX>
static cudaError_t dispatch(int nd, int dir, const SweepArgs& a, cudaStream_t s, bool prep)
{
    if (nd == 1) return go<1, 0, FLUX>(a, s, prep);
    if (nd == 2) return dir == 0 ? go<2, 0, FLUX>(a, s, prep) : go<2, 1, FLUX>(a, s, prep);
    if (dir == 0) return go<3, 0, FLUX>(a, s, prep);
    if (dir == 1) return go<3, 1, FLUX>(a, s, prep);
    return go<3, 2, FLUX>(a, s, prep);
}

cudaError_t launch_sweep_fp64(int nd, int dir, int flux, const SweepArgs& a, cudaStream_t s)
{
    return flux == FLUX_ROE ? dispatch<FLUX_ROE>(nd, dir, a, s, false)
                            : flux == FLUX_AUSM ? dispatch<FLUX_AUSM>(nd, dir, a, s, false)
                            : dispatch<FLUX_VANLEER>(nd, dir, a, s, false);
}

cudaError_t prepare_sweeps_fp64()
{
    // omega_k^(T) = delta_k d_k / sum_j delta_j d_j (Eq. 19), sum in k order
    cudaError_t e0 = fill_omega_table();
    if (e0 != cudaSuccess) return e0;
    SweepArgs a{};
    for (int nd = 1; nd <= 3; ++nd)
        for (int d = 0; d < nd; ++d)
            for (int f = 0; f < 3; ++f) {
                cudaError_t e = f == 0 ? dispatch<FLUX_ROE>(nd, d, a, 0, true)
                                       : f == 1 ? dispatch<FLUX_VANLEER>(nd, d, a, 0, true)
                                       : dispatch<FLUX_AUSM>(nd, d, a, 0, true);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

}  // namespace wcns
