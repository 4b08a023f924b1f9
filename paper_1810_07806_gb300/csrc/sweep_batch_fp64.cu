// sweep_batch_fp64.cu -- FP64 instances of the batched sweep: one launch covers
// the tiles of every instance of a batch (tile table), each tile reading its
// own instance's geometry, boundary rule and time step; or, persistent, as
// many CTAs as fit on the device taking tiles from a counter.
#include "wcns_internal.h"

namespace wcns {

template <int ND, int DIR, int FLUX>
static cudaError_t go(const SweepArgs& a, long long ntiles, cudaStream_t s, bool prepare)
{
    using G = TileGeom<double, ND, DIR, batch_cfg<double>(ND)>;
    auto k = sweep_kernel<double, double, ND, DIR, FLUX, true, batch_cfg<double>(ND)>;
    const size_t smem = G::smem_bytes();
    if (prepare) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static std::atomic<int> resident{0};
    return launch_tiles(k, G::THREADS, smem, a, ntiles, s, resident);
}

template <int FLUX>
static cudaError_t dispatch(int nd, int dir, const SweepArgs& a, long long ntiles, cudaStream_t s, bool prep)
{
    if (nd == 1) return go<1, 0, FLUX>(a, ntiles, s, prep);
    if (nd == 2) return dir == 0 ? go<2, 0, FLUX>(a, ntiles, s, prep) : go<2, 1, FLUX>(a, ntiles, s, prep);
    if (dir == 0) return go<3, 0, FLUX>(a, ntiles, s, prep);
    if (dir == 1) return go<3, 1, FLUX>(a, ntiles, s, prep);
    return go<3, 2, FLUX>(a, ntiles, s, prep);
}

cudaError_t launch_sweep_batch_fp64(int nd, int dir, int flux, const SweepArgs& a, long long ntiles,
                                     cudaStream_t s)
{
    return flux == FLUX_ROE ? dispatch<FLUX_ROE>(nd, dir, a, ntiles, s, false)
                            : flux == FLUX_AUSM ? dispatch<FLUX_AUSM>(nd, dir, a, ntiles, s, false)
                            : dispatch<FLUX_VANLEER>(nd, dir, a, ntiles, s, false);
}

cudaError_t prepare_sweeps_batch_fp64()
{
    cudaError_t e0 = fill_omega_table();   // this unit's Eq. 19 weight table
    if (e0 != cudaSuccess) return e0;
    SweepArgs a{};
    for (int nd = 1; nd <= 3; ++nd)
        for (int d = 0; d < nd; ++d)
            for (int f = 0; f < 3; ++f) {
                cudaError_t e = f == 0 ? dispatch<FLUX_ROE>(nd, d, a, 0, 0, true)
                                       : f == 1 ? dispatch<FLUX_VANLEER>(nd, d, a, 0, 0, true)
                                       : dispatch<FLUX_AUSM>(nd, d, a, 0, 0, true);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

}  // namespace wcns
