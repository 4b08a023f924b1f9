// wcns_noalloc.cu -- an FP64 SSP-RK3 step that allocates no device memory.
//
// For callers that cannot call cudaMalloc (all device memory already held
// by another allocator, or a loop that must make no allocation calls): the
// stage state and right-hand side of one step live in a static device
// buffer owned by the library instead of in a handle's scratch.  Every GPU
// that loads the library holds WCNS_NOALLOC_SCRATCH_BYTES of it until the
// process exits.  The caller still passes the state U.
#include <math.h>
#include <stdio.h>

#include <atomic>
#include <mutex>

#include "../../include/wcns.h"
#include "wcns_internal.h"

using namespace wcns;

// The shared scratch: [StepScalars | fallback counter | L | U1], 256-byte
// aligned parts.  In host code this name is only a stand-in for the
// symbol; kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[WCNS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t kHead = 512;   // StepScalars (256) + fallback counter (256)
constexpr int kMaxDevices = 64;
// Per device: the scratch's device address, published by g_ready (release
// store after the set-up, acquire load before use); g_setup serialises the
// set-up itself, so host threads making their first call at once neither
// race nor repeat it.
unsigned char* g_base[kMaxDevices];
std::atomic<bool> g_ready[kMaxDevices];
std::mutex g_setup;

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Largest node count whose two state-sized parts fit behind the header:
// kHead + 2 * round256(8 nv N) <= WCNS_NOALLOC_SCRATCH_BYTES.
long long max_nodes(int nv)
{
    const size_t part = ((size_t)WCNS_NOALLOC_SCRATCH_BYTES - kHead) / 2 & ~(size_t)255;
    return (long long)(part / ((size_t)nv * sizeof(double)));
}

wcns_status fail(wcns_status s, const char* msg)
{
    set_last_error(msg);
    return s;
}

wcns_status cuda_fail(cudaError_t e, const char* where)
{
    char buf[256];
    snprintf(buf, sizeof buf, "wcns_step_rk3_noalloc: %s: %s", where, cudaGetErrorString(e));
    set_last_error(buf);
    return WCNS_ERR_CUDA;
}

// Once per device, with that device current: the scratch's device address
// and the kernels' launch attributes.
cudaError_t setup_device(int dev)
{
    if (g_ready[dev].load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_setup);
    if (g_ready[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = prepare_sweeps_fp64();
    if (e != cudaSuccess) return e;
    g_base[dev] = static_cast<unsigned char*>(p);
    g_ready[dev].store(true, std::memory_order_release);
    return cudaSuccess;
}

}  // namespace

extern "C" wcns_status wcns_step_rk3_noalloc(const wcns_grid* g, double gamma,
                                             const wcns_scheme_params* prm, void* U, double dt,
                                             double* dt_used, void* stream)
{
    set_last_error(nullptr);
    if (!g || !prm || !U) return fail(WCNS_ERR_INVALID, "wcns_step_rk3_noalloc: null argument");
    if (g->ndim < 1 || g->ndim > 3) return fail(WCNS_ERR_INVALID, "ndim must be 1, 2 or 3");
    if (!(gamma > 1.0)) return fail(WCNS_ERR_INVALID, "gamma must exceed 1");
    if (prm->precision != WCNS_FP64)
        return fail(WCNS_ERR_INVALID, "wcns_step_rk3_noalloc: precision must be WCNS_FP64");
    if (const char* why = scheme_params_error(prm)) return fail(WCNS_ERR_INVALID, why);
    if (grid_has_single_grid_features(g))
        return fail(WCNS_ERR_INVALID, "wcns_step_rk3_noalloc: periodic and transmissive boundaries only, no body force");

    const int nd = g->ndim, nv = nd + 2;
    const long long cap = max_nodes(nv);
    int n[3] = {1, 1, 1}, periodic[3] = {0, 0, 0};
    double h[3] = {1, 1, 1}, inv_h[3] = {0, 0, 0};
    long long N = 1;
    for (int a = 0; a < nd; ++a) {
        const int per = g->bc[a][0] == WCNS_BC_PERIODIC;
        if ((g->bc[a][1] == WCNS_BC_PERIODIC) != per)
            return fail(WCNS_ERR_INVALID, "periodic must be set on both sides of an axis");
        for (int sd = 0; sd < 2; ++sd)
            if (g->bc[a][sd] != WCNS_BC_PERIODIC && g->bc[a][sd] != WCNS_BC_TRANSMISSIVE)
                return fail(WCNS_ERR_INVALID, "unknown boundary kind");
        if (g->n[a] < (per ? 1 : 2) || !(g->hi[a] > g->lo[a]))
            return fail(WCNS_ERR_INVALID, "bad node count or extent");
        n[a] = g->n[a];
        periodic[a] = per;
        h[a] = (g->hi[a] - g->lo[a]) / (per ? g->n[a] : g->n[a] - 1);
        inv_h[a] = 1.0 / h[a];
        // checked before the product, so that no node count can overflow
        if (N > cap / g->n[a]) {
            char buf[256];
            snprintf(buf, sizeof buf,
                     "wcns_step_rk3_noalloc: the grid does not fit the static scratch buffer of %u bytes "
                     "(at most %lld nodes for %d variables)",
                     WCNS_NOALLOC_SCRATCH_BYTES, cap, nv);
            return fail(WCNS_ERR_INVALID, buf);
        }
        N *= g->n[a];
    }
    if (nd == 3 && (n[1] > 65535 || n[2] > 65535)) return fail(WCNS_ERR_INVALID, "grid too large");
    const size_t state_bytes = (size_t)nv * (size_t)N * sizeof(double);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(WCNS_ERR_INVALID, "device index out of range");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    e = setup_device(dev);
    if (e != cudaSuccess) return cuda_fail(e, "device set-up");

    unsigned char* base = g_base[dev];
    StepScalars* sc = reinterpret_cast<StepScalars*>(base);
    long long* fallback = reinterpret_cast<long long*>(base + 256);
    double* L = reinterpret_cast<double*>(base + kHead);
    double* U1 = reinterpret_cast<double*>(base + kHead + round256(state_bytes));
    double* U0 = static_cast<double*>(U);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const SchemeConst K = make_scheme_const(prm, gamma);

    // the buffer keeps the previous call's contents: clear what must start at zero
    if ((e = launch_reset_clock(INFINITY, sc, s)) != cudaSuccess) return cuda_fail(e, "clock reset");
    if ((e = cudaMemsetAsync(fallback, 0, sizeof(long long), s)) != cudaSuccess)
        return cuda_fail(e, "counter reset");
    if (dt > 0.0) e = launch_set_dt(dt, 0, sc, s);
    else e = launch_cfl(nd, U0, N, h, gamma, prm->cfl, 0, sc, s);
    if (e != cudaSuccess) return cuda_fail(e, "time step");

    const long long M = (long long)nv * N;
    for (int stage = 1; stage <= 3; ++stage) {
        const double* in = stage == 1 ? U0 : U1;
        for (int d = 0; d < nd; ++d) {
            SweepArgs a{};
            a.U = in;
            a.L = L;
            a.N = N;
            a.n[0] = n[0];
            a.n[1] = n[1];
            a.n[2] = n[2];
            a.periodic = periodic[d];
            a.inv_h = inv_h[d];
            a.accumulate = d > 0;
            a.flags = nullptr;
            a.fallback = fallback;
            a.dt = &sc->dt;
            a.K = K;
            a.sqrt_eps_f = (float)sqrt(prm->eps);
            if ((e = launch_sweep_fp64(nd, d, prm->flux, a, s)) != cudaSuccess) return cuda_fail(e, "sweep");
        }
        if ((e = launch_rk_fp64(stage, U0, U1, L, M, sc, s)) != cudaSuccess) return cuda_fail(e, "stage");
    }
    if (dt_used) {
        if ((e = cudaMemcpyAsync(dt_used, &sc->dt, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "dt copy");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sync");
    }
    return WCNS_OK;
}
