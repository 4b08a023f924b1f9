// wcns_scalar.cu -- scalar conservation laws u_t + f(u)_x = 0 on periodic 1D
// grids: the accuracy tests of Sec. 3.2 (linear advection, f = u) and
// Sec. 3.3 (inviscid Burgers, f = u^2 / 2).  The midpoint flux is Eq. 6 over
// the node-to-midpoint interpolation of Sec. 2.2 (no characteristic
// projection: one field), the derivative Eq. 3, the time integrator SSP-RK3.
//
// One line is solved by one thread-block cluster.  CTA r of the cluster owns
// nodes [r seg, (r + 1) seg) in its shared memory for the whole call.  The
// 2 + 3 ghost nodes its faces need and the 3 + 2 ghost faces its nodes need
// are read from the owning CTAs' shared memory (distributed shared memory)
// after a cluster barrier, so a run of nsteps RK3 steps is one launch with
// two cluster barriers per stage and no global-memory traffic between the
// first load and the last store.  Arithmetic is FP64 in the fixed order of
// wcns_fp64.cuh (the order of the definitions: left-to-right sums,
// round-to-nearest, no contraction), so a result is a deterministic function
// of the input bits.
#include <cooperative_groups.h>

#include <math.h>

#include "../../include/wcns.h"
#include "wcns_fp64.cuh"
#include "wcns_internal.h"

namespace cg = cooperative_groups;

namespace wcns {
namespace {

constexpr int SC_THREADS = 128;
constexpr int SC_MAX_SEG = 6144;   // nodes per CTA: (4 seg + 14) doubles of shared memory

struct ScalarArgs {
    const double* uin;    // input lines (RHS mode)
    double* u;            // lines advanced in place (run mode)
    double* L;            // output RHS (RHS mode)
    long long ld;         // line stride in doubles
    int n;                // nodes per line (periodic)
    int seg;              // nodes per CTA
    double h, dt;
    int nsteps;
    SchemeConst K;
};

template <int KIND>
__device__ __forceinline__ double flux_of(double u)
{
    return KIND == WCNS_SCALAR_ADVECTION ? u : mul_(mul_(0.5, u), u);
}

// Eq. 6 at face j+1/2 from e[0..5] = u_{j-2} .. u_{j+3}: the left state
// interpolates e[0..4] about u_j, the right state the mirror e[5..1] about
// u_{j+1}; a = 1 (advection) or (u_L + u_R) / 2 (Burgers).
template <int KIND>
__device__ __forceinline__ double scalar_face(const double* e, const SchemeConst& K)
{
    double sl[5], sr[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        sl[m] = e[m];
        sr[m] = e[5 - m];
    }
    int flags;
    const double uL = interp_weights_fp64(sl, K, flags);
    const double uR = interp_weights_fp64(sr, K, flags);
    const double a = KIND == WCNS_SCALAR_ADVECTION ? 1.0 : mul_(0.5, add_(uL, uR));
    return mul_(0.5, sub_(add_(flux_of<KIND>(uR), flux_of<KIND>(uL)), mul_(fabs(a), sub_(uR, uL))));
}

__device__ __forceinline__ int wrap(long long g, int n)
{
    long long r = g % n;
    return (int)(r < 0 ? r + n : r);
}

// RUN = false: L = -f'(u) once.  RUN = true: nsteps SSP-RK3 steps in place.
template <int KIND, bool RUN>
__global__ void __launch_bounds__(SC_THREADS) scalar_kernel(const ScalarArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int csize = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const long long line = blockIdx.x / csize;
    const int tid = threadIdx.x;
    const int n = a.n, seg = a.seg;
    extern __shared__ double sm[];
    double* ue = sm;                    // [seg + 5]: 2 ghost nodes, owned nodes, 3 ghost nodes
    double* Fe = sm + (seg + 5);        // [seg + 5]: 3 ghost faces, owned faces, 2 ghost faces
    double* u0 = sm + 2 * (seg + 5);    // [seg]: state at the start of the RK3 step
    double* Fn = u0 + seg;              // [seg + 4]: node fluxes f(u), nodes lo-2 .. lo+cnt+1 (Eq. 4-5)
    const int diff = a.K.diff;
    const int lo = rank * seg;
    const int cnt = max(0, min(seg, n - lo));
    const double* gin = RUN ? a.u + line * a.ld : a.uin + line * a.ld;

    for (int l = tid; l < cnt; l += SC_THREADS) {
        const double v = gin[lo + l];
        ue[2 + l] = v;
        if (RUN) u0[l] = v;
    }
    const int stages = RUN ? 3 * a.nsteps : 1;
    for (int st = 0; st < stages; ++st) {
        cl.sync();   // every CTA's nodes of this stage are in place
        if (tid < 5 && cnt > 0) {
            const long long g = tid < 2 ? (long long)lo - 2 + tid : (long long)lo + cnt + (tid - 2);
            const int gi = wrap(g, n);
            const int owner = gi / seg;
            const double* r = cl.map_shared_rank(ue, owner);
            ue[tid < 2 ? tid : cnt + tid] = r[2 + gi - owner * seg];
        }
        __syncthreads();
        // face lo+l+1/2 reads nodes lo+l-2 .. lo+l+3 = ue[l .. l+5]
        for (int l = tid; l < cnt; l += SC_THREADS) Fe[3 + l] = scalar_face<KIND>(ue + l, a.K);
        if (diff != DIFF_MD)
            for (int m = tid; m < cnt + 4; m += SC_THREADS) Fn[m] = flux_of<KIND>(ue[m]);
        cl.sync();   // every CTA's faces are in place
        if (tid < 5 && cnt > 0) {
            const long long g = tid < 3 ? (long long)lo - 3 + tid : (long long)lo + cnt + (tid - 3);
            const int gi = wrap(g, n);
            const int owner = gi / seg;
            const double* r = cl.map_shared_rank(Fe, owner);
            Fe[tid < 3 ? tid : cnt + tid] = r[3 + gi - owner * seg];
        }
        __syncthreads();
        const int stage = st % 3;
        for (int l = tid; l < cnt; l += SC_THREADS) {
            // node i = lo+l: f[0..5] = faces i-5/2 .. i+5/2 = Fe[l .. l+5]
            const double* f = Fe + l;
            const double* fn = Fn + l;   // f(u) at nodes i-2 .. i+2
            const double fp =
                diff == DIFF_MD
                    ? add_(add_(mul_(MD_A1, sub_(f[3], f[2])), mul_(MD_A2, sub_(f[4], f[1]))),
                           mul_(MD_A3, sub_(f[5], f[0])))
                    : diff_alt_fp64(diff, f[1], f[2], f[3], f[4], sub_(fn[3], fn[1]), sub_(fn[4], fn[0]));
            const double Li = div_int_(-fp, a.h);
            if (!RUN) {
                a.L[line * a.ld + lo + l] = Li;
                continue;
            }
            const double v = add_(ue[2 + l], mul_(a.dt, Li));
            if (stage == 0) {
                ue[2 + l] = v;
            } else if (stage == 1) {
                ue[2 + l] = add_(mul_(0.75, u0[l]), mul_(0.25, v));
            } else {
                const double un = add_(div_int_(u0[l], 3.0), mul_(2.0 / 3.0, v));
                u0[l] = un;
                ue[2 + l] = un;
            }
        }
    }
    if (RUN)
        for (int l = tid; l < cnt; l += SC_THREADS) a.u[line * a.ld + lo + l] = u0[l];
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int KIND, bool RUN>
cudaError_t launch_one(const ScalarArgs& a, int count, int csize, cudaStream_t s)
{
    const size_t smem = (size_t)(4 * a.seg + 14) * sizeof(double);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((long long)count * csize));
    cfg.blockDim = dim3(SC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, scalar_kernel<KIND, RUN>, a);
}

template <int KIND, bool RUN>
cudaError_t prepare_one(int want_cluster, int* ok_cluster)
{
    auto k = scalar_kernel<KIND, RUN>;
    const int smem = (4 * SC_MAX_SEG + 14) * (int)sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (want_cluster > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *ok_cluster = 8;
            return cudaSuccess;
        }
        // can a cluster of want_cluster CTAs with the largest segment be placed?
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(want_cluster);
        cfg.blockDim = dim3(SC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = want_cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
        if (e != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            *ok_cluster = 8;
            return cudaSuccess;
        }
    }
    *ok_cluster = want_cluster;
    return cudaSuccess;
}

constexpr int kMaxDevices = 64;
int g_max_cluster[kMaxDevices];   // 0: device not prepared

// Prepares the four kernels on the current device (once) and returns the
// largest cluster size every one of them can use.
cudaError_t prepare(int* max_cluster)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (g_max_cluster[dev] == 0) {
        // this unit's copy of the Eq. 19 weights of the reduced stencil sets
        if ((e = fill_omega_table()) != cudaSuccess) return e;
        int c[4] = {16, 16, 16, 16};
        if ((e = prepare_one<0, false>(16, &c[0])) != cudaSuccess) return e;
        if ((e = prepare_one<0, true>(16, &c[1])) != cudaSuccess) return e;
        if ((e = prepare_one<1, false>(16, &c[2])) != cudaSuccess) return e;
        if ((e = prepare_one<1, true>(16, &c[3])) != cudaSuccess) return e;
        int m = 16;
        for (int i = 0; i < 4; ++i) m = c[i] < m ? c[i] : m;
        g_max_cluster[dev] = m;
    }
    *max_cluster = g_max_cluster[dev];
    return cudaSuccess;
}

// Smallest power-of-two cluster giving at most SC_THREADS nodes per CTA,
// capped at max_cluster; the segment then grows to cover the line.
void plan(int n, int max_cluster, int* csize, int* seg)
{
    int c = 1;
    while (c < max_cluster && (long long)c * SC_THREADS < n) c *= 2;
    *csize = c;
    *seg = (n + c - 1) / c;
}

wcns_status check_common(int kind, const wcns_scheme_params* prm, int n, double h, int count,
                         long long ld)
{
    if (!prm) return (set_last_error("null params"), WCNS_ERR_INVALID);
    if (kind != WCNS_SCALAR_ADVECTION && kind != WCNS_SCALAR_BURGERS)
        return (set_last_error("kind must be WCNS_SCALAR_ADVECTION or WCNS_SCALAR_BURGERS"),
                WCNS_ERR_INVALID);
    if (const char* why = scheme_params_error(prm)) return (set_last_error(why), WCNS_ERR_INVALID);
    if (prm->precision != WCNS_FP64)
        return (set_last_error("the scalar solver computes in FP64 only"), WCNS_ERR_INVALID);
    if (n < 1 || count < 1 || ld < n)
        return (set_last_error("need n >= 1, count >= 1, ld >= n"), WCNS_ERR_INVALID);
    if (!(h > 0.0) || !isfinite(h)) return (set_last_error("h must be positive"), WCNS_ERR_INVALID);
    if ((long long)count * 16 > 0x7fffffffLL)
        return (set_last_error("too many lines in one call"), WCNS_ERR_INVALID);
    return WCNS_OK;
}

wcns_status scalar_call(int kind, const wcns_scheme_params* prm, int n, double h, double t_end,
                        int nsteps, int count, const double* uin, double* u, double* L, long long ld,
                        bool run, void* stream)
{
    int maxc = 0;
    cudaError_t e = prepare(&maxc);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return WCNS_ERR_CUDA;
    }
    if ((long long)n > (long long)maxc * SC_MAX_SEG) {
        set_last_error("n exceeds wcns_scalar_max_nodes()");
        return WCNS_ERR_INVALID;
    }
    ScalarArgs a{};
    a.uin = uin;
    a.u = u;
    a.L = L;
    a.ld = ld;
    a.n = n;
    a.h = h;
    a.nsteps = nsteps;
    a.dt = run ? t_end / nsteps : 0.0;
    a.K = make_scheme_const(prm, 2.0);
    int csize = 1;
    plan(n, maxc, &csize, &a.seg);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (kind == WCNS_SCALAR_ADVECTION)
        e = run ? launch_one<0, true>(a, count, csize, s) : launch_one<0, false>(a, count, csize, s);
    else
        e = run ? launch_one<1, true>(a, count, csize, s) : launch_one<1, false>(a, count, csize, s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return WCNS_ERR_CUDA;
    }
    return WCNS_OK;
}

}  // namespace
}  // namespace wcns

using namespace wcns;

extern "C" int wcns_scalar_max_nodes(void)
{
    int maxc = 0;
    if (prepare(&maxc) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return maxc * SC_MAX_SEG;
}

extern "C" wcns_status wcns_scalar_rhs(int kind, const wcns_scheme_params* prm, int n, double h,
                                       int count, const double* u, long long ld, double* L,
                                       void* stream)
{
    set_last_error(nullptr);
    const wcns_status st = check_common(kind, prm, n, h, count, ld);
    if (st != WCNS_OK) return st;
    if (!u || !L) return (set_last_error("null array"), WCNS_ERR_INVALID);
    return scalar_call(kind, prm, n, h, 0.0, 0, count, u, nullptr, L, ld, false, stream);
}

extern "C" wcns_status wcns_scalar_run(int kind, const wcns_scheme_params* prm, int n, double h,
                                       double t_end, int nsteps, int count, double* u, long long ld,
                                       void* stream)
{
    set_last_error(nullptr);
    const wcns_status st = check_common(kind, prm, n, h, count, ld);
    if (st != WCNS_OK) return st;
    if (!u) return (set_last_error("null array"), WCNS_ERR_INVALID);
    if (nsteps < 0 || !(t_end >= 0.0) || !isfinite(t_end))
        return (set_last_error("need nsteps >= 0 and a finite t_end >= 0"), WCNS_ERR_INVALID);
    if (nsteps == 0) return WCNS_OK;
    return scalar_call(kind, prm, n, h, t_end, nsteps, count, nullptr, u, nullptr, ld, true, stream);
}
