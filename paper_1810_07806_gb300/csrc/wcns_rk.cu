// wcns_rk.cu -- time step and stage kernels: the CFL reduction (FP64), the
// SSP-RK3 stage combinations (Shu-Osher form, the third-order strong
// stability preserving method the paper cites for time integration) and the
// deterministic FP64 conservation totals.
#include <math.h>

#include "wcns_fp64.cuh"
#include "wcns_internal.h"

namespace wcns {

struct InvH {
    double v[3];
};

__device__ __forceinline__ float warp_maxf(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ double warp_max(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// lambda = max_i sum_d (|u_d| + c) / h_d over all nodes, FP64, each node in
// the fixed order c = sqrt(gamma p / rho), s = sum_d (|m_d / rho| + c) / h_d.
template <int ND>
__global__ void __launch_bounds__(256) cfl_reduce_kernel(const double* __restrict__ U, long long N,
                                                         InvH hh, double gamma, double gm1,
                                                         StepScalars* sc, int clip)
{
    if (clip && !(sc->t < sc->t_end)) return;   // finished: nothing to do
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double Ui[ND + 2];
#pragma unroll
        for (int v = 0; v < ND + 2; ++v) Ui[v] = U[v * N + i];
        const double c = sqrt_(div_(mul_(gamma, pressure_exact<ND>(Ui, gm1)), Ui[0]));
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < ND; ++a) {
            const double q = div_(add_(fabs(div_(Ui[1 + a], Ui[0])), c), hh.v[a]);
            s = a == 0 ? q : add_(s, q);
        }
        m = fmax(m, s);
    }
    m = warp_max(m);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        m = warp_max(m);
        if (threadIdx.x == 0)
            atomicMax(&sc->lam_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// The same lambda for the FP32 path: each node's wave-speed sum is evaluated
// in FP32 from the FP64 state and multiplied by (1 + 2^-16), an upper bound of
// its rounding error, so the step never exceeds the FP64 CFL bound; the
// maximum and dt stay FP64.  One pass over the state, no FP64 divisions.
// S (nullable) receives float(U), the first stage's input, from the same pass.
template <int ND>
__global__ void __launch_bounds__(256) cfl_reduce_fast_kernel(const double* __restrict__ U, long long N,
                                                              InvH hh, float gamma, StepScalars* sc,
                                                              int clip, float* __restrict__ S)
{
    if (clip && !(sc->t < sc->t_end)) return;
    float m = 0.f;
    const float gm1 = gamma - 1.f;
    const double rr = sc->ref_rho, er = sc->ref_E;
    float ih[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) ih[a] = (float)(1.0 / hh.v[a]);
    // one node: its wave-speed sum, and (S non-null) its float(U - U_r)
    auto node = [&](double rho_d, const double (&mv_d)[ND], double E_d, float (&out)[ND + 2]) {
        const float rho = f64_to_f32_ftz(rho_d);
        const float ir = __frcp_rn(rho);
        float m2 = 0.f, s = 0.f;
        float vel[ND];
#pragma unroll
        for (int a = 0; a < ND; ++a) {
            const float mv = f64_to_f32_ftz(mv_d[a]);
            out[1 + a] = mv;
            m2 = fmaf(mv, mv, m2);
            vel[a] = fabsf(mv) * ir;
        }
        const float E = f64_to_f32_ftz(E_d);
        if (S != nullptr) {
            // the first stage's input, relative to the reference state
            out[0] = f64_to_f32_ftz(rho_d - rr);
            out[ND + 1] = f64_to_f32_ftz(E_d - er);
        }
        const float p = gm1 * fmaf(-0.5f * m2, ir, E);
        const float c = sqrtf(gamma * p * ir);
#pragma unroll
        for (int a = 0; a < ND; ++a) s = fmaf(vel[a] + c, ih[a], s);
        return s;
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // two nodes per thread and step with 16-byte loads (8-byte stores) where
    // the arrays allow it
    const bool pairs = (N & 1) == 0 && (reinterpret_cast<unsigned long long>(U) & 15ull) == 0 &&
                       (reinterpret_cast<unsigned long long>(S) & 7ull) == 0;
    if (pairs) {
        for (long long k = i0; k < N / 2; k += stride) {
            const long long i = 2 * k;
            const double2 r2 = *reinterpret_cast<const double2*>(U + i);
            const double2 e2 = *reinterpret_cast<const double2*>(U + (ND + 1) * N + i);
            double2 m2[ND];
#pragma unroll
            for (int a = 0; a < ND; ++a) m2[a] = *reinterpret_cast<const double2*>(U + (1 + a) * N + i);
            double mx[ND], my[ND];
#pragma unroll
            for (int a = 0; a < ND; ++a) { mx[a] = m2[a].x; my[a] = m2[a].y; }
            float ox[ND + 2], oy[ND + 2];
            m = fmaxf(m, node(r2.x, mx, e2.x, ox));
            m = fmaxf(m, node(r2.y, my, e2.y, oy));
            if (S != nullptr) {
#pragma unroll
                for (int v = 0; v < ND + 2; ++v) *reinterpret_cast<float2*>(S + v * N + i) = make_float2(ox[v], oy[v]);
            }
        }
    } else {
        for (long long i = i0; i < N; i += stride) {
            double mv[ND];
#pragma unroll
            for (int a = 0; a < ND; ++a) mv[a] = U[(1 + a) * N + i];
            float o[ND + 2];
            m = fmaxf(m, node(U[i], mv, U[(ND + 1) * N + i], o));
            if (S != nullptr) {
#pragma unroll
                for (int v = 0; v < ND + 2; ++v) S[v * N + i] = o[v];
            }
        }
    }
    // the maximum in FP32, scaled once by 1 + 2^-16 (exact on a float, and
    // it commutes with the max)
    m = warp_maxf(m);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        m = warp_maxf(m);
        if (threadIdx.x == 0)
            atomicMax(&sc->lam_bits, (unsigned long long)__double_as_longlong((double)m * (1.0 + 1.0 / 65536.0)));
    }
}

// dt = CFL / lambda, clipped so the step lands on t_end.
__global__ void cfl_finalize_kernel(StepScalars* sc, double cfl, int clip)
{
    const double t = sc->t;
    const double lam = __longlong_as_double((long long)sc->lam_bits);
    sc->lam_bits = 0ull;   // ready for the next reduction
    if (clip && !(t < sc->t_end)) { sc->dt = 0.0; return; }
    double dt = div_(cfl, lam);
    if (clip && add_(t, dt) > sc->t_end) dt = sub_(sc->t_end, t);
    sc->t = add_(t, dt);
    sc->dt = dt;
    sc->steps += 1ull;
}

__global__ void set_dt_kernel(StepScalars* sc, double dt, int clip)
{
    const double t = sc->t;
    if (clip && !(t < sc->t_end)) { sc->dt = 0.0; return; }
    if (clip && add_(t, dt) > sc->t_end) dt = sub_(sc->t_end, t);
    sc->t = add_(t, dt);
    sc->dt = dt;
    sc->steps += 1ull;
}

__global__ void reset_clock_kernel(StepScalars* sc, double t_end)
{
    sc->dt = 0.0;
    sc->t = 0.0;
    sc->t_end = t_end;
    sc->lam_bits = 0ull;
    sc->steps = 0ull;
}

cudaError_t launch_reset_clock(double t_end, StepScalars* sc, cudaStream_t s)
{
    reset_clock_kernel<<<1, 1, 0, s>>>(sc, t_end);
    return cudaGetLastError();
}

static int reduce_blocks(long long N)
{
    long long b = (N + 255) / 256;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

cudaError_t launch_cfl(int nd, const double* U, long long N, const double* h, double gamma,
                       double cfl, int clip, StepScalars* sc, cudaStream_t s)
{
    InvH hh{{h[0], h[1], h[2]}};
    const double gm1 = gamma - 1.0;
    const int nb = reduce_blocks(N);
    if (nd == 1) cfl_reduce_kernel<1><<<nb, 256, 0, s>>>(U, N, hh, gamma, gm1, sc, clip);
    else if (nd == 2) cfl_reduce_kernel<2><<<nb, 256, 0, s>>>(U, N, hh, gamma, gm1, sc, clip);
    else cfl_reduce_kernel<3><<<nb, 256, 0, s>>>(U, N, hh, gamma, gm1, sc, clip);
    cfl_finalize_kernel<<<1, 1, 0, s>>>(sc, cfl, clip);
    return cudaGetLastError();
}

cudaError_t launch_cfl_fast(int nd, const double* U, long long N, const double* h, double gamma,
                            double cfl, int clip, StepScalars* sc, cudaStream_t s, float* S)
{
    InvH hh{{h[0], h[1], h[2]}};
    const int nb = reduce_blocks(N);
    if (nd == 1) cfl_reduce_fast_kernel<1><<<nb, 256, 0, s>>>(U, N, hh, (float)gamma, sc, clip, S);
    else if (nd == 2) cfl_reduce_fast_kernel<2><<<nb, 256, 0, s>>>(U, N, hh, (float)gamma, sc, clip, S);
    else cfl_reduce_fast_kernel<3><<<nb, 256, 0, s>>>(U, N, hh, (float)gamma, sc, clip, S);
    cfl_finalize_kernel<<<1, 1, 0, s>>>(sc, cfl, clip);
    return cudaGetLastError();
}

cudaError_t launch_set_dt(double dt, int clip, StepScalars* sc, cudaStream_t s)
{
    set_dt_kernel<<<1, 1, 0, s>>>(sc, dt, clip);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 stages
// U1 = U0 + dt L;  U1 = 3/4 U0 + 1/4 (U1 + dt L);  U0 = U0 / 3 + 2/3 (U1 + dt L),
// each sum and product rounded as written.
template <int STAGE>
__global__ void __launch_bounds__(256) rk_fp64_kernel(double* __restrict__ U0, double* __restrict__ U1,
                                                      const double* __restrict__ L, long long M,
                                                      const StepScalars* sc)
{
    const double dt = sc->dt;
    if (dt == 0.0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M;
         i += (long long)gridDim.x * blockDim.x) {
        const double l = L[i];
        if (STAGE == 1) {
            U1[i] = add_(U0[i], mul_(dt, l));
        } else if (STAGE == 2) {
            U1[i] = add_(mul_(0.75, U0[i]), mul_(0.25, add_(U1[i], mul_(dt, l))));
        } else {
            U0[i] = add_(div_(U0[i], 3.0), mul_(2.0 / 3.0, add_(U1[i], mul_(dt, l))));
        }
    }
}

static int stream_blocks(long long M)
{
    long long b = (M + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

cudaError_t launch_rk_fp64(int stage, double* U0, double* U1, const double* L, long long M,
                           const StepScalars* sc, cudaStream_t s)
{
    const int nb = stream_blocks(M);
    if (stage == 1) rk_fp64_kernel<1><<<nb, 256, 0, s>>>(U0, U1, L, M, sc);
    else if (stage == 2) rk_fp64_kernel<2><<<nb, 256, 0, s>>>(U0, U1, L, M, sc);
    else rk_fp64_kernel<3><<<nb, 256, 0, s>>>(U0, U1, L, M, sc);
    return cudaGetLastError();
}

// S = float(U - U_r): the single-precision input of a step's first stage
// (variable blockIdx.y; U_r = 0 without a clock).
__global__ void __launch_bounds__(256) to_fp32_kernel(const double* __restrict__ U, float* __restrict__ S,
                                                      long long N, int nv, const StepScalars* sc)
{
    if (sc != nullptr && f64_is_zero(sc->dt)) return;   // a finished run (sc may be null: always convert)
    const int v = blockIdx.y;
    double r = 0.0;
    if (sc != nullptr) r = v == 0 ? sc->ref_rho : (v == nv - 1 ? sc->ref_E : 0.0);
    const double* Uv = U + (long long)v * N;
    float* Sv = S + (long long)v * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        Sv[i] = f64_to_f32_ftz(Uv[i] - r);
}

cudaError_t launch_to_fp32(int nv, const double* U, float* S, long long N, const StepScalars* sc, cudaStream_t s)
{
    const int bx = (stream_blocks(N) + nv - 1) / nv;
    to_fp32_kernel<<<dim3(bx, nv), 256, 0, s>>>(U, S, N, nv, sc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reference state
// Order-preserving 64-bit keys of doubles (min/max by unsigned comparison).
__device__ __forceinline__ unsigned long long order_key(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_order_key(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

__global__ void ref_begin_kernel(StepScalars* sc)
{
    sc->ref_keys[0] = ~0ull;
    sc->ref_keys[1] = ~0ull;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y < x ? y : x;
    }
    return x;
}

// min rho and min p = (gamma - 1)(E - |m|^2 / (2 rho)) (FP64, fixed order)
// over the state; minima are exact, so the result does not depend on the
// reduction order (a batch instance and the same grid alone get the same).
template <int ND>
__global__ void __launch_bounds__(256) ref_reduce_kernel(const double* __restrict__ U, long long N, double gm1,
                                                         StepScalars* sc)
{
    unsigned long long kr = ~0ull, kp = ~0ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double Ui[ND + 2];
#pragma unroll
        for (int v = 0; v < ND + 2; ++v) Ui[v] = U[v * N + i];
        const unsigned long long a = order_key(Ui[0]), b = order_key(pressure_exact<ND>(Ui, gm1));
        kr = a < kr ? a : kr;
        kp = b < kp ? b : kp;
    }
    kr = warp_min_u64(kr);
    kp = warp_min_u64(kp);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&sc->ref_keys[0], kr);
        atomicMin(&sc->ref_keys[1], kp);
    }
}

__global__ void ref_finalize_kernel(StepScalars* sc, double gm1)
{
    const double rr = from_order_key(sc->ref_keys[0]);
    const double pr = from_order_key(sc->ref_keys[1]);
    const double er = div_(pr, gm1);
    sc->ref_rho = rr;
    sc->ref_E = er;
    sc->ref_rhof = (float)rr;
    sc->ref_Ef = (float)er;
    sc->ref_pf = (float)pr;
    sc->ref_hf = (float)add_(er, pr);
}

cudaError_t launch_reference(int nd, const double* U, long long N, double gamma, StepScalars* sc,
                             cudaStream_t s)
{
    const double gm1 = gamma - 1.0;
    const int nb = reduce_blocks(N);
    ref_begin_kernel<<<1, 1, 0, s>>>(sc);
    if (nd == 1) ref_reduce_kernel<1><<<nb, 256, 0, s>>>(U, N, gm1, sc);
    else if (nd == 2) ref_reduce_kernel<2><<<nb, 256, 0, s>>>(U, N, gm1, sc);
    else ref_reduce_kernel<3><<<nb, 256, 0, s>>>(U, N, gm1, sc);
    ref_finalize_kernel<<<1, 1, 0, s>>>(sc, gm1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- conservation
// Deterministic: block b sums a fixed slice in a fixed tree order; one block
// then sums the partials in index order.
int conserved_blocks(long long N)
{
    long long b = (N + 2047) / 2048;
    return (int)(b < 512 ? (b < 1 ? 1 : b) : 512);
}

__global__ void __launch_bounds__(256) conserved_partial_kernel(const double* __restrict__ U, long long N,
                                                                int nv, double* partials)
{
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < N ? lo + chunk : N;
    __shared__ double red[8];
    for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += U[v * N + i];
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            partials[v * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

__global__ void conserved_final_kernel(double* partials, int nb, int nv, double vol)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int v = 0; v < nv; ++v) {
            double t = 0.0;
            for (int b = 0; b < nb; ++b) t += partials[v * nb + b];
            partials[nv * nb + v] = t * vol;
        }
    }
}

cudaError_t launch_conserved(int nv, const double* U, long long N, double vol, double* partials,
                             int nblocks, cudaStream_t s)
{
    conserved_partial_kernel<<<nblocks, 256, 0, s>>>(U, N, nv, partials);
    conserved_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, nv, vol);
    return cudaGetLastError();
}

}  // namespace wcns
