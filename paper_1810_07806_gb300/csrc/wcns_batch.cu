// wcns_batch.cu -- the batch engine: many independent grids of one dimension
// and precision ("instances", each with its own size, boundary rules, time
// step and end time) advanced together.  Per RK stage one launch per
// direction covers the tiles of every instance (a tile table); the CFL
// reduction, the per-instance time-step rule and the stage combinations run
// over chunk tables.  One SSP-RK3 step of the whole batch is captured once
// as a CUDA graph and replayed until every instance has reached its end
// time.  Finished instances skip their work (dt = 0) until removed.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/wcns.h"
#include "wcns_fp64.cuh"
#include "wcns_internal.h"

namespace wcns {

struct NodeChunk {      // nodes [begin, begin + count) of one instance
    int inst;
    int count;
    long long begin;
    long long off;      // the instance's element offset and node count (copies
    long long N;        // of its BatchInst's, so the state loads need no other load)
};

struct ElemChunk {      // batch-array elements [begin, begin + count), one instance
    int inst;
    int count;
    long long begin;
};

constexpr int kNodeChunk = 1024;   // a multiple of the 256 threads of the time-step pass
constexpr int kElemChunk = 4096;
constexpr int kDtStride = (int)(sizeof(StepScalars) / sizeof(double));
static_assert(sizeof(StepScalars) % sizeof(double) == 0, "StepScalars must be a whole number of doubles");

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ double bwarp_max(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float bwarp_maxf(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Per-instance maximum wave-speed sum.  FP64 batches evaluate every node in
// the same fixed order as the single-grid rule (so a batched instance takes
// the same steps as the instance alone); FP32 batches use FP32 speeds rounded
// upward, with an FP64 maximum, and write float(U) of the instances that
// advance (the first stage's input) from the same pass.
template <int ND, bool FAST>
__global__ void __launch_bounds__(256) batch_cfl_kernel(const double* __restrict__ U,
                                                        const BatchInst* __restrict__ insts,
                                                        const NodeChunk* __restrict__ chunks,
                                                        double gamma, double gm1, StepScalars* sc,
                                                        float* __restrict__ S)
{
    const NodeChunk ch = chunks[blockIdx.x];
    // the state of this thread's nodes (at most KU: kNodeChunk = KU x 256),
    // loaded before anything else is waited for
    constexpr int KU = kNodeChunk / 256;
    const double* Ui = U + ch.off;
    const long long N = ch.N;
    double Uv[KU][ND + 2];
#pragma unroll
    for (int j = 0; j < KU; ++j) {
        const int k = threadIdx.x + j * 256;
        if (k < ch.count) {
#pragma unroll
            for (int v = 0; v < ND + 2; ++v) Uv[j][v] = Ui[v * N + ch.begin + k];
        }
    }
    // the instance still runs (one FP64 compare per block, not per thread:
    // the FP64 pipe runs at a small fraction of the FP32 rate)
    StepScalars* s = sc + ch.inst;
    __shared__ int s_run;
    if (threadIdx.x == 0) s_run = s->t < s->t_end;
    __syncthreads();
    if (!s_run) return;
    const BatchInst& I = insts[ch.inst];
    double m = 0.0;
    float mf = 0.f;
    const float gf = (float)gamma;
    const double rr = s->ref_rho, er = s->ref_E;
#pragma unroll
    for (int j = 0; j < KU; ++j) {
        const int k = threadIdx.x + j * 256;
        if (k >= ch.count) continue;
        const long long i = ch.begin + k;
        if constexpr (FAST) {
            // the same FP32 expressions as the single-grid rule; the stage
            // input is relative to the instance's reference state
            float Uf[ND + 2];
#pragma unroll
            for (int v = 0; v < ND + 2; ++v) {
                const double x = Uv[j][v];
                Uf[v] = f64_to_f32_ftz(x);
                const double r = v == 0 ? rr : (v == ND + 1 ? er : 0.0);
                S[ch.off + v * N + i] = (v == 0 || v == ND + 1) ? f64_to_f32_ftz(x - r) : Uf[v];
            }
            const float ir = __frcp_rn(Uf[0]);
            float m2 = 0.f, sum = 0.f, vel[ND];
#pragma unroll
            for (int a = 0; a < ND; ++a) {
                m2 = fmaf(Uf[1 + a], Uf[1 + a], m2);
                vel[a] = fabsf(Uf[1 + a]) * ir;
            }
            const float p = (gf - 1.f) * fmaf(-0.5f * m2, ir, Uf[ND + 1]);
            const float c = sqrtf(gf * p * ir);
#pragma unroll
            for (int a = 0; a < ND; ++a) sum = fmaf(vel[a] + c, I.inv_hf[a], sum);
            mf = fmaxf(mf, sum);
        } else {
            const double c = sqrt_(div_(mul_(gamma, pressure_exact<ND>(Uv[j], gm1)), Uv[j][0]));
            double sum = 0.0;
#pragma unroll
            for (int a = 0; a < ND; ++a) {
                const double q = div_(add_(fabs(div_(Uv[j][1 + a], Uv[j][0])), c), I.h[a]);
                sum = a == 0 ? q : add_(sum, q);
            }
            m = fmax(m, sum);
        }
    }
    if constexpr (FAST) {
        // the maximum in FP32, scaled once by 1 + 2^-16 (exact on a float,
        // and it commutes with the max): no FP64 work per thread
        mf = bwarp_maxf(mf);
        __shared__ float redf[8];
        if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = mf;
        __syncthreads();
        if (threadIdx.x < 32) {
            mf = threadIdx.x < (blockDim.x >> 5) ? redf[threadIdx.x] : 0.f;
            mf = bwarp_maxf(mf);
            if (threadIdx.x == 0)
                atomicMax(&s->lam_bits,
                          (unsigned long long)__double_as_longlong((double)mf * (1.0 + 1.0 / 65536.0)));
        }
        return;
    }
    m = bwarp_max(m);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        m = bwarp_max(m);
        if (threadIdx.x == 0) atomicMax(&s->lam_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// dt_i = CFL / lambda_i clipped to t_end_i (0 once finished); counts the
// instances that advance in this step.
__global__ void batch_finalize_kernel(StepScalars* sc, const int* __restrict__ slots, int nslots,
                                      double cfl, int* active)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nslots) return;
    StepScalars* s = sc + slots[k];
    const double t = s->t;
    const double lam = __longlong_as_double((long long)s->lam_bits);
    s->lam_bits = 0ull;
    if (!(t < s->t_end)) { s->dt = 0.0; return; }
    double dt = div_(cfl, lam);
    if (add_(t, dt) > s->t_end) dt = sub_(s->t_end, t);
    s->t = add_(t, dt);
    s->dt = dt;
    s->steps += 1ull;
    atomicAdd(active, 1);
}

template <int STAGE>
__global__ void __launch_bounds__(256) batch_rk_fp64_kernel(double* __restrict__ U0, double* __restrict__ U1,
                                                            const double* __restrict__ L,
                                                            const ElemChunk* __restrict__ chunks,
                                                            const StepScalars* __restrict__ sc)
{
    const ElemChunk ch = chunks[blockIdx.x];
    const double dt = sc[ch.inst].dt;
    if (dt == 0.0) return;
    for (int k = threadIdx.x; k < ch.count; k += blockDim.x) {
        const long long i = ch.begin + k;
        const double l = L[i];
        if (STAGE == 1) U1[i] = add_(U0[i], mul_(dt, l));
        else if (STAGE == 2) U1[i] = add_(mul_(0.75, U0[i]), mul_(0.25, add_(U1[i], mul_(dt, l))));
        else U0[i] = add_(div_(U0[i], 3.0), mul_(2.0 / 3.0, add_(U1[i], mul_(dt, l))));
    }
}

__global__ void set_clock_kernel(StepScalars* sc, double t_end)
{
    sc->dt = 0.0;
    sc->t = 0.0;
    sc->t_end = t_end;
    sc->lam_bits = 0ull;
    sc->steps = 0ull;
}

}  // namespace wcns

using namespace wcns;

// ---------------------------------------------------------------- engine
struct BatchSlot {
    bool used = false;
    int n[3] = {1, 1, 1};
    int periodic[3] = {0, 0, 0};
    double h[3] = {1, 1, 1};
    GridInfo G;            // boundary kinds, fixed states, body force
    long long N = 0;
    long long off = 0;     // element offset in the arenas
    long long elems = 0;   // reserved elements (nv * N rounded up)
    double t_end = 0.0;
};

struct wcns_batch {
    int ndim = 0, nv = 0, precision = 0, flux = 0;
    double gamma = 1.4, cfl = 0.5;
    SchemeConst K{};
    float sqrt_eps_f = 0.f;
    long long cap_elems = 0;
    int cap_slots = 0;
    // arenas and per-instance clocks
    double* U = nullptr;
    void* S = nullptr;      // FP64: stage state; FP32: stage input A (float)
    float* S2 = nullptr;    // FP32: stage input B
    void* L = nullptr;
    float* D = nullptr;
    StepScalars* sc = nullptr;
    int* active = nullptr;
    long long* fallback = nullptr;
    // tables
    BatchInst* d_insts = nullptr;
    int* d_slots = nullptr;
    BatchTile* d_tiles[3] = {nullptr, nullptr, nullptr};
    NodeChunk* d_nch = nullptr;
    ElemChunk* d_ech = nullptr;
    size_t cap_tiles[3] = {0, 0, 0}, cap_nch = 0, cap_ech = 0;
    long long ntiles[3] = {0, 0, 0};
    int nnch = 0, nech = 0, nslots_active = 0;
    std::vector<BatchSlot> slots;
    std::vector<std::pair<long long, long long>> free_ranges;   // [begin, end), sorted
    bool dirty = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;   // stream used only to record the step graph
    size_t bytes = 0;
    // sweep launch form: 0 = one CTA per tile (tile table), 1 = persistent
    // CTAs taking tiles from device counters (one counter per sweep of a step)
    int launch_mode = 0;
    unsigned int* work = nullptr;
    bool any_gravity = false;   // some instance has a body force (the last sweep adds it)
};

namespace {

wcns_status bfail(wcns_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

wcns_status bcuda(cudaError_t e, const char* where)
{
    return bfail(WCNS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define BCK(call, where)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bcuda(e_, where);       \
    } while (0)

template <typename T>
cudaError_t ensure(T*& p, size_t& cap, size_t need)
{
    if (need <= cap && p) return cudaSuccess;
    size_t n = std::max(need, cap * 2);
    if (n < 64) n = 64;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)&p, n * sizeof(T));
    if (e == cudaSuccess) cap = n;
    return e;
}

template <typename T, int ND, int DIR>
void add_tiles(std::vector<BatchTile>& out, int inst, const BatchSlot& s)
{
    using G = TileGeom<T, ND, DIR, batch_cfg<T>(ND)>;
    const int nd = s.n[DIR];
    const int ptiles = (nd + G::TS - 1) / G::TS;
    if (DIR == 0) {
        const long long rows = s.N / s.n[0];
        for (long long lf = 0; lf < rows; lf += G::TL)
            for (int pt = 0; pt < ptiles; ++pt) out.push_back(BatchTile{inst, pt * G::TS, (int)lf, 0});
    } else {
        const long long outer = s.N / ((long long)s.n[0] * nd);
        for (long long o = 0; o < outer; ++o)
            for (int pt = 0; pt < ptiles; ++pt)
                for (int xf = 0; xf < s.n[0]; xf += G::TL) out.push_back(BatchTile{inst, pt * G::TS, xf, (int)o});
    }
}

template <typename T>
void build_tiles(int nd, int dir, std::vector<BatchTile>& out, int inst, const BatchSlot& s)
{
    if (nd == 1) add_tiles<T, 1, 0>(out, inst, s);
    else if (nd == 2) { if (dir == 0) add_tiles<T, 2, 0>(out, inst, s); else add_tiles<T, 2, 1>(out, inst, s); }
    else if (dir == 0) add_tiles<T, 3, 0>(out, inst, s);
    else if (dir == 1) add_tiles<T, 3, 1>(out, inst, s);
    else add_tiles<T, 3, 2>(out, inst, s);
}

wcns_status rebuild(wcns_batch* b)
{
    const bool fp32 = b->precision == WCNS_FP32;
    std::vector<BatchInst> insts(b->cap_slots);
    std::vector<int> active;
    std::vector<BatchTile> tiles[3];
    std::vector<NodeChunk> nch;
    std::vector<ElemChunk> ech;
    bool any_gravity = false;
    for (int i = 0; i < b->cap_slots; ++i) {
        const BatchSlot& s = b->slots[i];
        BatchInst& I = insts[i];
        memset(&I, 0, sizeof I);
        if (!s.used) continue;
        active.push_back(i);
        I.off = s.off;
        I.N = s.N;
        for (int a = 0; a < 3; ++a) {
            I.n[a] = s.n[a];
            I.periodic[a] = s.periodic[a];
            I.h[a] = s.h[a];
            I.inv_h[a] = a < b->ndim ? 1.0 / s.h[a] : 0.0;
            I.inv_hf[a] = (float)I.inv_h[a];
            for (int sd = 0; sd < 2; ++sd) {
                I.bc[a][sd] = s.G.bc[a][sd];
                for (int v = 0; v < 5; ++v) I.bcs[a][sd][v] = s.G.bc_state[a][sd][v];
            }
            I.grav[a] = s.G.gravity[a];
        }
        I.has_grav = s.G.has_gravity ? 1 : 0;
        if (s.G.has_gravity) any_gravity = true;
        for (int d = 0; d < b->ndim; ++d) {
            if (fp32) build_tiles<float>(b->ndim, d, tiles[d], i, s);
            else build_tiles<double>(b->ndim, d, tiles[d], i, s);
        }
        for (long long k = 0; k < s.N; k += kNodeChunk)
            nch.push_back(NodeChunk{i, (int)std::min<long long>(kNodeChunk, s.N - k), k, s.off, s.N});
        const long long M = (long long)b->nv * s.N;
        for (long long k = 0; k < M; k += kElemChunk)
            ech.push_back(ElemChunk{i, (int)std::min<long long>(kElemChunk, M - k), s.off + k});
    }
    BCK(cudaMemcpy(b->d_insts, insts.data(), sizeof(BatchInst) * b->cap_slots, cudaMemcpyHostToDevice), "insts");
    if (!active.empty())
        BCK(cudaMemcpy(b->d_slots, active.data(), sizeof(int) * active.size(), cudaMemcpyHostToDevice), "slots");
    for (int d = 0; d < b->ndim; ++d) {
        BCK(ensure(b->d_tiles[d], b->cap_tiles[d], tiles[d].size()), "tile table");
        if (!tiles[d].empty())
            BCK(cudaMemcpy(b->d_tiles[d], tiles[d].data(), sizeof(BatchTile) * tiles[d].size(),
                           cudaMemcpyHostToDevice), "tile table");
        b->ntiles[d] = (long long)tiles[d].size();
    }
    BCK(ensure(b->d_nch, b->cap_nch, nch.size()), "node chunks");
    BCK(ensure(b->d_ech, b->cap_ech, ech.size()), "element chunks");
    if (!nch.empty())
        BCK(cudaMemcpy(b->d_nch, nch.data(), sizeof(NodeChunk) * nch.size(), cudaMemcpyHostToDevice), "chunks");
    if (!ech.empty())
        BCK(cudaMemcpy(b->d_ech, ech.data(), sizeof(ElemChunk) * ech.size(), cudaMemcpyHostToDevice), "chunks");
    b->nnch = (int)nch.size();
    b->nech = (int)ech.size();
    b->nslots_active = (int)active.size();
    b->any_gravity = any_gravity;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->dirty = false;
    return WCNS_OK;
}

constexpr int kWorkCounters = 16;   // >= 3 stages x 3 directions

cudaError_t sweeps(wcns_batch* b, const void* Uin, void* L, cudaStream_t s, int fuse_stage = 0,
                   float* S_out = nullptr, int counter0 = 0)
{
    const bool fp32 = b->precision == WCNS_FP32;
    for (int k = 0; k < b->ndim; ++k) {
        // FP32: z, y, x with the stage combination in the x sweep (as the
        // single-grid FP32 step); FP64: x, y, z, the oracle's order
        const int d = fuse_stage ? b->ndim - 1 - k : k;
        SweepArgs a{};
        a.U = Uin;
        a.L = L;
        a.accumulate = k > 0;
        a.fallback = b->fallback;
        a.K = b->K;
        a.sqrt_eps_f = b->sqrt_eps_f;
        a.insts = b->d_insts;
        a.tiles = b->d_tiles[d];
        a.inst_dt = &b->sc[0].dt;
        a.dt_stride = kDtStride;
        if (b->launch_mode == 1) {
            a.work = b->work + counter0 + k;
            a.ntiles = b->ntiles[d];
        }
        // the last sweep of an RHS adds the body force of the instances that
        // have one (as a single grid's last sweep)
        a.source = b->any_gravity && k == b->ndim - 1;
        if (fuse_stage && d == 0) {
            a.fuse_stage = fuse_stage;
            a.U0 = b->U;
            a.D = b->D;
            a.S_out = S_out;
        }
        // FP32 sweeps after the first of an RHS: programmatic dependents of
        // the previous one (as on single grids)
        a.pdl = fp32 && k > 0;
        cudaError_t e = fp32 ? launch_sweep_batch_fp32(b->ndim, d, b->flux, a, b->ntiles[d], s)
                             : launch_sweep_batch_fp64(b->ndim, d, b->flux, a, b->ntiles[d], s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One SSP-RK3 step of every instance (the captured sequence).
cudaError_t step_sequence(wcns_batch* b, cudaStream_t s)
{
    const bool fp32 = b->precision == WCNS_FP32;
    cudaError_t e = cudaMemsetAsync(b->active, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (b->launch_mode == 1 && (e = cudaMemsetAsync(b->work, 0, sizeof(unsigned int) * kWorkCounters, s)) != cudaSuccess)
        return e;
    if (b->nnch > 0) {
        const double gm1 = b->gamma - 1.0;
        float* S0 = fp32 ? (float*)b->S : nullptr;   // FP32: the first stage's input
        if (b->ndim == 1)
            fp32 ? batch_cfl_kernel<1, true><<<b->nnch, 256, 0, s>>>(b->U, b->d_insts, b->d_nch, b->gamma, gm1, b->sc, S0)
                 : batch_cfl_kernel<1, false><<<b->nnch, 256, 0, s>>>(b->U, b->d_insts, b->d_nch, b->gamma, gm1, b->sc, S0);
        else if (b->ndim == 2)
            fp32 ? batch_cfl_kernel<2, true><<<b->nnch, 256, 0, s>>>(b->U, b->d_insts, b->d_nch, b->gamma, gm1, b->sc, S0)
                 : batch_cfl_kernel<2, false><<<b->nnch, 256, 0, s>>>(b->U, b->d_insts, b->d_nch, b->gamma, gm1, b->sc, S0);
        else
            fp32 ? batch_cfl_kernel<3, true><<<b->nnch, 256, 0, s>>>(b->U, b->d_insts, b->d_nch, b->gamma, gm1, b->sc, S0)
                 : batch_cfl_kernel<3, false><<<b->nnch, 256, 0, s>>>(b->U, b->d_insts, b->d_nch, b->gamma, gm1, b->sc, S0);
    }
    if (b->nslots_active > 0)
        batch_finalize_kernel<<<(b->nslots_active + 127) / 128, 128, 0, s>>>(b->sc, b->d_slots, b->nslots_active,
                                                                           b->cfl, b->active);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (b->nech == 0) return cudaSuccess;
    if (!fp32) {
        double* U1 = (double*)b->S;
        double* L = (double*)b->L;
        if ((e = sweeps(b, b->U, L, s, 0, nullptr, 0)) != cudaSuccess) return e;
        batch_rk_fp64_kernel<1><<<b->nech, 256, 0, s>>>(b->U, U1, L, b->d_ech, b->sc);
        if ((e = sweeps(b, U1, L, s, 0, nullptr, 3)) != cudaSuccess) return e;
        batch_rk_fp64_kernel<2><<<b->nech, 256, 0, s>>>(b->U, U1, L, b->d_ech, b->sc);
        if ((e = sweeps(b, U1, L, s, 0, nullptr, 6)) != cudaSuccess) return e;
        batch_rk_fp64_kernel<3><<<b->nech, 256, 0, s>>>(b->U, U1, L, b->d_ech, b->sc);
    } else {
        // stage inputs A -> B -> A (A = float(U) from the time-step pass);
        // the x sweep of each stage applies the stage combination, stage 3
        // to the FP64 state
        float* A = (float*)b->S;
        float* B = b->S2;
        float* L = (float*)b->L;
        if ((e = sweeps(b, A, L, s, 1, B, 0)) != cudaSuccess) return e;
        if ((e = sweeps(b, B, L, s, 2, A, 3)) != cudaSuccess) return e;
        if ((e = sweeps(b, A, L, s, 3, nullptr, 6)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// per device and precision: the batched kernels' attributes are set
std::atomic<bool> prepared_batch[64][2];

}  // namespace

extern "C" {

wcns_status wcns_batch_create(int ndim, double gamma, const wcns_scheme_params* prm, long long max_nodes,
                              int max_instances, wcns_batch** out)
{
    set_last_error(nullptr);
    if (!prm || !out) return bfail(WCNS_ERR_INVALID, "wcns_batch_create: null argument");
    *out = nullptr;
    if (ndim < 1 || ndim > 3) return bfail(WCNS_ERR_INVALID, "ndim must be 1, 2 or 3");
    if (!(gamma > 1.0)) return bfail(WCNS_ERR_INVALID, "gamma must exceed 1");
    if (const char* why = scheme_params_error(prm)) return bfail(WCNS_ERR_INVALID, "%s", why);
    if (max_nodes < 1 || max_instances < 1) return bfail(WCNS_ERR_INVALID, "capacities must be positive");

    wcns_batch* b = new wcns_batch();
    b->ndim = ndim;
    b->nv = ndim + 2;
    b->precision = prm->precision;
    b->flux = prm->flux;
    b->gamma = gamma;
    b->cfl = prm->cfl;
    b->K = make_scheme_const(prm, gamma);
    b->sqrt_eps_f = (float)sqrt(prm->eps);
    b->cap_slots = max_instances;
    // each instance's block is rounded up to 64 elements
    b->cap_elems = (long long)b->nv * max_nodes + 64LL * max_instances;
    b->slots.resize(max_instances);
    b->free_ranges.push_back({0, b->cap_elems});

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { delete b; return bcuda(e, "cudaGetDevice"); }
    const bool fp32 = b->precision == WCNS_FP32;
    if (!prepared_batch[dev & 63][fp32]) {
        e = fp32 ? prepare_sweeps_batch_fp32() : prepare_sweeps_batch_fp64();
        if (e == cudaSuccess && fp32) e = prepare_sweeps_fp32_weights();
        if (e != cudaSuccess) { delete b; return bcuda(e, "prepare batched sweeps"); }
        prepared_batch[dev & 63][fp32] = true;
    }
    const size_t w = fp32 ? 4 : 8;
    const size_t M = (size_t)b->cap_elems;
    b->bytes = M * 8 + M * w * 2 + (fp32 ? M * 8 : 0) + sizeof(StepScalars) * max_instances +
               (sizeof(BatchInst) + sizeof(int) + sizeof(long long)) * max_instances + 64;
    e = cudaMalloc((void**)&b->U, M * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->S, M * w);
    if (e == cudaSuccess) e = cudaMalloc(&b->L, M * w);
    if (e == cudaSuccess && fp32) e = cudaMalloc((void**)&b->D, M * 4);
    if (e == cudaSuccess && fp32) e = cudaMalloc((void**)&b->S2, M * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->sc, sizeof(StepScalars) * max_instances);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->active, 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->work, sizeof(unsigned int) * kWorkCounters);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->fallback, sizeof(long long) * max_instances);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_insts, sizeof(BatchInst) * max_instances);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_slots, sizeof(int) * max_instances);
    if (e == cudaSuccess) e = cudaMemset(b->sc, 0, sizeof(StepScalars) * max_instances);
    if (e == cudaSuccess) e = cudaMemset(b->fallback, 0, sizeof(long long) * max_instances);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        const size_t need = b->bytes;
        wcns_batch_destroy(b);
        cudaGetLastError();
        return bfail(WCNS_ERR_NOMEM, "batch allocation of %zu bytes failed", need);
    }
    *out = b;
    return WCNS_OK;
}

wcns_status wcns_batch_destroy(wcns_batch* b)
{
    if (!b) return WCNS_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->U);
    cudaFree(b->S);
    cudaFree(b->L);
    cudaFree(b->D);
    cudaFree(b->S2);
    cudaFree(b->sc);
    cudaFree(b->active);
    cudaFree(b->work);
    cudaFree(b->fallback);
    cudaFree(b->d_insts);
    cudaFree(b->d_slots);
    for (int d = 0; d < 3; ++d) cudaFree(b->d_tiles[d]);
    cudaFree(b->d_nch);
    cudaFree(b->d_ech);
    delete b;
    return WCNS_OK;
}

size_t wcns_batch_bytes(const wcns_batch* b) { return b ? b->bytes : 0; }

wcns_status wcns_batch_add(wcns_batch* b, const wcns_grid* g, const double* U0, int u0_on_device,
                           double t_end, int* slot_out, void* stream)
{
    set_last_error(nullptr);
    if (!b || !g || !U0 || !slot_out) return bfail(WCNS_ERR_INVALID, "wcns_batch_add: null argument");
    if (g->ndim != b->ndim) return bfail(WCNS_ERR_INVALID, "grid dimension differs from the batch's");
    if (!(t_end >= 0.0)) return bfail(WCNS_ERR_INVALID, "t_end must be >= 0");
    // the single-grid rules: boundary kinds (transmissive, periodic,
    // reflecting, fixed state), node spacing, fixed states, body force
    BatchSlot s;
    char why[256];
    if (const char* msg = grid_error(g, b->gamma, s.G, why, sizeof why)) return bfail(WCNS_ERR_INVALID, "%s", msg);
    s.N = s.G.N;
    for (int a = 0; a < b->ndim; ++a) {
        s.n[a] = s.G.n[a];
        s.periodic[a] = s.G.periodic[a];
        s.h[a] = s.G.h[a];
    }
    if (b->ndim == 3 && (s.n[1] > 65535 || s.n[2] > 65535)) return bfail(WCNS_ERR_INVALID, "grid too large");
    int slot = -1;
    for (int i = 0; i < b->cap_slots; ++i)
        if (!b->slots[i].used) { slot = i; break; }
    if (slot < 0) return bfail(WCNS_ERR_BUSY, "no free instance slot");
    const long long M = (long long)b->nv * s.N;
    s.elems = (M + 63) / 64 * 64;
    long long off = -1;
    for (auto& r : b->free_ranges)
        if (r.second - r.first >= s.elems) {
            off = r.first;
            r.first += s.elems;
            break;
        }
    if (off < 0) return bfail(WCNS_ERR_NOMEM, "batch arena has no free range of %lld elements", s.elems);
    b->free_ranges.erase(std::remove_if(b->free_ranges.begin(), b->free_ranges.end(),
                                        [](const std::pair<long long, long long>& r) { return r.first >= r.second; }),
                         b->free_ranges.end());
    s.off = off;
    s.t_end = t_end;
    s.used = true;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaMemcpyAsync(b->U + off, U0, sizeof(double) * M,
                        u0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st), "initial state copy");
    set_clock_kernel<<<1, 1, 0, st>>>(b->sc + slot, t_end);
    BCK(cudaGetLastError(), "clock set");
    // the FP32 stage values' reference state, from the initial state (the
    // same rule and kernels as a single grid's first step)
    BCK(launch_reference(b->ndim, b->U + off, s.N, b->gamma, b->sc + slot, st), "reference state");
    BCK(cudaMemsetAsync(b->fallback + slot, 0, sizeof(long long), st), "fallback counter reset");
    b->slots[slot] = s;
    b->dirty = true;
    *slot_out = slot;
    return WCNS_OK;
}

wcns_status wcns_batch_remove(wcns_batch* b, int slot)
{
    set_last_error(nullptr);
    if (!b || slot < 0 || slot >= b->cap_slots || !b->slots[slot].used)
        return bfail(WCNS_ERR_INVALID, "wcns_batch_remove: bad slot");
    BatchSlot& s = b->slots[slot];
    b->free_ranges.push_back({s.off, s.off + s.elems});
    std::sort(b->free_ranges.begin(), b->free_ranges.end());
    std::vector<std::pair<long long, long long>> merged;
    for (auto& r : b->free_ranges) {
        if (!merged.empty() && merged.back().second == r.first) merged.back().second = r.second;
        else merged.push_back(r);
    }
    b->free_ranges.swap(merged);
    s = BatchSlot();
    b->dirty = true;
    return WCNS_OK;
}

wcns_status wcns_batch_step(wcns_batch* b, int nsteps, int* active_out, void* stream)
{
    set_last_error(nullptr);
    if (!b || nsteps < 0) return bfail(WCNS_ERR_INVALID, "wcns_batch_step: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    BCK(cudaGetLastError(), "pending CUDA error");
    if (b->dirty) {
        BCK(cudaStreamSynchronize(s), "sync before table rebuild");
        wcns_status st = rebuild(b);
        if (st != WCNS_OK) return st;
    }
    if (!b->exec && b->nslots_active > 0) {
        // record one step of the whole batch once; it is replayed every step
        BCK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = step_sequence(b, b->capture);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return bcuda(e, "capture step"); }
        if (e2 != cudaSuccess) return bcuda(e2, "end capture");
        b->graph = g;
        BCK(cudaGraphInstantiate(&b->exec, g, 0), "instantiate step graph");
    }
    for (int k = 0; k < nsteps && b->exec; ++k) BCK(cudaGraphLaunch(b->exec, s), "graph launch");
    if (active_out) {
        int act = 0;
        BCK(cudaMemcpyAsync(&act, b->active, sizeof(int), cudaMemcpyDeviceToHost, s), "active copy");
        BCK(cudaStreamSynchronize(s), "sync");
        *active_out = b->exec ? act : 0;
    }
    return WCNS_OK;
}

wcns_status wcns_batch_launch_mode(wcns_batch* b, int mode)
{
    set_last_error(nullptr);
    if (!b || mode < 0 || mode > 1) return bfail(WCNS_ERR_INVALID, "wcns_batch_launch_mode: bad argument");
    if (mode != b->launch_mode) {
        b->launch_mode = mode;
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    }
    return WCNS_OK;
}

wcns_status wcns_batch_autotune(wcns_batch* b, int steps, int* mode_out, double* ms_per_step, void* stream)
{
    set_last_error(nullptr);
    if (!b || steps < 1) return bfail(WCNS_ERR_INVALID, "wcns_batch_autotune: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    BCK(cudaGetLastError(), "pending CUDA error");
    if (b->dirty) {
        BCK(cudaStreamSynchronize(s), "sync before table rebuild");
        wcns_status st = rebuild(b);
        if (st != WCNS_OK) return st;
    }
    double ms[2] = {0.0, 0.0};
    if (b->nslots_active > 0) {
        // trial steps on the live batch; state, clocks and counters are saved
        // first and put back afterwards, so the results do not change
        const size_t ub = sizeof(double) * (size_t)b->cap_elems;
        const size_t cb = sizeof(StepScalars) * (size_t)b->cap_slots;
        const size_t fbb = sizeof(long long) * (size_t)b->cap_slots;
        char* save = nullptr;
        if (cudaMalloc((void**)&save, ub + cb + fbb) != cudaSuccess) {
            cudaGetLastError();
            return bfail(WCNS_ERR_NOMEM, "wcns_batch_autotune: no room to save the batch state");
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaMemcpyAsync(save, b->U, ub, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(save + ub, b->sc, cb, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(save + ub + cb, b->fallback, fbb, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        for (int mode = 0; mode < 2 && e == cudaSuccess; ++mode) {
            wcns_batch_launch_mode(b, mode);
            wcns_status st = wcns_batch_step(b, 1, nullptr, stream);   // capture + warm-up
            if (st != WCNS_OK) { e = cudaErrorUnknown; break; }
            e = cudaEventRecord(e0, s);
            for (int k = 0; k < steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            ms[mode] = t / steps;
            // restore (also after a failed trial, so the batch keeps its state)
            const cudaError_t r1 = cudaMemcpyAsync(b->U, save, ub, cudaMemcpyDeviceToDevice, s);
            const cudaError_t r2 = cudaMemcpyAsync(b->sc, save + ub, cb, cudaMemcpyDeviceToDevice, s);
            const cudaError_t r3 = cudaMemcpyAsync(b->fallback, save + ub + cb, fbb, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = r1 != cudaSuccess ? r1 : (r2 != cudaSuccess ? r2 : r3);
        }
        const cudaError_t es = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = es;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(save);
        if (e != cudaSuccess) return bcuda(e, "wcns_batch_autotune");
        wcns_batch_launch_mode(b, ms[1] < ms[0] ? 1 : 0);
    }
    if (mode_out) *mode_out = b->launch_mode;
    if (ms_per_step) { ms_per_step[0] = ms[0]; ms_per_step[1] = ms[1]; }
    return WCNS_OK;
}

wcns_status wcns_batch_run(wcns_batch* b, int max_steps, int check, int* steps_out, void* stream)
{
    set_last_error(nullptr);
    if (!b || max_steps < 0) return bfail(WCNS_ERR_INVALID, "wcns_batch_run: bad argument");
    if (check < 1) check = 1;
    int done = 0, active = 1;
    while (done < max_steps && active > 0) {
        const int k = std::min(check, max_steps - done);
        wcns_status st = wcns_batch_step(b, k, &active, stream);
        if (st != WCNS_OK) return st;
        done += k;
    }
    if (steps_out) *steps_out = done;
    return WCNS_OK;
}

wcns_status wcns_batch_read(wcns_batch* b, int slot, double* U_out, int out_on_device, double* t_out,
                            int* steps_out, void* stream)
{
    set_last_error(nullptr);
    if (!b || slot < 0 || slot >= b->cap_slots || !b->slots[slot].used)
        return bfail(WCNS_ERR_INVALID, "wcns_batch_read: bad slot");
    const BatchSlot& s = b->slots[slot];
    cudaStream_t st = (cudaStream_t)stream;
    if (U_out)
        BCK(cudaMemcpyAsync(U_out, b->U + s.off, sizeof(double) * b->nv * s.N,
                            out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st), "state copy");
    StepScalars sc;
    long long fell = 0;
    BCK(cudaMemcpyAsync(&sc, b->sc + slot, sizeof sc, cudaMemcpyDeviceToHost, st), "clock copy");
    BCK(cudaMemcpyAsync(&fell, b->fallback + slot, sizeof fell, cudaMemcpyDeviceToHost, st), "counter copy");
    BCK(cudaStreamSynchronize(st), "sync");
    if (t_out) *t_out = sc.t;
    if (steps_out) *steps_out = (int)sc.steps;
    if (fell > 0)
        return bfail(WCNS_ERR_NONPHYSICAL, "instance %d: %lld faces had rho <= 0 or p <= 0 and used first-order values",
                     slot, fell);
    return WCNS_OK;
}

}  // extern "C"

namespace wcns {
// For the serving loop: slots in use whose clock has reached t_end (one
// device-to-host copy of all clocks; synchronises the stream).
cudaError_t batch_finished_slots(wcns_batch* b, std::vector<int>& out, cudaStream_t s)
{
    out.clear();
    std::vector<StepScalars> clocks(b->cap_slots);
    cudaError_t e = cudaMemcpyAsync(clocks.data(), b->sc, sizeof(StepScalars) * b->cap_slots,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < b->cap_slots; ++i)
        if (b->slots[i].used && !(clocks[i].t < clocks[i].t_end)) out.push_back(i);
    return cudaSuccess;
}

int batch_active_count(const wcns_batch* b)
{
    int n = 0;
    for (const BatchSlot& s : b->slots) n += s.used ? 1 : 0;
    return n;
}

bool batch_fits(const wcns_batch* b, long long nodes)
{
    const long long need = ((long long)b->nv * nodes + 63) / 64 * 64;
    bool slot = false;
    for (const BatchSlot& s : b->slots) if (!s.used) { slot = true; break; }
    if (!slot) return false;
    for (const auto& r : b->free_ranges) if (r.second - r.first >= need) return true;
    return false;
}

long long batch_capacity_nodes(const wcns_batch* b) { return (b->cap_elems - 64LL * b->cap_slots) / b->nv; }
}  // namespace wcns
