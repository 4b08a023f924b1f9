// wcns_api.cu -- the C ABI of libwcns (declared in include/wcns.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/wcns.h"
#include "wcns_internal.h"

using namespace wcns;

struct wcns_handle {
    int ndim = 0, nv = 0;
    int n[3] = {1, 1, 1};
    long long N = 0;
    double h[3] = {1, 1, 1}, inv_h[3] = {0, 0, 0};
    int periodic[3] = {0, 0, 0};
    GridInfo G;                 // boundary kinds, fixed states, gravity
    double gamma = 1.4;
    wcns_scheme_params p{};
    SchemeConst K{};
    float sqrt_eps_f = 0.f;
    int device = 0;
    // device scratch
    void* L = nullptr;          // RHS, handle precision
    void* U1 = nullptr;         // FP64: stage state; FP32: stage sweep input A (float)
    float* S2 = nullptr;        // FP32: second stage input buffer B
    float* D = nullptr;         // FP32: stage increment
    StepScalars* sc = nullptr;
    long long* fallback = nullptr;
    double* partials = nullptr;
    int nblk_cons = 0;
    size_t bytes = 0;
    // tile configuration of each direction's FP32 sweep (set by wcns_autotune)
    int tile_cfg[3] = {0, 0, 0};
    // FP32: the reference state of the stage values is in sc (set at the
    // first step or advance)
    bool ref_set = false;
    // device copy of a host state (wcns_step_rk3_host), allocated on first use
    double* Udev = nullptr;
    // one RK3 step with the CFL rule as a CUDA graph, per state pointer:
    // [0] clock reset + step (wcns_step_rk3), [1] clipped step (wcns_advance);
    // captured on an internal stream, replayed on the caller's
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    const void* graph_U[2] = {nullptr, nullptr};
    // optional sweep timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev;    // pairs (start, end) around each RHS's sweeps
    size_t ev_used = 0;             // events recorded since the last read
    long long prof_sweeps = 0;      // sweep launches those pairs cover
};

static thread_local std::string g_err;

static wcns_status fail(wcns_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

static wcns_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(WCNS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);     \
    } while (0)

extern "C" {

const char* wcns_last_error(void) { return g_err.c_str(); }

const char* wcns_version(void) { return "wcns-gb300 0.1 (sm_103a)"; }

void wcns_default_params(wcns_scheme_params* p)
{
    if (!p) return;
    p->flux = WCNS_FLUX_ROE;
    p->diff = WCNS_DIFF_MD6;
    p->weights = WCNS_W_TENO;
    p->C = 1.0;
    p->eps = 1e-40;
    p->CT = 1e-5;
    p->q = 6;
    p->characteristic = 1;
    p->precision = WCNS_FP64;
    p->cfl = 0.5;
    p->entropy_fix = 0;
    p->eps_js = 1e-6;
}

// Per device: the sweep kernels' shared-memory attributes are set (atomic:
// two host threads creating their first handles at once may both set them,
// which is harmless, without a data race).
static std::atomic<bool> prepared_fp64[64], prepared_fp32[64];

wcns_status wcns_create(const wcns_grid* g, double gamma, const wcns_scheme_params* prm,
                        wcns_handle** out)
{
    g_err.clear();
    if (!g || !prm || !out) return fail(WCNS_ERR_INVALID, "wcns_create: null argument");
    *out = nullptr;
    if (g->ndim < 1 || g->ndim > 3) return fail(WCNS_ERR_INVALID, "ndim must be 1, 2 or 3");
    if (!(gamma > 1.0)) return fail(WCNS_ERR_INVALID, "gamma must exceed 1");
    if (const char* why = scheme_params_error(prm)) return fail(WCNS_ERR_INVALID, "%s", why);

    GridInfo G;
    char why[256];
    if (const char* msg = grid_error(g, gamma, G, why, sizeof why)) return fail(WCNS_ERR_INVALID, "%s", msg);
    wcns_handle* h = new wcns_handle();
    h->ndim = G.ndim;
    h->nv = G.nv;
    h->N = G.N;
    for (int a = 0; a < 3; ++a) {
        h->n[a] = G.n[a];
        h->periodic[a] = G.periodic[a];
        h->h[a] = G.h[a];
        h->inv_h[a] = G.inv_h[a];
    }
    h->G = G;
    // launch limits: the outer axis of the y and z sweeps is a grid z-dimension
    if ((h->ndim == 3 && (h->n[1] > 65535 || h->n[2] > 65535)) || h->N > (1LL << 40)) {
        delete h;
        return fail(WCNS_ERR_INVALID, "grid too large");
    }
    h->gamma = gamma;
    h->p = *prm;
    h->K = make_scheme_const(prm, gamma);
    h->sqrt_eps_f = (float)sqrt(prm->eps);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
    const bool fp32 = prm->precision == WCNS_FP32;
    const int slot = h->device & 63;
    if (!fp32 && !prepared_fp64[slot]) {
        e = prepare_sweeps_fp64();
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "prepare fp64 sweeps"); }
        prepared_fp64[slot] = true;
    }
    if (fp32 && !prepared_fp32[slot]) {
        e = prepare_sweeps_fp32();
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "prepare fp32 sweeps"); }
        prepared_fp32[slot] = true;
    }
    const size_t M = (size_t)h->nv * h->N;
    const size_t w = fp32 ? 4 : 8;
    h->nblk_cons = conserved_blocks(h->N);
    size_t bytes = M * w * 2 + (fp32 ? M * 8 : 0) + sizeof(StepScalars) + 64 +
                   sizeof(double) * (h->nblk_cons + 1) * h->nv;
    char* base = nullptr;
    e = cudaMalloc((void**)&base, bytes + 4096);
    if (e != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return fail(WCNS_ERR_NOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    size_t off = 0;
    auto carve = [&](size_t sz) { void* p = base + off; off = (off + sz + 255) & ~(size_t)255; return p; };
    h->L = carve(M * w);
    h->U1 = carve(M * w);
    if (fp32) h->D = (float*)carve(M * 4);
    if (fp32) h->S2 = (float*)carve(M * 4);
    h->sc = (StepScalars*)carve(sizeof(StepScalars));
    h->fallback = (long long*)carve(64);
    h->partials = (double*)carve(sizeof(double) * (h->nblk_cons + 1) * h->nv);
    h->bytes = bytes + 4096;
    e = cudaMemset(h->sc, 0, sizeof(StepScalars));
    if (e == cudaSuccess) e = cudaMemset(h->fallback, 0, 64);
    if (e != cudaSuccess) { cudaFree(base); delete h; return cuda_fail(e, "cudaMemset"); }
    *out = h;
    return WCNS_OK;
}

static void drop_graphs(wcns_handle* h)
{
    for (int k = 0; k < 2; ++k) {
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
        h->graph[k] = nullptr;
        h->graph_U[k] = nullptr;
    }
}

wcns_status wcns_destroy(wcns_handle* h)
{
    if (!h) return WCNS_OK;
    drop_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->Udev) cudaFree(h->Udev);
    cudaError_t e = cudaFree(h->L);
    delete h;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    return WCNS_OK;
}

size_t wcns_handle_bytes(const wcns_handle* h) { return h ? h->bytes : 0; }

size_t wcns_flags_bytes(const wcns_handle* h)
{
    if (!h) return 0;
    size_t s = 0;
    for (int d = 0; d < h->ndim; ++d) s += (size_t)h->nv * (h->N / h->n[d]) * (h->n[d] + 5);
    return s;
}

static size_t flags_offset(const wcns_handle* h, int d)
{
    size_t s = 0;
    for (int a = 0; a < d; ++a) s += (size_t)h->nv * (h->N / h->n[a]) * (h->n[a] + 5);
    return s;
}

static cudaError_t timed_event(wcns_handle* h, cudaStream_t s)
{
    if (h->ev_used == h->ev.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        h->ev.push_back(e);
    }
    return cudaEventRecord(h->ev[h->ev_used++], s);
}

// Evaluate L = RHS(U) with all directions; U and L in the handle precision.
// FP32 steps sweep the directions in reverse (z, y, x) and let the x sweep
// apply the SSP-RK3 stage combination (fuse_stage 1..3): U0 is the FP64
// state, D the FP32 increment, S_out the next stage's input.
static cudaError_t run_rhs(wcns_handle* h, const void* U, void* L, uint8_t* flags,
                           const double* dtp, cudaStream_t s, int fuse_stage = 0,
                           double* U0 = nullptr, float* S_out = nullptr)
{
    const bool fp32 = h->p.precision == WCNS_FP32;
    // FP32 sweeps after the first run as programmatic dependents of the
    // previous one (their staging and faces overlap its last wave); the time
    // of the whole RHS is then what the profile events can measure
    const bool pdl = fp32;
    cudaError_t e;
    if (h->profiling && (e = timed_event(h, s)) != cudaSuccess) return e;
    for (int k = 0; k < h->ndim; ++k) {
        const int d = fuse_stage ? h->ndim - 1 - k : k;
        SweepArgs a{};
        a.U = U;
        a.L = L;
        a.N = h->N;
        a.n[0] = h->n[0];
        a.n[1] = h->n[1];
        a.n[2] = h->n[2];
        a.periodic = h->periodic[d];
        a.inv_h = h->inv_h[d];
        a.inv_hf = (float)h->inv_h[d];
        a.accumulate = k > 0;
        a.flags = flags ? flags + flags_offset(h, d) : nullptr;
        a.fallback = h->fallback;
        a.dt = dtp;
        a.K = h->K;
        a.sqrt_eps_f = h->sqrt_eps_f;
        a.bc_lo = h->G.bc[d][0];
        a.bc_hi = h->G.bc[d][1];
        for (int sd = 0; sd < 2; ++sd)
            for (int v = 0; v < 5; ++v) a.bcs[sd][v] = h->G.bc_state[d][sd][v];
        if (h->G.has_gravity && k == h->ndim - 1) {   // the last sweep adds the source
            a.source = 1;
            for (int b = 0; b < 3; ++b) a.grav[b] = h->G.gravity[b];
        }
        if (fuse_stage && d == 0) {
            a.fuse_stage = fuse_stage;
            a.U0 = U0;
            a.D = h->D;
            a.S_out = S_out;
        }
        a.pdl = pdl && k > 0;
        e = fp32 ? launch_sweep_fp32(h->ndim, d, h->p.flux, h->tile_cfg[d], a, s)
                 : launch_sweep_fp64(h->ndim, d, h->p.flux, a, s);
        if (e != cudaSuccess) return e;
    }
    if (h->profiling) {
        if ((e = timed_event(h, s)) != cudaSuccess) return e;
        h->prof_sweeps += h->ndim;
    }
    return cudaSuccess;
}

wcns_status wcns_rhs(wcns_handle* h, const void* U, void* L, uint8_t* flags, void* stream)
{
    g_err.clear();
    if (!h || !U || !L) return fail(WCNS_ERR_INVALID, "wcns_rhs: null argument");
    CK(cudaGetLastError(), "pending CUDA error");
    CK(run_rhs(h, U, L, flags, nullptr, (cudaStream_t)stream),
       "wcns_rhs launch");
    return WCNS_OK;
}

// The three stages of one step after dt has been placed in h->sc.  In FP32
// mode the first stage reads float(U), converted here.
// converted: the FP32 first-stage input float(U) is already in place (the
// time-step pass wrote it).
static cudaError_t run_stages(wcns_handle* h, double* U, cudaStream_t s, bool converted = false)
{
    const long long M = (long long)h->nv * h->N;
    const double* dtp = &h->sc->dt;
    cudaError_t e;
    if (h->p.precision == WCNS_FP64) {
        double* U1 = (double*)h->U1;
        double* L = (double*)h->L;
        if ((e = run_rhs(h, U, L, nullptr, dtp, s)) != cudaSuccess) return e;
        if ((e = launch_rk_fp64(1, U, U1, L, M, h->sc, s)) != cudaSuccess) return e;
        if ((e = run_rhs(h, U1, L, nullptr, dtp, s)) != cudaSuccess) return e;
        if ((e = launch_rk_fp64(2, U, U1, L, M, h->sc, s)) != cudaSuccess) return e;
        if ((e = run_rhs(h, U1, L, nullptr, dtp, s)) != cudaSuccess) return e;
        return launch_rk_fp64(3, U, U1, L, M, h->sc, s);
    }
    // FP32: stage inputs A -> B -> A; the x sweep of stages 1 and 2 writes
    // the next one, stage 3 the FP64 state (the next step converts A anew)
    float* A = (float*)h->U1;
    float* B = h->S2;
    float* L = (float*)h->L;
    if (!converted && (e = launch_to_fp32(h->nv, U, A, h->N, h->sc, s)) != cudaSuccess) return e;
    if ((e = run_rhs(h, A, L, nullptr, dtp, s, 1, U, B)) != cudaSuccess) return e;
    if ((e = run_rhs(h, B, L, nullptr, dtp, s, 2, U, A)) != cudaSuccess) return e;
    return run_rhs(h, A, L, nullptr, dtp, s, 3, U, nullptr);
}

// The time step of a step: the fixed-order FP64 rule for the FP64 path (bit
// reproducible with the oracle), the FP32-evaluated speeds with an FP64 max
// for the FP32 path.
static cudaError_t step_cfl(wcns_handle* h, const double* U, int clip, cudaStream_t s)
{
    if (h->p.precision == WCNS_FP32)   // also writes float(U), the first stage's input
        return launch_cfl_fast(h->ndim, U, h->N, h->h, h->gamma, h->p.cfl, clip, h->sc, s, (float*)h->U1);
    return launch_cfl(h->ndim, U, h->N, h->h, h->gamma, h->p.cfl, clip, h->sc, s);
}

static cudaError_t reset_clock(wcns_handle* h, double t_end, cudaStream_t s)
{
    return launch_reset_clock(t_end, h->sc, s);
}

// FP32 handles: the reference state of the stage values, taken once from the
// first state the handle steps (stream-ordered, before any captured step).
static cudaError_t ensure_reference(wcns_handle* h, const void* U, cudaStream_t s)
{
    if (h->p.precision != WCNS_FP32 || h->ref_set) return cudaSuccess;
    const cudaError_t e = launch_reference(h->ndim, (const double*)U, h->N, h->gamma, h->sc, s);
    if (e == cudaSuccess) h->ref_set = true;
    return e;
}

// The graph of one CFL step on state U (kind 0: with the clock reset of
// wcns_step_rk3; kind 1: the clipped step of wcns_advance), captured on
// first use for this U.  Returns false (and leaves no error pending) when
// capture is not possible; the caller then launches directly.
static bool step_graph(wcns_handle* h, int kind, void* U)
{
    if (h->graph[kind] && h->graph_U[kind] == U) return true;
    if (h->graph[kind]) cudaGraphExecDestroy(h->graph[kind]);
    h->graph[kind] = nullptr;
    h->graph_U[kind] = nullptr;
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaError_t e = kind == 0 ? reset_clock(h, INFINITY, h->cap) : cudaSuccess;
    if (e == cudaSuccess) e = step_cfl(h, (const double*)U, kind, h->cap);
    if (e == cudaSuccess) e = run_stages(h, (double*)U, h->cap, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&h->graph[kind], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        h->graph[kind] = nullptr;
        cudaGetLastError();
        return false;
    }
    h->graph_U[kind] = U;
    return true;
}

wcns_status wcns_step_rk3(wcns_handle* h, void* U, double dt, double* dt_used, void* stream)
{
    g_err.clear();
    if (!h || !U) return fail(WCNS_ERR_INVALID, "wcns_step_rk3: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaGetLastError(), "pending CUDA error");
    // a synchronising step reports faces that fell back during it
    long long before = 0;
    if (dt_used) {
        CK(cudaMemcpyAsync(&before, h->fallback, sizeof before, cudaMemcpyDeviceToHost, s), "counter copy");
        CK(cudaStreamSynchronize(s), "sync");
    }
    CK(ensure_reference(h, U, s), "reference state");
    if (!(dt > 0.0) && !h->profiling && step_graph(h, 0, U)) {
        CK(cudaGraphLaunch(h->graph[0], s), "step graph");
    } else {
        CK(reset_clock(h, INFINITY, s), "reset clock");
        if (dt > 0.0) CK(launch_set_dt(dt, 0, h->sc, s), "set dt");
        else CK(step_cfl(h, (const double*)U, 0, s), "cfl");
        CK(run_stages(h, (double*)U, s, !(dt > 0.0)), "rk3 stages");
    }
    if (dt_used) {
        long long after = 0;
        CK(cudaMemcpyAsync(dt_used, &h->sc->dt, sizeof(double), cudaMemcpyDeviceToHost, s), "dt copy");
        CK(cudaMemcpyAsync(&after, h->fallback, sizeof after, cudaMemcpyDeviceToHost, s), "counter copy");
        CK(cudaStreamSynchronize(s), "sync");
        if (after > before)
            return fail(WCNS_ERR_NONPHYSICAL, "wcns_step_rk3: %lld faces had rho <= 0 or p <= 0 and used "
                        "first-order values", after - before);
    }
    return WCNS_OK;
}

wcns_status wcns_step_rk3_host(wcns_handle* h, double* U, int nsteps, void* stream)
{
    g_err.clear();
    if (!h || !U || nsteps < 0) return fail(WCNS_ERR_INVALID, "wcns_step_rk3_host: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaGetLastError(), "pending CUDA error");
    const size_t bytes = sizeof(double) * (size_t)h->nv * (size_t)h->N;
    if (!h->Udev) {
        if (cudaMalloc((void**)&h->Udev, bytes) != cudaSuccess) {
            h->Udev = nullptr;
            cudaGetLastError();
            return fail(WCNS_ERR_NOMEM, "wcns_step_rk3_host: cudaMalloc of %zu bytes failed", bytes);
        }
        h->bytes += bytes;
    }
    long long before = 0, after = 0;
    CK(cudaMemcpyAsync(&before, h->fallback, sizeof before, cudaMemcpyDeviceToHost, s), "counter copy");
    CK(cudaMemcpyAsync(h->Udev, U, bytes, cudaMemcpyHostToDevice, s), "state copy in");
    CK(ensure_reference(h, h->Udev, s), "reference state");
    for (int k = 0; k < nsteps; ++k) {
        if (!h->profiling && step_graph(h, 0, h->Udev)) {
            CK(cudaGraphLaunch(h->graph[0], s), "step graph");
        } else {
            CK(reset_clock(h, INFINITY, s), "reset clock");
            CK(step_cfl(h, h->Udev, 0, s), "cfl");
            CK(run_stages(h, h->Udev, s, true), "rk3 stages");
        }
    }
    CK(cudaMemcpyAsync(U, h->Udev, bytes, cudaMemcpyDeviceToHost, s), "state copy out");
    CK(cudaMemcpyAsync(&after, h->fallback, sizeof after, cudaMemcpyDeviceToHost, s), "counter copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (after > before)
        return fail(WCNS_ERR_NONPHYSICAL, "wcns_step_rk3_host: %lld faces had rho <= 0 or p <= 0 and used "
                    "first-order values", after - before);
    return WCNS_OK;
}

wcns_status wcns_advance(wcns_handle* h, void* U, double t_end, int max_steps, int check,
                         double* t_out, int* steps_out, void* stream)
{
    g_err.clear();
    if (!h || !U || !(t_end >= 0.0) || max_steps < 0)
        return fail(WCNS_ERR_INVALID, "wcns_advance: bad argument");
    if (check < 1) check = 1;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaGetLastError(), "pending CUDA error");
    CK(reset_clock(h, t_end, s), "reset clock");
    long long before = 0, after = 0;
    CK(ensure_reference(h, U, s), "reference state");
    CK(cudaMemcpyAsync(&before, h->fallback, sizeof before, cudaMemcpyDeviceToHost, s), "counter copy");
    CK(cudaStreamSynchronize(s), "sync");
    long long issued = 0;
    StepScalars cur{};
    while (issued < max_steps) {
        const long long left = max_steps - issued;
        const int batch = left < check ? (int)left : check;
        const bool use_graph = !h->profiling && step_graph(h, 1, U);
        for (int k = 0; k < batch; ++k) {
            if (use_graph) {
                CK(cudaGraphLaunch(h->graph[1], s), "step graph");
            } else {
                CK(step_cfl(h, (const double*)U, 1, s), "cfl");
                CK(run_stages(h, (double*)U, s, true), "rk3 stages");
            }
        }
        issued += batch;
        CK(cudaMemcpyAsync(&cur, h->sc, sizeof cur, cudaMemcpyDeviceToHost, s), "clock copy");
        CK(cudaMemcpyAsync(&after, h->fallback, sizeof after, cudaMemcpyDeviceToHost, s), "counter copy");
        CK(cudaStreamSynchronize(s), "sync");
        if (cur.t >= t_end) break;
    }
    if (t_out) *t_out = cur.t;
    if (steps_out) *steps_out = (int)cur.steps;
    if (after > before)
        return fail(WCNS_ERR_NONPHYSICAL, "wcns_advance: %lld faces had rho <= 0 or p <= 0 and used "
                    "first-order values", after - before);
    return WCNS_OK;
}

wcns_status wcns_conserved(wcns_handle* h, const void* U, double* out, void* stream)
{
    g_err.clear();
    if (!h || !U || !out) return fail(WCNS_ERR_INVALID, "wcns_conserved: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    double vol = 1.0;
    for (int a = 0; a < h->ndim; ++a) vol *= h->h[a];
    CK(launch_conserved(h->nv, (const double*)U, h->N, vol, h->partials, h->nblk_cons, s), "conserved");
    CK(cudaMemcpyAsync(out, h->partials + (size_t)h->nv * h->nblk_cons, sizeof(double) * h->nv,
                       cudaMemcpyDeviceToHost, s), "conserved copy");
    CK(cudaStreamSynchronize(s), "sync");
    return WCNS_OK;
}

wcns_status wcns_cfl_dt(wcns_handle* h, const void* U, double* dt, void* stream)
{
    g_err.clear();
    if (!h || !U || !dt) return fail(WCNS_ERR_INVALID, "wcns_cfl_dt: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(reset_clock(h, INFINITY, s), "reset clock");
    CK(launch_cfl(h->ndim, (const double*)U, h->N, h->h, h->gamma, h->p.cfl, 0, h->sc, s), "cfl");
    CK(cudaMemcpyAsync(dt, &h->sc->dt, sizeof(double), cudaMemcpyDeviceToHost, s), "dt copy");
    CK(cudaStreamSynchronize(s), "sync");
    return WCNS_OK;
}

wcns_status wcns_fallback_count(wcns_handle* h, long long* count, int reset, void* stream)
{
    g_err.clear();
    if (!h || !count) return fail(WCNS_ERR_INVALID, "wcns_fallback_count: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(count, h->fallback, sizeof(long long), cudaMemcpyDeviceToHost, s), "copy");
    if (reset) CK(cudaMemsetAsync(h->fallback, 0, sizeof(long long), s), "reset");
    CK(cudaStreamSynchronize(s), "sync");
    return WCNS_OK;
}

wcns_status wcns_profile(wcns_handle* h, int enable)
{
    g_err.clear();
    if (!h) return fail(WCNS_ERR_INVALID, "wcns_profile: null handle");
    h->profiling = enable != 0;
    return WCNS_OK;
}

wcns_status wcns_profile_read(wcns_handle* h, double* sweep_ms, long long* sweep_launches)
{
    g_err.clear();
    if (!h || !sweep_ms || !sweep_launches) return fail(WCNS_ERR_INVALID, "wcns_profile_read: null argument");
    double tot = 0.0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        CK(cudaEventSynchronize(h->ev[i + 1]), "event sync");
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]), "event time");
        tot += ms;
    }
    *sweep_ms = tot;
    *sweep_launches = h->prof_sweeps;
    h->ev_used = 0;
    h->prof_sweeps = 0;
    return WCNS_OK;
}

int wcns_launches_per_step(const wcns_handle* h, int cfl_step)
{
    if (!h) return 0;
    // clock reset + (CFL reduction and finalize | set dt) + stages: FP64 3 x
    // (sweeps + stage combine); FP32 3 x sweeps (the last sweep of each stage
    // applies the combination) plus a state conversion when dt is given (the
    // CFL pass converts the state otherwise)
    const int stages =
        h->p.precision == WCNS_FP32 ? (cfl_step ? 0 : 1) + 3 * h->ndim : 3 * (h->ndim + 1);
    return 1 + (cfl_step ? 2 : 1) + stages;
}

}  // extern "C"

namespace wcns {
// Message for wcns_last_error() from entry points defined in other files.
void set_last_error(const char* msg)
{
    if (msg) g_err = msg;
    else g_err.clear();
}
}  // namespace wcns

extern "C" wcns_status wcns_autotune(wcns_handle* h, const void* U, int* chosen, void* stream)
{
    using namespace wcns;
    set_last_error(nullptr);
    if (!h || !U) return fail(WCNS_ERR_INVALID, "wcns_autotune: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    drop_graphs(h);   // captured steps hold the old tile shapes
    // the comparison weights have one tile configuration; TENO has three
    if (h->p.precision == WCNS_FP32 && h->ndim >= 2 && h->p.weights == WCNS_W_TENO) {
        float* A = (float*)h->U1;
        CK(launch_to_fp32(h->nv, (const double*)U, A, h->N, nullptr, s), "autotune state");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        for (int d = 0; d < h->ndim; ++d) {
            float best = 1e30f;
            int pick = 0;
            for (int cfg = 0; cfg < 3; ++cfg) {
                SweepArgs a{};
                a.U = A;
                a.L = h->L;
                a.N = h->N;
                for (int k = 0; k < 3; ++k) a.n[k] = h->n[k];
                a.periodic = h->periodic[d];
                a.inv_h = h->inv_h[d];
                a.inv_hf = (float)h->inv_h[d];
                a.accumulate = d != h->ndim - 1;   // as in a step: the first sweep writes L
                a.fallback = h->fallback;
                a.K = h->K;
                a.sqrt_eps_f = h->sqrt_eps_f;
                a.bc_lo = h->G.bc[d][0];
                a.bc_hi = h->G.bc[d][1];
                for (int sd = 0; sd < 2; ++sd)
                    for (int v = 0; v < 5; ++v) a.bcs[sd][v] = h->G.bc_state[d][sd][v];
                CK(launch_sweep_fp32(h->ndim, d, h->p.flux, cfg, a, s), "autotune warm-up");
                CK(cudaEventRecord(e0, s), "event");
                for (int r = 0; r < 3; ++r) CK(launch_sweep_fp32(h->ndim, d, h->p.flux, cfg, a, s), "autotune");
                CK(cudaEventRecord(e1, s), "event");
                CK(cudaEventSynchronize(e1), "event");
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1), "event");
                if (ms < best) { best = ms; pick = cfg; }
            }
            h->tile_cfg[d] = pick;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CK(cudaMemsetAsync(h->fallback, 0, sizeof(long long), s), "counter reset");
    }
    if (chosen)
        for (int d = 0; d < 3; ++d) chosen[d] = d < h->ndim ? h->tile_cfg[d] : 0;
    return WCNS_OK;
}

extern "C" wcns_status wcns_tile_config(wcns_handle* h, const int* set, int* get)
{
    using namespace wcns;
    set_last_error(nullptr);
    if (!h) return fail(WCNS_ERR_INVALID, "wcns_tile_config: null handle");
    if (set) {
        for (int d = 0; d < h->ndim; ++d)
            if (set[d] < 0 || set[d] > 2) return fail(WCNS_ERR_INVALID, "tile configuration must be 0, 1 or 2");
        if (h->p.precision == WCNS_FP32 && h->ndim >= 2)
            for (int d = 0; d < h->ndim; ++d) h->tile_cfg[d] = set[d];
        drop_graphs(h);   // captured steps hold the old tile shapes
    }
    if (get)
        for (int d = 0; d < 3; ++d) get[d] = d < h->ndim ? h->tile_cfg[d] : 0;
    return WCNS_OK;
}
