// wcns_serve.cu -- the serving loop: solve requests arrive at any time, are
// admitted into resident batches as device memory and slots allow, advance
// together with everything already running (continuous batching: requests
// join and leave at RK-step boundaries), and are returned as they finish.
//
// One worker thread per server owns the GPU work: each tick it (1) admits
// queued requests in arrival order while the HBM budget, a slot and a free
// arena range allow, (2) advances every non-empty batch by a fixed number of
// graph-replayed steps, (3) copies finished states to the host, queues their
// results and frees their slots.  Batches are created per scheme class
// (dimension, precision, flux, constants, gamma, CFL) with arenas sized from
// the budget.  The C ABI calls (submit, poll) only touch host queues.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/wcns.h"
#include "wcns_internal.h"

using namespace wcns;

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    uint64_t ticket;
    wcns_request req;          // U0 points into `state`
    std::vector<double> state;
    double t_submit;
};

struct Running {
    uint64_t ticket;
    uint64_t tag;
    int ndim, n[3], precision;
    double t_submit, t_admit;
    long long nodes;
};

// Requests share a batch when every scheme constant and gamma agree.
using ClassKey = std::tuple<int, int, int, double, double, double, double, int, double, int, double, int>;

struct ClassBatch {
    wcns_batch* b = nullptr;
    size_t bytes = 0;
    std::map<int, Running> running;   // slot -> request
    // GPU time of one RK3 step of the class (smoothed), from events around
    // its steps in the last tick
    double ms_per_step = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int stepped = 0;                  // steps issued in the current tick
};

constexpr int kMaxTickScale = 64;     // a cheap class takes at most 64x the base steps

ClassKey key_of(const wcns_request& r)
{
    const wcns_scheme_params& p = r.params;
    return ClassKey(r.grid.ndim, p.precision, p.flux, p.C, p.eps, p.CT, p.cfl, p.q, r.gamma, p.weights,
                    p.weights == WCNS_W_JS ? p.eps_js : 0.0, p.diff);
}

size_t bytes_per_node(int ndim, int precision)
{
    const size_t nv = ndim + 2;
    return nv * (8 + (precision == WCNS_FP32 ? 4 + 4 + 4 + 4 : 8 + 8));
}

}  // namespace

struct wcns_server {
    wcns_server_config cfg{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> pending;
    std::deque<wcns_result> done;
    bool stop = false;
    uint64_t next_ticket = 1;
    // worker-owned
    std::map<ClassKey, ClassBatch> classes;
    size_t bytes_in_use = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::thread worker;
    wcns_status worker_status = WCNS_OK;
    // statistics
    long long admitted = 0, completed = 0, ticks = 0, steps = 0;
    int max_queue = 0, max_running = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

wcns_status sfail(wcns_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

void finish(wcns_server* sv, wcns_result r)
{
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->done.push_back(r);
    sv->cv_done.notify_all();
}

wcns_result failed_result(const Pending& p, wcns_status st, double now)
{
    wcns_result r;
    memset(&r, 0, sizeof r);
    r.ticket = p.ticket;
    r.tag = p.req.tag;
    r.status = st;
    r.ndim = p.req.grid.ndim;
    for (int a = 0; a < 3; ++a) r.n[a] = p.req.grid.n[a];
    r.precision = p.req.params.precision;
    r.t_submit = p.t_submit;
    r.t_admit = now;
    r.t_done = now;
    return r;
}

long long nodes_of(const wcns_grid& g)
{
    long long N = 1;
    for (int a = 0; a < g.ndim; ++a) N *= g.n[a];
    return N;
}

// Admit what fits; returns the number admitted.
int admit(wcns_server* sv)
{
    std::deque<Pending> batch;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        batch.swap(sv->pending);
    }
    int admitted = 0;
    std::deque<Pending> keep;
    for (auto& p : batch) {
        const ClassKey key = key_of(p.req);
        const long long N = nodes_of(p.req.grid);
        auto it = sv->classes.find(key);
        if (it == sv->classes.end()) {
            // a new class: its arena gets an equal share of the budget not yet
            // reserved, at most max_nodes_per_class nodes, at least this request
            const size_t bpn = bytes_per_node(p.req.grid.ndim, p.req.params.precision);
            const size_t free_bytes = sv->cfg.hbm_budget_bytes > sv->bytes_in_use
                                          ? sv->cfg.hbm_budget_bytes - sv->bytes_in_use : 0;
            long long cap = (long long)(free_bytes / 2 / bpn);
            if (sv->cfg.max_nodes_per_class > 0 && cap > sv->cfg.max_nodes_per_class)
                cap = sv->cfg.max_nodes_per_class;
            if (cap < N) cap = (long long)(free_bytes / bpn);
            if (cap < N) {
                if (sv->classes.empty() || (long long)(sv->cfg.hbm_budget_bytes / bpn) < N) {
                    finish(sv, failed_result(p, WCNS_ERR_NOMEM, sv->now()));   // can never fit
                } else {
                    keep.push_back(std::move(p));
                }
                continue;
            }
            ClassBatch cb;
            wcns_scheme_params prm = p.req.params;
            wcns_status st = wcns_batch_create(p.req.grid.ndim, p.req.gamma, &prm, cap,
                                               sv->cfg.max_instances_per_class, &cb.b);
            if (st != WCNS_OK) {
                finish(sv, failed_result(p, st, sv->now()));
                continue;
            }
            cb.bytes = wcns_batch_bytes(cb.b);
            sv->bytes_in_use += cb.bytes;
            it = sv->classes.emplace(key, cb).first;
        }
        ClassBatch& cb = it->second;
        if (N > batch_capacity_nodes(cb.b)) {
            finish(sv, failed_result(p, WCNS_ERR_NOMEM, sv->now()));   // larger than the class arena
            continue;
        }
        if (!batch_fits(cb.b, N)) {
            keep.push_back(std::move(p));
            continue;
        }
        int slot = -1;
        wcns_status st = wcns_batch_add(cb.b, &p.req.grid, p.state.data(), 0, p.req.t_end, &slot, sv->stream);
        if (st != WCNS_OK) {
            finish(sv, failed_result(p, st, sv->now()));
            continue;
        }
        Running r;
        r.ticket = p.ticket;
        r.tag = p.req.tag;
        r.ndim = p.req.grid.ndim;
        for (int a = 0; a < 3; ++a) r.n[a] = p.req.grid.n[a];
        r.precision = p.req.params.precision;
        r.t_submit = p.t_submit;
        r.t_admit = sv->now();
        r.nodes = N;
        cb.running[slot] = r;
        ++admitted;
        ++sv->admitted;
    }
    if (!keep.empty()) {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (auto it = keep.rbegin(); it != keep.rend(); ++it) sv->pending.push_front(std::move(*it));
    }
    return admitted;
}

void retire(wcns_server* sv)
{
    std::vector<int> fin;
    for (auto& kv : sv->classes) {
        ClassBatch& cb = kv.second;
        if (cb.running.empty()) continue;
        if (batch_finished_slots(cb.b, fin, sv->stream) != cudaSuccess) {
            sv->worker_status = WCNS_ERR_CUDA;
            return;
        }
        for (int slot : fin) {
            auto rit = cb.running.find(slot);
            if (rit == cb.running.end()) continue;
            const Running& ru = rit->second;
            wcns_result r;
            memset(&r, 0, sizeof r);
            r.ticket = ru.ticket;
            r.tag = ru.tag;
            r.ndim = ru.ndim;
            for (int a = 0; a < 3; ++a) r.n[a] = ru.n[a];
            r.precision = ru.precision;
            r.U = (double*)malloc(sizeof(double) * (ru.ndim + 2) * ru.nodes);
            int steps = 0;
            double t = 0.0;
            wcns_status st = r.U ? wcns_batch_read(cb.b, slot, r.U, 0, &t, &steps, sv->stream) : WCNS_ERR_NOMEM;
            r.status = st;
            r.t = t;
            r.steps = steps;
            r.t_submit = ru.t_submit;
            r.t_admit = ru.t_admit;
            r.t_done = sv->now();
            wcns_batch_remove(cb.b, slot);
            cb.running.erase(rit);
            ++sv->completed;
            finish(sv, r);
        }
    }
}

void worker_main(wcns_server* sv)
{
    cudaSetDevice(sv->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            bool busy = false;
            for (auto& kv : sv->classes) busy = busy || !kv.second.running.empty();
            if (!busy)
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                                     [&] { return sv->stop || !sv->pending.empty(); });
            if (sv->stop) break;
            sv->max_queue = std::max<int>(sv->max_queue, (int)sv->pending.size());
        }
        admit(sv);
        // Time-fair ticks: the most expensive class advances steps_per_tick
        // steps, a cheaper class as many more as fit in the same GPU time (at
        // most kMaxTickScale times as many), so cheap requests are not held
        // to the step rate of expensive ones.  Results do not depend on how
        // the steps are grouped.
        double slowest = 0.0;
        for (auto& kv : sv->classes)
            if (!kv.second.running.empty()) slowest = std::max(slowest, kv.second.ms_per_step);
        int running = 0;
        for (auto& kv : sv->classes) {
            ClassBatch& cb = kv.second;
            cb.stepped = 0;
            if (cb.running.empty()) continue;
            running += (int)cb.running.size();
            const int base = sv->cfg.steps_per_tick;
            int n = base;
            if (cb.ms_per_step > 0.0 && slowest > 0.0) {
                const double want = base * slowest / cb.ms_per_step;
                n = (int)std::min<double>(std::max<double>(want, base), (double)base * kMaxTickScale);
            }
            if (!cb.ev0 && (cudaEventCreate(&cb.ev0) != cudaSuccess || cudaEventCreate(&cb.ev1) != cudaSuccess))
                sv->worker_status = WCNS_ERR_CUDA;
            if (cb.ev0) cudaEventRecord(cb.ev0, sv->stream);
            if (wcns_batch_step(cb.b, n, nullptr, sv->stream) != WCNS_OK) sv->worker_status = WCNS_ERR_CUDA;
            if (cb.ev1) cudaEventRecord(cb.ev1, sv->stream);
            cb.stepped = n;
            sv->steps += n;
        }
        sv->max_running = std::max(sv->max_running, running);
        if (running) {
            ++sv->ticks;
            retire(sv);
            for (auto& kv : sv->classes) {
                ClassBatch& cb = kv.second;
                float ms = 0.f;
                if (cb.stepped > 0 && cb.ev1 && cudaEventSynchronize(cb.ev1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, cb.ev0, cb.ev1) == cudaSuccess) {
                    const double per = ms / cb.stepped;
                    cb.ms_per_step = cb.ms_per_step > 0.0 ? 0.5 * (cb.ms_per_step + per) : per;
                }
            }
        }
        if (sv->worker_status != WCNS_OK) break;
    }
    // fail what is still queued or running
    std::deque<Pending> left;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        left.swap(sv->pending);
    }
    for (auto& p : left) finish(sv, failed_result(p, WCNS_ERR_BUSY, sv->now()));
}

}  // namespace

extern "C" {

void wcns_server_default_config(wcns_server_config* c)
{
    if (!c) return;
    c->hbm_budget_bytes = (size_t)8 << 30;
    c->max_instances_per_class = 256;
    c->max_nodes_per_class = 0;
    c->steps_per_tick = 16;
}

wcns_status wcns_server_create(const wcns_server_config* cfg, wcns_server** out)
{
    set_last_error(nullptr);
    if (!cfg || !out) return sfail(WCNS_ERR_INVALID, "wcns_server_create: null argument");
    if (cfg->hbm_budget_bytes == 0 || cfg->max_instances_per_class < 1 || cfg->steps_per_tick < 1)
        return sfail(WCNS_ERR_INVALID, "wcns_server_create: bad configuration");
    wcns_server* sv = new wcns_server();
    sv->cfg = *cfg;
    sv->t0 = Clock::now();
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete sv;
        return sfail(WCNS_ERR_CUDA, "wcns_server_create: %s", cudaGetErrorString(e));
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return WCNS_OK;
}

wcns_status wcns_batch_submit(wcns_server* sv, const wcns_request* req, uint64_t* ticket)
{
    set_last_error(nullptr);
    if (!sv || !req || !req->U0) return sfail(WCNS_ERR_INVALID, "wcns_batch_submit: null argument");
    const wcns_grid& g = req->grid;
    if (g.ndim < 1 || g.ndim > 3) return sfail(WCNS_ERR_INVALID, "ndim must be 1, 2 or 3");
    for (int a = 0; a < g.ndim; ++a)
        if (g.n[a] < 1) return sfail(WCNS_ERR_INVALID, "bad node count");
    if (!(req->t_end >= 0.0)) return sfail(WCNS_ERR_INVALID, "t_end must be >= 0");
    if (!(req->gamma > 1.0)) return sfail(WCNS_ERR_INVALID, "gamma must exceed 1");
    if (const char* why = scheme_params_error(&req->params)) return sfail(WCNS_ERR_INVALID, "%s", why);
    {
        GridInfo G;
        char why[256];
        if (const char* msg = grid_error(&g, req->gamma, G, why, sizeof why))
            return sfail(WCNS_ERR_INVALID, "%s", msg);
    }
    Pending p;
    p.req = *req;
    const long long N = nodes_of(g);
    p.state.assign(req->U0, req->U0 + (size_t)(g.ndim + 2) * N);
    p.req.U0 = p.state.data();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return sfail(WCNS_ERR_BUSY, "server is shutting down");
        p.ticket = sv->next_ticket++;
        p.t_submit = sv->now();
        if (ticket) *ticket = p.ticket;
        sv->pending.push_back(std::move(p));
    }
    sv->cv_work.notify_all();
    return WCNS_OK;
}

wcns_status wcns_serve_poll(wcns_server* sv, wcns_result* out, int max, int* n_out, int timeout_us)
{
    set_last_error(nullptr);
    if (!sv || !out || !n_out || max < 1) return sfail(WCNS_ERR_INVALID, "wcns_serve_poll: bad argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done.empty() && timeout_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !sv->done.empty(); });
    int n = 0;
    while (n < max && !sv->done.empty()) {
        out[n++] = sv->done.front();
        sv->done.pop_front();
    }
    *n_out = n;
    if (n == 0 && sv->worker_status != WCNS_OK) return sfail(sv->worker_status, "serving loop stopped");
    return n == 0 && timeout_us > 0 ? WCNS_ERR_TIMEOUT : WCNS_OK;
}

void wcns_result_free(wcns_result* r)
{
    if (r && r->U) {
        free(r->U);
        r->U = nullptr;
    }
}

wcns_status wcns_server_stats(wcns_server* sv, wcns_server_stats_t* st)
{
    if (!sv || !st) return sfail(WCNS_ERR_INVALID, "wcns_server_stats: null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    st->queued = (int)sv->pending.size();
    st->completed = sv->completed;
    st->admitted = sv->admitted;
    st->ticks = sv->ticks;
    st->steps = sv->steps;
    st->max_queue = sv->max_queue;
    st->max_running = sv->max_running;
    st->bytes_reserved = sv->bytes_in_use;
    return WCNS_OK;
}

wcns_status wcns_server_destroy(wcns_server* sv)
{
    if (!sv) return WCNS_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& kv : sv->classes) {
        wcns_batch_destroy(kv.second.b);
        if (kv.second.ev0) cudaEventDestroy(kv.second.ev0);
        if (kv.second.ev1) cudaEventDestroy(kv.second.ev1);
    }
    for (auto& r : sv->done) wcns_result_free(&r);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    delete sv;
    return WCNS_OK;
}

}  // extern "C"
