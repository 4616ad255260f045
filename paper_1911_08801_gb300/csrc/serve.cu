// Serving loop: as-S_N solve requests are admitted by device-memory footprint, their flux state
// stays on the device, and the steps of every admitted solve run together as one batch
// (continuous batching: requests that arrive while others are on the device join at the next
// chunk boundary, finished solves leave and free their memory).
//
// One host thread owns the device work.  Per iteration it (1) admits queued requests in arrival
// order while the slot limit and the footprint budget allow, setting each up (quadrature, cross
// sections, kernel matrix K built in FP64 on the device, initial state) on a set-up stream;
// (2) advances every admitted solve by up to `chunk` explicit steps with one persistent launch
// per step (the batch path: Sec. 3.2 step, members at their own step sizes and counts);
// (3) waits for the chunk, and for each solve that reached its step count copies the scalar flux
// (Sec. 2.2) to the host result, records the latency and frees the solve.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "problem.h"
#include "trace.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    int64_t id = 0;
    assn_request spec{};
    std::vector<double> sa, ss, q;
    std::vector<float> psi0;
    size_t footprint = 0;
    Clock::time_point t_submit;
};

struct Active {
    Request req;
    assn_problem* p = nullptr;
    bool in_batch = false;
    int remaining = 0;
    Clock::time_point t_admit;
};

struct Result {
    int status = ASSN_OK;
    std::string error;
    std::vector<double> phi;
    double latency_s = 0, queue_s = 0;
    bool done = false;
};

}  // namespace

struct assn_server {
    int dev = 0;
    int precision = ASSN_BF16;
    size_t budget = 0;
    int max_active = 0;
    int chunk = 8;
    int use_graph = 1;
    cudaStream_t setup = nullptr;
    assn_batch* batch = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::map<int64_t, Result> results;
    std::set<int64_t> cancel;            // admitted requests to retire at the next chunk boundary
    bool stopping = false;
    int64_t next_id = 1;

    // loop-owned
    std::vector<Active> active;
    size_t in_use = 0;

    // statistics (under mu)
    int64_t submitted = 0, completed = 0, failed = 0, max_active_seen = 0, launches = 0;
    size_t peak_bytes = 0;
    double busy_s = 0, updates = 0;
    std::vector<double> latencies;
    Clock::time_point t_first_submit, t_last_done;
    bool any = false;
    int64_t n_active_pub = 0, n_queued_pub = 0;

    std::thread loop;
};

namespace {

thread_local std::string g_server_error;

// Server calls come from several host threads: messages are kept per calling thread.
int sfail(assn_server*, int status, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int sfail(assn_server*, int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_server_error = buf;
    return status;
}

int padq(int Q) { return (Q + 63) / 64 * 64; }

// Set up one admitted request: a problem on the set-up stream with its quadrature, cross
// sections, K and initial state.  Returns a status; on error *out is NULL and msg is set.
int setup_problem(assn_server* s, const Request& r, assn_problem** out, std::string& msg) {
    *out = nullptr;
    const assn_request& q = r.spec;
    assn_problem* p = nullptr;
    int st = assn_create(&p, q.nx, q.ny, q.x0, q.x1, q.y0, q.y1, s->precision, s->setup);
    if (st) {
        msg = assn_last_error(nullptr);
        return st;
    }
    st = assn_set_product_quadrature(p, q.n_polar, q.n_azim);
    if (!st) st = assn_set_cross_sections(p, r.sa.data(), r.ss.data(), r.q.data());
    if (!st) st = assn_set_artificial_scattering(p, q.sigma_as, q.eps, q.kernel_kind, q.normalisation);
    if (!st) {
        if (q.init_kind == ASSN_INIT_LINE_SOURCE) st = assn_init_line_source(p, q.delta, q.floor_value);
        else if (q.init_kind == ASSN_INIT_STATE) st = assn_set_state_f32(p, r.psi0.data());
        // ASSN_INIT_ZERO: the state is zero after the quadrature is set
    }
    if (st) {
        msg = assn_last_error(p);
        assn_destroy(p);
        return st;
    }
    *out = p;
    return ASSN_OK;
}

void finish(assn_server* s, Active& a, int status, const std::string& msg) {
    Result res;
    res.status = status;
    res.error = msg;
    if (status == ASSN_OK) {
        res.phi.resize((size_t)a.req.spec.nx * a.req.spec.ny);
        int st = assn_scalar_flux(a.p, res.phi.data());
        if (st) {
            res.status = st;
            res.error = assn_last_error(a.p);
            res.phi.clear();
        }
    }
    const auto now = Clock::now();
    res.latency_s = std::chrono::duration<double>(now - a.req.t_submit).count();
    res.queue_s = std::chrono::duration<double>(a.t_admit - a.req.t_submit).count();
    res.done = true;
    if (a.p) {
        if (a.in_batch) assn_batch_remove(s->batch, a.p);
        a.in_batch = false;
        assn_destroy(a.p);
        a.p = nullptr;
    }
    s->in_use -= a.req.footprint;
    std::lock_guard<std::mutex> g(s->mu);
    if (res.status == ASSN_OK) {
        ++s->completed;
        s->latencies.push_back(res.latency_s);
        s->updates += (double)a.req.spec.nx * a.req.spec.ny * a.req.spec.n_polar * a.req.spec.n_azim * a.req.spec.nsteps;
    } else {
        ++s->failed;
    }
    s->t_last_done = now;
    s->cancel.erase(a.req.id);
    s->results[a.req.id] = std::move(res);
    s->cv_done.notify_all();
}

void loop_main(assn_server* s) {
    cudaSetDevice(s->dev);
    while (true) {
        // ---- admission (arrival order; stop at the first request that does not fit)
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->active.empty())
                s->cv_work.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
            if (s->stopping && s->queue.empty() && s->active.empty()) break;
            size_t used = s->in_use;
            int slots = s->max_active - (int)s->active.size();
            while (!s->queue.empty() && slots > 0 && used + s->queue.front().footprint <= s->budget) {
                used += s->queue.front().footprint;
                admit.push_back(std::move(s->queue.front()));
                s->queue.pop_front();
                --slots;
            }
        }
        assn::TraceRange admit_range("serving admission");
        for (Request& r : admit) {
            Active a;
            a.t_admit = Clock::now();
            a.req = std::move(r);
            s->in_use += a.req.footprint;
            std::string msg;
            int st = setup_problem(s, a.req, &a.p, msg);
            if (!st && a.req.spec.nsteps > 0) {
                st = assn_batch_add(s->batch, a.p, 0, a.req.spec.dt);
                if (st) msg = assn_batch_last_error(s->batch);
                else a.in_batch = true;
            }
            if (st) {
                finish(s, a, st, msg);
                continue;
            }
            a.remaining = a.req.spec.nsteps;
            if (a.remaining == 0) {
                finish(s, a, ASSN_OK, "");
                continue;
            }
            s->active.push_back(std::move(a));
        }
        {   // cancelled while admitted: retire before the next chunk
            std::vector<int64_t> drop;
            {
                std::lock_guard<std::mutex> g(s->mu);
                for (const Active& a : s->active)
                    if (s->cancel.count(a.req.id)) drop.push_back(a.req.id);
            }
            if (!drop.empty()) {
                std::vector<Active> keep;
                for (Active& a : s->active) {
                    if (std::find(drop.begin(), drop.end(), a.req.id) != drop.end())
                        finish(s, a, ASSN_ERR_CANCELLED, "cancelled");
                    else
                        keep.push_back(std::move(a));
                }
                s->active.swap(keep);
            }
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->peak_bytes = std::max(s->peak_bytes, s->in_use);
            s->max_active_seen = std::max<int64_t>(s->max_active_seen, (int64_t)s->active.size());
            s->n_active_pub = (int64_t)s->active.size();
            s->n_queued_pub = (int64_t)s->queue.size();
        }
        if (s->active.empty()) continue;

        // ---- one chunk of steps for every active solve
        assn::TraceRange chunk_range("serving chunk");
        const auto t0 = Clock::now();
        int st = ASSN_OK;
        for (Active& a : s->active) {
            st = assn_batch_set_steps(s->batch, a.p, std::min(a.remaining, s->chunk), a.req.spec.dt);
            if (st) break;
        }
        int nmax = 0;
        for (Active& a : s->active) nmax = std::max(nmax, std::min(a.remaining, s->chunk));
        if (!st) st = assn_batch_run(s->batch, s->use_graph);
        if (!st) st = assn_batch_sync(s->batch);
        const double dt_busy = std::chrono::duration<double>(Clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->busy_s += dt_busy;
            if (!st) s->launches += nmax;
        }
        if (st) {   // a failed chunk fails every active solve (their states are unknown)
            const std::string msg = assn_batch_last_error(s->batch);
            for (Active& a : s->active) finish(s, a, st, msg);
            s->active.clear();
            continue;
        }
        std::vector<Active> keep;
        for (Active& a : s->active) {
            a.remaining -= std::min(a.remaining, s->chunk);
            if (a.remaining == 0) finish(s, a, ASSN_OK, "");
            else keep.push_back(std::move(a));
        }
        s->active.swap(keep);
    }
}

}  // namespace

extern "C" {

int assn_footprint_bytes(int nx, int ny, int Q, int precision, size_t* bytes) {
    if (!bytes || nx < 1 || ny < 1 || Q < 1 || Q > ASSN_MAX_Q || precision < ASSN_FP64 || precision > ASSN_BF16X2)
        return ASSN_ERR_ARG;
    const size_t ncell = (size_t)nx * ny, Qp = (size_t)padq(Q), Mp = (Qp + 127) / 128 * 128;
    const size_t elem = precision == ASSN_FP64 ? 8 : 4;
    size_t b = 2 * ncell * Qp * elem + 4 * 4096; // ping-pong state and its guard regions
    b += ncell * 32 + ncell * 8;                 // cell constants, FP64 staging for the scalar flux
    b += (size_t)Q * Q * 8 + Qp * 64;            // FP64 K, per-ordinate constants
    if (precision == ASSN_FP64) b += Qp * Qp * 8;
    else if (precision == ASSN_FP32) b += Qp * Qp * 4;
    else b += Mp * Qp * 2 * (precision == ASSN_BF16 ? 1 : 2);   // BF16 G; hi + lo (BF16X3, BF16X2); TF32 words
    b += (size_t)1 << 20;                        // small buffers, descriptors, allocation rounding
    *bytes = (b + ((size_t)2 << 20) - 1) / ((size_t)2 << 20) * ((size_t)2 << 20);
    return ASSN_OK;
}

int assn_server_create(assn_server** out, int precision, size_t hbm_budget_bytes, int max_active, int chunk_steps,
                       int use_graph) {
    if (!out) return sfail(nullptr, ASSN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (precision != ASSN_BF16 && precision != ASSN_BF16X3)
        return sfail(nullptr, ASSN_ERR_UNSUPPORTED, "the server steps the tensor-core precisions (BF16, BF16X3)");
    if (max_active < 1 || max_active > 1024) return sfail(nullptr, ASSN_ERR_ARG, "max_active must be 1..1024");
    if (chunk_steps < 1) return sfail(nullptr, ASSN_ERR_ARG, "chunk_steps must be >= 1");
    assn_server* s = new (std::nothrow) assn_server();
    if (!s) return sfail(nullptr, ASSN_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&s->dev);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->setup, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return sfail(nullptr, ASSN_ERR_CUDA, "server create: %s", cudaGetErrorString(e));
    }
    int st = assn_batch_create(&s->batch, nullptr);
    if (st) {
        cudaStreamDestroy(s->setup);
        delete s;
        return sfail(nullptr, st, "server batch: %s", assn_batch_last_error(nullptr));
    }
    s->precision = precision;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.85 * (double)free_b);
    s->max_active = max_active;
    s->chunk = chunk_steps;
    s->use_graph = use_graph;
    s->loop = std::thread(loop_main, s);
    *out = s;
    return ASSN_OK;
}

int assn_server_submit(assn_server* s, const assn_request* r, int64_t* id) {
    if (!s || !r || !id) return sfail(s, ASSN_ERR_ARG, "NULL argument");
    *id = 0;
    const int Q = r->n_polar * r->n_azim;
    if (r->nx < 1 || r->ny < 1 || r->n_polar < 1 || r->n_azim < 1 || Q > ASSN_MAX_Q || r->nsteps < 0 ||
        !(r->dt > 0) || !r->sigma_a || !r->sigma_s || !r->q)
        return sfail(s, ASSN_ERR_ARG, "invalid request");
    if (r->init_kind != ASSN_INIT_LINE_SOURCE && r->init_kind != ASSN_INIT_ZERO && r->init_kind != ASSN_INIT_STATE)
        return sfail(s, ASSN_ERR_ARG, "unknown init_kind %d", r->init_kind);
    if (r->init_kind == ASSN_INIT_STATE && !r->psi0) return sfail(s, ASSN_ERR_ARG, "psi0 is NULL");
    Request req;
    req.spec = *r;
    const size_t ncell = (size_t)r->nx * r->ny;
    req.sa.assign(r->sigma_a, r->sigma_a + ncell);
    req.ss.assign(r->sigma_s, r->sigma_s + ncell);
    req.q.assign(r->q, r->q + ncell);
    if (r->init_kind == ASSN_INIT_STATE) req.psi0.assign(r->psi0, r->psi0 + ncell * Q);
    req.spec.sigma_a = req.spec.sigma_s = req.spec.q = nullptr;
    req.spec.psi0 = nullptr;
    assn_footprint_bytes(r->nx, r->ny, Q, s->precision, &req.footprint);
    if (req.footprint > s->budget)
        return sfail(s, ASSN_ERR_OOM, "request needs %zu bytes, more than the whole budget %zu", req.footprint,
                     s->budget);
    req.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stopping) return sfail(s, ASSN_ERR_STATE, "server is stopping");
        req.id = s->next_id++;
        *id = req.id;
        if (!s->any) {
            s->t_first_submit = req.t_submit;
            s->any = true;
        }
        ++s->submitted;
        s->results[req.id] = Result{};
        s->queue.push_back(std::move(req));
    }
    s->cv_work.notify_one();
    return ASSN_OK;
}

int assn_server_wait(assn_server* s, int64_t id, double timeout_s, double* phi_host, double* latency_s,
                     double* queue_s) {
    if (!s) return sfail(s, ASSN_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(id);
    if (it == s->results.end()) return sfail(s, ASSN_ERR_ARG, "unknown request id %lld", (long long)id);
    auto ready = [&] { return s->results[id].done; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return sfail(s, ASSN_ERR_TIMEOUT, "request %lld not finished", (long long)id);
    }
    Result res = std::move(s->results[id]);
    s->results.erase(id);
    lk.unlock();
    if (latency_s) *latency_s = res.latency_s;
    if (queue_s) *queue_s = res.queue_s;
    if (res.status != ASSN_OK) return sfail(s, res.status, "request %lld: %s", (long long)id, res.error.c_str());
    if (phi_host) std::copy(res.phi.begin(), res.phi.end(), phi_host);
    return ASSN_OK;
}

int assn_server_cancel(assn_server* s, int64_t id) {
    if (!s) return sfail(s, ASSN_ERR_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->results.find(id);
        if (it == s->results.end()) return sfail(s, ASSN_ERR_ARG, "unknown request id %lld", (long long)id);
        if (it->second.done) return sfail(s, ASSN_ERR_STATE, "request %lld has finished", (long long)id);
        auto q = std::find_if(s->queue.begin(), s->queue.end(), [&](const Request& r) { return r.id == id; });
        if (q == s->queue.end()) {   // admitted (or being admitted): the loop retires it
            s->cancel.insert(id);
            return ASSN_OK;
        }
        Result res;
        res.status = ASSN_ERR_CANCELLED;
        res.error = "cancelled before admission";
        res.latency_s = std::chrono::duration<double>(Clock::now() - q->t_submit).count();
        res.queue_s = res.latency_s;
        res.done = true;
        s->queue.erase(q);
        ++s->failed;
        it->second = std::move(res);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();
    return ASSN_OK;
}

int assn_server_get_stats(assn_server* s, assn_server_stats* out) {
    if (!s || !out) return sfail(s, ASSN_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    assn_server_stats st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.failed = s->failed;
    st.active = s->n_active_pub;
    st.queued = (int64_t)s->queue.size();
    st.max_active_seen = s->max_active_seen;
    st.launches = s->launches;
    st.busy_s = s->busy_s;
    st.updates = s->updates;
    st.wall_s = s->any ? std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count() : 0.0;
    st.updates_per_s = st.wall_s > 0 ? s->updates / st.wall_s : 0.0;
    st.budget_bytes = (int64_t)s->budget;
    st.peak_bytes = (int64_t)s->peak_bytes;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double f) {   // nearest rank
            size_t k = (size_t)ceil(f * (double)v.size());
            return v[std::min(v.size() - 1, k > 0 ? k - 1 : 0)];
        };
        st.p50_latency_s = pct(0.50);
        st.p99_latency_s = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st.mean_latency_s = sum / (double)v.size();
    }
    *out = st;
    return ASSN_OK;
}

int assn_server_destroy(assn_server* s) {
    if (!s) return ASSN_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->loop.joinable()) s->loop.join();
    cudaSetDevice(s->dev);
    assn_batch_destroy(s->batch);
    cudaStreamDestroy(s->setup);
    delete s;
    return ASSN_OK;
}

const char* assn_server_last_error(void) { return g_server_error.c_str(); }

}  // extern "C"
