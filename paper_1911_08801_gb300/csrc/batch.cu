// Batched stepping of several as-S_N problems (uneven grids, ordinate counts and kernel widths)
// by the persistent tensor-core kernel, optionally as a CUDA graph, and the tile-shape autotuner.
//
// Every launch advances each member whose device step counter is below its target by one
// explicit step (Sec. 3: upwind transport, collision and isotropic scattering, and the
// artificial-scattering contraction of Sec. 3.2 in one pass) or, for a batch of the paper's
// explicit scheme (Sec. 3.1, Heun + minmod), by one of the two stages of a Heun step; members that
// reached their target are skipped on the device, so a run of max(launches per member) launches,
// captured once as a graph, completes every member at its own step count with no host round trip
// in between.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "problem.h"
#include "trace.h"

using namespace assn;

struct assn_batch {
    int dev = 0;
    int precision = -1;                 // of the members (BF16 or BF16X3; TF32 or BF16X2 if all are paired)
    int scheme = -1;                    // of the members (forward-Euler upwind or Heun + minmod)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    struct Member {
        assn_problem* p;
        int nsteps;
        double dt;
        // stepped by its own paired-SM launches (the kernel its steps run alone), not in a class
        bool paired = false;
    };
    std::vector<Member> members;
    // Members grouped by padded ordinate count Qp: each class has its own plan, tile width and
    // launch per step, so every class runs at the tile width that suits its ordinate count and on
    // the kernel instance compiled for its ordinate stride.
    struct Class {
        int Qp = 0;
        std::vector<int> idx;           // member indices
        Tc2Plan* plan = nullptr;
        std::vector<int> targets;
        int nt = 0;                     // requested tile width (0 = automatic)
        TcRings rings;                  // requested rings (zero fields automatic)
        int nmax = 0;                   // launches per run
    };
    std::vector<Class> classes;
    bool planned = false;
    cudaGraphExec_t graph = nullptr;    // one run: every class's launches
    std::vector<int> graph_shape;       // nmax per class the graph was captured for
    unsigned int* d_err = nullptr;
    cudaEvent_t done = nullptr;
    // side streams for the launch chains of the classes and of the paired members (created when
    // first needed): forked from the batch stream by `fork`, joined back by `join`, so that one
    // chain's launches overlap the tails of the others'
    static constexpr int kSide = 8;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
    int want_nt = 0;                    // 0 = automatic (per class)
    int grouping = 0;                   // 0: one class per padded ordinate count; 1: one class
    TcRings want_rings;                 // zero fields automatic (per class)
    bool tuned = false;                 // classes carry autotuned tilings
    std::string err;
    int64_t launches = 0;
};

namespace {

thread_local std::string g_batch_error;

int bfail(assn_batch* b, int status, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int bfail(assn_batch* b, int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf; else g_batch_error = buf;
    return status;
}

#define BK(b, call)                                                                                    \
    do {                                                                                               \
        cudaError_t _e = (call);                                                                       \
        if (_e != cudaSuccess)                                                                         \
            return bfail((b), _e == cudaErrorMemoryAllocation ? ASSN_ERR_OOM : ASSN_ERR_CUDA, "%s: %s", \
                         #call, cudaGetErrorString(_e));                                               \
    } while (0)

// Launches per time step of the batch's scheme (a Heun step is two stage launches).
int launches_per_step(const assn_batch* b) { return b->scheme == ASSN_SCHEME_HEUN_MINMOD ? 2 : 1; }

void drop_graph(assn_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_shape.clear();
}

// Forget plans (membership, dt or tiling changed); tuned tilings are kept unless `untune`.
void drop_plan(assn_batch* b, bool untune = true) {
    drop_graph(b);
    for (auto& c : b->classes)
        if (c.plan) tc2_plan_destroy(c.plan);
    if (untune) {
        b->classes.clear();
        b->tuned = false;
    } else {
        for (auto& c : b->classes) c.plan = nullptr;
    }
    b->planned = false;
}

// Group members into classes by Qp, or all into one class keyed by the largest Qp (keeps tilings
// of existing classes).
void group(assn_batch* b) {
    std::vector<assn_batch::Class> old;
    old.swap(b->classes);
    int qmax = 0;
    for (auto& m : b->members) qmax = std::max(qmax, m.p->Qp);
    for (size_t i = 0; i < b->members.size(); ++i) {
        // with one class per ordinate count, a member whose steps run on the paired-SM kernel keeps
        // it: its launches join the batch's sequence (and graph) beside the class launches
        b->members[i].paired = !b->grouping && problem_paired(b->members[i].p);
        if (b->members[i].paired) continue;
        const int Qp = b->grouping ? qmax : b->members[i].p->Qp;
        auto it = std::find_if(b->classes.begin(), b->classes.end(), [&](const assn_batch::Class& c) { return c.Qp == Qp; });
        if (it == b->classes.end()) {
            assn_batch::Class c;
            c.Qp = Qp;
            for (auto& o : old)
                if (o.Qp == Qp) { c.nt = o.nt; c.rings = o.rings; }
            b->classes.push_back(c);
            it = b->classes.end() - 1;
        }
        it->idx.push_back((int)i);
    }
    std::sort(b->classes.begin(), b->classes.end(),
              [](const assn_batch::Class& x, const assn_batch::Class& y) { return x.Qp > y.Qp; });
}

// ---------------------------------------------------------------------------------------------
// Autotuner: times one launch of each candidate tiling (tile width NT, ring depths) on the
// problems' current states, writing into scratch buffers so no state changes, and keeps the
// fastest.  Results are cached per (precision, multiset of grid size x ordinate stride).

struct TuneKey {
    std::string s;
    bool operator<(const TuneKey& o) const { return s < o.s; }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, TcRings>> g_tune_cache;

TuneKey tune_key(const std::vector<Tc2Problem>& probs, bool split) {
    std::vector<std::pair<int, int>> v;
    for (const Tc2Problem& p : probs) v.push_back({p.nx * p.ny, p.Qp});
    std::sort(v.begin(), v.end());
    std::string s = split ? "x3" : "b1";
    char buf[48];
    for (auto& e : v) {
        snprintf(buf, sizeof buf, ":%dx%d", e.first, e.second);
        s += buf;
    }
    return TuneKey{s};
}

// probs: descriptions of the problems as they will be stepped (buf[parity] is read); par[i] the
// parity of problem i's current state.  Candidates: every tile width that fits TMEM, each with the
// automatic rings and a few other ring shapes (duplicates of an already timed layout skipped).
// Returns cudaSuccess and the best (nt, rings), or an error; ms_out gets the best launch time.
cudaError_t autotune(const std::vector<Tc2Problem>& probs, const std::vector<int>& par, bool split,
                     cudaStream_t s, int* nt_out, TcRings* rings_out, float* ms_out, bool use_cache) {
    const TuneKey key = tune_key(probs, split);
    if (use_cache) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *nt_out = it->second.first;
            *rings_out = it->second.second;
            if (ms_out) *ms_out = -1.0f;
            return cudaSuccess;
        }
    }
    const int n = (int)probs.size();
    int MBmax = 1;
    for (const Tc2Problem& p : probs) MBmax = std::max(MBmax, p.Mp / 128);
    std::vector<float*> scratch(n, nullptr);
    int* d_cnt = nullptr;
    unsigned int* d_err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaSuccess;
    float best = INFINITY;
    int best_nt = 0;
    TcRings best_r;
    do {
        for (int i = 0; i < n && err == cudaSuccess; ++i)
            err = cudaMalloc(&scratch[i], (size_t)probs[i].nx * probs[i].ny * probs[i].Qp * sizeof(float));
        if (err != cudaSuccess) break;
        if ((err = cudaMalloc(&d_cnt, sizeof(int) * n)) != cudaSuccess) break;
        if ((err = cudaMalloc(&d_err, sizeof(unsigned int))) != cudaSuccess) break;
        if ((err = cudaMemsetAsync(d_err, 0, sizeof(unsigned int), s)) != cudaSuccess) break;
        if ((err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess) break;
        std::vector<Tc2Problem> trial(probs);
        for (int i = 0; i < n; ++i) {
            // counter 0 -> read buf[0] (the current state), write buf[1] (scratch)
            trial[i].buf[0] = probs[i].buf[par[i]];
            trial[i].buf[1] = scratch[i];
            trial[i].counter = d_cnt + i;
            trial[i].target = 1;
        }
        const TcRings shapes[] = {TcRings{}, TcRings{3, 3, 3, 2}, TcRings{2, 2, 0, 4}, TcRings{3, 3, 0, 4},
                                  TcRings{2, 2, 0, 1}, TcRings{3, 3, 0, 1}};
        std::vector<std::pair<int, TcRings>> seen;
        for (int nt = 32; nt <= 256 && err == cudaSuccess; nt *= 2) {
            if (2 * MBmax * nt > 512) break;
            for (const TcRings& want : shapes) {
                Tc2Plan* plan = nullptr;
                cudaError_t ce = tc2_plan_create(&plan, trial.data(), n, split, nt, want);
                if (ce == cudaErrorNotSupported) continue;
                if (ce != cudaSuccess) { err = ce; break; }
                const TcRings got = tc2_plan_rings(plan);
                bool dup = false;
                for (auto& v : seen)
                    dup = dup || (v.first == nt && v.second.SS == got.SS && v.second.SB == got.SB &&
                                  v.second.SA == got.SA && v.second.MPR == got.MPR);
                if (dup) {
                    tc2_plan_destroy(plan);
                    continue;
                }
                seen.push_back({nt, got});
                float tot = 0.0f;
                for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
                    err = cudaMemsetAsync(d_cnt, 0, sizeof(int) * n, s);
                    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
                    if (err == cudaSuccess) err = launch_step_tc2(plan, d_err, n == 1 ? 0 : -1, s);
                    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
                    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tot += ms;   // first launch is the warm-up
                }
                tc2_plan_destroy(plan);
                if (err != cudaSuccess) break;
                unsigned int flag = 0;
                err = cudaMemcpy(&flag, d_err, sizeof flag, cudaMemcpyDeviceToHost);
                if (err == cudaSuccess && flag) err = cudaErrorLaunchTimeout;
                if (err != cudaSuccess) break;
                if (tot / 3.0f < best) {
                    best = tot / 3.0f;
                    best_nt = nt;
                    best_r = got;
                }
            }
        }
    } while (false);
    for (float* p : scratch)
        if (p) cudaFree(p);
    if (d_cnt) cudaFree(d_cnt);
    if (d_err) cudaFree(d_err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    if (best_nt == 0) return cudaErrorNotSupported;
    *nt_out = best_nt;
    *rings_out = best_r;
    if (ms_out) *ms_out = best;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = {best_nt, best_r};
    return cudaSuccess;
}

// Builds the per-class plans for the current membership (targets from each member's state and
// nsteps), or only refreshes the targets when the plans exist.
// The one-CTA kernel has no TF32 or BF16X2 form: such a batch must leave every member paired.
int check_classes(assn_batch* b) {
    if (!b->classes.empty() && (b->precision == ASSN_TF32 || b->precision == ASSN_BF16X2))
        return bfail(b, ASSN_ERR_UNSUPPORTED,
                     "the one-launch grouping steps every member on the one-CTA kernel, which has no TF32 or "
                     "BF16X2 form");
    return ASSN_OK;
}

int ensure_batch_plan(assn_batch* b) {
    if (!b->planned) {
        group(b);
        if (int r = check_classes(b)) return r;
        for (auto& m : b->members)
            if (m.paired) {
                const int r = problem_pair_plan(m.p, m.dt);
                if (r) return bfail(b, r, "batch: paired-SM plan: %s", assn_last_error(m.p));
            }
        for (auto& c : b->classes) {
            std::vector<Tc2Problem> d;
            for (int i : c.idx) {
                const assn_batch::Member& m = b->members[i];
                d.push_back(problem_tc2(m.p, m.dt, m.p->cur + launches_per_step(b) * m.nsteps));
            }
            const int nt = b->want_nt ? b->want_nt : c.nt;
            const bool user = b->want_rings.SS || b->want_rings.SB || b->want_rings.SA || b->want_rings.MPR;
            cudaError_t e = tc2_plan_create(&c.plan, d.data(), (int)d.size(), b->precision == ASSN_BF16X3, nt,
                                            user ? b->want_rings : c.rings);
            if (e == cudaErrorNotSupported)
                return bfail(b, ASSN_ERR_UNSUPPORTED, "batch: tiling not supported for Qp = %d (tile %d)", c.Qp, nt);
            BK(b, e);
        }
        b->planned = true;
    }
    for (auto& c : b->classes) {
        c.targets.resize(c.idx.size());
        c.nmax = 0;
        for (size_t k = 0; k < c.idx.size(); ++k) {
            const assn_batch::Member& m = b->members[c.idx[k]];
            c.targets[k] = m.p->cur + launches_per_step(b) * m.nsteps;
            c.nmax = std::max(c.nmax, launches_per_step(b) * m.nsteps);
        }
        BK(b, tc2_plan_set_targets(c.plan, c.targets.data(), b->stream));
    }
    return ASSN_OK;
}

int index_of(const assn_batch* b, const assn_problem* p) {
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i].p == p) return (int)i;
    return -1;
}

}  // namespace

extern "C" {

int assn_batch_create(assn_batch** out, void* cuda_stream) {
    if (!out) return bfail(nullptr, ASSN_ERR_ARG, "out is NULL");
    *out = nullptr;
    assn_batch* b = new (std::nothrow) assn_batch();
    if (!b) return bfail(nullptr, ASSN_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            b->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        bfail(nullptr, e == cudaErrorMemoryAllocation ? ASSN_ERR_OOM : ASSN_ERR_CUDA, "batch create: %s",
              cudaGetErrorString(e));
        if (b->d_err) cudaFree(b->d_err);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return e == cudaErrorMemoryAllocation ? ASSN_ERR_OOM : ASSN_ERR_CUDA;
    }
    *out = b;
    return ASSN_OK;
}

int assn_batch_destroy(assn_batch* b) {
    if (!b) return ASSN_OK;
    cudaSetDevice(b->dev);
    cudaStreamSynchronize(b->stream);
    drop_plan(b);
    if (b->d_err) cudaFree(b->d_err);
    if (b->done) cudaEventDestroy(b->done);
    if (b->fork) cudaEventDestroy(b->fork);
    for (int s = 0; s < assn_batch::kSide; ++s) {
        if (b->join[s]) cudaEventDestroy(b->join[s]);
        if (b->side[s]) cudaStreamDestroy(b->side[s]);
    }
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return ASSN_OK;
}

int assn_batch_add(assn_batch* b, assn_problem* p, int nsteps, double dt) {
    if (!b || !p) return bfail(b, ASSN_ERR_ARG, "batch or problem is NULL");
    if (nsteps < 0) return bfail(b, ASSN_ERR_ARG, "nsteps < 0");
    if (!p->tensor()) return bfail(b, ASSN_ERR_UNSUPPORTED, "batches step the tensor-core precisions only");
    if (p->scheme != ASSN_SCHEME_EULER_UPWIND && p->scheme != ASSN_SCHEME_HEUN_MINMOD)
        return bfail(b, ASSN_ERR_UNSUPPORTED, "batches take the explicit schemes (forward-Euler upwind, Heun + minmod)");
    if (b->precision >= 0 && p->precision != b->precision)
        return bfail(b, ASSN_ERR_ARG, "all members of a batch share one precision");
    if (b->scheme >= 0 && p->scheme != b->scheme)
        return bfail(b, ASSN_ERR_ARG, "all members of a batch share one scheme");
    if (p->dev != b->dev) return bfail(b, ASSN_ERR_ARG, "problem lives on another device");
    if (index_of(b, p) >= 0) return bfail(b, ASSN_ERR_ARG, "problem is already a member");
    if ((int)b->members.size() >= 1024) return bfail(b, ASSN_ERR_ARG, "a batch holds at most 1024 problems");
    const int r = problem_prepare(p, dt);
    if (r) return bfail(b, r, "member: %s", p->err.c_str());
    if (p->paired_only() && !(problem_paired(p) && problem_pair_supported(p)))
        return bfail(b, ASSN_ERR_UNSUPPORTED,
                     "TF32 and BF16X2 members run on the paired-SM kernel only (193..256 or 449..512 ordinates)");
    b->precision = p->precision;
    b->scheme = p->scheme;
    b->members.push_back({p, nsteps, dt});
    drop_plan(b);
    return ASSN_OK;
}

int assn_batch_set_steps(assn_batch* b, assn_problem* p, int nsteps, double dt) {
    if (!b || !p) return bfail(b, ASSN_ERR_ARG, "batch or problem is NULL");
    const int i = index_of(b, p);
    if (i < 0) return bfail(b, ASSN_ERR_ARG, "problem is not a member");
    if (nsteps < 0) return bfail(b, ASSN_ERR_ARG, "nsteps < 0");
    if (dt != b->members[i].dt) {
        const int r = problem_prepare(p, dt);
        if (r) return bfail(b, r, "member: %s", p->err.c_str());
        b->members[i].dt = dt;
        drop_plan(b, false);   // dt is baked into the descriptors
    }
    b->members[i].nsteps = nsteps;
    return ASSN_OK;
}

int assn_batch_remove(assn_batch* b, assn_problem* p) {
    if (!b || !p) return bfail(b, ASSN_ERR_ARG, "batch or problem is NULL");
    const int i = index_of(b, p);
    if (i < 0) return bfail(b, ASSN_ERR_ARG, "problem is not a member");
    BK(b, cudaStreamSynchronize(b->stream));
    b->members.erase(b->members.begin() + i);
    if (b->members.empty()) b->precision = b->scheme = -1;
    drop_plan(b);
    return ASSN_OK;
}

int assn_batch_set_tiling(assn_batch* b, int tile_cells, int stages) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    if (tile_cells != 0 && tile_cells != 32 && tile_cells != 64 && tile_cells != 128 && tile_cells != 256)
        return bfail(b, ASSN_ERR_ARG, "tile_cells must be 0, 32, 64, 128 or 256");
    if (stages != 0 && (stages < 2 || stages > 8)) return bfail(b, ASSN_ERR_ARG, "stages must be 0 or 2..8");
    b->want_nt = tile_cells;
    b->want_rings = TcRings{stages, stages, stages, 0};
    drop_plan(b);
    return ASSN_OK;
}

int assn_batch_set_grouping(assn_batch* b, int one_launch) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    if (one_launch != 0 && one_launch != 1) return bfail(b, ASSN_ERR_ARG, "one_launch must be 0 or 1");
    if (one_launch != b->grouping) {
        b->grouping = one_launch;
        drop_plan(b);
    }
    return ASSN_OK;
}

int assn_batch_autotune(assn_batch* b, int use_cache, int* tile_cells, int* stages, double* ms_per_launch) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    if (b->members.empty()) return bfail(b, ASSN_ERR_STATE, "batch has no members");
    BK(b, cudaSetDevice(b->dev));
    for (auto& m : b->members) {   // the tuner reads the members' current states
        if (m.p->stream != b->stream) {
            BK(b, cudaStreamSynchronize(m.p->stream));
        }
    }
    drop_plan(b);
    group(b);
    if (int r = check_classes(b)) return r;
    double total_ms = 0.0;
    bool all_cached = true;
    for (auto& c : b->classes) {
        std::vector<Tc2Problem> d;
        std::vector<int> par;
        for (int i : c.idx) {
            d.push_back(problem_tc2(b->members[i].p, b->members[i].dt, 1));
            par.push_back(b->members[i].p->cur);
        }
        int nt = 0;
        TcRings rr;
        float ms = 0.0f;
        cudaError_t e = autotune(d, par, b->precision == ASSN_BF16X3, b->stream, &nt, &rr, &ms, use_cache != 0);
        if (e == cudaErrorLaunchTimeout) return bfail(b, ASSN_ERR_TIMEOUT, "autotune: a bounded device wait gave up");
        if (e == cudaErrorNotSupported) return bfail(b, ASSN_ERR_UNSUPPORTED, "autotune: no tiling fits Qp = %d", c.Qp);
        BK(b, e);
        c.nt = nt;
        c.rings = rr;
        if (ms >= 0.0f) { total_ms += ms; all_cached = false; }
    }
    b->want_nt = 0;
    b->want_rings = TcRings{};
    b->tuned = true;
    // report the class with the most ordinate blocks (the first); none when every member is paired
    if (tile_cells) *tile_cells = b->classes.empty() ? 0 : b->classes[0].nt;
    if (stages) *stages = b->classes.empty() ? 0 : b->classes[0].rings.SA;
    if (ms_per_launch) *ms_per_launch = all_cached ? -1.0 : total_ms;
    return ASSN_OK;
}

int assn_batch_run(assn_batch* b, int use_graph) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    TraceRange tr("assn_batch_run");
    if (b->members.empty()) return ASSN_OK;
    BK(b, cudaSetDevice(b->dev));
    const int lps = launches_per_step(b);
    int nmax = 0;
    for (auto& m : b->members) nmax = std::max(nmax, lps * m.nsteps);
    if (nmax == 0) return ASSN_OK;
    // order after each member's pending work; set each device counter to the member's parity
    for (auto& m : b->members) {
        assn_problem* p = m.p;
        if (p->stream != b->stream) {
            BK(b, cudaEventRecord(b->done, p->stream));
            BK(b, cudaStreamWaitEvent(b->stream, b->done, 0));
        }
        if (p->counter_host != p->cur) {
            p->counter_host = p->cur;
            BK(b, cudaMemcpyAsync(p->d_counter, &p->counter_host, sizeof(int), cudaMemcpyHostToDevice, b->stream));
        }
    }
    int r = ensure_batch_plan(b);
    if (r) return r;
    std::vector<int> shape;   // what a captured graph is specific to
    for (auto& c : b->classes) shape.push_back(c.nmax);
    int nlaunch = 0;
    for (int v : shape) nlaunch += v;
    int npaired = 0;
    for (auto& m : b->members)
        if (m.paired) {   // (the launches' buffers follow from the member's current one)
            shape.push_back(lps * m.nsteps);
            shape.push_back(m.p->cur);
            nlaunch += lps * m.nsteps;
            ++npaired;
        }
    const int nchain = npaired + (int)b->classes.size();   // independent launch chains
    const int nside = std::min(nchain, (int)assn_batch::kSide);
    if (nside > 0 && !b->fork) {
        BK(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (int s = 0; s < assn_batch::kSide; ++s) {
            BK(b, cudaStreamCreateWithFlags(&b->side[s], cudaStreamNonBlocking));
            BK(b, cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming));
        }
    }
    auto enqueue = [&]() -> cudaError_t {
        // each class's chain of launches (one per step; Heun: per stage) and each paired member's
        // chain on a side stream forked from the batch stream, round robin
        cudaError_t e = cudaSuccess;
        if (nside > 0) {
            e = cudaEventRecord(b->fork, b->stream);
            for (int s = 0; s < nside && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->side[s], b->fork, 0);
        }
        int j = 0;
        for (auto& c : b->classes) {
            cudaStream_t s = b->side[j++ % nside];
            for (int k = 0; k < c.nmax && e == cudaSuccess; ++k)
                e = lps == 2 ? launch_heun_stage_tc2(c.plan, b->d_err, -1, nullptr, 0.0f, 1.0f, s)
                             : launch_step_tc2(c.plan, b->d_err, -1, s);
        }
        for (auto& m : b->members) {
            if (!m.paired) continue;
            cudaStream_t s = b->side[j++ % nside];
            const int cur0 = m.p->cur;
            for (int k = 0; k < lps * m.nsteps && e == cudaSuccess; ++k) {
                if (lps == 2)   // a Heun step ends in the buffer it started from
                    e = problem_pair_launch(m.p, m.dt, (k & 1) ? cur0 ^ 1 : cur0, k & 1, b->d_err, s);
                else
                    e = problem_pair_launch(m.p, m.dt, (cur0 + k) & 1, -1, b->d_err, s);
            }
        }
        for (int s = 0; s < nside; ++s) {   // joined even after an error, so that a capture can end
            cudaError_t e2 = cudaEventRecord(b->join[s], b->side[s]);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(b->stream, b->join[s], 0);
            if (e == cudaSuccess) e = e2;
        }
        return e;
    };
    if (use_graph) {
        if (!b->graph || b->graph_shape != shape) {
            drop_graph(b);
            cudaGraph_t g = nullptr;
            BK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue();
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            BK(b, e);
            b->graph_shape = shape;
        }
        BK(b, cudaGraphLaunch(b->graph, b->stream));
    } else {
        BK(b, enqueue());
    }
    b->launches += nlaunch;
    BK(b, cudaEventRecord(b->done, b->stream));
    for (auto& m : b->members) {
        assn_problem* p = m.p;
        p->counter_host = p->cur + lps * m.nsteps;
        p->cur = p->counter_host & 1;
        p->launches += lps * m.nsteps;
        if (m.paired)   // the paired-SM kernel leaves the device step counter alone: set it
            BK(b, cudaMemcpyAsync(p->d_counter, &p->counter_host, sizeof(int), cudaMemcpyHostToDevice, b->stream));
        if (p->stream != b->stream) BK(b, cudaStreamWaitEvent(p->stream, b->done, 0));
    }
    return ASSN_OK;
}

int assn_batch_sync(assn_batch* b) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    BK(b, cudaSetDevice(b->dev));
    BK(b, cudaStreamSynchronize(b->stream));
    unsigned int f = 0;
    BK(b, cudaMemcpy(&f, b->d_err, sizeof f, cudaMemcpyDeviceToHost));
    if (f) {
        BK(b, cudaMemset(b->d_err, 0, sizeof f));
        return bfail(b, ASSN_ERR_TIMEOUT, "batch step: a bounded device wait gave up (flag 0x%x)%s", f,
                     (f & 0x80000000u) ? "; work in flight did not drain, treat the CUDA context as suspect" : "");
    }
    return ASSN_OK;
}

int assn_batch_info(assn_batch* b, int* members, int* tile_cells, int* stages, int* total_tiles,
                    int64_t* launches) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    if (members) *members = (int)b->members.size();
    int nt = 0, st = 0, cols = 0, tiles = 0;
    size_t sm = 0;
    if (!b->members.empty()) {
        BK(b, cudaSetDevice(b->dev));
        int r = ensure_batch_plan(b);
        if (r) return r;
        if (!b->classes.empty()) tc2_plan_describe(b->classes[0].plan, &nt, &st, &cols, &sm);
        for (auto& c : b->classes) tiles += tc2_plan_total_tiles(c.plan);
    }
    if (tile_cells) *tile_cells = nt;
    if (stages) *stages = st;
    if (total_tiles) *total_tiles = tiles;
    if (launches) *launches = b->launches;
    return ASSN_OK;
}

int assn_batch_class_info(assn_batch* b, int k, int* ordinate_stride, int* members, int* tile_cells, int* stages,
                          int* tiles) {
    if (!b) return bfail(b, ASSN_ERR_ARG, "batch is NULL");
    if (!b->members.empty()) {
        BK(b, cudaSetDevice(b->dev));
        int r = ensure_batch_plan(b);
        if (r) return r;
    }
    if (k < 0 || k >= (int)b->classes.size()) return bfail(b, ASSN_ERR_ARG, "class %d of %d", k, (int)b->classes.size());
    const assn_batch::Class& c = b->classes[k];
    int nt = 0, st = 0, cols = 0;
    size_t sm = 0;
    tc2_plan_describe(c.plan, &nt, &st, &cols, &sm);
    if (ordinate_stride) *ordinate_stride = c.Qp;
    if (members) *members = (int)c.idx.size();
    if (tile_cells) *tile_cells = nt;
    if (stages) *stages = st;
    if (tiles) *tiles = tc2_plan_total_tiles(c.plan);
    return ASSN_OK;
}

int assn_batch_classes(assn_batch* b, int* nclass) {
    if (!b || !nclass) return bfail(b, ASSN_ERR_ARG, "NULL argument");
    *nclass = 0;
    if (!b->members.empty()) {
        BK(b, cudaSetDevice(b->dev));
        int r = ensure_batch_plan(b);
        if (r) return r;
    }
    *nclass = (int)b->classes.size();
    return ASSN_OK;
}

const char* assn_batch_last_error(const assn_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

// Single problem: tune its tiling the same way and apply it (assn_set_tiling with the result).
int assn_autotune(assn_problem* p, double dt, int use_cache, int* tile_cells, int* stages, double* ms_per_step) {
    if (!p) return ASSN_ERR_ARG;
    if (!p->tensor()) return problem_fail(p, ASSN_ERR_UNSUPPORTED, "autotune applies to the tensor-core precisions");
    if (p->paired_only())
        return problem_fail(p, ASSN_ERR_UNSUPPORTED,
                            "autotune tunes the persistent one-CTA kernel, which has no TF32 or BF16X2 form");
    int r = problem_prepare(p, dt);
    if (r) return r;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return problem_fail(p, ASSN_ERR_CUDA, cudaGetErrorString(e));
    std::vector<Tc2Problem> d{problem_tc2(p, dt, 1)};
    std::vector<int> par{p->cur};
    int nt = 0;
    TcRings rr;
    float ms = 0.0f;
    e = autotune(d, par, p->precision == ASSN_BF16X3, p->stream, &nt, &rr, &ms, use_cache != 0);
    if (e == cudaErrorLaunchTimeout) return problem_fail(p, ASSN_ERR_TIMEOUT, "autotune: a bounded device wait gave up");
    if (e == cudaErrorNotSupported) return problem_fail(p, ASSN_ERR_UNSUPPORTED, "autotune: no tiling fits");
    if (e != cudaSuccess) return problem_fail(p, ASSN_ERR_CUDA, cudaGetErrorString(e));
    r = assn_set_tiling(p, nt, 0, 0);
    if (r) return r;
    r = assn_set_rings(p, rr.SS, rr.SB, rr.SA, rr.MPR);
    if (r) return r;
    const int st = rr.SA;
    if (tile_cells) *tile_cells = nt;
    if (stages) *stages = st;
    if (ms_per_step) *ms_per_step = ms;
    return ASSN_OK;
}

}  // extern "C"
