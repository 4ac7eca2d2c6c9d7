// Serving loop: BnB instances (problem (intro_sparse_glm) of §1, each certified
// by the hybrid loop of Fig. 1) admitted as they arrive and solved together.
//
// Requests wait in a FIFO.  A request is admitted when a slot is free
// (max_active) and its device footprint (the exact byte count kglm_create
// will allocate, its device-resident open-node queue included) fits in what
// the admitted requests leave of the HBM budget.  Its X and node queue then
// live on the device, and one scheduler thread runs rounds: every running
// request's next node batch is selected on the device, the selected batches
// are evaluated together -- the FISTA iterations of the BF16 requests as
// shared launches (one grouped S = X V + link, one grouped G = X^T R and one
// prox over all of their nodes per iteration), the others with their own
// launches on the same stream -- and each request's batch is closed,
// branched and merged into its queue on the device.  A request that arrives
// while others run is admitted at the next round that has a slot and memory
// for it: continuous batching at node-batch granularity.  Each request's
// nodes see the same arithmetic whatever else shares the launches (its tiles,
// split-K slices and node-level work depend on its own shapes only), so its
// result does not depend on the mix.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"
#include "kglm.h"

using namespace kglm;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    int64_t id = 0;
    kglm_desc d{};
    std::vector<double> X, y;
    kglm_request_info info{};
};

}  // namespace

struct kglm_server {
    kglm_server_desc d{};
    int device = 0;
    int64_t budget = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;        // queue or capacity changed
    std::condition_variable cv_done;   // a request finished
    std::deque<Req*> pending;
    std::map<int64_t, Req*> reqs;
    int64_t next_id = 1, used = 0, peak_used = 0, submitted = 0, finished = 0;
    int active = 0, peak_active = 0;
    bool stopping = false;
    std::atomic<int> cancel{0};
    std::thread scheduler;
    cudaStream_t stream = nullptr;     // every request's context runs on it
    int64_t rounds = 0, round_batches = 0, shared_launches = 0;
    std::string err = "no error";
};

namespace {

double since(const kglm_server* s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

// The scheduler: one host thread runs rounds over the admitted requests.  A
// round admits what the queue, the slots and the budget allow (each admitted
// request gets a context on the server's stream with its open-node queue on
// the device, and starts its search), selects the next node batch of every
// running request on the device, evaluates all selected batches together
// (serve_evaluate: the iterations of the BF16 requests as shared launches),
// and closes, branches and merges each request's batch on the device.  A
// request whose queue is empty (or whose time limit passed) is finished: its
// result is published and its memory returns to the budget.
struct Running {
    Req* r = nullptr;
    kglm_ctx* ctx = nullptr;
    ServeSolve* sv = nullptr;
    Clock::time_point t_start;
};

// Publish a finished request and release its slot and memory (the caller holds no lock).
void publish(kglm_server* s, Running& a, const kglm_request_info& info) {
    std::vector<double>().swap(a.r->X);   // the host copy is no longer needed
    std::vector<double>().swap(a.r->y);
    std::lock_guard<std::mutex> g(s->mu);
    a.r->info = info;
    a.r->info.t_done = since(s);
    s->used -= a.r->info.device_bytes;
    --s->active;
    ++s->finished;
    s->cv_done.notify_all();
}

void fail(kglm_server* s, Running& a, kglm_status st, const char* msg) {
    kglm_request_info info = a.r->info;
    info.state = KGLM_REQ_FAILED;
    info.status = st;
    snprintf(info.message, sizeof(info.message), "%s", msg);
    if (a.sv) serve_free(a.sv);
    a.sv = nullptr;
    if (a.ctx) kglm_destroy(a.ctx);
    a.ctx = nullptr;
    publish(s, a, info);
}

void finish(kglm_server* s, Running& a, bool stopped, bool cancelled) {
    SolveResult res;
    const kglm_status st = serve_finish(a.sv, stopped, &res);
    a.sv = nullptr;
    if (st != KGLM_OK) {
        fail(s, a, st, kglm_last_error(a.ctx));
        return;
    }
    kglm_request_info info = a.r->info;
    info.opt = res.opt;
    info.gap = res.gap;
    info.nodes = res.nodes;
    info.batches = res.batches;
    for (int t = 0; t < KGLM_MAX_K; ++t) info.support[t] = t < (int)res.support.size() ? res.support[t] : -1;
    info.state = cancelled ? KGLM_REQ_CANCELLED : KGLM_REQ_DONE;
    info.status = KGLM_OK;
    kglm_destroy(a.ctx);
    a.ctx = nullptr;
    publish(s, a, info);
}

// Context and search of an admitted request on the server's stream.
bool start(kglm_server* s, Running& a) {
    kglm_desc d = a.r->d;
    d.hbm_budget = a.r->info.device_bytes + 65536;   // the admitted share (plus rounding of small arrays)
    kglm_status st = kglm_create(&d, a.r->X.data(), a.r->y.data(), s->stream, &a.ctx);
    if (st != KGLM_OK) {
        a.ctx = nullptr;
        fail(s, a, st, kglm_last_error(nullptr));
        return false;
    }
    st = serve_begin(a.ctx, d.max_batch, &a.sv);
    if (st != KGLM_OK) {
        fail(s, a, st, kglm_last_error(a.ctx));
        return false;
    }
    a.t_start = Clock::now();
    return true;
}

void scheduler_main(kglm_server* s) {
    cudaSetDevice(s->device);
    std::vector<Running> run;
    for (;;) {
        std::vector<Running> admitted;
        bool stop = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (run.empty()) s->cv.wait(lk, [&] { return s->stopping || !s->pending.empty(); });
            stop = s->stopping;
            while (!stop && !s->pending.empty() && (int)(run.size() + admitted.size()) < s->d.max_active &&
                   s->used + s->pending.front()->info.device_bytes <= s->budget) {
                Req* r = s->pending.front();
                s->pending.pop_front();
                s->used += r->info.device_bytes;
                s->peak_used = std::max(s->peak_used, s->used);
                s->peak_active = std::max(s->peak_active, ++s->active);
                r->info.state = KGLM_REQ_RUNNING;
                r->info.t_admit = since(s);
                Running a;
                a.r = r;
                admitted.push_back(a);
            }
        }
        for (Running& a : admitted)
            if (start(s, a)) run.push_back(a);
        if (stop || s->cancel.load()) {
            for (Running& a : run) finish(s, a, true, true);
            return;
        }
        if (run.empty()) continue;
        // select every running request's next batch; finished ones leave
        std::vector<Running> next;
        std::vector<kglm_ctx*> sel;
        std::vector<size_t> who;
        for (Running& a : run) {
            const double el = std::chrono::duration<double>(Clock::now() - a.t_start).count();
            if (s->d.time_limit_s > 0 && el > s->d.time_limit_s) {
                finish(s, a, true, false);
                continue;
            }
            int m = 0;
            const kglm_status st = serve_select(a.sv, &m);
            if (st != KGLM_OK) {
                fail(s, a, st, kglm_last_error(a.ctx));
                continue;
            }
            if (m == 0) {
                finish(s, a, false, false);
                continue;
            }
            who.push_back(next.size());
            next.push_back(a);
            sel.push_back(a.ctx);
        }
        run.swap(next);
        if (sel.empty()) continue;
        int64_t shared = 0;
        const kglm_status st = serve_evaluate(sel.data(), (int)sel.size(), s->d.iters, s->d.check_every, &shared);
        if (st != KGLM_OK) {
            const std::string msg = kglm_last_error(sel[0]);
            for (Running& a : run) fail(s, a, st, msg.c_str());
            run.clear();
            continue;
        }
        std::vector<Running> keep;
        for (Running& a : run) {
            const kglm_status su = serve_update(a.sv);
            if (su != KGLM_OK) fail(s, a, su, kglm_last_error(a.ctx));
            else keep.push_back(a);
        }
        run.swap(keep);
        {
            std::lock_guard<std::mutex> g(s->mu);
            ++s->rounds;
            s->round_batches += (int64_t)sel.size();
            s->shared_launches += shared;
        }
    }
}

bool finished_state(int32_t st) {
    return st == KGLM_REQ_DONE || st == KGLM_REQ_FAILED || st == KGLM_REQ_CANCELLED;
}

}  // namespace

extern "C" {

kglm_status kglm_server_create(const kglm_server_desc* desc, kglm_server** out) {
    if (!out) return KGLM_EINVAL;
    *out = nullptr;
    if (!desc || desc->max_active < 1 || desc->max_active > 256 || desc->iters < 1 || desc->check_every < 0 ||
        desc->hbm_budget < 0 || desc->batch_cap < 0)
        return KGLM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KGLM_ECUDA;
    }
    int64_t budget = desc->hbm_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return KGLM_ECUDA;
        }
        budget = (int64_t)(0.8 * (double)fr);
    }
    kglm_server* s = new (std::nothrow) kglm_server();
    if (!s) return KGLM_ENOMEM;
    s->d = *desc;
    if (s->d.batch_cap == 0) s->d.batch_cap = 4096;
    s->device = dev;
    s->budget = budget;
    s->t0 = Clock::now();
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s->stream = nullptr;
        kglm_server_destroy(s);
        return KGLM_ECUDA;
    }
    try {
        s->scheduler = std::thread(scheduler_main, s);
    } catch (...) {
        kglm_server_destroy(s);
        return KGLM_ENOMEM;
    }
    *out = s;
    return KGLM_OK;
}

kglm_status kglm_server_submit(kglm_server* s, const kglm_desc* desc, const double* X, const double* y,
                               int64_t* id) {
    if (!s || !desc || !X || !y || !id) return KGLM_EINVAL;
    kglm_desc d = *desc;
    d.hbm_budget = 0;
    if (d.max_batch == 0) {
        // App. E.4: the largest power-of-two batch that fits this request's share
        const int64_t share = s->budget / std::max(1, s->d.max_active);
        int32_t m = 0;
        kglm_desc q = d;
        q.max_batch = 1;
        const kglm_status st = kglm_suggest_batch(&q, share, s->d.batch_cap, &m);
        if (st == KGLM_ENOMEM) {
            // less than a share: the smallest batch, if it fits the whole budget
            m = 1;
        } else if (st != KGLM_OK) {
            std::lock_guard<std::mutex> g(s->mu);
            s->err = "submit: desc rejected";
            return st;
        }
        d.max_batch = m;
    }
    // the request's open nodes stay on the device: by default as many as a quarter
    // of one slot's share of the budget holds (two buffers of masks, bound, id and
    // slot per node), at most 1 GiB or 2^22 nodes and at least 64 batches
    if (s->d.open_cap > 0) {
        d.open_cap = s->d.open_cap;
    } else {
        const int64_t per = 2 * (20 + 8 * ((d.p + 31) / 32));
        const int64_t bytes = std::min<int64_t>(1LL << 30, s->budget / (4 * std::max(1, s->d.max_active)));
        d.open_cap = std::max<int64_t>(64 * (int64_t)d.max_batch, std::min<int64_t>(1 << 22, bytes / per));
    }
    int64_t bytes = 0;
    kglm_status st = kglm_estimate_bytes(&d, &bytes);
    if (st != KGLM_OK) {
        std::lock_guard<std::mutex> g(s->mu);
        s->err = "submit: desc rejected";
        return st;
    }
    if (bytes > s->budget) {
        std::lock_guard<std::mutex> g(s->mu);
        s->err = "submit: the instance needs more device memory than the server's whole budget";
        return KGLM_ENOMEM;
    }
    Req* r = new (std::nothrow) Req();
    if (!r) return KGLM_ENOMEM;
    try {
        r->X.assign(X, X + (size_t)d.n * (size_t)d.p);
        r->y.assign(y, y + (size_t)d.n);
    } catch (...) {
        delete r;
        return KGLM_ENOMEM;
    }
    r->d = d;
    r->info.state = KGLM_REQ_QUEUED;
    r->info.status = KGLM_OK;
    r->info.opt = INFINITY;
    r->info.gap = INFINITY;
    for (int t = 0; t < KGLM_MAX_K; ++t) r->info.support[t] = -1;
    r->info.device_bytes = bytes;
    r->info.batch = d.max_batch;
    r->info.t_admit = -1;
    r->info.t_done = -1;
    r->info.message[0] = 0;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stopping) {
            delete r;
            return KGLM_ESTATE;
        }
        r->id = s->next_id++;
        r->info.t_submit = since(s);
        s->reqs[r->id] = r;
        s->pending.push_back(r);
        ++s->submitted;
        *id = r->id;
    }
    s->cv.notify_all();
    return KGLM_OK;
}

kglm_status kglm_server_info(kglm_server* s, int64_t id, kglm_request_info* info) {
    if (!s || !info) return KGLM_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return KGLM_EINVAL;
    *info = it->second->info;
    return KGLM_OK;
}

kglm_status kglm_server_wait(kglm_server* s, int64_t id, double timeout_s, kglm_request_info* info) {
    if (!s) return KGLM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return KGLM_EINVAL;
    Req* r = it->second;
    auto done = [&] { return finished_state(r->info.state); };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return KGLM_ETIMEOUT;
    } else {
        s->cv_done.wait(lk, done);
    }
    if (info) *info = r->info;
    return KGLM_OK;
}

kglm_status kglm_server_drain(kglm_server* s, double timeout_s) {
    if (!s) return KGLM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] { return s->finished == s->submitted; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) return KGLM_ETIMEOUT;
    } else {
        s->cv_done.wait(lk, done);
    }
    return KGLM_OK;
}

kglm_status kglm_server_stats(kglm_server* s, kglm_server_stats_t* out) {
    if (!s || !out) return KGLM_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    out->submitted = s->submitted;
    out->finished = s->finished;
    out->queued = (int64_t)s->pending.size();
    out->active = s->active;
    out->peak_active = s->peak_active;
    out->bytes_in_use = s->used;
    out->peak_bytes = s->peak_used;
    out->budget = s->budget;
    out->elapsed_s = since(s);
    out->rounds = s->rounds;
    out->round_batches = s->round_batches;
    out->shared_launches = s->shared_launches;
    return KGLM_OK;
}

const char* kglm_server_last_error(kglm_server* s) {
    if (!s) return "null server";
    std::lock_guard<std::mutex> g(s->mu);
    return s->err.c_str();
}

void kglm_server_destroy(kglm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stopping = true;
    }
    s->cancel.store(1);
    s->cv.notify_all();
    if (s->scheduler.joinable()) s->scheduler.join();
    if (s->stream) cudaStreamDestroy(s->stream);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
