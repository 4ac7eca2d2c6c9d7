// Serving loop: BnB instances (problem (intro_sparse_glm) of §1, each certified
// by the hybrid loop of Fig. 1) admitted as they arrive, solved concurrently.
//
// Requests wait in a FIFO.  A request is admitted when a worker is free and
// its device footprint (the exact byte count kglm_create will allocate) fits
// in what the admitted requests leave of the HBM budget; it then gets its own
// context, stream and host worker thread, so its node batches run on the
// device while other requests' batches do (kernels of different streams share
// the SMs) and its host-side tree work overlaps their device work.  When it
// finishes, its memory returns to the budget and the next request in line is
// admitted: continuous batching at request granularity.  Every request runs
// the same deterministic kernels in the same order as kglm_solve alone, so
// its result does not depend on the mix.
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
    std::vector<std::thread> workers;
    std::string err = "no error";
};

namespace {

double since(const kglm_server* s) { return std::chrono::duration<double>(Clock::now() - s->t0).count(); }

// Solve one admitted request on its own context and stream (no lock held;
// the result is published by the caller under the lock).
kglm_request_info run_request(kglm_server* s, Req* r, kglm_request_info in) {
    kglm_desc d = r->d;
    d.hbm_budget = in.device_bytes + 65536;   // the admitted share (plus rounding of small arrays)
    kglm_ctx* ctx = nullptr;
    kglm_status st = kglm_create(&d, r->X.data(), r->y.data(), nullptr, &ctx);
    const char* msg = st == KGLM_OK ? "" : kglm_last_error(nullptr);
    if (st == KGLM_OK) {
        SolveResult res;
        st = solve_cancellable(ctx, d.max_batch, s->d.iters, s->d.check_every, s->d.time_limit_s, &s->cancel, &res);
        if (st != KGLM_OK) msg = kglm_last_error(ctx);
        if (st == KGLM_OK) {
            in.opt = res.opt;
            in.gap = res.gap;
            in.nodes = res.nodes;
            in.batches = res.batches;
            for (int t = 0; t < KGLM_MAX_K; ++t) in.support[t] = t < (int)res.support.size() ? res.support[t] : -1;
            in.state = res.cancelled ? KGLM_REQ_CANCELLED : KGLM_REQ_DONE;
        }
        if (st != KGLM_OK) snprintf(in.message, sizeof(in.message), "%s", msg);
        kglm_destroy(ctx);
    } else {
        snprintf(in.message, sizeof(in.message), "%s", msg);
    }
    if (st != KGLM_OK) in.state = KGLM_REQ_FAILED;
    in.status = st;
    std::vector<double>().swap(r->X);   // the host copy is no longer needed
    std::vector<double>().swap(r->y);
    return in;
}

void worker_main(kglm_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] {
            return s->stopping || (!s->pending.empty() && s->used + s->pending.front()->info.device_bytes <= s->budget);
        });
        if (s->stopping) return;
        Req* r = s->pending.front();
        s->pending.pop_front();
        s->used += r->info.device_bytes;
        s->peak_used = std::max(s->peak_used, s->used);
        s->peak_active = std::max(s->peak_active, ++s->active);
        r->info.state = KGLM_REQ_RUNNING;
        r->info.t_admit = since(s);
        const kglm_request_info start = r->info;
        s->cv.notify_all();   // another worker may admit the next one
        lk.unlock();
        const kglm_request_info res = run_request(s, r, start);
        lk.lock();
        r->info = res;
        r->info.t_done = since(s);
        s->used -= r->info.device_bytes;
        --s->active;
        ++s->finished;
        s->cv.notify_all();
        s->cv_done.notify_all();
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
    try {
        for (int w = 0; w < desc->max_active; ++w) s->workers.emplace_back(worker_main, s);
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
    for (auto& t : s->workers)
        if (t.joinable()) t.join();
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
