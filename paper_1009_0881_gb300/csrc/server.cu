// Serving form: continuous batching of NMF solves on one GPU (include/nmf.h).
//
// Requests queue in arrival order.  `slots` worker threads each own an
// nmf_handle (stream + workspace).  A free worker takes the longest run of
// requests from the queue head (at most kMaxBatch) whose combined workspace,
// with the workspaces the other slots hold, fits in the HBM budget, and solves
// them as one nmf_solve_batch (one CUDA graph, a branch per request).  An idle
// worker whose workspace keeps the head from fitting releases it.  Requests
// that arrive while others are on the GPU start as soon as a slot and memory
// free up; their kernels overlap with the running ones (one stream per slot,
// concurrent branches inside a batch).
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nmf.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxBatch = 16;

struct Request {
    nmf_problem* prob = nullptr;
    int64_t ticket = 0;
    size_t bytes = 0;  // workspace of this request alone
    int status = NMF_EBUSY;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

}  // namespace

struct nmf_server_s {
    int device = 0;
    size_t budget = 0;
    std::vector<nmf_handle> handles;
    std::vector<size_t> held;  // workspace bytes held by each slot
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::unordered_map<int64_t, Request*> all;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_ticket = 0;
    int64_t running = 0, completed = 0;
    nmf_handle sizer = nullptr;  // workspace estimates (used under mu)
    int max_batch = kMaxBatch;   // requests a slot takes at once (NMF_SERVE_MAX_BATCH)

    size_t held_except(int i) const {
        size_t s = 0;
        for (size_t j = 0; j < held.size(); ++j)
            if ((int)j != i) s += held[j];
        return s;
    }
    bool fits(int i, size_t bytes) const {
        return budget == 0 || held_except(i) + std::max(held[i], bytes) <= budget;
    }
    // Workspace of the first `count` queued requests solved together.
    size_t group_bytes(int count) {
        std::vector<nmf_problem> g(count);
        for (int k = 0; k < count; ++k) g[k] = *queue[k]->prob;
        const int64_t b = nmf_workspace_bytes(sizer, g.data(), count);
        return b < 0 ? SIZE_MAX : (size_t)b;
    }
};

namespace {

void worker_loop(nmf_server_s* s, int i) {
    std::unique_lock<std::mutex> lk(s->mu);
    std::vector<Request*> batch;
    std::vector<nmf_problem> probs;
    for (;;) {
        s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
        if (s->queue.empty()) {
            if (s->stop) return;
            continue;
        }
        if (!s->fits(i, s->queue.front()->bytes)) {
            // this slot is idle: give its workspace back so the head can fit, then
            // wait for running requests to finish (and their slots to do the same)
            if (s->held[i] > 0) {
                lk.unlock();
                nmf_release_workspace(s->handles[i]);
                lk.lock();
                s->held[i] = 0;
                s->cv.notify_all();
                continue;
            }
            s->cv.wait_for(lk, std::chrono::milliseconds(1));
            continue;
        }
        // the longest run from the head that fits together
        int count = 1;
        size_t bytes = s->queue.front()->bytes;
        const int most = std::min<int>(s->max_batch, (int)s->queue.size());
        while (count < most) {
            const size_t b = s->group_bytes(count + 1);
            if (!s->fits(i, b)) break;
            bytes = b;
            ++count;
        }
        batch.assign(s->queue.begin(), s->queue.begin() + count);
        s->queue.erase(s->queue.begin(), s->queue.begin() + count);
        s->held[i] = std::max(s->held[i], bytes);
        s->running += count;
        lk.unlock();
        probs.resize(count);
        for (int k = 0; k < count; ++k) probs[k] = *batch[k]->prob;
        const int rc = nmf_solve_batch(s->handles[i], probs.data(), count);
        lk.lock();
        const Clock::time_point now = Clock::now();
        for (int k = 0; k < count; ++k) {
            Request* r = batch[k];
            r->prob->status = probs[k].status;
            r->prob->sweeps_run = probs[k].sweeps_run;
            r->prob->objective = probs[k].objective;
            r->status = probs[k].status != NMF_OK ? probs[k].status : rc;
            r->done = true;
            r->t_done = now;
        }
        s->running -= count;
        s->completed += count;
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

int nmf_server_create(nmf_server* out, int device, size_t hbm_budget_bytes, int slots, nmf_precision prec) {
    if (!out || slots < 1 || slots > 64) return NMF_EINVAL;
    *out = nullptr;
    nmf_server_s* s = new nmf_server_s;
    s->device = device;
    s->budget = hbm_budget_bytes;
    for (int i = 0; i < slots; ++i) {
        nmf_handle h = nullptr;
        const int rc = nmf_create(&h, device, 0, prec);
        if (rc) {
            for (nmf_handle x : s->handles) nmf_destroy(x);
            delete s;
            return rc;
        }
        s->handles.push_back(h);
    }
    if (nmf_create(&s->sizer, device, 0, prec)) {
        for (nmf_handle x : s->handles) nmf_destroy(x);
        delete s;
        return NMF_ECUDA;
    }
    s->held.assign(slots, 0);
    if (const char* e = std::getenv("NMF_SERVE_MAX_BATCH")) {
        const int v = std::atoi(e);
        if (v >= 1) s->max_batch = std::min(v, kMaxBatch);
    }
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_loop, s, i);
    *out = s;
    return NMF_OK;
}

int64_t nmf_server_submit(nmf_server s, nmf_problem* prob) {
    if (!s || !prob) return NMF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t bytes = nmf_workspace_bytes(s->sizer, prob, 1);
    if (bytes < 0) return bytes;
    if (s->budget && (size_t)bytes > s->budget) return NMF_ENOMEM;
    Request* r = new Request;
    r->prob = prob;
    r->bytes = (size_t)bytes;
    r->t_submit = Clock::now();
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    s->cv.notify_all();
    return r->ticket;
}

int nmf_server_poll(nmf_server s, int64_t ticket, int wait_ms, double* latency_ms) {
    if (!s) return NMF_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return NMF_EINVAL;
    Request* r = it->second;
    if (!r->done) {
        if (wait_ms < 0)
            s->cv.wait(lk, [&] { return r->done; });
        else if (wait_ms > 0)
            s->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; });
    }
    if (!r->done) return NMF_EBUSY;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    const int st = r->status;
    s->all.erase(it);
    delete r;
    return st;
}

int nmf_server_stats(nmf_server s, int64_t* queued, int64_t* running, int64_t* completed, int64_t* bytes_held) {
    if (!s) return NMF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = s->running;
    if (completed) *completed = s->completed;
    if (bytes_held) {
        size_t b = 0;
        for (size_t h : s->held) b += h;
        *bytes_held = (int64_t)b;
    }
    return NMF_OK;
}

void nmf_server_destroy(nmf_server s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
        s->stop = true;
        s->cv.notify_all();
    }
    for (std::thread& t : s->workers) t.join();
    for (nmf_handle h : s->handles) nmf_destroy(h);
    nmf_destroy(s->sizer);
    for (auto& kv : s->all) delete kv.second;
    delete s;
}

}  // extern "C"
