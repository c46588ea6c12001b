// Serving loop: continuous batching of optimization requests over several
// concurrent device batches.
//
// A server owns `slots` contexts, each with its own CUDA stream and device
// workspace.  Requests are copied and queued on submit.  Whenever a slot is
// free, the queue's head forms its next device batch: requests join in
// arrival order while the batch stays within max_batch queries and the
// slot's memo budget (admission by memo memory).  Batches of different slots
// run concurrently on the GPU, so requests that arrive while others are on
// the device start as soon as a slot frees up instead of waiting for one
// global batch.  Progress is driven by the caller (submit / poll): no thread
// of the library runs in the background.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mpdp.h"
#include "mpdp_launch.h"
#include "mpdp_persist.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int n = 0, m = 0;
    std::vector<double> card;
    std::vector<mpdp_edge> edges;
    Clock::time_point t_submit;
    Clock::time_point t_done;
    int state = 0;  // 0 queued, 1 on the device, 2 done
    int status = MPDP_OK;
    double cost = 0.0;
    std::vector<mpdp_plan_node> nodes;
};

struct Slot {
    mpdp_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<int64_t> tickets;
    std::vector<int64_t> handles;
};

}  // namespace

struct mpdp_server {
    int device = 0;
    mpdp_server_config cfg{};
    std::vector<Slot> slots;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Request> reqs;
    std::deque<int64_t> unreported;  // finished, not yet returned by a poll
    int64_t next_ticket = 0;
    int running = 0;
    mpdp::PersistEngine* engine = nullptr;  // persistent mode
    std::vector<int> free_slots;            // persistent mode: query slots without a request
};

namespace {

const mpdp_server_config kDefaultServer = {4, 256, 0, {MPDP_MEMO_DENSE, MPDP_ENUM_AUTO, 64, 1, 0, 32,
                                                       MPDP_FILTER_CONNECTED, 8, 4, 1, 18}, 0, 0};
constexpr size_t kDefaultSlotBudget = (size_t)16 << 30;

size_t slot_budget(const mpdp_server* s)
{
    return s->cfg.slot_budget_bytes ? (size_t)s->cfg.slot_budget_bytes : kDefaultSlotBudget;
}

// Move finished batches' plans into their requests.
int collect(mpdp_server* s, Slot& sl, Clock::time_point now)
{
    const int count = (int)sl.handles.size();
    std::vector<mpdp_plan_node> nodes((size_t)count * MPDP_PLAN_STRIDE);
    std::vector<int32_t> nn(count), st(count);
    std::vector<double> cost(count);
    const int rc = mpdp_get_plans(sl.ctx, sl.handles.data(), count, nodes.data(), MPDP_PLAN_STRIDE, nn.data(),
                                  cost.data(), st.data(), nullptr);
    for (int i = 0; i < count; i++) {
        Request& r = s->reqs[sl.tickets[i]];
        s->unreported.push_back(sl.tickets[i]);
        r.state = 2;
        r.t_done = now;
        r.status = st[i];
        r.cost = cost[i];
        r.nodes.assign(nodes.begin() + (size_t)i * MPDP_PLAN_STRIDE,
                       nodes.begin() + (size_t)i * MPDP_PLAN_STRIDE + nn[i]);
    }
    sl.busy = false;
    sl.tickets.clear();
    sl.handles.clear();
    s->running--;
    return rc == MPDP_ERR_BAD_HANDLE ? MPDP_ERR_INTERNAL : MPDP_OK;
}

// Form and enqueue the next batch of a free slot from the queue's head.
int launch(mpdp_server* s, Slot& sl)
{
    std::vector<int> ns, ms;
    std::vector<int64_t> take;
    const size_t budget = slot_budget(s);
    while (!s->queue.empty() && (int)take.size() < s->cfg.max_batch) {
        const Request& r = s->reqs[s->queue.front()];
        ns.push_back(r.n);
        ms.push_back(r.m);
        if (mpdp::batch_workspace_bytes(ns.data(), ms.data(), (int)ns.size(), s->cfg.kernel) > budget) {
            ns.pop_back();
            ms.pop_back();
            break;
        }
        take.push_back(s->queue.front());
        s->queue.pop_front();
    }
    if (take.empty()) return MPDP_OK;
    std::vector<mpdp_query> qs(take.size());
    for (size_t i = 0; i < take.size(); i++) {
        const Request& r = s->reqs[take[i]];
        mpdp_query& q = qs[i];
        memset(&q, 0, sizeof(q));
        q.n_rels = r.n;
        q.n_edges = r.m;
        q.card = r.card.data();
        q.edges = r.edges.empty() ? nullptr : r.edges.data();
        q.cost_model = MPDP_COST_COUT;
        q.mode = MPDP_MODE_EXACT;
    }
    sl.handles.assign(take.size(), -1);
    const int rc = mpdp_optimize_batch(sl.ctx, qs.data(), (int)qs.size(), sl.handles.data());
    if (rc != MPDP_OK) {
        // the batch was rejected whole: report it on every request
        for (int64_t t : take) {
            Request& r = s->reqs[t];
            r.state = 2;
            r.status = rc;
            r.t_done = Clock::now();
            s->unreported.push_back(t);
        }
        sl.handles.clear();
        return MPDP_OK;
    }
    for (int64_t t : take) s->reqs[t].state = 1;
    sl.tickets = take;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    sl.busy = true;
    s->running++;
    return MPDP_OK;
}

// Persistent mode: collect finished requests, hand queued ones to free slots.
int progress_persistent(mpdp_server* s)
{
    std::vector<mpdp::PersistResult> fin;
    int rc = mpdp::persist_poll(s->engine, fin);
    if (rc != MPDP_OK) return rc;
    const Clock::time_point now = Clock::now();
    for (mpdp::PersistResult& f : fin) {
        Request& r = s->reqs[f.ticket];
        r.state = 2;
        r.t_done = now;
        r.status = f.status;
        r.cost = f.cost;
        r.nodes = std::move(f.nodes);
        s->unreported.push_back(f.ticket);
        s->free_slots.push_back(f.slot);
        s->running--;
    }
    while (!s->queue.empty() && !s->free_slots.empty()) {
        const int64_t t = s->queue.front();
        Request& r = s->reqs[t];
        const int slot = s->free_slots.back();
        rc = mpdp::persist_submit(s->engine, slot, t, r.n, r.m, r.card.data(), r.edges.empty() ? nullptr : r.edges.data());
        if (rc != MPDP_OK) return rc;
        s->free_slots.pop_back();
        s->queue.pop_front();
        r.state = 1;
        s->running++;
    }
    return MPDP_OK;
}

int progress(mpdp_server* s, int64_t* done, int32_t cap, int32_t* count)
{
    if (s->engine) {
        const int rc = progress_persistent(s);
        if (rc != MPDP_OK) return rc;
        int found = 0;
        while (done && found < cap && !s->unreported.empty()) {
            done[found++] = s->unreported.front();
            s->unreported.pop_front();
        }
        if (count) *count = found;
        return MPDP_OK;
    }
    const Clock::time_point now = Clock::now();
    for (Slot& sl : s->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            cudaGetLastError();
            return MPDP_ERR_CUDA;
        }
        const int rc = collect(s, sl, now);
        if (rc != MPDP_OK) return rc;
    }
    for (Slot& sl : s->slots) {
        if (s->queue.empty()) break;
        if (sl.busy) continue;
        const int rc = launch(s, sl);
        if (rc != MPDP_OK) return rc;
    }
    // report finished tickets, oldest first; the rest wait for the next poll
    int found = 0;
    while (done && found < cap && !s->unreported.empty()) {
        done[found++] = s->unreported.front();
        s->unreported.pop_front();
    }
    if (count) *count = found;
    return MPDP_OK;
}

}  // namespace

extern "C" {

int mpdp_server_default_config(mpdp_server_config* cfg)
{
    if (!cfg) return MPDP_ERR_INVALID_ARG;
    *cfg = kDefaultServer;
    return MPDP_OK;
}

int mpdp_server_create(mpdp_server** out, int device, const mpdp_server_config* cfg)
{
    if (!out) return MPDP_ERR_INVALID_ARG;
    *out = nullptr;
    const mpdp_server_config c = cfg ? *cfg : kDefaultServer;
    if (c.persistent != 0 && c.persistent != 1) return MPDP_ERR_INVALID_ARG;
    if (c.persistent) {
        if (c.slots < 1 || c.slots > 1024) return MPDP_ERR_INVALID_ARG;
    } else if (c.slots < 1 || c.slots > 16 || c.max_batch < 1 || c.max_batch > 1024) {
        return MPDP_ERR_INVALID_ARG;
    }
    mpdp_server* s = new mpdp_server();
    s->device = device;
    s->cfg = c;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return MPDP_ERR_CUDA;
    }
    if (c.persistent) {
        const int max_rels = mpdp::persist_max_rels(c.slot_budget_bytes);
        const int rc = max_rels < 2 ? MPDP_ERR_INVALID_ARG
                                    : mpdp::persist_create(&s->engine, device, c.slots, max_rels, c.kernel);
        if (rc != MPDP_OK) {
            delete s;
            return rc;
        }
        for (int i = c.slots - 1; i >= 0; i--) s->free_slots.push_back(i);
        *out = s;
        return MPDP_OK;
    }
    s->slots.resize(c.slots);
    int rc = MPDP_OK;
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            rc = MPDP_ERR_CUDA;
            break;
        }
        rc = mpdp_create(&sl.ctx, device, slot_budget(s), sl.stream);
        if (rc != MPDP_OK) break;
        rc = mpdp_set_config(sl.ctx, &c.kernel);
        if (rc != MPDP_OK) break;
    }
    if (rc != MPDP_OK) {
        mpdp_server_destroy(s);
        return rc;
    }
    *out = s;
    return MPDP_OK;
}

void mpdp_server_destroy(mpdp_server* s)
{
    if (!s) return;
    if (s->engine) mpdp::persist_destroy(s->engine);
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ctx) mpdp_destroy(sl.ctx);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    cudaGetLastError();
    delete s;
}

int mpdp_server_submit(mpdp_server* s, const mpdp_query* q, int64_t* ticket)
{
    if (!s || !q || !ticket) return MPDP_ERR_INVALID_ARG;
    *ticket = -1;
    const int n = q->n_rels, m = q->n_edges;
    if (q->mode != MPDP_MODE_EXACT) return MPDP_ERR_INVALID_ARG;
    // the checks a batch would apply, here, so that one bad request cannot
    // get a whole batch rejected
    const int vrc = mpdp::validate_host_query(q);
    if (vrc != MPDP_OK) return vrc;
    if (s->engine ? n > mpdp::persist_max_rels(s->engine)
                  : mpdp::batch_workspace_bytes(&n, &m, 1, s->cfg.kernel) > slot_budget(s))
        return MPDP_ERR_ADMISSION;
    if (cudaSetDevice(s->device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    const int64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.n = n;
    r.m = m;
    r.card.assign(q->card, q->card + n);
    r.edges.assign(q->edges, q->edges + m);
    r.t_submit = Clock::now();
    s->queue.push_back(t);
    *ticket = t;
    return progress(s, nullptr, 0, nullptr);
}

int mpdp_server_poll(mpdp_server* s, int64_t* done, int32_t cap, int32_t* count)
{
    if (!s || cap < 0 || (cap > 0 && !done)) return MPDP_ERR_INVALID_ARG;
    if (count) *count = 0;
    if (cudaSetDevice(s->device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    return progress(s, done, cap, count);
}

int mpdp_server_drain(mpdp_server* s)
{
    if (!s) return MPDP_ERR_INVALID_ARG;
    if (cudaSetDevice(s->device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    if (s->engine) {
        // the kernel finishes every request it holds; bounded wait
        const Clock::time_point limit = Clock::now() + std::chrono::seconds(300);
        while (!s->queue.empty() || s->running > 0) {
            const int rc = progress(s, nullptr, 0, nullptr);
            if (rc != MPDP_OK) return rc;
            if (Clock::now() > limit) return MPDP_ERR_TIMEOUT;
            if (s->running > 0) std::this_thread::sleep_for(std::chrono::microseconds(5));
        }
        return MPDP_OK;
    }
    while (!s->queue.empty() || s->running > 0) {
        for (Slot& sl : s->slots)
            if (sl.busy && cudaEventSynchronize(sl.done) != cudaSuccess) {
                cudaGetLastError();
                return MPDP_ERR_CUDA;
            }
        const int rc = progress(s, nullptr, 0, nullptr);
        if (rc != MPDP_OK) return rc;
    }
    return MPDP_OK;
}

int mpdp_server_pending(const mpdp_server* s, int32_t* queued, int32_t* running)
{
    if (!s) return MPDP_ERR_INVALID_ARG;
    if (queued) *queued = (int32_t)s->queue.size();
    if (running && s->engine) {
        *running = mpdp::persist_busy(s->engine);
        return MPDP_OK;
    }
    if (running) {
        int r = 0;
        for (const Slot& sl : s->slots) r += sl.busy ? (int)sl.tickets.size() : 0;
        *running = r;
    }
    return MPDP_OK;
}

int mpdp_server_result(mpdp_server* s, int64_t ticket, mpdp_plan_node* nodes, int32_t cap, int32_t* n_nodes,
                       double* cost, double* latency_us)
{
    if (!s) return MPDP_ERR_INVALID_ARG;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return MPDP_ERR_BAD_HANDLE;
    Request& r = it->second;
    if (r.state != 2) return MPDP_ERR_NOT_READY;
    const int status = r.status;
    if (status == MPDP_OK) {
        if (nodes && cap < (int)r.nodes.size()) return MPDP_ERR_BUFFER_TOO_SMALL;
        if (nodes) memcpy(nodes, r.nodes.data(), r.nodes.size() * sizeof(mpdp_plan_node));
        if (n_nodes) *n_nodes = (int32_t)r.nodes.size();
        if (cost) *cost = r.cost;
    }
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    s->reqs.erase(it);
    return status;
}

}  // extern "C"
