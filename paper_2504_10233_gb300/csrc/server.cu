// Serving loop: continuous batching of walk requests with streaming edge
// updates integrated at epoch boundaries (the paper integrates all updates
// before each walk, Section 6 (ii)).
//
// A worker thread owns the graph.  Updates queue up and are applied as one
// batch once no walk launch is in flight; that starts a new epoch.  Walk
// requests are admitted while walker slots and device memory allow; requests
// admitted together share one persistent launch in request mode (each keeps
// its own seed, policy and local walker ids, so its paths are the same alone
// and in the mix), and up to `concurrent_launches` launches overlap on the
// device on separate streams.  Completion is observed with events (no device
// spin-waits); every host wait is bounded by the caller's timeout.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "bingo_host.h"

using namespace bingo;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    std::vector<uint32_t> starts;
    bingo_policy pol{};
    uint64_t seed = 0;
    double t_arrival = 0, t_admit = -1, t_done = -1;
    uint64_t epoch = 0;
    std::vector<uint32_t> paths, plen;
    int state = 0;  // 0 queued, 1 running, 2 done
    bingo_status status = BINGO_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t walkers = 0;
    uint32_t stride = 0;
    std::vector<Request*> reqs;
    Buf starts, paths, plen, pols, req_off, req_key, queue;
    std::vector<uint64_t> h_off, h_key;
    std::vector<bingo_policy> h_pol;
    std::vector<uint32_t> h_starts;
};

}  // namespace

struct bingo_server {
    bingo_graph* g = nullptr;
    bingo_server_config cfg{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    bool paused = false;       // bingo_server_pause: no admissions while set
    double t_created = 0;
    std::deque<bingo_update> updates;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1, epoch = 0, update_seq = 0;
    double updates_since = 0;  // arrival of the oldest queued update
    std::vector<Slot> slots;
    uint64_t inflight = 0;
    cudaStream_t ustream = nullptr;
    // stats
    uint64_t requests_done = 0, walkers_done = 0, steps_done = 0, updates_applied = 0, epochs = 0;
    std::vector<double> lat_ms;
    bingo_status worker_error = BINGO_OK;
};

namespace {

void complete_slot(bingo_server* S, Slot& sl) {
    // results: rows of the merged launch (stride sl.stride) into each request's buffers
    for (size_t ri = 0; ri < sl.reqs.size(); ri++) {
        Request* r = sl.reqs[ri];
        const uint32_t rs = r->pol.max_len + 1;
        const uint64_t n = r->starts.size();
        r->paths.resize(n * rs);
        r->plen.resize(n);
        const uint64_t off = sl.h_off[ri];
        cudaError_t e = cudaSuccess;
        if (n) {
            e = cudaMemcpy2D(r->paths.data(), rs * 4, (uint32_t*)sl.paths.p + off * sl.stride, sl.stride * 4, rs * 4, n,
                             cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(r->plen.data(), (uint32_t*)sl.plen.p + off, n * 4, cudaMemcpyDeviceToHost);
        }
        uint64_t steps = 0;
        for (uint32_t x : r->plen) steps += x - 1;
        std::lock_guard<std::mutex> lk(S->mu);
        r->status = e == cudaSuccess ? BINGO_OK : BINGO_E_CUDA;
        r->t_done = now_s();
        r->state = 2;
        S->requests_done++;
        S->walkers_done += n;
        S->steps_done += steps;
        S->lat_ms.push_back((r->t_done - r->t_arrival) * 1e3);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->inflight -= sl.walkers;
    sl.busy = false;
    sl.reqs.clear();
    S->cv_done.notify_all();
}

bool launch_slot(bingo_server* S, Slot& sl, std::vector<Request*>& batch, uint64_t epoch) {
    bingo_graph* g = S->g;
    uint64_t total = 0;
    uint32_t stride = 1;
    sl.h_off.clear();
    sl.h_key.clear();
    sl.h_pol.clear();
    sl.h_starts.clear();
    for (Request* r : batch) {
        sl.h_off.push_back(total);
        sl.h_key.push_back(r->seed);
        sl.h_pol.push_back(r->pol);
        sl.h_starts.insert(sl.h_starts.end(), r->starts.begin(), r->starts.end());
        total += r->starts.size();
        stride = std::max(stride, r->pol.max_len + 1);
    }
    sl.h_off.push_back(total);
    if (ensure(sl.starts, 4 * total + 4) || ensure(sl.paths, 4ull * total * stride + 4) || ensure(sl.plen, 4 * total + 4) ||
        ensure(sl.pols, sizeof(bingo_policy) * batch.size()) || ensure(sl.req_off, 8 * sl.h_off.size()) ||
        ensure(sl.req_key, 8 * batch.size()) || ensure(sl.queue, 64))
        return false;
    cudaStream_t s = sl.stream;
    cudaMemcpyAsync(sl.starts.p, sl.h_starts.data(), 4 * total, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sl.pols.p, sl.h_pol.data(), sizeof(bingo_policy) * batch.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sl.req_off.p, sl.h_off.data(), 8 * sl.h_off.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sl.req_key.p, sl.h_key.data(), 8 * batch.size(), cudaMemcpyHostToDevice, s);
    WalkReq q;
    q.nwalkers = total;
    q.starts = (const uint32_t*)sl.starts.p;
    q.dev_pols = (const bingo_policy*)sl.pols.p;
    q.npol = (uint32_t)batch.size();
    q.stride = stride;
    q.paths = (uint32_t*)sl.paths.p;
    q.plen = (uint32_t*)sl.plen.p;
    q.mode = BINGO_WALK_PERSISTENT;
    q.pad = true;
    q.queue = (unsigned long long*)sl.queue.p;
    q.req_off = (const uint64_t*)sl.req_off.p;
    q.req_key = (const uint64_t*)sl.req_key.p;
    q.nreq = (uint32_t)batch.size();
    if (walk_launch(g, q, s) != BINGO_OK) return false;
    cudaEventRecord(sl.done, s);
    sl.stride = stride;
    sl.walkers = total;
    sl.reqs = batch;
    sl.busy = true;
    const double ta = now_s();
    for (Request* r : batch) {
        r->state = 1;
        r->epoch = epoch;
        r->t_admit = ta;
    }
    return true;
}

void worker_main(bingo_server* S) {
    cudaSetDevice(S->g->device);
    const uint64_t max_walkers = S->cfg.max_inflight_walkers;
    const bool merge = !(S->cfg.flags & BINGO_SERVER_NO_MERGE);
    for (;;) {
        // 1. completions
        for (Slot& sl : S->slots)
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) complete_slot(S, sl);
        std::unique_lock<std::mutex> lk(S->mu);
        bool any_busy = false;
        for (Slot& sl : S->slots) any_busy |= sl.busy;
        if (S->stop && S->queue.empty() && S->updates.empty() && !any_busy) break;
        // 2. epoch boundary: apply queued updates once no launch reads the graph.  While launches are
        // in flight, admission continues until the oldest queued update has waited update_delay_us.
        const bool updates_due =
            !S->updates.empty() && (now_s() - S->updates_since) * 1e6 >= (double)S->cfg.update_delay_us;
        if (!S->updates.empty() && (updates_due || S->queue.empty())) {
            if (!any_busy) {
                const size_t nb = std::min<size_t>(S->updates.size(), S->cfg.max_update_batch);
                std::vector<bingo_update> batch(S->updates.begin(), S->updates.begin() + nb);
                S->updates.erase(S->updates.begin(), S->updates.begin() + nb);
                lk.unlock();
                bingo_update_stats st;
                bingo_status rc = bingo_apply_updates(S->g, batch.data(), batch.size(), S->ustream, &st);
                lk.lock();
                if (rc != BINGO_OK && S->worker_error == BINGO_OK) S->worker_error = rc;
                S->updates_applied += nb;
                S->epoch++;
                S->epochs++;
                S->updates_since = now_s();  // what remains queued now waits from this epoch on
                S->cv_done.notify_all();
                continue;
            }
        }
        if (!S->queue.empty() && !updates_due && !S->paused) {
            // 3. admission into a free slot
            Slot* free_slot = nullptr;
            for (Slot& sl : S->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            if (free_slot) {
                size_t fr = 0, tt = 0;
                cudaMemGetInfo(&fr, &tt);
                std::vector<Request*> batch;
                uint64_t w = 0, bytes = 0;
                while (!S->queue.empty()) {
                    Request* r = S->queue.front();
                    const uint64_t n = r->starts.size();
                    const uint64_t need = n * 4ull * (r->pol.max_len + 3);
                    if (!batch.empty() && (!merge || S->inflight + w + n > max_walkers || batch.size() >= 4096)) break;
                    // walker slots: a request waits for in-flight launches to free enough of them
                    if (batch.empty() && S->inflight + n > max_walkers && S->inflight > 0) break;
                    // device memory: a request is admitted only if its launch buffers leave hbm_reserve_bytes free;
                    // otherwise it waits (for launches or other users of the device to free memory)
                    if (bytes + need + S->cfg.hbm_reserve_bytes > fr) break;
                    batch.push_back(r);
                    S->queue.pop_front();
                    w += n;
                    bytes += need;
                }
                if (!batch.empty()) {
                    const uint64_t ep = S->epoch;
                    S->inflight += w;
                    lk.unlock();
                    const bool ok = launch_slot(S, *free_slot, batch, ep);
                    lk.lock();
                    if (!ok) {
                        S->inflight -= w;
                        for (Request* r : batch) {
                            r->state = 2;
                            r->status = BINGO_E_OOM;
                        }
                        S->cv_done.notify_all();
                    }
                    continue;
                }
            }
        }
        // 4. idle: wait for new work or poll launches
        S->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 2000));
    }
}

}  // namespace

extern "C" {

bingo_status bingo_server_create(bingo_graph* g, const bingo_server_config* cfg, bingo_server** out) {
    if (!g || !out) { set_error("NULL argument"); return BINGO_E_INVALID; }
    if (g->part) { set_error("server: a partition graph walks only through bingo_part_walk"); return BINGO_E_STATE; }
    bingo_server* S = new bingo_server();
    S->g = g;
    if (cfg) S->cfg = *cfg;
    if (!S->cfg.max_inflight_walkers) S->cfg.max_inflight_walkers = 4ull << 20;
    if (!S->cfg.hbm_reserve_bytes) S->cfg.hbm_reserve_bytes = 1ull << 30;
    if (!S->cfg.max_update_batch) S->cfg.max_update_batch = 65536;
    if (!S->cfg.concurrent_launches) S->cfg.concurrent_launches = 4;
    if (!S->cfg.max_len_cap) S->cfg.max_len_cap = 128;
    if (!S->cfg.update_delay_us) S->cfg.update_delay_us = 1000;
    S->t_created = now_s();
    S->slots.resize(S->cfg.concurrent_launches);
    for (Slot& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            set_error("server: stream/event creation failed");
            return BINGO_E_CUDA;
        }
    }
    cudaStreamCreateWithFlags(&S->ustream, cudaStreamNonBlocking);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return BINGO_OK;
}

bingo_status bingo_server_destroy(bingo_server* S) {
    if (!S) return BINGO_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot& sl : S->slots) {
        Buf* bs[] = {&sl.starts, &sl.paths, &sl.plen, &sl.pols, &sl.req_off, &sl.req_key, &sl.queue};
        for (Buf* b : bs) release(*b);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (S->ustream) cudaStreamDestroy(S->ustream);
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
    return BINGO_OK;
}

bingo_status bingo_server_submit_updates(bingo_server* S, const bingo_update* ups, uint64_t n, uint64_t* epoch) {
    if (!S || (n && !ups)) { set_error("NULL argument"); return BINGO_E_INVALID; }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { set_error("server stopping"); return BINGO_E_STATE; }
        if (S->updates.empty() && n) S->updates_since = now_s();
        for (uint64_t i = 0; i < n; i++) S->updates.push_back(ups[i]);
        if (epoch) *epoch = S->epoch + 1;
    }
    S->cv_work.notify_all();
    return BINGO_OK;
}

bingo_status bingo_server_submit_walk(bingo_server* S, const uint32_t* starts, uint64_t nwalkers,
                                      const bingo_policy* pol, uint64_t seed, uint64_t* ticket) {
    if (!S || !pol || !ticket || (nwalkers && !starts)) { set_error("NULL argument"); return BINGO_E_INVALID; }
    if (pol->kind > BINGO_NODE2VEC || pol->max_len > S->cfg.max_len_cap || nwalkers > S->cfg.max_inflight_walkers) {
        set_error("request exceeds server limits (kind, max_len cap %u, walker slots)", S->cfg.max_len_cap);
        return BINGO_E_INVALID;
    }
    if (pol->kind == BINGO_NODE2VEC && S->g->G.eh_mask == 0) {
        set_error("node2vec requests need the edge index: run one node2vec walk before starting the server");
        return BINGO_E_STATE;
    }
    Request* r = new Request();
    r->starts.assign(starts, starts + nwalkers);
    r->pol = *pol;
    r->seed = seed;
    r->t_arrival = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { delete r; set_error("server stopping"); return BINGO_E_STATE; }
        r->ticket = S->next_ticket++;
        S->reqs[r->ticket] = r;
        S->queue.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();
    return BINGO_OK;
}

bingo_status bingo_server_wait(bingo_server* S, uint64_t ticket, uint32_t timeout_ms, uint32_t* paths,
                               uint32_t* path_len, uint64_t* epoch) {
    if (!S) { set_error("NULL server"); return BINGO_E_INVALID; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return BINGO_E_INVALID; }
    Request* r = it->second;
    if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state == 2; })) {
        set_error("request %llu not done within %u ms", (unsigned long long)ticket, timeout_ms);
        return BINGO_E_TIMEOUT;
    }
    const bingo_status st = r->status;
    if (paths && !r->paths.empty()) memcpy(paths, r->paths.data(), 4 * r->paths.size());
    if (path_len && !r->plen.empty()) memcpy(path_len, r->plen.data(), 4 * r->plen.size());
    if (epoch) *epoch = r->epoch;
    S->reqs.erase(it);
    delete r;
    if (st != BINGO_OK) set_error("request failed");
    return st;
}

bingo_status bingo_server_drain(bingo_server* S, uint32_t timeout_ms) {
    if (!S) { set_error("NULL server"); return BINGO_E_INVALID; }
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        bool busy = false;
        for (Slot& sl : S->slots) busy |= sl.busy;
        if (S->queue.empty() && S->updates.empty() && !busy) break;
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            set_error("drain timed out");
            return BINGO_E_TIMEOUT;
        }
    }
    if (S->worker_error != BINGO_OK) {
        set_error("an update batch failed inside the server");
        return S->worker_error;
    }
    return BINGO_OK;
}

bingo_status bingo_server_pause(bingo_server* S, uint32_t paused) {
    if (!S) { set_error("NULL server"); return BINGO_E_INVALID; }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
    }
    S->cv_work.notify_all();
    return BINGO_OK;
}

bingo_status bingo_server_request_get(bingo_server* S, uint64_t ticket, bingo_server_request_info* out) {
    if (!S || !out) { set_error("NULL argument"); return BINGO_E_INVALID; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return BINGO_E_INVALID; }
    const Request* r = it->second;
    memset(out, 0, sizeof(*out));
    out->state = (uint32_t)r->state;
    out->status = (uint32_t)r->status;
    out->walkers = r->starts.size();
    out->epoch = r->epoch;
    const auto ms = [&](double t) { return t < 0 ? -1.0 : (t - S->t_created) * 1e3; };
    out->submit_ms = ms(r->t_arrival);
    out->admit_ms = ms(r->t_admit);
    out->done_ms = ms(r->t_done);
    return BINGO_OK;
}

bingo_status bingo_server_stats_get(bingo_server* S, bingo_server_stats* out) {
    if (!S || !out) { set_error("NULL argument"); return BINGO_E_INVALID; }
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->requests_done = S->requests_done;
    out->walkers_done = S->walkers_done;
    out->steps_done = S->steps_done;
    out->updates_applied = S->updates_applied;
    out->epochs = S->epochs;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t i = (size_t)std::min<double>(v.size() - 1, std::max<double>(0, p * (v.size() - 1) + 0.5));
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double x : v) s += x;
        out->mean_ms = s / v.size();
    }
    return BINGO_OK;
}

}  // extern "C"
