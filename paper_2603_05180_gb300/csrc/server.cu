// Continuous-batching query server over one index (the engine's serving
// extension; the paper has no serving loop).  Host runtime in C++: requests arrive one at a
// time from any thread; a dispatcher thread takes the oldest waiting requests as
// one batch whatever their parameters (one crisp_search with per-query
// parameters), admits it when a stream slot is free and the search's scratch
// fits the memory budget, and runs copy-in, crisp_search and copy-out on that
// slot's stream.  Batches on different slots overlap on the
// GPU; completions are found by polling each slot's event.  Every request keeps
// its arrival and completion time, from which p50 / p99 latency follow.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    std::vector<float> q;
    crisp_search_params p;
    int state = 0;                  // 0 waiting, 1 on the GPU, 2 done, 3 failed
    crisp_status err = CRISP_OK;
    std::string msg;
    std::vector<int64_t> ids;
    std::vector<float> d2;
    crisp_query_stats st{};
    Clock::time_point t_arrive, t_done;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    int32_t ko = 0;                 // result row length of the batch (its largest k)
    size_t scratch = 0;
    float *hQ = nullptr, *hD = nullptr, *dQ = nullptr, *dD = nullptr;
    int64_t *hI = nullptr, *dI = nullptr;
    crisp_query_stats *hS = nullptr, *dS = nullptr;
};

}  // namespace

struct crisp_server {
    const crisp_index *ix = nullptr;
    crisp_server_params prm{};
    int device = 0;
    std::vector<Slot> slots;
    std::deque<uint64_t> waiting;   // waiting requests, oldest first
    size_t n_waiting = 0;
    std::unordered_map<uint64_t, Req> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t scratch_in_use = 0, scratch_peak = 0;
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_requests = 0;
    std::vector<double> lat_us;
};

static void release_slot_buffers(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.hQ);
    cudaFreeHost(s.hI);
    cudaFreeHost(s.hD);
    cudaFreeHost(s.hS);
    cudaFree(s.dQ);
    cudaFree(s.dI);
    cudaFree(s.dD);
    cudaFree(s.dS);
    if (s.event) cudaEventDestroy(s.event);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

// Collect finished batches: results to their requests, slot and scratch freed.
static bool reap(crisp_server *sv) {
    bool any = false;
    for (Slot &s : sv->slots) {
        if (!s.busy) continue;
        cudaError_t e = cudaEventQuery(s.event);
        if (e == cudaErrorNotReady) continue;
        const Clock::time_point now = Clock::now();
        for (size_t i = 0; i < s.tickets.size(); ++i) {
            Req &r = sv->reqs[s.tickets[i]];
            if (e != cudaSuccess) {
                r.state = 3;
                r.err = CRISP_ECUDA;
                r.msg = cudaGetErrorString(e);
                sv->failed++;
                continue;
            }
            r.ids.assign(s.hI + i * s.ko, s.hI + i * s.ko + r.p.k);
            r.d2.assign(s.hD + i * s.ko, s.hD + i * s.ko + r.p.k);
            r.st = s.hS[i];
            r.state = 2;
            r.t_done = now;
            sv->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_arrive).count());
            sv->completed++;
        }
        sv->scratch_in_use -= s.scratch;
        s.busy = false;
        s.tickets.clear();
        any = true;
    }
    if (any) sv->cv_done.notify_all();
    return any;
}

// Admit the oldest waiting requests (arrival order, up to max_batch, any mix of
// parameters) onto a free slot.
static bool admit(crisp_server *sv) {
    if (sv->n_waiting == 0) return false;
    Slot *free_slot = nullptr;
    bool any_busy = false;
    for (Slot &s : sv->slots) {
        if (!s.busy && !free_slot) free_slot = &s;
        any_busy |= s.busy;
    }
    if (!free_slot) return false;
    const int32_t n = (int32_t)std::min<size_t>(sv->waiting.size(), (size_t)sv->prm.max_batch);
    std::vector<crisp_search_params> prm((size_t)n);
    int32_t ko = 1;
    for (int32_t i = 0; i < n; ++i) {
        prm[i] = sv->reqs[sv->waiting[i]].p;
        ko = std::max(ko, prm[i].k);
    }
    size_t need = 0;
    crisp_status st = crisp_search_scratch_bytes(sv->ix, n, prm.data(), n, &need);
    if (st == CRISP_OK && any_busy && sv->scratch_in_use + need > (size_t)sv->prm.scratch_budget) return false;
    std::vector<uint64_t> batch(sv->waiting.begin(), sv->waiting.begin() + n);
    sv->waiting.erase(sv->waiting.begin(), sv->waiting.begin() + n);   // the requests leave the queue either way
    sv->n_waiting -= (size_t)n;
    Slot &s = *free_slot;
    const int32_t D = sv->ix->D;
    for (int32_t i = 0; i < n; ++i) memcpy(s.hQ + (size_t)i * D, sv->reqs[batch[i]].q.data(), sizeof(float) * D);
    cudaError_t e = cudaSuccess;
    if (st == CRISP_OK) {
        e = cudaMemcpyAsync(s.dQ, s.hQ, sizeof(float) * (size_t)n * D, cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess) st = crisp_search(sv->ix, s.dQ, n, prm.data(), n, s.dI, s.dD, ko, s.dS, s.stream);
        else st = CRISP_ECUDA;
    }
    if (st == CRISP_OK) {
        e = cudaMemcpyAsync(s.hI, s.dI, sizeof(int64_t) * (size_t)n * ko, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.hD, s.dD, sizeof(float) * (size_t)n * ko, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.hS, s.dS, sizeof(crisp_query_stats) * n, cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.event, s.stream);
        if (e != cudaSuccess) st = CRISP_ECUDA;
    }
    if (st != CRISP_OK) {
        const char *m = crisp_last_error();
        for (uint64_t t : batch) {
            Req &r = sv->reqs[t];
            r.state = 3;
            r.err = st;
            r.msg = m ? m : "";
            sv->failed++;
        }
        sv->cv_done.notify_all();
        return true;
    }
    for (uint64_t t : batch) sv->reqs[t].state = 1;
    s.busy = true;
    s.tickets = batch;
    s.ko = ko;
    s.scratch = need;
    sv->scratch_in_use += need;
    sv->scratch_peak = std::max(sv->scratch_peak, sv->scratch_in_use);
    sv->batches++;
    sv->batched_requests += n;
    return true;
}

static void run(crisp_server *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool busy = false;
        for (Slot &s : sv->slots) busy |= s.busy;
        if (sv->stop && sv->n_waiting == 0 && !busy) break;
        bool progress = reap(sv);
        while (admit(sv)) progress = true;
        if (!progress) {
            busy = false;
            for (Slot &s : sv->slots) busy |= s.busy;
            // poll the GPU every 20 us while work is in flight, else sleep until a submit
            if (busy) sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

extern "C" crisp_status crisp_server_create(const crisp_index *ix, const crisp_server_params *p, crisp_server **out) {
    CRISP_REQUIRE(ix && p && out, "crisp_server_create: null pointer");
    CRISP_REQUIRE(p->streams >= 1 && p->streams <= 64, "crisp_server_create: streams outside [1, 64]");
    CRISP_REQUIRE(p->max_batch >= 1, "crisp_server_create: max_batch < 1");
    CRISP_REQUIRE(p->scratch_budget >= 0, "crisp_server_create: scratch_budget < 0");
    crisp_server *sv = new crisp_server();
    sv->ix = ix;
    sv->prm = *p;
    sv->device = ix->device;
    cudaSetDevice(sv->device);
    if (sv->prm.scratch_budget == 0) {
        // default: half the device memory free now, between 8 and 64 GiB
        size_t free_b = 0, total_b = 0;
        int64_t b = (int64_t)8 << 30;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
            b = std::min<int64_t>(std::max<int64_t>(b, (int64_t)(free_b / 2)), (int64_t)64 << 30);
        else cudaGetLastError();
        sv->prm.scratch_budget = b;
    }
    sv->slots.resize(p->streams);
    const size_t B = (size_t)p->max_batch, D = (size_t)ix->D, KO = CRISP_KOUT_MAX;
    for (Slot &s : sv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&s.hQ, sizeof(float) * B * D);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&s.hI, sizeof(int64_t) * B * KO);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&s.hD, sizeof(float) * B * KO);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&s.hS, sizeof(crisp_query_stats) * B);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.dQ, sizeof(float) * B * D);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.dI, sizeof(int64_t) * B * KO);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.dD, sizeof(float) * B * KO);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s.dS, sizeof(crisp_query_stats) * B);
        if (e != cudaSuccess) {
            for (Slot &x : sv->slots) release_slot_buffers(x);
            delete sv;
            return crisp_cuda_fail(e, "crisp_server_create", __FILE__, __LINE__);
        }
    }
    sv->worker = std::thread(run, sv);
    *out = sv;
    return CRISP_OK;
}

static crisp_status submit_at(crisp_server *sv, const float *q, const crisp_search_params *p, Clock::time_point t_arrive,
                              uint64_t *ticket) {
    size_t probe = 0;
    crisp_status st = crisp_search_scratch_bytes(sv->ix, 1, p, 1, &probe);   // validates the parameters
    if (st) return st;
    Req r;
    r.q.assign(q, q + sv->ix->D);
    r.p = *p;
    r.t_arrive = t_arrive;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        CRISP_REQUIRE(!sv->stop, "crisp_server_submit: server is stopping");
        *ticket = sv->next_ticket++;
        sv->reqs.emplace(*ticket, std::move(r));
        sv->waiting.push_back(*ticket);
        sv->n_waiting++;
        sv->submitted++;
    }
    sv->cv_work.notify_one();
    return CRISP_OK;
}

extern "C" crisp_status crisp_server_submit(crisp_server *sv, const float *q, const crisp_search_params *p,
                                            uint64_t *ticket) {
    CRISP_REQUIRE(sv && q && p && ticket, "crisp_server_submit: null pointer");
    return submit_at(sv, q, p, Clock::now(), ticket);
}

extern "C" crisp_status crisp_server_replay(crisp_server *sv, const float *Q, int32_t nq, int64_t n,
                                            const int32_t *qidx, const crisp_search_params *params,
                                            int32_t n_params, const int32_t *pidx, const double *arrival_us, int32_t kmax,
                                            int64_t *ids, float *sqdist, double *latency_us, double *wall_us) {
    CRISP_REQUIRE(sv && Q && qidx && params && pidx && arrival_us && ids && sqdist && latency_us,
                  "crisp_server_replay: null pointer");
    CRISP_REQUIRE(nq >= 1 && n >= 0 && kmax >= 1 && n_params >= 1,
                  "crisp_server_replay: nq < 1, n < 0, kmax < 1 or n_params < 1");
    for (int64_t i = 0; i < n; ++i) {
        CRISP_REQUIRE(qidx[i] >= 0 && qidx[i] < nq, "crisp_server_replay: qidx[%lld] outside [0, nq)", (long long)i);
        CRISP_REQUIRE(pidx[i] >= 0 && pidx[i] < n_params, "crisp_server_replay: pidx[%lld] outside [0, n_params)",
                      (long long)i);
        CRISP_REQUIRE(params[pidx[i]].k <= kmax, "crisp_server_replay: request %lld has k > kmax", (long long)i);
        CRISP_REQUIRE(i == 0 || arrival_us[i] >= arrival_us[i - 1], "crisp_server_replay: arrivals not sorted");
    }
    const int32_t D = sv->ix->D;
    std::vector<uint64_t> tickets((size_t)n);
    const Clock::time_point t0 = Clock::now();
    // open loop: request i enters at t0 + arrival_us[i] whatever the server's state;
    // its latency counts from that scheduled time even if this thread runs late
    for (int64_t i = 0; i < n; ++i) {
        const Clock::time_point due = t0 + std::chrono::nanoseconds((int64_t)(arrival_us[i] * 1e3));
        while (Clock::now() < due) {
            if (due - Clock::now() > std::chrono::microseconds(200)) std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        crisp_status st = submit_at(sv, Q + (size_t)qidx[i] * D, &params[pidx[i]], due, &tickets[(size_t)i]);
        if (st) {
            for (int64_t j = 0; j < i; ++j) crisp_server_wait(sv, tickets[(size_t)j], -1, nullptr, nullptr, nullptr, nullptr);
            return st;
        }
    }
    crisp_status first_err = CRISP_OK;
    for (int64_t i = 0; i < n; ++i) {
        int64_t *oi = ids + (size_t)i * kmax;
        float *od = sqdist + (size_t)i * kmax;
        for (int32_t j = 0; j < kmax; ++j) {
            oi[j] = -1;
            od[j] = INFINITY;
        }
        latency_us[i] = NAN;
        crisp_status st = crisp_server_wait(sv, tickets[(size_t)i], -1, oi, od, nullptr, &latency_us[i]);
        if (st && !first_err) first_err = st;
    }
    if (wall_us) *wall_us = std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    return first_err;
}

extern "C" crisp_status crisp_server_wait(crisp_server *sv, uint64_t ticket, int32_t timeout_ms, int64_t *ids,
                                          float *sqdist, crisp_query_stats *stats, double *latency_us) {
    CRISP_REQUIRE(sv, "crisp_server_wait: null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    CRISP_REQUIRE(it != sv->reqs.end(), "crisp_server_wait: unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (it->second.state < 2) {
        if (timeout_ms >= 0 && Clock::now() >= deadline) {
            crisp_set_error("crisp_server_wait: request %llu not finished within %d ms", (unsigned long long)ticket,
                            timeout_ms);
            return CRISP_ETIMEOUT;
        }
        if (timeout_ms >= 0) sv->cv_done.wait_until(lk, deadline);
        else sv->cv_done.wait(lk);
        it = sv->reqs.find(ticket);
    }
    Req &r = it->second;
    crisp_status st = r.state == 2 ? CRISP_OK : r.err;
    if (st == CRISP_OK) {
        if (ids) memcpy(ids, r.ids.data(), sizeof(int64_t) * r.ids.size());
        if (sqdist) memcpy(sqdist, r.d2.data(), sizeof(float) * r.d2.size());
        if (stats) *stats = r.st;
        if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_arrive).count();
    } else {
        crisp_set_error("crisp_server_wait: request %llu failed: %s", (unsigned long long)ticket, r.msg.c_str());
    }
    sv->reqs.erase(it);
    return st;
}

extern "C" crisp_status crisp_server_get_stats(crisp_server *sv, crisp_server_stats *out) {
    CRISP_REQUIRE(sv && out, "crisp_server_get_stats: null pointer");
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof *out);
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->batches = sv->batches;
    out->mean_batch = sv->batches ? (double)sv->batched_requests / (double)sv->batches : 0.0;
    out->scratch_peak = (int64_t)sv->scratch_peak;
    if (!sv->lat_us.empty()) {
        std::vector<double> v = sv->lat_us;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        out->p50_us = q(0.50);
        out->p99_us = q(0.99);
        out->max_us = v.back();
        double s = 0.0;
        for (double x : v) s += x;
        out->mean_us = s / (double)v.size();
    }
    return CRISP_OK;
}

extern "C" crisp_status crisp_server_reset_stats(crisp_server *sv) {
    CRISP_REQUIRE(sv, "crisp_server_reset_stats: null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->lat_us.clear();
    sv->completed = sv->failed = sv->batches = sv->batched_requests = 0;
    sv->submitted = sv->n_waiting;
    sv->scratch_peak = sv->scratch_in_use;
    return CRISP_OK;
}

extern "C" void crisp_server_destroy(crisp_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot &s : sv->slots) release_slot_buffers(s);
    delete sv;
}
