// server.cu -- continuous batching of independent NSGA-III runs on one GPU.
//
// Requests (m, d, N, divisions, generations, options) arrive at any time
// through nsga3_server_submit.  One worker thread owns the device work:
//   - admission: requests are taken in arrival order while a slot is free
//     and the device-memory budget can hold the run's workspace; a run's
//     context is carved out of one pre-allocated arena, so admission and
//     release never call cudaMalloc / cudaFree (cudaFree would synchronise
//     the whole device and stall every other run);
//   - execution: every admitted run owns a slot stream and advances by
//     chunks of generations (one CUDA-graph launch per generation), at most
//     two chunks queued per run, so runs of different sizes overlap on the
//     device and a new run starts as soon as it is admitted;
//   - completion: when a run's last chunk has finished, its population is
//     copied to host memory, its context is destroyed (workspace back to the
//     arena) and the slot is reused at once.
// Each run's random numbers depend only on its own seed and generation
// counter (Philox), so a run's result is the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "nsga3.h"
#include "runtime.h"

// ------------------------------------------------------------ arena ----
DeviceArena::DeviceArena(void* base, size_t bytes) : base_(static_cast<char*>(base)), cap_(bytes / kAlign * kAlign)
{
    if (cap_) free_[0] = cap_;
}

void* DeviceArena::alloc(size_t bytes)
{
    const size_t b = round_up(bytes ? bytes : 1);
    std::lock_guard<std::mutex> lk(mu_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < b) continue;
        const size_t off = it->first, rest = it->second - b;
        free_.erase(it);
        if (rest) free_[off + b] = rest;
        live_[off] = b;
        used_ += b;
        return base_ + off;
    }
    return nullptr;
}

void DeviceArena::release(void* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    const size_t off = static_cast<size_t>(static_cast<char*>(p) - base_);
    auto lv = live_.find(off);
    if (lv == live_.end()) return;
    size_t start = off, size = lv->second;
    used_ -= size;
    live_.erase(lv);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && next->first == off + size) {
        size += next->second;
        next = free_.erase(next);
    }
    if (next != free_.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == start) {
            start = prev->first;
            size += prev->second;
            free_.erase(prev);
        }
    }
    free_[start] = size;
}

size_t DeviceArena::in_use() const
{
    std::lock_guard<std::mutex> lk(mu_);
    return used_;
}

size_t DeviceArena::largest_free() const
{
    std::lock_guard<std::mutex> lk(mu_);
    size_t b = 0;
    for (const auto& f : free_) b = std::max(b, f.second);
    return b;
}

// ----------------------------------------------------------- server ----
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    nsga3_request r{};
    std::vector<float> W;
    size_t bytes = 0;
    double t_submit = 0;
};

struct Result {
    nsga3_run_info info{};
    std::vector<float> X, F;
    std::vector<int32_t> rank;
};

struct Chunk {
    cudaEvent_t ev;
    int gens;
};

struct Active {
    Request q;
    nsga3_ctx* ctx = nullptr;
    int slot = -1;
    int launched = 0, finished = 0;
    double t_admit = 0;
    std::deque<Chunk> inflight;
    nsga3_status st = NSGA3_OK;
    std::string msg;
};

}  // namespace

struct nsga3_server {
    int device = 0;
    void* arena_mem = nullptr;
    DeviceArena* arena = nullptr;
    int max_active = 1, chunk = 1;
    Clock::time_point t0;
    std::vector<cudaStream_t> slots;
    std::vector<int> free_slots;
    std::vector<cudaEvent_t> free_events;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;      // guarded by mu
    std::map<int64_t, Result> done;   // guarded by mu
    std::deque<int64_t> unclaimed;    // completed ids not yet returned by wait
    int64_t next_id = 0;
    bool stop = false;
    std::string err;

    // statistics (guarded by mu)
    int64_t submitted = 0, admitted = 0, completed = 0, peak_active = 0, n_active = 0, launches = 0;
    uint64_t peak_bytes = 0;

    std::thread worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void set_err(nsga3_server* s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = buf;
}

void copy_msg(nsga3_run_info& info, const std::string& m)
{
    snprintf(info.message, sizeof info.message, "%s", m.c_str());
}

void publish(nsga3_server* s, int64_t id, Result&& r)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->done[id] = std::move(r);
    s->unclaimed.push_back(id);
    s->completed += 1;
    s->cv_done.notify_all();
}

Result failed_result(const Request& q, nsga3_status st, const std::string& msg, double now)
{
    Result r;
    r.info.status = st;
    r.info.m = q.r.m;
    r.info.d = q.r.d;
    r.info.N = q.r.N;
    r.info.generations = q.r.generations;
    r.info.workspace_bytes = q.bytes;
    r.info.t_submit = q.t_submit;
    r.info.t_admit = -1.0;
    r.info.t_done = now;
    copy_msg(r.info, msg);
    return r;
}

cudaEvent_t take_event(nsga3_server* s)
{
    if (!s->free_events.empty()) {
        cudaEvent_t e = s->free_events.back();
        s->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Finishes a run whose queued work has completed (or failed): result to
// host memory, context destroyed without a device-wide synchronisation.
void retire(nsga3_server* s, Active& a)
{
    cudaStream_t st = s->slots[a.slot];
    Result r;
    r.info.m = a.q.r.m;
    r.info.d = a.q.r.d;
    r.info.N = a.q.r.N;
    r.info.generations = a.q.r.generations;
    r.info.workspace_bytes = a.q.bytes;
    r.info.t_submit = a.q.t_submit;
    r.info.t_admit = a.t_admit;
    nsga3_status status = a.st;
    std::string msg = a.msg;
    long long launches = 0;
    if (!status) {
        const int N = a.q.r.N;
        r.X.resize((size_t)N * a.q.r.d);
        r.F.resize((size_t)N * a.q.r.m);
        r.rank.resize(N);
        status = nsga3_get_population(a.ctx, r.X.data(), r.F.data(), r.rank.data(), st);
        if (!status) status = nsga3_sync(a.ctx, st);  // waits for the copies, reads the device status
        if (!status) status = ctx_launches(a.ctx, (void*)st, &launches);
        if (status) msg = nsga3_last_error(a.ctx);
    }
    cudaStreamSynchronize(st);
    cudaGetLastError();
    for (auto& c : a.inflight) s->free_events.push_back(c.ev);
    a.inflight.clear();
    ctx_destroy(a.ctx, false);
    a.ctx = nullptr;
    s->free_slots.push_back(a.slot);
    r.info.status = status;
    r.info.t_done = s->now();
    copy_msg(r.info, msg);
    if (status) {
        r.X.clear();
        r.F.clear();
        r.rank.clear();
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->n_active -= 1;
        s->launches += launches;
    }
    publish(s, a.q.id, std::move(r));
}

void worker_main(nsga3_server* s)
{
    cudaSetDevice(s->device);
    std::vector<Active> active;
    bool mem_changed = true;
    for (;;) {
        bool progress = false;
        // ---- admission, in arrival order
        for (;;) {
            Request q;
            {
                std::unique_lock<std::mutex> lk(s->mu);
                if (s->stop) {
                    while (!s->pending.empty()) {
                        Request c = std::move(s->pending.front());
                        s->pending.pop_front();
                        lk.unlock();
                        publish(s, c.id, failed_result(c, NSGA3_ESTATE, "server shut down before admission", s->now()));
                        lk.lock();
                    }
                    break;
                }
                if (s->pending.empty() || s->free_slots.empty()) break;
                const Request& h = s->pending.front();
                if (h.bytes <= s->arena->capacity()) {
                    if (!mem_changed) break;
                    if (s->arena->in_use() + h.bytes > s->arena->capacity()) {
                        mem_changed = false;
                        break;
                    }
                }
                q = std::move(s->pending.front());
                s->pending.pop_front();
            }
            if (q.bytes > s->arena->capacity()) {
                publish(s, q.id, failed_result(q, NSGA3_ENOMEM, "workspace exceeds the server's memory budget",
                                               s->now()));
                progress = true;
                continue;
            }
            nsga3_opts o = q.r.opts;
            o.W = q.W.empty() ? nullptr : q.W.data();
            nsga3_ctx* ctx = nullptr;
            std::string cerr;
            nsga3_status cst = ctx_create(q.r.m, q.r.d, q.r.N, q.r.ref_divisions, &o, s->arena, &ctx, &cerr,
                                          s->max_active > 1);
            if (cst == NSGA3_ENOMEM) {
                // fragmented arena: keep the request at the head, retry after a release
                std::lock_guard<std::mutex> lk(s->mu);
                s->pending.push_front(std::move(q));
                mem_changed = false;
                break;
            }
            if (cst) {
                publish(s, q.id, failed_result(q, cst, cerr, s->now()));
                progress = true;
                continue;
            }
            Active a;
            a.q = std::move(q);
            a.ctx = ctx;
            a.slot = s->free_slots.back();
            s->free_slots.pop_back();
            a.t_admit = s->now();
            a.st = nsga3_init(ctx, s->slots[a.slot]);
            if (a.st) a.msg = nsga3_last_error(ctx);
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->admitted += 1;
                s->n_active += 1;
                s->peak_active = std::max(s->peak_active, s->n_active);
                s->peak_bytes = std::max<uint64_t>(s->peak_bytes, s->arena->in_use());
            }
            active.push_back(std::move(a));
            progress = true;
        }
        // ---- launches: keep two chunks queued per run
        for (auto& a : active) {
            while (!a.st && a.inflight.size() < 2 && a.launched < a.q.r.generations) {
                const int g = std::min(s->chunk, a.q.r.generations - a.launched);
                cudaStream_t st = s->slots[a.slot];
                a.st = nsga3_run(a.ctx, g, st);
                if (a.st) {
                    a.msg = nsga3_last_error(a.ctx);
                    break;
                }
                cudaEvent_t ev = take_event(s);
                if (!ev || cudaEventRecord(ev, st) != cudaSuccess) {
                    cudaGetLastError();
                    a.st = NSGA3_ECUDA;
                    a.msg = "event record failed";
                    if (ev) s->free_events.push_back(ev);
                    break;
                }
                a.inflight.push_back({ev, g});
                a.launched += g;
                progress = true;
            }
        }
        // ---- completions
        for (size_t i = 0; i < active.size();) {
            Active& a = active[i];
            while (!a.inflight.empty()) {
                cudaError_t e = cudaEventQuery(a.inflight.front().ev);
                if (e == cudaErrorNotReady) break;
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    a.st = NSGA3_ECUDA;
                    a.msg = cudaGetErrorString(e);
                }
                a.finished += a.inflight.front().gens;
                s->free_events.push_back(a.inflight.front().ev);
                a.inflight.pop_front();
                progress = true;
            }
            bool stopping;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                stopping = s->stop;
            }
            const bool complete = a.finished >= a.q.r.generations;
            if (complete || (a.st && a.inflight.empty()) || stopping) {
                if (stopping && !complete && !a.st) {
                    a.st = NSGA3_ESTATE;
                    a.msg = "server shut down before the run finished";
                }
                retire(s, a);
                mem_changed = true;
                active.erase(active.begin() + i);
                progress = true;
                continue;
            }
            ++i;
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && active.empty() && s->pending.empty()) break;
            if (!progress) {
                if (active.empty())
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                }
            }
        }
    }
}

}  // namespace

extern "C" {

nsga3_status nsga3_server_create(uint64_t memory_budget, int max_active, int gens_per_launch, nsga3_server** out)
{
    if (!out || max_active < 1 || max_active > 1024 || gens_per_launch < 1 || memory_budget < DeviceArena::kAlign)
        return NSGA3_EINVAL;
    *out = nullptr;
    nsga3_server* s = new nsga3_server();
    s->t0 = Clock::now();
    s->max_active = max_active;
    s->chunk = gens_per_launch;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return NSGA3_ECUDA;
    }
    if (cudaMalloc(&s->arena_mem, memory_budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return NSGA3_ENOMEM;
    }
    s->arena = new DeviceArena(s->arena_mem, memory_budget);
    for (int i = 0; i < max_active; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        s->slots.push_back(st);
        s->free_slots.push_back(max_active - 1 - i);
    }
    if ((int)s->slots.size() != max_active) {
        for (auto st : s->slots) cudaStreamDestroy(st);
        cudaFree(s->arena_mem);
        delete s->arena;
        delete s;
        return NSGA3_ECUDA;
    }
    std::reverse(s->free_slots.begin(), s->free_slots.end());
    s->worker = std::thread(worker_main, s);
    *out = s;
    return NSGA3_OK;
}

nsga3_status nsga3_server_submit(nsga3_server* s, const nsga3_request* req, int64_t* id)
{
    if (!s || !req || !id) return NSGA3_EINVAL;
    Request q;
    q.r = *req;
    size_t bytes = 0;
    std::string err;
    nsga3_status st = ctx_workspace_bytes(req->m, req->d, req->N, req->ref_divisions, &req->opts, 0, &bytes, &err);
    if (st) {
        set_err(s, "submit: %s", err.c_str());
        return st;
    }
    if (req->generations < 0 || !req->opts.W || req->opts.problem != 0) {
        set_err(s, "submit: generations must be >= 0 and opts.W set (softmax-simplex problem only)");
        return NSGA3_EINVAL;
    }
    q.W.assign(req->opts.W, req->opts.W + (size_t)req->m * (req->m - 1));
    q.r.opts.W = nullptr;
    q.bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return NSGA3_ESTATE;
        q.id = s->next_id++;
        q.t_submit = s->now();
        *id = q.id;
        s->pending.push_back(std::move(q));
        s->submitted += 1;
    }
    s->cv_work.notify_one();
    return NSGA3_OK;
}

nsga3_status nsga3_server_wait(nsga3_server* s, int timeout_ms, int64_t* id)
{
    if (!s || !id) return NSGA3_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    *id = -1;
    auto ready = [&] { return !s->unclaimed.empty(); };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (s->unclaimed.empty()) return NSGA3_OK;
    *id = s->unclaimed.front();
    s->unclaimed.pop_front();
    return NSGA3_OK;
}

nsga3_status nsga3_server_fetch(nsga3_server* s, int64_t id, float* X, float* F, int32_t* rank,
                                nsga3_run_info* info)
{
    if (!s) return NSGA3_EINVAL;
    Result r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->done.find(id);
        if (it == s->done.end()) return NSGA3_EINVAL;
        r = std::move(it->second);
        s->done.erase(it);
        auto u = std::find(s->unclaimed.begin(), s->unclaimed.end(), id);
        if (u != s->unclaimed.end()) s->unclaimed.erase(u);
    }
    if (info) *info = r.info;
    if (X && !r.X.empty()) memcpy(X, r.X.data(), r.X.size() * sizeof(float));
    if (F && !r.F.empty()) memcpy(F, r.F.data(), r.F.size() * sizeof(float));
    if (rank && !r.rank.empty()) memcpy(rank, r.rank.data(), r.rank.size() * sizeof(int32_t));
    return (nsga3_status)r.info.status;
}

nsga3_status nsga3_server_get_stats(nsga3_server* s, nsga3_server_stats* st)
{
    if (!s || !st) return NSGA3_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->active = s->n_active;
    st->pending = (int64_t)s->pending.size();
    st->peak_active = s->peak_active;
    st->launches = s->launches;
    st->budget_bytes = s->arena->capacity();
    st->bytes_in_use = s->arena->in_use();
    st->peak_bytes = s->peak_bytes;
    return NSGA3_OK;
}

double nsga3_server_now(const nsga3_server* s) { return s ? s->now() : 0.0; }

const char* nsga3_server_last_error(const nsga3_server* s) { return s ? s->err.c_str() : ""; }

void nsga3_server_destroy(nsga3_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->slots) cudaStreamDestroy(st);
    for (auto e : s->free_events) cudaEventDestroy(e);
    cudaFree(s->arena_mem);
    cudaGetLastError();
    delete s->arena;
    delete s;
}

}  // extern "C"
