// Serving with continuous batching.
//
// Requests (one query each, with their own k and ef) are submitted from any
// thread.  A scheduler thread keeps up to n_streams micro-batches in flight,
// each on its own CUDA stream with its own device slot buffers.  Whenever a
// slot is free it admits pending requests, first come first served, while
// their device reservation fits the HBM budget: the query, its result
// rows, and the per-query search state sized by its ef (result set, visited
// hash).  A micro-batch holds requests of one ef class (the class of the
// oldest pending request), so short searches do not wait for long ones.
// Admitted requests are uploaded, searched with the class launch, and copied
// back; completion is detected with an event and the results handed to
// aqr_poll.  New requests are therefore admitted while
// earlier micro-batches are still on the GPU and their work overlaps on the
// device.  Each query's result depends only on the query, (k, ef) and the
// index, so a request gets the same answer alone or in any mix.
//
// Waits: poll waits at most its timeout; stop lets the micro-batches already
// on the GPU finish (finite kernels) and then joins the scheduler.
#include <cuda_runtime.h>
#include <stdint.h>
#include <sys/prctl.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "aqr_internal.h"

namespace aqr {

constexpr int kClassesS = kClasses;

namespace {
using Clock = std::chrono::steady_clock;
constexpr int kServeKMax = 128;  // k_stride of the serving slots

struct Request {
    uint64_t ticket;
    int32_t k, ef;
    std::vector<float> q;
    Clock::time_point t_submit, t_launch, t_done;
    int64_t bytes = 0;
    int batch = 0;
    bool done = false;
    std::vector<int64_t> ids;
    std::vector<float> dists;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaStream_t side[kClassesS] = {};
    cudaEvent_t ev_fork[1] = {};
    cudaEvent_t ev_join[kClassesS] = {};
    cudaEvent_t done = nullptr;
    float* dq = nullptr;
    int32_t* dk = nullptr;
    int32_t* def = nullptr;
    int64_t* dperm = nullptr;
    int64_t* dids = nullptr;
    float* ddists = nullptr;
    unsigned int* work = nullptr;
    unsigned long long* counters = nullptr;
    float* hq = nullptr;
    int32_t* hk = nullptr;
    int32_t* hef = nullptr;
    int64_t* hperm = nullptr;
    int64_t* hids = nullptr;
    float* hdists = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    int64_t bytes = 0;
};

}  // namespace

struct Ctx::Serve {
    aqr_serve_config cfg{};
    std::vector<Slot> slots;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    bool dead = false;          // the scheduler left on a host exception
    bool inject_fault = false;  // test hook: throw at the next pass
    bool thread_error = false;
    std::string error;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    int64_t budget = 0, in_use = 0;
};

namespace {

int64_t request_bytes(const Ctx* c, int k, int ef) {
    const int64_t ef_eff = std::max(k, ef);
    const int64_t cap = ef_class_cap((int)ef_eff);
    // query (FP32 + codes), result rows, result set W and visited hash of its class
    return (int64_t)c->ix.ldx * 4 + c->ix.dp + (int64_t)kServeKMax * 12 + cap * 8 +
           (cap <= 64 ? 1024 : cap <= 256 ? 2048 : 4096) * 4;
}

void free_slot(Slot& sl) {
    if (sl.s) cudaStreamSynchronize(sl.s);
    for (int i = 0; i < kClassesS; ++i) {
        if (sl.side[i]) cudaStreamDestroy(sl.side[i]);
        if (sl.ev_join[i]) cudaEventDestroy(sl.ev_join[i]);
    }
    if (sl.ev_fork[0]) cudaEventDestroy(sl.ev_fork[0]);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.s) cudaStreamDestroy(sl.s);
    cudaFree(sl.dq);
    cudaFree(sl.dk);
    cudaFree(sl.def);
    cudaFree(sl.dperm);
    cudaFree(sl.dids);
    cudaFree(sl.ddists);
    cudaFree(sl.work);
    cudaFree(sl.counters);
    cudaFreeHost(sl.hq);
    cudaFreeHost(sl.hk);
    cudaFreeHost(sl.hef);
    cudaFreeHost(sl.hperm);
    cudaFreeHost(sl.hids);
    cudaFreeHost(sl.hdists);
    sl = Slot();
}

cudaError_t alloc_slot(Slot& sl, int B, int d) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
    for (int i = 0; i < kClassesS && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&sl.side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_fork[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dq, (size_t)B * d * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dk, (size_t)B * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.def, (size_t)B * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dperm, (size_t)B * 8);
    if (e == cudaSuccess) e = cudaMalloc(&sl.dids, (size_t)B * kServeKMax * 8);
    if (e == cudaSuccess) e = cudaMalloc(&sl.ddists, (size_t)B * kServeKMax * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl.work, sizeof(unsigned int) * kClassesS);
    if (e == cudaSuccess) e = cudaMalloc(&sl.counters, sizeof(unsigned long long) * C_NUM);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.hq, (size_t)B * d * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.hk, (size_t)B * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.hef, (size_t)B * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.hperm, (size_t)B * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.hids, (size_t)B * kServeKMax * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.hdists, (size_t)B * kServeKMax * 4);
    return e;
}

// Hand a finished slot's results to its requests.  Called with sv->mu held.
void complete_slot(Ctx::Serve* sv, Slot& sl) {
    const auto now = Clock::now();
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
        auto it = sv->reqs.find(sl.tickets[i]);
        if (it == sv->reqs.end()) continue;
        Request& r = it->second;
        r.ids.assign(sl.hids + i * kServeKMax, sl.hids + i * kServeKMax + r.k);
        r.dists.assign(sl.hdists + i * kServeKMax, sl.hdists + i * kServeKMax + r.k);
        r.t_done = now;
        r.done = true;
    }
    sv->in_use -= sl.bytes;
    sl.bytes = 0;
    sl.tickets.clear();
    sl.busy = false;
}

void scheduler_loop(Ctx* c) {
    // The polls below sleep a few microseconds; the default timer slack of a
    // thread (50 us on Linux) would stretch each sleep by that much, which
    // every request would wait on top of its search.
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
    Ctx::Serve* sv = c->serve;
    cudaSetDevice(c->device);
    const int d = c->ix.d;
    const int B = sv->cfg.max_batch;
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        if (sv->inject_fault) {
            sv->inject_fault = false;
            throw std::bad_alloc();
        }
        // retire finished micro-batches
        bool any_busy = false;
        for (Slot& sl : sv->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaSuccess) {
                complete_slot(sv, sl);
                sv->cv_done.notify_all();
            } else if (q != cudaErrorNotReady) {
                sv->thread_error = true;
                sv->error = std::string("serving: ") + cudaGetErrorString(q);
                complete_slot(sv, sl);
                sv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        if (sv->stop && !any_busy) break;
        // admit into a free slot
        Slot* free_sl = nullptr;
        for (Slot& sl : sv->slots)
            if (!sl.busy) {
                free_sl = &sl;
                break;
            }
        if (!sv->stop && free_sl && !sv->pending.empty()) {
            Slot& sl = *free_sl;
            int m = 0;
            int64_t bytes = 0;
            // One ef class per micro-batch: the class of the oldest pending
            // request, then the later requests of that class in arrival
            // order (the others keep their place), so that a short search is
            // never held back by a long one in the same batch.
            int cls = -1;
            std::deque<uint64_t> rest;
            while (!sv->pending.empty()) {
                const uint64_t tk = sv->pending.front();
                sv->pending.pop_front();
                auto it = sv->reqs.find(tk);
                if (it == sv->reqs.end()) continue;  // cancelled
                Request& r = it->second;
                const int rc = class_index(ef_class_cap(std::max(r.k, r.ef)));
                if (cls < 0) cls = rc;
                if (rc != cls || m >= B || sv->in_use + bytes + r.bytes > sv->budget) {
                    rest.push_back(tk);
                    if (m >= B || (rc == cls && sv->in_use + bytes + r.bytes > sv->budget)) break;
                    continue;
                }
                std::memcpy(sl.hq + (size_t)m * d, r.q.data(), (size_t)d * 4);
                sl.hk[m] = r.k;
                sl.hef[m] = r.ef;
                r.t_launch = Clock::now();
                sl.tickets.push_back(r.ticket);
                bytes += r.bytes;
                ++m;
            }
            // put back what was passed over, ahead of the unscanned requests
            while (!rest.empty()) {
                sv->pending.push_front(rest.back());
                rest.pop_back();
            }
            if (m > 0) {
                for (uint64_t t : sl.tickets) sv->reqs[t].batch = m;
                sl.busy = true;
                sl.bytes = bytes;
                sv->in_use += bytes;
                lk.unlock();
                std::vector<int64_t> perm;
                ClassPlan plan;
                NvtxRange range("aqr.serve_batch");
                plan_classes(m, sl.hk, sl.hef, perm, plan);
                std::memcpy(sl.hperm, perm.data(), (size_t)m * 8);
                cudaError_t e = cudaMemcpyAsync(sl.dq, sl.hq, (size_t)m * d * 4, cudaMemcpyHostToDevice, sl.s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(sl.dk, sl.hk, (size_t)m * 4, cudaMemcpyHostToDevice, sl.s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(sl.def, sl.hef, (size_t)m * 4, cudaMemcpyHostToDevice, sl.s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(sl.dperm, sl.hperm, (size_t)m * 8, cudaMemcpyHostToDevice, sl.s);
                if (e == cudaSuccess) {
                    std::lock_guard<std::mutex> g(c->cfg_mu);  // parameters, configurations
                    e = enqueue_classes(c, sl.dq, m, plan, sl.dk, sl.def, sl.dperm, kServeKMax, sl.dids,
                                        sl.ddists, sl.work, sl.counters, sl.s, sl.side, sl.ev_fork,
                                        sl.ev_join);
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(sl.hids, sl.dids, (size_t)m * kServeKMax * 8, cudaMemcpyDeviceToHost, sl.s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(sl.hdists, sl.ddists, (size_t)m * kServeKMax * 4, cudaMemcpyDeviceToHost, sl.s);
                if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.s);
                lk.lock();
                if (e != cudaSuccess) {
                    sv->thread_error = true;
                    sv->error = std::string("serving launch: ") + cudaGetErrorString(e);
                    cudaStreamSynchronize(sl.s);
                    complete_slot(sv, sl);
                    sv->cv_done.notify_all();
                }
                continue;
            }
        }
        // nothing to do right now: wait for a submit or poll the slots again
        const bool idle = !any_busy && (sv->pending.empty() || !free_sl);
        if (idle && !sv->stop) {
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        } else if (any_busy) {
            // micro-batches on the GPU: poll their events again after a few
            // microseconds, with the lock free for submitters meanwhile
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(5));
            lk.lock();
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(sv->cfg.batch_wait_us));
            lk.lock();
        }
    }
}

// The scheduler thread: an exception (host memory) must not leave it.  It
// then marks the service dead (aqr_submit refuses new requests with
// AQR_ERR_CUDA), waits for the micro-batches still on the GPU (finite
// kernels) and gives their slots and bytes back, and completes every
// request not yet finished with the scheduler's error, so that pollers see
// AQR_ERR_CUDA instead of waiting.
void scheduler(Ctx* c) {
    try {
        scheduler_loop(c);
    } catch (...) {
        Ctx::Serve* sv = c->serve;
        std::lock_guard<std::mutex> g(sv->mu);
        sv->dead = true;
        sv->stop = true;
        sv->thread_error = true;
        sv->error = "serving: the scheduler stopped (out of host memory)";
        for (Slot& sl : sv->slots) {
            if (!sl.busy) continue;
            cudaStreamSynchronize(sl.s);
            sv->in_use -= sl.bytes;
            sl.bytes = 0;
            sl.tickets.clear();
            sl.busy = false;
        }
        sv->pending.clear();
        for (auto& kv : sv->reqs) kv.second.done = true;
        sv->cv_done.notify_all();
    }
}

}  // namespace

void serve_shutdown(Ctx* c) {
    Ctx::Serve* sv = c->serve;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->th.joinable()) sv->th.join();
    for (Slot& sl : sv->slots) free_slot(sl);
    delete sv;
    c->serve = nullptr;
}

}  // namespace aqr

using namespace aqr;

extern "C" aqr_status aqr_serve_start(aqr_ctx* ctx, const aqr_serve_config* cfg) {
    if (!ctx || !cfg) return AQR_ERR_INVALID_ARG;
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    if (ctx->serve) return fail(ctx, AQR_ERR_BUSY, "serving already started");
    if (cfg->max_batch < 1 || cfg->max_batch > 65536 || cfg->n_streams < 1 || cfg->n_streams > 16 ||
        cfg->hbm_budget < 0 || cfg->max_pending < 1 || cfg->batch_wait_us < 0)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_serve_start: bad configuration");
    cudaSetDevice(ctx->device);
    Ctx::Serve* sv = new Ctx::Serve();
    sv->cfg = *cfg;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    sv->budget = cfg->hbm_budget > 0 ? cfg->hbm_budget : (int64_t)(fr / 4);
    sv->slots.resize(cfg->n_streams);
    for (Slot& sl : sv->slots) {
        cudaError_t e = alloc_slot(sl, cfg->max_batch, ctx->ix.d);
        if (e != cudaSuccess) {
            for (Slot& s2 : sv->slots) free_slot(s2);
            delete sv;
            return cuda_fail(ctx, e, "aqr_serve_start slots");
        }
    }
    ctx->serve = sv;
    sv->th = std::thread(scheduler, (Ctx*)ctx);
    return AQR_OK;
}

extern "C" aqr_status aqr_submit(aqr_ctx* ctx, const float* query_host, int32_t k, int32_t ef,
                                 uint64_t* ticket) {
    if (!ctx || !query_host || !ticket) return AQR_ERR_INVALID_ARG;
    Ctx::Serve* sv = ctx->serve;
    if (!sv) return AQR_ERR_BUSY;
    if (k < 1 || ef < 1 || k > kServeKMax || ef_class_cap(std::max(k, ef)) == 0)
        return AQR_ERR_INVALID_ARG;
    Request r;
    r.k = k;
    r.ef = ef;
    r.q.assign(query_host, query_host + ctx->ix.d);
    r.bytes = request_bytes(ctx, k, ef);
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->dead) return fail(ctx, AQR_ERR_CUDA, sv->error);
        if (sv->stop) return AQR_ERR_BUSY;
        if (r.bytes > sv->budget) return AQR_ERR_NO_MEMORY;
        if ((int64_t)sv->pending.size() >= sv->cfg.max_pending) return AQR_ERR_BUSY;
        r.ticket = sv->next_ticket++;
        r.t_submit = Clock::now();
        *ticket = r.ticket;
        sv->pending.push_back(r.ticket);
        sv->reqs.emplace(r.ticket, std::move(r));
    }
    sv->cv_work.notify_one();
    return AQR_OK;
}

extern "C" aqr_status aqr_poll(aqr_ctx* ctx, uint64_t ticket, int64_t* ids_host, float* dists_host,
                               aqr_request_stats* st_host, int64_t timeout_us) {
    if (!ctx || !ids_host || !dists_host) return AQR_ERR_INVALID_ARG;
    Ctx::Serve* sv = ctx->serve;
    if (!sv) return AQR_ERR_BUSY;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return AQR_ERR_INVALID_ARG;
    if (!it->second.done && timeout_us > 0) {
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&]() {
            auto j = sv->reqs.find(ticket);
            return j == sv->reqs.end() || j->second.done;
        });
        it = sv->reqs.find(ticket);
        if (it == sv->reqs.end()) return AQR_ERR_INVALID_ARG;
    }
    if (!it->second.done) return AQR_ERR_NOT_READY;
    Request& r = it->second;
    std::memcpy(ids_host, r.ids.data(), r.ids.size() * 8);
    std::memcpy(dists_host, r.dists.data(), r.dists.size() * 4);
    if (st_host) {
        st_host->queue_us = std::chrono::duration<double, std::micro>(r.t_launch - r.t_submit).count();
        st_host->latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
        st_host->batch_size = r.batch;
    }
    const bool err = sv->thread_error;
    sv->reqs.erase(it);
    if (err) return fail(ctx, AQR_ERR_CUDA, sv->error);
    return AQR_OK;
}

extern "C" aqr_status aqr_cancel(aqr_ctx* ctx, uint64_t ticket) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    Ctx::Serve* sv = ctx->serve;
    if (!sv) return AQR_ERR_BUSY;
    std::lock_guard<std::mutex> g(sv->mu);
    for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it)
        if (*it == ticket) {
            sv->pending.erase(it);
            sv->reqs.erase(ticket);
            return AQR_OK;
        }
    return sv->reqs.count(ticket) ? AQR_ERR_NOT_READY : AQR_ERR_INVALID_ARG;
}

extern "C" aqr_status aqr_serve_inject_host_fault(aqr_ctx* ctx) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    Ctx::Serve* sv = ctx->serve;
    if (!sv) return AQR_ERR_BUSY;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->inject_fault = true;
    }
    sv->cv_work.notify_all();
    return AQR_OK;
}

extern "C" aqr_status aqr_serve_stop(aqr_ctx* ctx) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!ctx->serve) return AQR_OK;
    serve_shutdown(ctx);
    return AQR_OK;
}

// Open-loop load generator on the calling thread: request i is submitted
// when arrival_us[i] microseconds have passed since the call began, and
// finished requests are collected (non-blocking polls, oldest first) between
// submissions; returns when every request has completed.
extern "C" aqr_status aqr_serve_replay(aqr_ctx* ctx, const float* queries_host, int64_t n,
                                       const int32_t* k, const int32_t* ef,
                                       const double* arrival_us, int32_t k_stride,
                                       int64_t* ids_host, float* dists_host,
                                       aqr_request_stats* stats_host, int64_t timeout_us) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!ctx->serve) return fail(ctx, AQR_ERR_BUSY, "aqr_serve_replay: serving not started");
    if (n < 0 || k_stride < 1 || k_stride > kServeKMax || timeout_us < 0)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_serve_replay: bad sizes");
    if (n == 0) return AQR_OK;
    if (!queries_host || !k || !ef || !arrival_us || !ids_host || !dists_host || !stats_host)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_serve_replay: null pointer");
    for (int64_t i = 0; i < n; ++i)
        if (k[i] < 1 || k[i] > k_stride || !(arrival_us[i] >= 0.0) ||
            (i > 0 && arrival_us[i] < arrival_us[i - 1]))
            return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_serve_replay: bad k or arrival times");
    const int64_t d = ctx->ix.d;
    std::vector<uint64_t> tickets((size_t)n);
    std::vector<char> done((size_t)n, 0);
    int64_t next_submit = 0, next_done = 0;
    const Clock::time_point t0 = Clock::now();
    const Clock::time_point deadline = t0 + std::chrono::microseconds(
        (int64_t)arrival_us[n - 1] + timeout_us);
    while (next_done < n) {
        const Clock::time_point now = Clock::now();
        const double now_us = std::chrono::duration<double, std::micro>(now - t0).count();
        while (next_submit < n && arrival_us[next_submit] <= now_us) {
            const int64_t i = next_submit;
            aqr_status st = aqr_submit(ctx, queries_host + i * d, k[i], ef[i], &tickets[(size_t)i]);
            if (st == AQR_ERR_BUSY) break;  // pending queue full: retry on the next pass
            if (st != AQR_OK) return st;
            ++next_submit;
        }
        // collect: the oldest outstanding requests, a bounded window per pass
        int polled = 0;
        for (int64_t j = next_done; j < next_submit && polled < 64; ++j) {
            if (done[(size_t)j]) continue;
            ++polled;
            aqr_status st = aqr_poll(ctx, tickets[(size_t)j], ids_host + j * k_stride,
                                     dists_host + j * k_stride, stats_host + j, 0);
            if (st == AQR_OK) {
                for (int32_t t = k[j]; t < k_stride; ++t) {
                    ids_host[j * k_stride + t] = -1;
                    dists_host[j * k_stride + t] = __builtin_huge_valf();
                }
                done[(size_t)j] = 1;
            } else if (st != AQR_ERR_NOT_READY) {
                return st;
            }
        }
        while (next_done < n && done[(size_t)next_done]) ++next_done;
        if (now > deadline) return fail(ctx, AQR_ERR_TIMEOUT, "aqr_serve_replay: requests not finished");
    }
    return AQR_OK;
}
