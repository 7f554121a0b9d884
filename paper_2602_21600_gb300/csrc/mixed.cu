// Mixed batches: queries with their own k and ef in one call.
//
// Queries are bucketed by ef class (max(ef, k) <= 64, 128, 256, 512, 1024);
// each class runs as one persistent launch of the search kernel with its
// per-warp result set sized for the class, longest ef first inside the
// class.  The class launches are forked onto parallel streams so that they
// share the GPU.  The whole sequence (per-query parameter upload, counter
// reset, fork, launches, join) is captured once into a CUDA graph and
// replayed while the call signature is unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "aqr_internal.h"

namespace aqr {

// Host bucketing: permutation of query rows grouped by class, descending
// ef_eff inside a class (longest first keeps the persistent warps busy).
void plan_classes(int64_t n, const int32_t* k, const int32_t* ef, std::vector<int64_t>& perm,
                  ClassPlan& plan) {
    perm.resize(n);
    std::iota(perm.begin(), perm.end(), 0);
    auto eff = [&](int64_t i) { return std::max(k[i], ef[i]); };
    auto cls = [&](int64_t i) {
        int c = 0;
        int cap = 64;
        while (eff(i) > cap) {
            cap <<= 1;
            ++c;
        }
        return c;
    };
    std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) {
        int ca = cls(a), cb = cls(b);
        if (ca != cb) return ca < cb;
        return eff(a) > eff(b);
    });
    plan = ClassPlan();
    for (int64_t i = 0; i < n; ++i) plan.count[cls(perm[i])]++;
    int64_t acc = 0;
    for (int c = 0; c < kClasses; ++c) {
        plan.first[c] = acc;
        acc += plan.count[c];
    }
}

// Enqueue the class launches of one mixed batch on `s` (forking onto the
// given side streams).  dk / def / dperm are device arrays already holding
// the per-query k, ef and the permutation.  work must have kClasses slots.
cudaError_t enqueue_classes(Ctx* c, const float* q, int64_t n, const ClassPlan& plan,
                            const int32_t* dk, const int32_t* def, const int64_t* dperm,
                            int k_stride, int64_t* ids, float* dists, unsigned int* work,
                            unsigned long long* counters, cudaStream_t s,
                            cudaStream_t* side, cudaEvent_t* ev_fork, cudaEvent_t* ev_join) {
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned int) * kClasses, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * C_NUM, s);
    if (e != cudaSuccess) return e;
    int used = 0;
    for (int cl = 0; cl < kClasses; ++cl)
        if (plan.count[cl]) ++used;
    if (used == 0) return cudaSuccess;
    e = cudaEventRecord(ev_fork[0], s);
    int si = 0;
    for (int cl = 0; cl < kClasses && e == cudaSuccess; ++cl) {
        if (!plan.count[cl]) continue;
        cudaStream_t cs = side[si];
        e = cudaStreamWaitEvent(cs, ev_fork[0], 0);
        if (e != cudaSuccess) break;
        SearchArgs a = base_args(c);
        a.q = q;
        a.ldq = c->ix.d;
        a.nq = plan.count[cl];
        a.q_index = dperm + plan.first[cl];
        a.q_k = dk;
        a.q_ef = def;
        a.k_stride = k_stride;
        a.ids = ids;
        a.dists = dists;
        a.work = work + cl;
        a.counters = counters;
        a.kc = c->kcfg[cl];
        e = launch_search(a, 64 << cl, false, c->num_sms, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_join[si], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join[si], 0);
        ++si;
    }
    return e;
}

struct Ctx::Mixed {
    int64_t cap = 0;
    int32_t* dk = nullptr;
    int32_t* def = nullptr;
    int64_t* dperm = nullptr;
    // pinned staging: k, ef, perm
    int32_t* hk = nullptr;
    int32_t* hef = nullptr;
    int64_t* hperm = nullptr;
    unsigned int* work = nullptr;
    cudaStream_t side[kClasses] = {};
    cudaEvent_t ev_fork[1] = {};
    cudaEvent_t ev_join[kClasses] = {};
    cudaEvent_t staged = nullptr;  // last upload from the pinned staging done
    cudaStream_t cap_stream = nullptr;  // capture stream (the caller's may be the legacy stream)
    cudaGraphExec_t exec = nullptr;
    // signature of the captured graph
    int64_t g_n = -1;
    ClassPlan g_plan;
    const float* g_q = nullptr;
    int64_t* g_ids = nullptr;
    float* g_dists = nullptr;
    int g_kstride = 0;
    uint64_t g_gen = 0;  // Ctx::config_gen at capture
};

void mixed_release(Ctx* c) {
    Ctx::Mixed* m = c->mixed;
    if (!m) return;
    if (m->exec) cudaGraphExecDestroy(m->exec);
    cudaFree(m->dk);
    cudaFree(m->def);
    cudaFree(m->dperm);
    cudaFree(m->work);
    cudaFreeHost(m->hk);
    cudaFreeHost(m->hef);
    cudaFreeHost(m->hperm);
    for (int i = 0; i < kClasses; ++i) {
        if (m->side[i]) cudaStreamDestroy(m->side[i]);
        if (m->ev_join[i]) cudaEventDestroy(m->ev_join[i]);
    }
    if (m->ev_fork[0]) cudaEventDestroy(m->ev_fork[0]);
    if (m->staged) cudaEventDestroy(m->staged);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    delete m;
    c->mixed = nullptr;
}

static cudaError_t mixed_init(Ctx* c) {
    if (c->mixed) return cudaSuccess;
    Ctx::Mixed* m = new Ctx::Mixed();
    c->mixed = m;
    cudaError_t e = cudaMalloc(&m->work, sizeof(unsigned int) * kClasses);
    for (int i = 0; i < kClasses && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&m->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->ev_join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->ev_fork[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    return e;
}

static cudaError_t mixed_reserve(Ctx::Mixed* m, int64_t n) {
    if (n <= m->cap) return cudaSuccess;
    cudaEventSynchronize(m->staged);
    cudaFree(m->dk);
    cudaFree(m->def);
    cudaFree(m->dperm);
    cudaFreeHost(m->hk);
    cudaFreeHost(m->hef);
    cudaFreeHost(m->hperm);
    m->dk = m->def = nullptr;
    m->dperm = nullptr;
    m->hk = m->hef = nullptr;
    m->hperm = nullptr;
    m->cap = 0;
    if (m->exec) {
        cudaGraphExecDestroy(m->exec);
        m->exec = nullptr;
    }
    cudaError_t e = cudaMalloc(&m->dk, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->def, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->dperm, n * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&m->hk, n * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&m->hef, n * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&m->hperm, n * 8);
    if (e == cudaSuccess) m->cap = n;
    return e;
}

}  // namespace aqr

using namespace aqr;

extern "C" aqr_status aqr_search_mixed(aqr_ctx* ctx, const float* queries_dev, int64_t n,
                                       const int32_t* k_host, const int32_t* ef_host,
                                       int32_t k_stride, int64_t* ids_dev, float* dists_dev,
                                       void* stream) {
    NvtxRange range("aqr.search_mixed");
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    if (n < 0 || n > 0x7FFFFFFF || k_stride < 1)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_search_mixed: bad sizes");
    if (n == 0) return AQR_OK;
    if (!queries_dev || !k_host || !ef_host || !ids_dev || !dists_dev)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_search_mixed: null pointer");
    for (int64_t i = 0; i < n; ++i) {
        aqr_status st = check_k_ef(ctx, k_host[i], ef_host[i]);
        if (st != AQR_OK) return st;
        if (k_host[i] > k_stride) return fail(ctx, AQR_ERR_INVALID_ARG, "k > k_stride");
    }
    cudaSetDevice(ctx->device);
    cudaError_t e = mixed_init(ctx);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_search_mixed init");
    Ctx::Mixed* m = ctx->mixed;
    e = mixed_reserve(m, n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_search_mixed buffers");
    std::vector<int64_t> perm;
    ClassPlan plan;
    plan_classes(n, k_host, ef_host, perm, plan);
    cudaStream_t s = (cudaStream_t)stream;
    // staging buffers may still feed the previous call's upload
    e = cudaEventSynchronize(m->staged);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_search_mixed staging");
    std::memcpy(m->hk, k_host, n * 4);
    std::memcpy(m->hef, ef_host, n * 4);
    std::memcpy(m->hperm, perm.data(), n * 8);
    e = cudaMemcpyAsync(m->dk, m->hk, n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->def, m->hef, n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->dperm, m->hperm, n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(m->staged, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_search_mixed upload");
    // the captured kernels carry the index, the search parameters and the
    // kernel configurations by value: replay only at the same generation
    const bool same = m->exec && m->g_gen == ctx->config_gen && m->g_n == n &&
                      m->g_q == queries_dev && m->g_ids == ids_dev && m->g_dists == dists_dev &&
                      m->g_kstride == k_stride && std::memcmp(&m->g_plan, &plan, sizeof(plan)) == 0;
    if (!same) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
        cudaError_t ee = enqueue_classes(ctx, queries_dev, n, plan, m->dk, m->def, m->dperm, k_stride,
                                         ids_dev, dists_dev, m->work, ctx->d_counters, m->cap_stream,
                                         m->side, m->ev_fork, m->ev_join);
        e = cudaStreamEndCapture(m->cap_stream, &g);
        if (ee != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(ctx, ee != cudaSuccess ? ee : e, "capture mixed batch");
        }
        if (m->exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(m->exec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(m->exec);
                m->exec = nullptr;
            }
        }
        if (!m->exec) e = cudaGraphInstantiate(&m->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            m->exec = nullptr;
            return cuda_fail(ctx, e, "instantiate mixed batch graph");
        }
        m->g_gen = ctx->config_gen;
        m->g_n = n;
        m->g_q = queries_dev;
        m->g_ids = ids_dev;
        m->g_dists = dists_dev;
        m->g_kstride = k_stride;
        m->g_plan = plan;
    }
    ctx->last_stream = s;
    e = cudaGraphLaunch(m->exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch mixed batch graph");
    return AQR_OK;
}
