// C ABI: contexts, parameters, index loading and export, search entry points.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <memory>
#include <tuple>
#include <new>
#include <vector>

#include "aqr_internal.h"

namespace aqr {

void DeviceIndex::release() {
    cudaFree(codes);
    cudaFree(x);
    cudaFree(adj0);
    cudaFree(upper_base);
    cudaFree(upper);
    cudaFree(qmin);
    cudaFree(qscale);
    cudaFree(qinv);
    *this = DeviceIndex();
}

aqr_status fail(Ctx* c, aqr_status st, const std::string& msg) {
    if (c) c->last_error = msg;
    return st;
}

aqr_status cuda_fail(Ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? AQR_ERR_NO_MEMORY : AQR_ERR_CUDA, m);
}

Ctx::~Ctx() {}

std::mutex& kernel_attr_mutex() {
    static std::mutex m;
    return m;
}

// Resident blocks per SM of a kernel at a block size and dynamic shared
// memory, computed once per device and remembered: serving launches small
// batches at a high rate, and the occupancy query is the costly host call
// of a launch.  Call with kernel_attr_mutex() held.
cudaError_t kernel_occupancy(const void* kern, int threads, int smem, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::map<std::tuple<int, const void*, int, int>, int> occ;
    const auto key = std::make_tuple(dev, kern, threads, smem);
    auto it = occ.find(key);
    if (it == occ.end()) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem);
        if (e != cudaSuccess) return e;
        it = occ.emplace(key, n).first;
    }
    *per_sm = it->second;
    return cudaSuccess;
}

static void release_host_bufs(Ctx* c) {
    cudaFree(c->h_qbuf_dev);
    cudaFree(c->h_ids_dev);
    cudaFree(c->h_dists_dev);
    c->h_qbuf_dev = nullptr;
    c->h_ids_dev = nullptr;
    c->h_dists_dev = nullptr;
    c->h_cap = 0;
    c->h_cap_k = 0;
    c->h_cap_d = 0;
}

// Fill a default parameter block (Table 3, row "0.97+").
static aqr_search_params defaults() {
    aqr_search_params p;
    p.m_ef = 3;
    p.rerank_pct = 40;
    p.n_coarse = 0;
    p.n_rerank = 0;
    p.tau_gap = 0.010f;
    p.tau_ratio = 1.008f;
    p.eps = 1e-6f;
    return p;
}

int class_index(int cap) {
    int i = 0;
    while ((64 << i) < cap) ++i;
    return i;
}

// Validate (k, ef) against the index and the kernel's ef classes.
aqr_status check_k_ef(Ctx* c, int32_t k, int32_t ef) {
    if (k < 1 || ef < 1) return fail(c, AQR_ERR_INVALID_ARG, "k and ef must be >= 1");
    int ef_eff = std::max(k, ef);
    if (ef_class_cap(ef_eff) == 0)
        return fail(c, AQR_ERR_INVALID_ARG, "max(ef, k) must be <= 1024");
    return AQR_OK;
}

SearchArgs base_args(Ctx* c) {
    const DeviceIndex& ix = c->ix;
    SearchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.codes = ix.codes;
    a.x = ix.x;
    a.adj0 = ix.adj0;
    a.upper = ix.upper;
    a.upper_base = ix.upper_base;
    a.qmin = ix.qmin;
    a.qscale = ix.qscale;
    a.qinv = ix.qinv;
    a.n = ix.n;
    a.d = ix.d;
    a.dp = ix.dp;
    a.ldx = ix.ldx;
    a.R0p = ix.R0p;
    a.R1p = ix.R1p;
    a.entry = ix.entry;
    a.max_level = ix.max_level;
    a.m_ef = c->params.m_ef;
    a.rerank_pct = c->params.rerank_pct;
    a.n_coarse = c->params.n_coarse;
    a.n_rerank = c->params.n_rerank;
    a.tau_gap = c->params.tau_gap;
    a.tau_ratio = c->params.tau_ratio;
    a.eps = c->params.eps;
    a.counters = c->d_counters;
    a.error = c->d_error;
    return a;
}

// One uniform-(k, ef) search launch: reset counters, launch.
aqr_status run_search(Ctx* c, const float* q, int64_t n, int32_t k, int32_t ef, int64_t* ids,
                      float* dists, uint8_t* exact, const aqr_trace* tr, bool plain,
                      cudaStream_t s) {
    NvtxRange range(plain ? "aqr.search_plain_f32" : "aqr.search");
    if (!c->has_index) return fail(c, AQR_ERR_NO_INDEX, "no index loaded");
    aqr_status st = check_k_ef(c, k, ef);
    if (st != AQR_OK) return st;
    if (n < 0 || n > 0x7FFFFFFF) return fail(c, AQR_ERR_INVALID_ARG, "n out of range");
    if (n > 0 && (!q || !ids || !dists)) return fail(c, AQR_ERR_INVALID_ARG, "null pointer");
    int ef_eff = std::max(k, ef);
    if (tr && (tr->c_ids || tr->c_dist || tr->a_ids || tr->a_dist) && tr->cap_c < ef_eff)
        return fail(c, AQR_ERR_INVALID_ARG, "trace cap_c < max(ef, k)");
    if (tr && tr->exp_seq && tr->cap_exp < 1)
        return fail(c, AQR_ERR_INVALID_ARG, "trace cap_exp < 1");
    c->last_stream = s;
    // each launch takes its own work counter, so that up to kMaxLaunchSlots
    // launches on different streams may overlap without sharing one
    unsigned int* work = c->d_work + (c->work_next++ % kMaxLaunchSlots);
    cudaError_t e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * C_NUM, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    if (n == 0) return AQR_OK;
    SearchArgs a = base_args(c);
    a.q = q;
    a.ldq = c->ix.d;
    a.nq = n;
    a.k = k;
    a.ef = ef;
    a.k_stride = k;
    a.ids = ids;
    a.dists = dists;
    a.exact = exact;
    if (tr) a.tr = *tr;
    // the autotuned configurations belong to the quantised path; the plain
    // comparison path runs with its automatic configuration
    if (!plain) a.kc = c->kcfg[class_index(ef_class_cap(ef_eff))];
    a.work = work;
    e = launch_search(a, ef_class_cap(ef_eff), plain, c->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "search launch");
    return AQR_OK;
}

}  // namespace aqr

using namespace aqr;

extern "C" {

const char* aqr_status_string(aqr_status s) {
    switch (s) {
        case AQR_OK: return "ok";
        case AQR_ERR_INVALID_ARG: return "invalid argument";
        case AQR_ERR_NO_MEMORY: return "out of memory";
        case AQR_ERR_NO_INDEX: return "no index loaded";
        case AQR_ERR_CUDA: return "CUDA error";
        case AQR_ERR_TIMEOUT: return "timeout";
        case AQR_ERR_BAD_FILE: return "bad index file";
        case AQR_ERR_BUSY: return "busy";
        case AQR_ERR_NOT_READY: return "not ready";
        case AQR_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

const char* aqr_last_error(aqr_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

aqr_status aqr_default_search_params(aqr_search_params* out) {
    if (!out) return AQR_ERR_INVALID_ARG;
    *out = defaults();
    return AQR_OK;
}

aqr_status aqr_search_params_for_recall(double target_recall, aqr_search_params* out,
                                        int32_t* ef_out) {
    if (!out || !(target_recall > 0.0 && target_recall <= 1.0)) return AQR_ERR_INVALID_ARG;
    // Table 3: coarse candidates, rerank K, gap and ratio thresholds, EF multiplier
    struct Row {
        int32_t coarse, rerank;
        float gap, ratio;
        int32_t mult;
    };
    static const Row rows[4] = {{35, 12, 0.020f, 1.015f, 2},
                                {45, 16, 0.015f, 1.012f, 2},
                                {55, 20, 0.012f, 1.010f, 3},
                                {70, 28, 0.010f, 1.008f, 3}};
    const Row& r = rows[target_recall < 0.90 ? 0 : target_recall < 0.95 ? 1
                        : target_recall < 0.97 ? 2 : 3];
    *out = defaults();
    out->n_coarse = r.coarse;
    out->n_rerank = r.rerank;
    out->tau_gap = r.gap;
    out->tau_ratio = r.ratio;
    out->m_ef = r.mult;
    if (ef_out) *ef_out = r.coarse * r.mult;
    return AQR_OK;
}

aqr_status aqr_create(aqr_ctx** out, int32_t device) {
    if (!out) return AQR_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return AQR_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return AQR_ERR_CUDA;
    aqr_ctx* c = new (std::nothrow) aqr_ctx();
    if (!c) return AQR_ERR_NO_MEMORY;
    c->device = device;
    c->params = defaults();
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&c->d_work, sizeof(unsigned int) * kMaxLaunchSlots);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counters, sizeof(unsigned long long) * C_NUM);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_knn_tensor, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(c->d_knn_tensor, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(c->d_error, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, sizeof(unsigned long long) * C_NUM);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        aqr_destroy(c);
        return e == cudaErrorMemoryAllocation ? AQR_ERR_NO_MEMORY : AQR_ERR_CUDA;
    }
    *out = c;
    return AQR_OK;
}

aqr_status aqr_destroy(aqr_ctx* ctx) {
    if (!ctx) return AQR_OK;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    mixed_release(ctx);
    cudaDeviceSynchronize();
    ctx->ix.release();
    release_host_bufs(ctx);
    cudaFree(ctx->d_work);
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_knn_tensor);
    cudaFree(ctx->d_error);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return AQR_OK;
}

aqr_status aqr_set_search_params(aqr_ctx* ctx, const aqr_search_params* p) {
    if (!ctx || !p) return AQR_ERR_INVALID_ARG;
    if (p->m_ef < 1 || p->rerank_pct < 0 || p->rerank_pct > 100 || p->n_coarse < 0 ||
        p->n_rerank < 0 || !(p->eps > 0.0f) || std::isnan(p->tau_gap) || std::isnan(p->tau_ratio))
        return fail(ctx, AQR_ERR_INVALID_ARG, "search parameters out of range");
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    ctx->params = *p;
    ++ctx->config_gen;
    return AQR_OK;
}

aqr_status aqr_quantize(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d, int64_t ldx,
                        const float* min_dev, const float* scale_dev, uint8_t* codes_dev,
                        int64_t ldc, void* stream) {
    NvtxRange range("aqr.quantize");
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (n < 0 || d <= 0 || ldx < d || ldc < d)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_quantize: bad sizes");
    if (n > 0 && (!x_dev || !min_dev || !scale_dev || !codes_dev))
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_quantize: null pointer");
    cudaError_t e = launch_encode(x_dev, n, d, ldx, min_dev, scale_dev, codes_dev, ldc,
                                  (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "encode launch");
    return AQR_OK;
}

}  // extern "C"

// ---- index file --------------------------------------------------------------

namespace {

struct Reader {
    FILE* f;
    uint64_t h = 1469598103934665603ull;
    bool ok = true;
    bool get(void* p, size_t bytes) {
        if (!ok) return false;
        if (bytes && std::fread(p, 1, bytes, f) != bytes) return ok = false;
        const uint8_t* b = (const uint8_t*)p;
        for (size_t i = 0; i < bytes; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
        return true;
    }
};

template <class T>
cudaError_t dev_alloc(T** p, size_t count, int64_t* bytes) {
    *bytes += (int64_t)(count * sizeof(T));
    return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

// Upload host arrays (file layout) into the padded device layout.
aqr_status upload_index(Ctx* c, DeviceIndex& ix, const float* mn, const float* sc,
                        const uint8_t* codes, const float* x, const uint32_t* adj0,
                        const int64_t* ub, const uint32_t* up) {
    const int64_t n = ix.n;
    cudaError_t e = cudaSuccess;
#define AQR_TRY(expr) \
    do {              \
        e = (expr);   \
        if (e != cudaSuccess) goto bad; \
    } while (0)
    {
        AQR_TRY(dev_alloc(&ix.codes, (size_t)n * ix.dp, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.x, (size_t)n * ix.ldx, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.adj0, (size_t)n * ix.R0p, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.upper_base, (size_t)n, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.upper, (size_t)std::max<int64_t>(ix.n_upper, 1) * ix.R1p, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.qmin, (size_t)ix.d, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.qscale, (size_t)ix.d, &ix.bytes));
        AQR_TRY(dev_alloc(&ix.qinv, (size_t)ix.d, &ix.bytes));
        AQR_TRY(cudaMemset(ix.codes, 0, (size_t)n * ix.dp));
        AQR_TRY(cudaMemset(ix.x, 0, (size_t)n * ix.ldx * 4));
        AQR_TRY(cudaMemset(ix.adj0, 0xFF, (size_t)n * ix.R0p * 4));
        AQR_TRY(cudaMemset(ix.upper, 0xFF, (size_t)std::max<int64_t>(ix.n_upper, 1) * ix.R1p * 4));
        if (codes) AQR_TRY(cudaMemcpy2D(ix.codes, ix.dp, codes, ix.d, ix.d, n, cudaMemcpyHostToDevice));
        if (x) AQR_TRY(cudaMemcpy2D(ix.x, (size_t)ix.ldx * 4, x, (size_t)ix.d * 4, (size_t)ix.d * 4, n,
                                    cudaMemcpyHostToDevice));
        if (adj0) AQR_TRY(cudaMemcpy2D(ix.adj0, (size_t)ix.R0p * 4, adj0, (size_t)ix.R0 * 4,
                                       (size_t)ix.R0 * 4, n, cudaMemcpyHostToDevice));
        if (ub) {
            std::vector<int32_t> ub32(n);
            for (int64_t i = 0; i < n; ++i) ub32[i] = (int32_t)ub[i];
            AQR_TRY(cudaMemcpy(ix.upper_base, ub32.data(), n * 4, cudaMemcpyHostToDevice));
        }
        if (up && ix.n_upper)
            AQR_TRY(cudaMemcpy2D(ix.upper, (size_t)ix.R1p * 4, up, (size_t)ix.R1 * 4,
                                 (size_t)ix.R1 * 4, ix.n_upper, cudaMemcpyHostToDevice));
        std::vector<float> inv(ix.d);
        for (int j = 0; j < ix.d; ++j) inv[j] = (float)(1.0 / (double)sc[j]);
        AQR_TRY(cudaMemcpy(ix.qmin, mn, ix.d * 4, cudaMemcpyHostToDevice));
        AQR_TRY(cudaMemcpy(ix.qscale, sc, ix.d * 4, cudaMemcpyHostToDevice));
        AQR_TRY(cudaMemcpy(ix.qinv, inv.data(), ix.d * 4, cudaMemcpyHostToDevice));
        ix.h_min.assign(mn, mn + ix.d);
        ix.h_scale.assign(sc, sc + ix.d);
        return AQR_OK;
    }
#undef AQR_TRY
bad:
    ix.release();
    return cuda_fail(c, e, "index upload");
}

}  // namespace

namespace aqr {
// Shapes derived from (n, d, M_i); used by the loader and the GPU builder.
aqr_status init_index_shape(Ctx* c, DeviceIndex& ix, int64_t n, int d, int M_i) {
    if (n < 1 || n > 0x7FFFFFFE || d < 1 || d > 2048 || M_i < 2 || M_i > 64)
        return fail(c, AQR_ERR_INVALID_ARG, "index shape out of range (n < 2^31, d <= 2048, 2 <= M_i <= 64)");
    ix.n = n;
    ix.d = d;
    ix.dp = round_up(d, 16);
    ix.ldx = round_up(d, 4);
    ix.M_i = M_i;
    ix.R0 = 2 * M_i;
    ix.R1 = M_i;
    ix.R0p = round_up(ix.R0, 32);
    ix.R1p = round_up(ix.R1, 32);
    return AQR_OK;
}
aqr_status upload_index_arrays(Ctx* c, DeviceIndex& ix, const float* mn, const float* sc,
                               const uint8_t* codes, const float* x, const uint32_t* adj0,
                               const int64_t* ub, const uint32_t* up) {
    return upload_index(c, ix, mn, sc, codes, x, adj0, ub, up);
}
}  // namespace aqr

static aqr_status load_graph_impl(aqr_ctx* ctx, const char* path) {
    if (!ctx || !path) return AQR_ERR_INVALID_ARG;
    if (ctx->serve)
        return fail(ctx, AQR_ERR_BUSY, "aqr_load_graph: stop serving before replacing the index");
    cudaSetDevice(ctx->device);
    std::unique_ptr<FILE, int (*)(FILE*)> file(std::fopen(path, "rb"), &std::fclose);
    FILE* f = file.get();
    if (!f) return fail(ctx, AQR_ERR_BAD_FILE, std::string("cannot open ") + path);
    Reader r{f};
    char magic[8];
    uint32_t version = 0, d = 0, M_i = 0, R0 = 0, R1 = 0, entry = 0, ef_c = 0;
    int32_t max_level = 0;
    uint64_t n = 0, n_upper = 0;
    double s_dist = 0, delta = 0, eta = 0;
    r.get(magic, 8);
    r.get(&version, 4);
    r.get(&d, 4);
    r.get(&n, 8);
    r.get(&M_i, 4);
    r.get(&R0, 4);
    r.get(&R1, 4);
    r.get(&entry, 4);
    r.get(&max_level, 4);
    r.get(&ef_c, 4);
    r.get(&n_upper, 8);
    r.get(&s_dist, 8);
    r.get(&delta, 8);
    r.get(&eta, 8);
    auto bad = [&](const std::string& m) {
        return fail(ctx, AQR_ERR_BAD_FILE, std::string(path) + ": " + m);
    };
    if (!r.ok || std::memcmp(magic, "AQRIDX01", 8) != 0) return bad("bad magic or short header");
    if (version != 1) return bad("unsupported version");
    if (d < 1 || d > 2048 || n < 1 || n > 0x7FFFFFFEull || M_i < 2 || M_i > 64 || R0 != 2 * M_i ||
        R1 != M_i || entry >= n || max_level < 0 || max_level > 64 || n_upper > n * 64ull)
        return bad("header fields out of range");
    // The header fixes the payload size: a file shorter than that is refused
    // before anything sized by the header is allocated.
    {
        const long here = std::ftell(f);
        if (here < 0 || std::fseek(f, 0, SEEK_END) != 0) return bad("cannot size the file");
        const long end = std::ftell(f);
        if (end < 0 || std::fseek(f, here, SEEK_SET) != 0) return bad("cannot size the file");
        const unsigned long long need = 8ull * d + 5ull * n * d + 4ull * n * R0 + 8ull * n +
                                        4ull * n_upper * R1 + 8ull;  // ... + checksum
        if ((unsigned long long)(end - here) < need) return bad("shorter than its header says");
    }
    DeviceIndex ix;
    if (init_index_shape(ctx, ix, (int64_t)n, (int)d, (int)M_i) != AQR_OK) return bad("shape");
    ix.entry = entry;
    ix.max_level = max_level;
    ix.ef_c = (int)ef_c;
    ix.n_upper = (int64_t)n_upper;
    ix.s_dist = s_dist;
    ix.delta = delta;
    ix.eta = eta;
    std::vector<float> mn(d), sc(d);
    std::vector<uint8_t> codes((size_t)n * d);
    std::vector<float> x((size_t)n * d);
    std::vector<uint32_t> adj0((size_t)n * R0);
    std::vector<int64_t> ub(n);
    std::vector<uint32_t> up((size_t)n_upper * R1);
    r.get(mn.data(), 4 * d);
    r.get(sc.data(), 4 * d);
    r.get(codes.data(), codes.size());
    r.get(x.data(), 4 * x.size());
    r.get(adj0.data(), 4 * adj0.size());
    r.get(ub.data(), 8 * ub.size());
    r.get(up.data(), 4 * up.size());
    uint64_t want = r.h, got = 0;
    if (!r.ok || std::fread(&got, 1, 8, f) != 8) return bad("truncated");
    if (got != want) return bad("checksum mismatch");
    file.reset();
    // Structural checks: ids in range, upper rows in range.
    for (uint32_t v : adj0)
        if (v != kNoId && v >= n) return fail(ctx, AQR_ERR_BAD_FILE, "adjacency id out of range");
    for (uint32_t v : up)
        if (v != kNoId && v >= n) return fail(ctx, AQR_ERR_BAD_FILE, "upper id out of range");
    // No row names a node twice: the search evaluates the new neighbours of
    // one expansion together, so a repeated id would enter W twice.
    {
        std::vector<uint64_t> stamp(n, ~0ull);
        auto rows_unique = [&](const std::vector<uint32_t>& a, size_t R, uint64_t first) {
            for (size_t r = 0; r < a.size() / R; ++r)
                for (size_t t = 0; t < R; ++t) {
                    const uint32_t v = a[r * R + t];
                    if (v == kNoId) continue;
                    if (stamp[v] == first + r) return false;
                    stamp[v] = first + r;
                }
            return true;
        };
        if (!rows_unique(adj0, R0, 0) || !rows_unique(up, R1, n))
            return fail(ctx, AQR_ERR_BAD_FILE, "an adjacency row names a node twice");
    }
    // Upper rows are laid out node by node in id order: node i owns rows
    // [ub[i], ub[next]) and its level is their count.  Every id listed in a
    // layer-lc row must itself reach layer lc, so that the search only reads
    // rows that exist.
    std::vector<int32_t> lvl(n, 0);
    {
        int64_t expect = 0, prev = -1;
        for (uint64_t i = 0; i < n; ++i) {
            if (ub[i] == -1) continue;
            // rows start at 0 and each owner's block follows the previous one
            if ((prev < 0 && ub[i] != 0) || ub[i] < expect || ub[i] >= (int64_t)n_upper)
                return fail(ctx, AQR_ERR_BAD_FILE, "upper_base not contiguous in id order");
            if (prev >= 0) lvl[prev] = (int32_t)(ub[i] - ub[prev]);
            prev = (int64_t)i;
            expect = ub[i] + 1;
        }
        if (prev >= 0) lvl[prev] = (int32_t)((int64_t)n_upper - ub[prev]);
        if (prev < 0 && n_upper != 0) return fail(ctx, AQR_ERR_BAD_FILE, "orphan upper rows");
        for (uint64_t i = 0; i < n; ++i)
            if (ub[i] < -1 || lvl[i] < 0 || lvl[i] > max_level)
                return fail(ctx, AQR_ERR_BAD_FILE, "upper_base out of range");
        int32_t top = 0;
        for (uint64_t i = 0; i < n; ++i) top = std::max(top, lvl[i]);
        if (top != max_level || lvl[entry] != max_level)
            return fail(ctx, AQR_ERR_BAD_FILE, "entry point is not on the top level");
        for (uint64_t i = 0; i < n; ++i)
            for (int32_t lc = 1; lc <= lvl[i]; ++lc)
                for (uint32_t t = 0; t < R1; ++t) {
                    uint32_t e = up[(size_t)(ub[i] + lc - 1) * R1 + t];
                    if (e != kNoId && lvl[e] < lc)
                        return fail(ctx, AQR_ERR_BAD_FILE, "upper list names a node below its layer");
                }
    }
    for (int j = 0; j < (int)d; ++j)
        if (!(sc[j] > 0.0f) || !std::isfinite(mn[j]))
            return fail(ctx, AQR_ERR_BAD_FILE, "quantiser parameters out of range");
    IndexGuard guard(ix);  // device arrays released unless the index is committed
    aqr_status st = upload_index(ctx, ix, mn.data(), sc.data(), codes.data(), x.data(), adj0.data(),
                                 ub.data(), up.data());
    if (st != AQR_OK) return st;
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    ctx->ix.release();
    guard.commit();
    ctx->ix = std::move(ix);
    ctx->has_index = true;
    ++ctx->config_gen;
    return AQR_OK;
}

// Host allocations sized by the file become AQR_ERR_NO_MEMORY, not an
// exception through the C boundary.
extern "C" aqr_status aqr_load_graph(aqr_ctx* ctx, const char* path) {
    try {
        return load_graph_impl(ctx, path);
    } catch (const std::bad_alloc&) {
        return fail(ctx, AQR_ERR_NO_MEMORY, "aqr_load_graph: out of host memory");
    }
}

extern "C" aqr_status aqr_index_info_get(aqr_ctx* ctx, aqr_index_info* out) {
    if (!ctx || !out) return AQR_ERR_INVALID_ARG;
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    const DeviceIndex& ix = ctx->ix;
    out->n = ix.n;
    out->d = ix.d;
    out->d_pad = ix.dp;
    out->M_i = ix.M_i;
    out->R0 = ix.R0;
    out->R1 = ix.R1;
    out->ef_c = ix.ef_c;
    out->max_level = ix.max_level;
    out->entry = ix.entry;
    out->n_upper = ix.n_upper;
    out->s_dist = ix.s_dist;
    out->device_bytes = ix.bytes;
    return AQR_OK;
}

extern "C" aqr_status aqr_export_graph(aqr_ctx* ctx, uint32_t* adj0_host, int64_t* upper_base_host,
                                       uint32_t* upper_host, uint8_t* codes_host,
                                       int32_t* entry_level_host) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    cudaSetDevice(ctx->device);
    const DeviceIndex& ix = ctx->ix;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && adj0_host)
        e = cudaMemcpy2D(adj0_host, (size_t)ix.R0 * 4, ix.adj0, (size_t)ix.R0p * 4, (size_t)ix.R0 * 4,
                         ix.n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && upper_base_host) {
        std::vector<int32_t> ub(ix.n);
        e = cudaMemcpy(ub.data(), ix.upper_base, ix.n * 4, cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < ix.n; ++i) upper_base_host[i] = ub[i];
    }
    if (e == cudaSuccess && upper_host && ix.n_upper)
        e = cudaMemcpy2D(upper_host, (size_t)ix.R1 * 4, ix.upper, (size_t)ix.R1p * 4, (size_t)ix.R1 * 4,
                         ix.n_upper, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && codes_host)
        e = cudaMemcpy2D(codes_host, ix.d, ix.codes, ix.dp, ix.d, ix.n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "export");
    if (entry_level_host) {
        entry_level_host[0] = (int32_t)ix.entry;
        entry_level_host[1] = ix.max_level;
    }
    return AQR_OK;
}

// ---- search ------------------------------------------------------------------

extern "C" aqr_status aqr_search(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k,
                                 int32_t ef, int64_t* ids_dev, float* dists_dev, void* stream) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    return run_search(ctx, queries_dev, n, k, ef, ids_dev, dists_dev, nullptr, nullptr, false,
                      (cudaStream_t)stream);
}

extern "C" aqr_status aqr_search_trace(aqr_ctx* ctx, const float* queries_dev, int64_t n,
                                       int32_t k, int32_t ef, int64_t* ids_dev, float* dists_dev,
                                       uint8_t* exact_dev, const aqr_trace* trace, void* stream) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    return run_search(ctx, queries_dev, n, k, ef, ids_dev, dists_dev, exact_dev, trace, false,
                      (cudaStream_t)stream);
}

extern "C" aqr_status aqr_search_plain_f32(aqr_ctx* ctx, const float* queries_dev, int64_t n,
                                           int32_t k, int32_t ef, int64_t* ids_dev,
                                           float* dists_dev, void* stream) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    return run_search(ctx, queries_dev, n, k, ef, ids_dev, dists_dev, nullptr, nullptr, true,
                      (cudaStream_t)stream);
}

extern "C" aqr_status aqr_search_host(aqr_ctx* ctx, const float* queries_host, int64_t n,
                                      int32_t k, int32_t ef, int64_t* ids_host,
                                      float* dists_host) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!queries_host || !ids_host || !dists_host)))
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_search_host: bad arguments");
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    aqr_status st = check_k_ef(ctx, k, ef);
    if (st != AQR_OK) return st;
    cudaSetDevice(ctx->device);
    // a new index may have another d: the query buffer follows it
    if (n > ctx->h_cap || k > ctx->h_cap_k || ctx->ix.d != ctx->h_cap_d) {
        cudaStreamSynchronize(ctx->own_stream);
        release_host_bufs(ctx);
        int64_t cap = std::max<int64_t>(n, 1);
        int ck = std::max(k, 16);
        cudaError_t e = cudaMalloc(&ctx->h_qbuf_dev, (size_t)cap * ctx->ix.d * 4);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_ids_dev, (size_t)cap * ck * 8);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->h_dists_dev, (size_t)cap * ck * 4);
        if (e != cudaSuccess) {
            release_host_bufs(ctx);
            return cuda_fail(ctx, e, "aqr_search_host buffers");
        }
        ctx->h_cap = cap;
        ctx->h_cap_k = ck;
        ctx->h_cap_d = ctx->ix.d;
    }
    cudaStream_t s = ctx->own_stream;
    cudaError_t e = cudaMemcpyAsync(ctx->h_qbuf_dev, queries_host, (size_t)n * ctx->ix.d * 4,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "H2D");
    st = run_search(ctx, ctx->h_qbuf_dev, n, k, ef, ctx->h_ids_dev, ctx->h_dists_dev, nullptr,
                    nullptr, false, s);
    if (st != AQR_OK) return st;
    e = cudaMemcpyAsync(ids_host, ctx->h_ids_dev, (size_t)n * k * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dists_host, ctx->h_dists_dev, (size_t)n * k * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_search_host");
    return AQR_OK;
}

extern "C" aqr_status aqr_get_stats(aqr_ctx* ctx, aqr_stats* out) {
    if (!ctx || !out) return AQR_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    unsigned long long h[C_NUM];
    int err = 0;
    cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(h, ctx->d_counters, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&err, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost);
    unsigned int tc = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&tc, ctx->d_knn_tensor, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_get_stats");
    out->knn_tensor = tc ? 1 : 0;
    const int64_t d = ctx->has_index ? ctx->ix.d : 0;
    out->queries = (int64_t)h[C_QUERIES];
    out->expansions = (int64_t)h[C_EXPANSIONS];
    out->dist_evals = (int64_t)h[C_EVALS];
    out->adj_entries = (int64_t)h[C_ADJ];
    out->stage2_evals = (int64_t)h[C_STAGE2];
    out->exact_evals = (int64_t)h[C_EXACT];
    out->early_exits = (int64_t)h[C_ET];
    out->device_errors = err;
    out->l0_evals = (int64_t)h[C_EVALS_L0];
    out->algo_bytes = out->queries * 4 * d + 4 * out->adj_entries + d * out->dist_evals +
                      d * out->stage2_evals + 4 * d * out->exact_evals;
    return AQR_OK;
}

extern "C" aqr_status aqr_bruteforce_knn(aqr_ctx* ctx, const float* base_dev, int64_t n, int32_t d,
                                         const float* q_dev, int64_t nq, int32_t k,
                                         const int64_t* self_ids_dev, int64_t* ids_dev,
                                         float* dists_dev, void* stream) {
    NvtxRange range("aqr.bruteforce_knn");
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (n < 1 || d < 1 || nq < 0 || k < 1 || k > 128 || n > 0xFFFFFFFEll)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_bruteforce_knn: bad sizes (k <= 128)");
    if (nq > 0 && (!base_dev || !q_dev || !ids_dev || !dists_dev))
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_bruteforce_knn: null pointer");
    cudaError_t e = launch_knn(base_dev, n, d, q_dev, nq, k, self_ids_dev, ids_dev, dists_dev,
                               ctx->num_sms, (cudaStream_t)stream, ctx->d_knn_tensor);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "knn launch");
    return AQR_OK;
}



extern "C" aqr_status aqr_set_kernel_config(aqr_ctx* ctx, int32_t ef, int32_t k,
                                            const aqr_kernel_config* cfg) {
    if (!ctx || !cfg) return AQR_ERR_INVALID_ARG;
    aqr_status st = check_k_ef(ctx, k, ef);
    if (st != AQR_OK) return st;
    if ((cfg->hash_slots != 0 && (cfg->hash_slots < 64 || cfg->hash_slots > 16384)) ||
        cfg->tile_rows < 0 || cfg->tile_rows > 32 || cfg->team_lanes < 0 || cfg->team_lanes > 2 ||
        (cfg->hash_tag_bits != 0 && cfg->hash_tag_bits != 16 && cfg->hash_tag_bits != 32) ||
        (cfg->warps_per_block != 0 && cfg->warps_per_block != 4 && cfg->warps_per_block != 11) ||
        (cfg->warps_per_query != 0 && cfg->warps_per_query != 1 && cfg->warps_per_query != 2 &&
         cfg->warps_per_query != 4))
        return fail(ctx, AQR_ERR_INVALID_ARG, "kernel configuration out of range");
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    ctx->kcfg[class_index(ef_class_cap(std::max(ef, k)))] = *cfg;
    ++ctx->config_gen;
    return AQR_OK;
}

namespace {

// Kernel configurations the autotuner times for one ef class: the automatic
// one and variations of hash size, tile, lanes per candidate, block shape
// and warps per query.
std::vector<aqr_kernel_config> tune_candidates(const Ctx* c) {
    std::vector<aqr_kernel_config> cands;
    const bool lane_ok = c->ix.dp <= 256;
    for (int team : {1, 2}) {
        if (team == 1 && !lane_ok) continue;
        cands.push_back(aqr_kernel_config{0, 0, team, 0, 0, 0});  // the automatic configuration
        for (int hs : {256, 512, 1024, 2048, 4096})
            for (int tile : {24, 32}) cands.push_back(aqr_kernel_config{hs, tile, team, 0, 0, 0});
        for (int hs : {384, 768}) cands.push_back(aqr_kernel_config{hs, 32, team, 32, 0, 0});
    }
    if (lane_ok)  // blocks of 11 warps, three per SM: the tile that fits, or smaller ones
        for (int hs : {0, 512, 1024})
            for (int tile : {0, 16, 20, 24})
                cands.push_back(aqr_kernel_config{hs, tile, 1, 0, 11, 0});
    for (int g : {2, 4})  // several warps per query
        for (int hs : {0, 1024, 2048})
            for (int tile : {0, 4, 16}) cands.push_back(aqr_kernel_config{hs, tile, 0, 0, 0, g});
    return cands;
}

// Times every candidate configuration on the batch (best of two timed runs
// after one warm-up, CUDA events on the context's stream) for the ef class
// of max(ef, k); leaves that class configured with the fastest and returns
// it with its time.  The automatic configuration (the first candidate) is
// kept unless another one is at least 2% faster, so that near-ties do not
// flip the choice from run to run.  ids / dists: [n, k] device scratch.
cudaError_t tune_class(Ctx* ctx, const float* q, int64_t n, int32_t k, int32_t ef, int64_t* ids,
                       float* dists, cudaEvent_t e0, cudaEvent_t e1, aqr_kernel_config* best_cfg,
                       float* best_ms) {
    const int ci = class_index(ef_class_cap(std::max(ef, k)));
    const aqr_kernel_config saved = ctx->kcfg[ci];
    const auto set_cfg = [&](const aqr_kernel_config& kc) {
        std::lock_guard<std::mutex> g(ctx->cfg_mu);
        ctx->kcfg[ci] = kc;
        ++ctx->config_gen;
    };
    const std::vector<aqr_kernel_config> cands = tune_candidates(ctx);
    float best = 1e30f;
    aqr_kernel_config best_c = saved;
    cudaStream_t s = ctx->own_stream;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) {
        set_cfg(cands[i]);
        float t_min = 1e30f;
        aqr_status st = AQR_OK;
        for (int rep = 0; rep < 3; ++rep) {
            if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
            st = run_search(ctx, q, n, k, ef, ids, dists, nullptr, nullptr, false, s);
            if (st != AQR_OK) break;  // configuration does not launch (e.g. shared memory)
            if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t_min = std::min(t_min, ms);
        }
        if (e == cudaSuccess && st == AQR_OK && t_min < (i == 0 ? best : 0.98f * best)) {
            best = t_min;
            best_c = cands[i];
        }
    }
    set_cfg(e == cudaSuccess ? best_c : saved);
    *best_cfg = best_c;
    *best_ms = best;
    return e;
}

struct TuneBuffers {
    int64_t* ids = nullptr;
    float* dists = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t alloc(int64_t n, int k) {
        cudaError_t e = cudaMalloc(&ids, (size_t)n * k * 8);
        if (e == cudaSuccess) e = cudaMalloc(&dists, (size_t)n * k * 4);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        return e;
    }
    ~TuneBuffers() {
        cudaFree(ids);
        cudaFree(dists);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

}  // namespace

extern "C" aqr_status aqr_autotune(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k,
                                   int32_t ef, aqr_kernel_config* chosen) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    aqr_status st = check_k_ef(ctx, k, ef);
    if (st != AQR_OK) return st;
    if (n < 1 || !queries_dev) return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_autotune: empty batch");
    cudaSetDevice(ctx->device);
    TuneBuffers tb;
    cudaError_t e = tb.alloc(n, k);
    aqr_kernel_config best_cfg{};
    float best_ms = 0;
    if (e == cudaSuccess) e = tune_class(ctx, queries_dev, n, k, ef, tb.ids, tb.dists, tb.e0, tb.e1,
                                         &best_cfg, &best_ms);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "aqr_autotune");
    if (chosen) *chosen = best_cfg;
    return AQR_OK;
}

// Recall@k of ids [n, k] against the first k of each row of gt [n, stride].
static double recall_at_k(const std::vector<int64_t>& ids, const int64_t* gt, int64_t n, int k,
                          int stride) {
    int64_t hit = 0;
    std::vector<int64_t> a(k), b(k);
    for (int64_t i = 0; i < n; ++i) {
        std::copy(ids.begin() + i * k, ids.begin() + i * k + k, a.begin());
        std::copy(gt + i * stride, gt + i * stride + k, b.begin());
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        for (int x = 0, y = 0; x < k && y < k;) {
            if (a[x] == b[y]) {
                if (a[x] >= 0) ++hit;
                ++x;
                ++y;
            } else if (a[x] < b[y]) {
                ++x;
            } else {
                ++y;
            }
        }
    }
    return (double)hit / ((double)n * k);
}

static aqr_status autotune_recall_impl(aqr_ctx* ctx, const float* queries_dev, int64_t n, int32_t k,
                                       const int64_t* gt, int32_t gt_stride, double target,
                                       const int32_t* efs, int32_t n_ef, aqr_tune_result* out,
                                       double* sweep) {
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (!ctx->has_index) return fail(ctx, AQR_ERR_NO_INDEX, "no index loaded");
    if (n < 1 || !queries_dev || !gt || !efs || !out || n_ef < 1 || k < 1 || gt_stride < k ||
        !(target > 0.0 && target <= 1.0))
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_autotune_recall: bad arguments");
    for (int i = 0; i < n_ef; ++i) {
        aqr_status st = check_k_ef(ctx, k, efs[i]);
        if (st != AQR_OK) return st;
        if (i > 0 && efs[i] <= efs[i - 1])
            return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_autotune_recall: ef list not ascending");
    }
    cudaSetDevice(ctx->device);
    // shortlist policies: m_ef in {3, 2, 1}, N_rerank 40% of N_c (Table 3's
    // rerank / coarse ratio) or all of N_c
    struct Pol {
        int m_ef, pct;
    };
    static const Pol pols[6] = {{3, 40}, {3, 100}, {2, 40}, {2, 100}, {1, 40}, {1, 100}};
    const aqr_search_params saved = ctx->params;
    aqr_kernel_config saved_k[kClasses];
    for (int i = 0; i < kClasses; ++i) saved_k[i] = ctx->kcfg[i];
    const auto set_pol = [&](const Pol& p) {
        aqr_search_params sp = saved;
        sp.m_ef = p.m_ef;
        sp.rerank_pct = p.pct;
        sp.n_coarse = 0;
        sp.n_rerank = 0;
        std::lock_guard<std::mutex> g(ctx->cfg_mu);
        ctx->params = sp;
        ++ctx->config_gen;
        return sp;
    };
    if (sweep)
        for (int i = 0; i < 6 * n_ef; ++i) sweep[i] = -1.0;
    TuneBuffers tb;
    cudaError_t e = tb.alloc(n, k);
    std::vector<int64_t> h_ids((size_t)n * k);
    struct Cand {
        int pol, ef;
        double recall;
    };
    std::vector<Cand> cands;
    Cand best_any{-1, 0, -1.0};
    cudaStream_t s = ctx->own_stream;
    for (int pi = 0; pi < 6 && e == cudaSuccess; ++pi) {
        set_pol(pols[pi]);
        for (int j = 0; j < n_ef; ++j) {
            aqr_status st = run_search(ctx, queries_dev, n, k, efs[j], tb.ids, tb.dists, nullptr,
                                       nullptr, false, s);
            if (st != AQR_OK) {
                std::lock_guard<std::mutex> g(ctx->cfg_mu);
                ctx->params = saved;
                return st;
            }
            e = cudaMemcpyAsync(h_ids.data(), tb.ids, h_ids.size() * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            const double r = recall_at_k(h_ids, gt, n, k, gt_stride);
            if (sweep) sweep[pi * n_ef + j] = r;
            if (r > best_any.recall) best_any = Cand{pi, efs[j], r};
            if (r >= target) {
                cands.push_back(Cand{pi, efs[j], r});
                break;
            }
        }
    }
    if (e == cudaSuccess && cands.empty() && best_any.pol >= 0) cands.push_back(best_any);
    aqr_tune_result best{};
    best.ms = 1e30;
    for (const Cand& c : cands) {
        if (e != cudaSuccess) break;
        const aqr_search_params sp = set_pol(pols[c.pol]);
        aqr_kernel_config kc{};
        float ms = 0;
        e = tune_class(ctx, queries_dev, n, k, c.ef, tb.ids, tb.dists, tb.e0, tb.e1, &kc, &ms);
        if (e == cudaSuccess && ms < best.ms) {
            best.params = sp;
            best.ef = c.ef;
            best.kernel = kc;
            best.recall = c.recall;
            best.ms = ms;
            best.reached = c.recall >= target ? 1 : 0;
        }
    }
    // the candidates' tuning set their classes: only the winner's keeps it
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    for (int i = 0; i < kClasses; ++i) ctx->kcfg[i] = saved_k[i];
    ++ctx->config_gen;
    if (e != cudaSuccess) {
        ctx->params = saved;
        return cuda_fail(ctx, e, "aqr_autotune_recall");
    }
    ctx->params = best.params;
    ctx->kcfg[class_index(ef_class_cap(std::max(best.ef, k)))] = best.kernel;
    *out = best;
    return AQR_OK;
}

// Host vectors of the sweep become AQR_ERR_NO_MEMORY, not an exception
// through the C boundary.
extern "C" aqr_status aqr_autotune_recall(aqr_ctx* ctx, const float* queries_dev, int64_t n,
                                          int32_t k, const int64_t* gt_ids_host, int32_t gt_stride,
                                          double target_recall, const int32_t* ef_list_host,
                                          int32_t n_ef, aqr_tune_result* out,
                                          double* sweep_recall_host) {
    try {
        return autotune_recall_impl(ctx, queries_dev, n, k, gt_ids_host, gt_stride, target_recall,
                                    ef_list_host, n_ef, out, sweep_recall_host);
    } catch (const std::bad_alloc&) {
        return fail(ctx, AQR_ERR_NO_MEMORY, "aqr_autotune_recall: out of host memory");
    }
}
