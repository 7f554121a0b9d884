// Internal declarations shared by the translation units of libaqr.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/aqr.h"
#include <nvtx3/nvToolsExt.h>

namespace aqr {

// NVTX range in the library's own domain ("aqr") around an entry point,
// for profilers; a no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) {
        static nvtxDomainHandle_t dom = nvtxDomainCreateA("aqr");
        nvtxEventAttributes_t at = {};
        at.version = NVTX_VERSION;
        at.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        at.messageType = NVTX_MESSAGE_TYPE_ASCII;
        at.message.ascii = name;
        dom_ = dom;
        nvtxDomainRangePushEx(dom_, &at);
    }
    ~NvtxRange() { nvtxDomainRangePop(dom_); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
    nvtxDomainHandle_t dom_;
};

constexpr uint32_t kNoId = 0xFFFFFFFFu;
constexpr unsigned long long kKeyEmpty = ~0ull;

// Device-resident index (Alg. 1 output): codes, FP32 store, layer-0 lists,
// upper-layer lists and the quantiser parameters.
struct DeviceIndex {
    int64_t n = 0;
    int d = 0;
    int dp = 0;      // code row bytes (d rounded up to 16)
    int ldx = 0;     // FP32 row stride in floats (d rounded up to 4)
    int M_i = 0;
    int R0 = 0, R1 = 0;    // list capacities (2 M_i, M_i)
    int R0p = 0, R1p = 0;  // row strides (capacities rounded up to 32 entries)
    int ef_c = 0;
    int max_level = -1;
    uint32_t entry = kNoId;
    int64_t n_upper = 0;
    double s_dist = 0, delta = 0, eta = 0;
    uint8_t* codes = nullptr;       // [n, dp]
    float* x = nullptr;             // [n, ldx]
    uint32_t* adj0 = nullptr;       // [n, R0p]
    int32_t* upper_base = nullptr;  // [n], -1 if level 0
    uint32_t* upper = nullptr;      // [n_upper, R1p]
    float* qmin = nullptr;          // [d]
    float* qscale = nullptr;        // [d]
    float* qinv = nullptr;          // [d] 1/scale_j (FP32) for the Stage-2 decode
    std::vector<float> h_min, h_scale;
    int64_t bytes = 0;
    void release();
};

// Releases a local DeviceIndex on every way out of its scope (an error
// return or a host exception) unless commit() handed it over first.
struct IndexGuard {
    DeviceIndex& ix;
    bool kept = false;
    explicit IndexGuard(DeviceIndex& i) : ix(i) {}
    ~IndexGuard() {
        if (!kept) ix.release();
    }
    void commit() { kept = true; }
    IndexGuard(const IndexGuard&) = delete;
    IndexGuard& operator=(const IndexGuard&) = delete;
};

// Device counters of one search launch (aggregated with atomics).
enum Counter {
    C_QUERIES = 0,
    C_EXPANSIONS,
    C_EVALS,
    C_ADJ,
    C_STAGE2,
    C_EXACT,
    C_ET,
    C_EVALS_L0,
    C_NUM
};

struct Ctx {
    int device = 0;
    int num_sms = 0;
    std::string last_error;
    aqr_search_params params{};
    aqr_kernel_config kcfg[5] = {};  // per ef class
    DeviceIndex ix;
    bool has_index = false;
    // small device scratch: work counters (one per concurrent class launch),
    // stats counters, error word
    unsigned int* d_work = nullptr;           // [kMaxLaunchSlots]
    unsigned int work_next = 0;               // next d_work counter (round robin per launch)
    unsigned long long* d_counters = nullptr; // [C_NUM]
    int* d_error = nullptr;
    unsigned int* d_knn_tensor = nullptr;     // 1: the last kNN ran on the tensor cores
    cudaStream_t last_stream = nullptr;
    // host-path buffers (aqr_search_host)
    float* h_qbuf_dev = nullptr;
    int64_t* h_ids_dev = nullptr;
    float* h_dists_dev = nullptr;
    int64_t h_cap = 0;
    int h_cap_k = 0;
    int h_cap_d = 0;  // query width the host-path buffers were sized for
    cudaStream_t own_stream = nullptr;
    // mixed-batch graph cache and serving state (opaque)
    struct Mixed;
    struct Serve;
    Mixed* mixed = nullptr;  // owned; freed by mixed_release
    Serve* serve = nullptr;  // owned; freed by serve_shutdown
    // The serving scheduler thread reads the search parameters and kernel
    // configurations: their writers hold cfg_mu, and so does the scheduler
    // while it builds a micro-batch's launch arguments.  config_gen counts
    // changes of the parameters, the configurations and the index; a cached
    // launch graph (the mixed-ef batch) is replayed only at the generation it
    // was captured in.
    std::mutex cfg_mu;
    uint64_t config_gen = 0;
    ~Ctx();
};

constexpr int kMaxLaunchSlots = 16;

// Per-launch arguments of the search kernel.
// Geometry of the per-query visited hash: `sets` sets of 8 bytes in shared
// memory, each four 16-bit tags (tag16; sets a power of two) or two 32-bit
// ids.  tag16 hashes ids to B = log2(id_mask + 1) bits, B - tag_bits of
// which select the set.
struct HashGeom {
    int sets;
    int tag16;
    int tag_bits;
    uint32_t id_mask;
};

struct SearchArgs {
    // index
    const uint8_t* codes;
    const float* x;
    const uint32_t* adj0;
    const uint32_t* upper;
    const int32_t* upper_base;
    const float* qmin;
    const float* qscale;
    const float* qinv;
    int64_t n;
    int d, dp, ldx, R0p, R1p;
    uint32_t entry;
    int max_level;
    // queries
    const float* q;
    int64_t ldq;
    int64_t nq;             // queries in this launch
    const int64_t* q_index; // optional: launch slot -> query row
    const int32_t* q_k;     // optional per-query k (indexed by query row)
    const int32_t* q_ef;    // optional per-query ef
    int k, ef;              // uniform values when q_k / q_ef are null
    int k_stride;           // output row stride
    // parameters
    int m_ef, rerank_pct, n_coarse, n_rerank;
    float tau_gap, tau_ratio, eps;
    // outputs
    int64_t* ids;
    float* dists;
    uint8_t* exact;
    aqr_trace tr;
    // kernel configuration (0 = automatic)
    aqr_kernel_config kc;
    // scratch
    unsigned int* work;
    unsigned long long* counters;
    int* error;
};

// cudaFuncSetAttribute (the dynamic shared-memory limit) is process-wide
// state of a kernel: a launch that relies on the size it set holds this lock
// from the set to the launch, so that a launch of the same kernel from
// another thread (the serving scheduler, another context) that sets a
// smaller size cannot come between them.
std::mutex& kernel_attr_mutex();
// Resident blocks per SM of kern (remembered per device, block size and
// dynamic shared memory); call with kernel_attr_mutex() held.
cudaError_t kernel_occupancy(const void* kern, int threads, int smem, int* per_sm);

// Launchers (return cudaError_t from the launch).
cudaError_t launch_search(const SearchArgs& a, int ef_cap, bool plain_f32, int num_sms,
                          cudaStream_t s);
cudaError_t launch_encode(const float* x, int64_t n, int d, int64_t ldx, const float* mn,
                          const float* sc, uint8_t* codes, int64_t ldc, cudaStream_t s);
// path_out (device word, may be null): 1 when the tensor-core pass produced
// the distances, 0 when the CUDA-core tiles did.
cudaError_t launch_knn(const float* base, int64_t n, int d, const float* q, int64_t nq, int k,
                       const int64_t* self_ids, int64_t* ids, float* dists, int num_sms,
                       cudaStream_t s, unsigned int* path_out = nullptr);
int ef_class_cap(int ef_eff);  // 64..1024, or 0 if too large
int class_index(int cap);       // 64 -> 0, 128 -> 1, ...

aqr_status run_search(Ctx* c, const float* q, int64_t n, int32_t k, int32_t ef, int64_t* ids,
                      float* dists, uint8_t* exact, const aqr_trace* tr, bool plain, cudaStream_t s);
SearchArgs base_args(Ctx* c);
aqr_status check_k_ef(Ctx* c, int32_t k, int32_t ef);

// Mixed batches: per-class bucketing and the class launches (mixed.cu).
constexpr int kClasses = 5;  // ef classes 64, 128, 256, 512, 1024
struct ClassPlan {
    int64_t count[kClasses] = {0, 0, 0, 0, 0};
    int64_t first[kClasses] = {0, 0, 0, 0, 0};
};
void plan_classes(int64_t n, const int32_t* k, const int32_t* ef, std::vector<int64_t>& perm,
                  ClassPlan& plan);
cudaError_t enqueue_classes(Ctx* c, const float* q, int64_t n, const ClassPlan& plan,
                            const int32_t* dk, const int32_t* def, const int64_t* dperm,
                            int k_stride, int64_t* ids, float* dists, unsigned int* work,
                            unsigned long long* counters, cudaStream_t s, cudaStream_t* side,
                            cudaEvent_t* ev_fork, cudaEvent_t* ev_join);
void serve_shutdown(Ctx* c);
void mixed_release(Ctx* c);

// Error helpers.
aqr_status fail(Ctx* c, aqr_status st, const std::string& msg);
aqr_status cuda_fail(Ctx* c, cudaError_t e, const char* what);

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace aqr

struct aqr_ctx : public aqr::Ctx {};
