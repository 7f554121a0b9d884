// Top-k merge for database sharding: the base set is split into S shards,
// each searched on its own graph, and the per-query result lists are merged.
// The paper has no sharding; the merge keeps the final ranking of Alg. 2
// (ascending distance, ties by id) over the union of the shards' lists, with
// shard-local ids turned into global ones by the shard's id offset.
//
// One warp per query, one lane per shard (S <= 32).  Every shard's list is
// sorted by (distance, id) with padding (id < 0) at its end, so the merge
// repeatedly takes the smallest list head by a warp arg-min and advances
// that list: k steps of a 5-level shuffle reduction, no shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "aqr_internal.h"

namespace aqr {
namespace {

constexpr int kMaxShards = 32;

struct ShardOffsets {
    int64_t v[kMaxShards];
};

// (d, id) < (d2, id2) lexicographically; exhausted heads carry id INT64_MAX.
__device__ __forceinline__ bool head_less(float d, int64_t id, float d2, int64_t id2) {
    return d < d2 || (d == d2 && id < id2);
}

__global__ void merge_topk_kernel(const float* __restrict__ dists, const int64_t* __restrict__ ids,
                                  int S, int64_t n, int k, ShardOffsets off,
                                  int64_t* __restrict__ ids_out, float* __restrict__ dists_out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < n;
         q += warps) {
        // this lane's list: shard `lane`, row q
        const int64_t base = ((int64_t)lane * n + q) * k;
        int pos = 0;
        float hd = INFINITY;
        int64_t hid = INT64_MAX;
        auto load_head = [&]() {
            hd = INFINITY;
            hid = INT64_MAX;
            if (lane < S && pos < k) {
                const int64_t id = ids[base + pos];
                if (id >= 0) {
                    hd = dists[base + pos];
                    hid = id + off.v[lane];
                }
            }
        };
        load_head();
        for (int t = 0; t < k; ++t) {
            float bd = hd;
            int64_t bid = hid;
            int bl = lane;
#pragma unroll
            for (int m = 16; m; m >>= 1) {
                const float od = __shfl_xor_sync(0xFFFFFFFFu, bd, m);
                const int64_t oid = (int64_t)__shfl_xor_sync(0xFFFFFFFFu, (unsigned long long)bid, m);
                const int ol = __shfl_xor_sync(0xFFFFFFFFu, bl, m);
                if (head_less(od, oid, bd, bid) || (od == bd && oid == bid && ol < bl)) {
                    bd = od;
                    bid = oid;
                    bl = ol;
                }
            }
            if (lane == 0) {
                const bool have = bid != INT64_MAX;
                ids_out[q * k + t] = have ? bid : -1;
                dists_out[q * k + t] = have ? bd : INFINITY;
            }
            if (bid == INT64_MAX) {
                // every list is exhausted: pad the rest
                for (int u = t + 1 + lane; u < k; u += 32) {
                    ids_out[q * k + u] = -1;
                    dists_out[q * k + u] = INFINITY;
                }
                break;
            }
            if (lane == bl) {
                ++pos;
                load_head();
            }
        }
    }
}

}  // namespace
}  // namespace aqr

using namespace aqr;

extern "C" aqr_status aqr_merge_topk(aqr_ctx* ctx, const float* dists_dev, const int64_t* ids_dev,
                                     int32_t S, int64_t n, int32_t k,
                                     const int64_t* id_offsets_host, int64_t* ids_out_dev,
                                     float* dists_out_dev, void* stream) {
    NvtxRange range("aqr.merge_topk");
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (S < 1 || S > kMaxShards || n < 0 || k < 1 || k > 1024)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_merge_topk: need 1 <= S <= 32, 1 <= k <= 1024");
    if (n == 0) return AQR_OK;
    if (!dists_dev || !ids_dev || !ids_out_dev || !dists_out_dev)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_merge_topk: null pointer");
    ShardOffsets off{};
    for (int s = 0; s < S; ++s) {
        off.v[s] = id_offsets_host ? id_offsets_host[s] : 0;
        if (off.v[s] < 0) return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_merge_topk: negative offset");
    }
    cudaSetDevice(ctx->device);
    const int threads = 256;
    const int64_t want = (n + 7) / 8;
    const int64_t grid = std::min<int64_t>(want, (int64_t)ctx->num_sms * 8);
    merge_topk_kernel<<<(unsigned)grid, threads, 0, (cudaStream_t)stream>>>(
        dists_dev, ids_dev, S, n, k, off, ids_out_dev, dists_out_dev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AQR_OK : cuda_fail(ctx, e, "aqr_merge_topk");
}
