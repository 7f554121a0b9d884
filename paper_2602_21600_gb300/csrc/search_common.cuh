// Pieces of the batched query kernel shared by its one-warp form
// (search.cu) and its several-warps-per-query form (search_group.cu): the
// staging-tile stride and the shared-memory layouts; and the Stage 2 / Stage
// 3 row loops of the group form (the one-warp kernel keeps the same loops
// inline, where they compile without spills at its register bound).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "aqr_internal.h"
#include "beam.cuh"

namespace aqr {

int search_team_width(int dp);
int search_stage_bytes(int dp, int ldx, bool lane_path);

// Row stride of the lane path's staging tile: unpadded, swizzled rows when
// they span a multiple of 8 chunks, else an odd number of chunks.
__host__ __device__ inline int search_lane_stride(int dp) {
    const int ch = dp / 16;
    return (ch & 7) == 0 ? dp : (ch | 1) * 16;
}

constexpr int kWarps = 4;  // warps per block
constexpr int kThreads = kWarps * 32;
// Wide lane kernel: blocks of 11 warps at 56 registers, three per SM, i.e.
// 33 resident queries per SM instead of at most 32 (28 by shared memory at
// the default tile).  A batch finishes in rounds of one query per resident
// warp; on 152 SMs 10,000 queries take two rounds instead of three.
constexpr int kWideWarps = 11;
constexpr int kWideBlocks = 3;

struct WarpLayout {
    int ef_cap, rmax, surv, stg, qf;  // surv: survivor slots (team evaluators only);
                                      // qf: FP32 query (plain path) or query codes bytes
    HashGeom hg;                      // visited hash, 8 * hg.sets bytes
    __host__ __device__ int bytes() const {
        return ((ef_cap * 8 + hg.sets * 8 + rmax * 4 + surv * 8 + stg + qf) + 15) & ~15;
    }
};

// Several warps per query (quantised path): a block of kWarps warps holds
// kWarps / G groups.  Per group: the result set W, the visited hash (the
// FP32 query after Stage 1), the survivor lists and the group scalars;
// per warp of the group: its candidate list, staging tile and query codes.
struct GroupLayout {
    int ef_cap, rmax, smax, stg, qf, G;
    HashGeom hg;
    __host__ __device__ int shared_bytes() const {
        return (ef_cap * 8 + hg.sets * 8 + G * smax * 8 + dev::GS_NUM * 4 + 15) & ~15;
    }
    __host__ __device__ int warp_bytes() const { return (rmax * 4 + stg + qf + 15) & ~15; }
    __host__ __device__ int bytes() const { return shared_bytes() + G * warp_bytes(); }
};


// Launch of the several-warps-per-query kernel (search_group.cu), G in
// {2, 4}: lane selects one lane per candidate in Stage 1, tw is the team
// width of the row size.
cudaError_t launch_group(const SearchArgs& a, const GroupLayout& gl, bool lane, int tw,
                         int num_sms, cudaStream_t s);

namespace dev {
// Stage 2 (Alg. 2) for the entries W[lo, hi): asymmetric distance of the
// FP32 query qf to each candidate's decoded code x~_j = code_j / scale_j +
// min_j (FP32 fma with the precomputed 1 / scale_j), TEAM lanes per
// candidate (asym_partial_s), rows staged into stg (stg_bytes) round by
// round at the stride of stage2_stride; each entry's key becomes (d^a, id).
template <int TEAM>
__device__ __forceinline__ void stage2_rows(const uint8_t* codes, int d, int dp, u64* W, int lo,
                                            int hi, unsigned char* stg, int stg_bytes,
                                            const float* qf, const float* s_min,
                                            const float* s_inv, uint64_t pol) {
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31, tl = lane & (TEAM - 1), team = lane / TEAM;
    const int st2 = stage2_stride(dp, TEAM);
    const int nw = (d + 3) >> 2;
    const int cap2 = stg_bytes / st2;
    const int win2 = prefetch_window(cap2, dp);
    for (int base = lo; base < hi; base += cap2) {
        const int nr = min(cap2, hi - base);
        const u64* Wb = W + base;
        // rows [base, base + win2) prefetched once this round is issued
        const int pf = base > lo ? min(hi, base - cap2 + win2) : lo;
        prefetch_rows_l2(codes, dp, W + pf, min(hi, base + win2) - pf);
        stage_rows<TEAM, 0, true>(stg, st2, codes, dp, [&](int r) { return key_id(Wb[r]); }, nr,
                                  pol);
        for (int b2 = 0; b2 < nr; b2 += NT) {
            const int i = b2 + team;
            const int r = i < nr ? i : 0;
            const uint32_t v = key_id(W[base + r]);
            float acc = asym_partial_s<TEAM>((const uint32_t*)(stg + (size_t)r * st2), qf, s_inv,
                                             s_min, tl, nw);
            acc = team_sum_f32<TEAM>(acc);
            __syncwarp();
            if (i < nr && tl == 0) W[base + i] = ((u64)__float_as_uint(acc) << 32) | ((u64)v << 1);
        }
        __syncwarp();
    }
}

// Stage 3 (Alg. 2) for W[lo, hi): exact FP32 squared L2 to the FP32 rows
// (fma accumulation, fixed butterfly), keys become (d^e, id) with the
// exact flag set.
template <int TEAM>
__device__ __forceinline__ void stage3_rows(const float* x, int ldx, u64* W, int lo, int hi,
                                            unsigned char* stg, int stg_bytes, const float* qf,
                                            uint64_t pol) {
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31, tl = lane & (TEAM - 1), team = lane / TEAM;
    const int xrow = ldx * 4, ngroups = ldx >> 2;
    const int cap3 = stg_bytes / xrow;
    const int win3 = prefetch_window(cap3, xrow);
    for (int base = lo; base < hi; base += cap3) {
        const int nr = min(cap3, hi - base);
        const u64* Wb = W + base;
        const int pf = base > lo ? min(hi, base - cap3 + win3) : lo;
        prefetch_rows_l2((const unsigned char*)x, xrow, W + pf, min(hi, base + win3) - pf);
        stage_rows<TEAM, 0, true>(stg, xrow, (const unsigned char*)x, xrow,
                                  [&](int r) { return key_id(Wb[r]); }, nr, pol);
        for (int b2 = 0; b2 < nr; b2 += NT) {
            const int i = b2 + team;
            const int r = i < nr ? i : 0;
            const uint32_t v = key_id(W[base + r]);
            float acc = f32_partial_s((const float4*)(stg + (size_t)r * xrow), qf, tl, TEAM, ngroups);
            acc = team_sum_f32<TEAM>(acc);
            __syncwarp();
            if (i < nr && tl == 0)
                W[base + i] = ((u64)__float_as_uint(acc) << 32) | ((u64)v << 1) | 1ull;
        }
        __syncwarp();
    }
}


}  // namespace dev
}  // namespace aqr
