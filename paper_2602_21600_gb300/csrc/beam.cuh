// Warp-level HNSW primitives shared by the query kernel and the graph
// builder: code distances, the greedy step, the ef-bounded layer search and
// the candidate staging they use.  One warp works on one query / node.
//
// Beam-search formulation.  With the strict total order (distance, id),
// HNSW's SEARCH-LAYER (Malkov & Yashunin, Alg. 2: candidate heap C, result
// heap W, stop when the best candidate is worse than the worst result)
// expands exactly the sequence "the smallest not-yet-expanded element of W"
// until every element of W is expanded, and W after one expansion is the
// ef smallest of W and the new neighbours, whatever order those are
// inserted in.  So a warp evaluates all neighbours of one expanded node at
// once, keeps those better than the current worst, and merges them into the
// sorted W; expansion order and W equal the textbook algorithm's.
//
// Visited set: a set-associative hash of node ids in shared memory that
// forgets on collision.  Forgetting is harmless: a re-evaluated node is
// either still in W (dropped as a duplicate in the merge) or worse than the
// current worst of W, which only decreases, so it is rejected again.  It
// never reports an unvisited node as visited: a set holds either whole ids
// or quotient tags that, with the set number, determine the id.
//
// Memory: the rows of all new neighbours of one expansion are copied into a
// per-warp shared staging buffer with 16-byte cp.async copies issued at
// once (one memory latency per expansion instead of one per candidate
// round), then the distances are computed from shared memory.
//
// Keys: 64-bit (distance:32 | id:31 | flag:1); ordering keys orders by
// (distance, id).  The flag marks "expanded" during the search.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace aqr {
namespace dev {

typedef unsigned long long u64;

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr u64 kEmpty = ~0ull;

// Bounds checks of the checked build (-DAQR_CHECKED): AQR_IN(err, cond) is
// the constant true in the normal build; in the checked build a false cond
// records the source line in the error word (the first one wins) and the
// guarded access is skipped.
__device__ __forceinline__ bool check_fail(int* err, int line) {
    if (err) atomicCAS(err, 0, 100000 + line);
    return false;
}
#ifdef AQR_CHECKED
#define AQR_IN(err, cond) ((cond) ? true : ::aqr::dev::check_fail((err), __LINE__))
#else
#define AQR_IN(err, cond) true
#endif
constexpr int kMaxChunks = 4;  // 16-byte code chunks per lane (d <= 64 * TEAM)

__device__ __forceinline__ u64 make_key(uint32_t dist, uint32_t id) {
    return ((u64)dist << 32) | ((u64)id << 1);
}
__device__ __forceinline__ uint32_t key_id(u64 k) { return (uint32_t)(k >> 1) & 0x7FFFFFFFu; }
__device__ __forceinline__ uint32_t key_hi(u64 k) { return (uint32_t)(k >> 32); }

__device__ __forceinline__ u64 shfl_u64(u64 v, int src) {
    uint32_t lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)v, src);
    uint32_t hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), src);
    return ((u64)hi << 32) | lo;
}
__device__ __forceinline__ u64 shfl_xor_u64(u64 v, int m) {
    uint32_t lo = __shfl_xor_sync(0xFFFFFFFFu, (uint32_t)v, m);
    uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), m);
    return ((u64)hi << 32) | lo;
}
__device__ __forceinline__ u64 warp_min_u64(u64 v) {
#pragma unroll
    for (int m = 16; m; m >>= 1) {
        u64 o = shfl_xor_u64(v, m);
        v = o < v ? o : v;
    }
    return v;
}
template <int TEAM>
__device__ __forceinline__ uint32_t team_sum_u32(uint32_t v) {
#pragma unroll
    for (int m = TEAM / 2; m; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    return v;
}
// Fixed butterfly order: every lane of a team ends with the same FP32 sum,
// and the sum does not depend on which warp or launch computed it.
template <int TEAM>
__device__ __forceinline__ float team_sum_f32(float v) {
#pragma unroll
    for (int m = TEAM / 2; m; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    return v;
}

__device__ __forceinline__ uint32_t sq_diff_u8x4(uint32_t a, uint32_t b, uint32_t acc) {
    uint32_t t = __vabsdiffu4(a, b);
    return __dp4a(t, t, acc);
}

// Encode of one value (Alg. 1): FP32 subtract, FP32 multiply, clip
// to [0, 255] (NaN -> 0), round half to even.
__device__ __forceinline__ uint32_t encode1(float v, float mn, float sc) {
    float t = __fmul_rn(__fsub_rn(v, mn), sc);
    t = fminf(fmaxf(t, 0.0f), 255.0f);
    return (uint32_t)__float2int_rn(t);
}

// Codes of chunk c (dimensions 16c .. 16c + 15, zero from d on) of a query,
// four to a 32-bit word, lowest dimension in the lowest byte.  The words are
// selected by value so that they stay in registers.
__device__ __forceinline__ uint4 encode_chunk(const float* qv, const float* mn, const float* sc,
                                              int c, int d) {
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
#pragma unroll 1
    for (int h = 0; h < 4; ++h) {
        uint32_t wh = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = c * 16 + 4 * h + u;
            const uint32_t code = j < d ? encode1(__ldg(qv + j), __ldg(mn + j), __ldg(sc + j)) : 0u;
            wh |= code << (8 * u);
        }
        w0 = h == 0 ? wh : w0;
        w1 = h == 1 ? wh : w1;
        w2 = h == 2 ? wh : w2;
        w3 = h == 3 ? wh : w3;
    }
    return make_uint4(w0, w1, w2, w3);
}

// ---- 16-byte asynchronous global -> shared copies ------------------------
// 16-byte global -> shared copy (s: shared-window address); HINT: with the
// L2 eviction-priority policy pol (createpolicy), decided at compile time so
// that no copy tests it.
template <bool HINT>
__device__ __forceinline__ void cp_async16(unsigned s, const void* gsrc, uint64_t pol) {
    if (HINT)
        asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s),
                     "l"(gsrc), "l"(pol)
                     : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// L2 policies: code rows are re-read by every query and should stay in L2;
// FP32 rows of the final re-rank are read once per query.
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Copy the rows named by id(0..cnt-1) of a row-major array (row_bytes per
// row, a multiple of 16; rows 16-byte aligned) into the staging buffer, row r
// at stg + r * stride, its chunk c in slot c ^ (r & swz) (swz = 0: in
// order).  Groups of G lanes copy one row each, lane j of a group the
// 16-byte chunks j, j + G, ... (coalesced row reads, no division).  NCH > 0
// fixes the row at NCH chunks (row_bytes is then ignored): the copy loop
// unrolls with no runtime bound, which matters on the hottest staging path.
// Warp-collective; returns when the rows are visible to the whole warp.
template <int G, int NCH, bool HINT, class IdFn>
__device__ __forceinline__ void stage_rows(unsigned char* stg, int stride, const unsigned char* base,
                                           int row_bytes, IdFn id, int cnt, uint64_t pol,
                                           int swz = 0) {
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31;
    const int g = lane / G, j = lane % G;
    const int rb = NCH ? NCH * 16 : row_bytes;
    const unsigned s0 = (unsigned)__cvta_generic_to_shared(stg);
    for (int r = g; r < cnt; r += NG) {
        const unsigned char* src = base + (int64_t)id(r) * rb;
        const unsigned dst = s0 + (unsigned)(r * stride);
        const int x = r & swz;
        if (NCH) {
#pragma unroll
            for (int t = 0; t < (NCH + G - 1) / G; ++t) {
                const int c = j + G * t;
                if (NCH % G == 0 || c < NCH)
                    cp_async16<HINT>(dst + (unsigned)((c ^ x) << 4), src + (c << 4), pol);
            }
        } else {
            const int nch = rb >> 4;
            for (int c = j; c < nch; c += G)
                cp_async16<HINT>(dst + (unsigned)((c ^ x) << 4), src + (c << 4), pol);
        }
    }
    cp_async_wait_all();
    __syncwarp();
}

// L2 prefetch of the rows of a row-major array (row_bytes per row) named by
// the keys W[0, cnt): one prefetch per 128-byte line, the lines spread over
// the warp's lanes.  Fire and forget (no registers or shared memory held):
// Stages 2-3 issue it some rounds ahead of the rows' staging copies, which
// then find them in L2 instead of waiting for DRAM.
__device__ __forceinline__ void prefetch_rows_l2(const unsigned char* base, int row_bytes,
                                                 const u64* W, int cnt) {
    const int lane = threadIdx.x & 31;
    const int lpr = (row_bytes + 127) / 128 + 1;  // lines touched by a row at any offset
    for (int t = lane; t < cnt * lpr; t += 32) {
        const int r = t / lpr, l = t - r * lpr;
        prefetch_l2(base + (int64_t)key_id(W[r]) * row_bytes + min(l * 128, row_bytes - 1));
    }
}
// Rows Stages 2-3 keep prefetched ahead of the one being staged: at least
// two rounds, else up to 32 KB.
__device__ __forceinline__ int prefetch_window(int cap_rows, int row_bytes) {
    return max(2 * cap_rows, 32768 / row_bytes);
}

// ---- distances of staged rows ----------------------------------------------
// Partial squared code distance over this lane's 16-byte chunks
// c = tl + TEAM * i of a row in shared memory; qc holds the probe's chunks.
template <int TEAM>
__device__ __forceinline__ uint32_t code_partial_s(const uint4* row, const uint4 (&qc)[kMaxChunks],
                                                   int tl, int nchunks) {
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kMaxChunks; ++i) {
        const int c = tl + TEAM * i;
        if (c < nchunks) {
            const uint4 b = row[c];
            acc = sq_diff_u8x4(qc[i].x, b.x, acc);
            acc = sq_diff_u8x4(qc[i].y, b.y, acc);
            acc = sq_diff_u8x4(qc[i].z, b.z, acc);
            acc = sq_diff_u8x4(qc[i].w, b.w, acc);
        }
    }
    return acc;
}
// Same on a row in global memory (read-only path).
template <int TEAM>
__device__ __forceinline__ uint32_t code_partial_g(const uint4* row, const uint4 (&qc)[kMaxChunks],
                                                   int tl, int nchunks) {
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kMaxChunks; ++i) {
        const int c = tl + TEAM * i;
        if (c < nchunks) {
            const uint4 b = __ldg(row + c);
            acc = sq_diff_u8x4(qc[i].x, b.x, acc);
            acc = sq_diff_u8x4(qc[i].y, b.y, acc);
            acc = sq_diff_u8x4(qc[i].z, b.z, acc);
            acc = sq_diff_u8x4(qc[i].w, b.w, acc);
        }
    }
    return acc;
}

template <int TEAM>
__device__ __forceinline__ void load_chunks(const uint8_t* row, uint4 (&qc)[kMaxChunks], int tl,
                                            int nchunks) {
#pragma unroll
    for (int i = 0; i < kMaxChunks; ++i) {
        const int c = tl + TEAM * i;
        qc[i] = c < nchunks ? __ldg((const uint4*)row + c) : make_uint4(0, 0, 0, 0);
    }
}

// Partial FP32 squared distance over this lane's float4 groups of a row in
// shared memory (qf: the FP32 query in shared memory, 16-byte aligned and
// zero-padded).
__device__ __forceinline__ float f32_partial_s(const float4* row, const float* qf, int tl,
                                               int team_w, int ngroups) {
    float acc = 0.0f;
    for (int g = tl; g < ngroups; g += team_w) {
        const float4 b = row[g];
        const float* qq = qf + 4 * g;
        const float t0 = qq[0] - b.x, t1 = qq[1] - b.y, t2 = qq[2] - b.z, t3 = qq[3] - b.w;
        acc = fmaf(t0, t0, acc);
        acc = fmaf(t1, t1, acc);
        acc = fmaf(t2, t2, acc);
        acc = fmaf(t3, t3, acc);
    }
    return acc;
}

// Byte u of w as an exact float: the byte goes into the low mantissa bits
// of 2^23 (bit pattern 0x4B000000), and subtracting 2^23 leaves the byte's
// value (exact for 0..255).  Two full-rate instructions instead of an
// integer-to-float conversion.
__device__ __forceinline__ float byte_as_float(uint32_t w, int u) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650u | (unsigned)u)) - 8388608.0f;
}

// Stage 2 (Alg. 2), partial asymmetric distance over this lane's 32-bit
// words w = tl + TEAM * i < nw of a staged code row (four dimensions j =
// 4w .. 4w + 3 each): decoded value x~_j = fma(code_j, 1 / scale_j, min_j),
// (q_j - x~_j)^2 accumulated by fma, dimensions in ascending order within
// the lane.  qf, s_inv, s_min: FP32 query and constants in shared memory,
// 16-byte aligned, zero from d on (such dimensions add exactly +0, whatever
// their code byte), so nw = ceil(d / 4) needs no per-dimension test.  The
// TEAM lanes of a candidate read consecutive words: with the row stride of
// stage2_stride the rows read together sit in distinct banks.
template <int TEAM>
__device__ __forceinline__ float asym_partial_s(const uint32_t* row, const float* qf,
                                                const float* s_inv, const float* s_min, int tl,
                                                int nw) {
    const float4* q4 = (const float4*)qf;
    const float4* i4 = (const float4*)s_inv;
    const float4* m4 = (const float4*)s_min;
    float acc = 0.0f;
#pragma unroll 1
    for (int w = tl; w < nw; w += TEAM) {
        const uint32_t c = row[w];
        const float4 q = q4[w], iv = i4[w], mn = m4[w];
        const float d0 = q.x - fmaf(byte_as_float(c, 0), iv.x, mn.x);
        const float d1 = q.y - fmaf(byte_as_float(c, 1), iv.y, mn.y);
        const float d2 = q.z - fmaf(byte_as_float(c, 2), iv.z, mn.z);
        const float d3 = q.w - fmaf(byte_as_float(c, 3), iv.w, mn.w);
        acc = fmaf(d0, d0, acc);
        acc = fmaf(d1, d1, acc);
        acc = fmaf(d2, d2, acc);
        acc = fmaf(d3, d3, acc);
    }
    return acc;
}

// Row stride of the Stage-2 staging tile: the smallest multiple of 16 bytes
// >= dp whose word count is an odd multiple of TEAM.  The 32 / TEAM rows a
// warp reads at once then start TEAM * (odd * t mod 32 / TEAM) banks apart,
// i.e. in distinct groups of TEAM banks.
__host__ __device__ inline int stage2_stride(int dp, int team) {
    if (team >= 32) return dp;
    int s = dp;
    while ((s / 4) % (2 * team) != team) s += 16;
    return s;
}

// Quantised-path evaluator, one lane per candidate (code rows up to 256
// bytes).  Lanes reading the same chunk of 8 consecutive staged rows must
// hit distinct 16-byte bank groups: rows of a multiple of 8 chunks are
// stored unpadded with chunk c of row r in slot c ^ (r & 7) (swz = 7);
// other rows use a stride of an odd number of chunks (swz = 0).  The query
// codes sit in shared memory (broadcast reads).  The integer distance is
// sum(q^2) + sum(x^2) - 2 sum(q x), each sum an exact dp4a accumulation.
// NCH > 0 fixes the row at NCH chunks at compile time (nchunks == NCH):
// the kernel then holds one copy loop and one distance loop instead of
// the runtime choice among four, a smaller hot loop for the instruction
// cache.  NCH = 0 chooses at run time.
template <int NCH = 0>
struct CodeLaneEvalT {
    const uint8_t* codes;
    int dp, nchunks, stride, cap_rows, swz;
    unsigned char* stg;
    const uint4* qs;  // query codes, nchunks x 16 bytes
    uint32_t qq;      // sum of squared query codes
    uint64_t pol;     // L2 policy of code-row copies
    // Two lanes per row, each copying every other 16-byte chunk: a lane
    // touches 1/16 of the rows (one id load and one address per row) for
    // the same number of copies as wider groups.
    // Rows of 6, 8 and 16 chunks (d = 96, 128, 256) take a copy loop
    // unrolled for their width.
    __device__ __forceinline__ void stage(const uint32_t* ids, int cnt) {
        const auto id = [&](int r) { return ids[r]; };
        if constexpr (NCH > 0) {
            stage_rows<2, NCH, true>(stg, stride, codes, dp, id, cnt, pol, swz);
            return;
        }
        switch (nchunks) {
            case 6: stage_rows<2, 6, true>(stg, stride, codes, dp, id, cnt, pol, swz); break;
            case 8: stage_rows<2, 8, true>(stg, stride, codes, dp, id, cnt, pol, swz); break;
            case 16: stage_rows<2, 16, true>(stg, stride, codes, dp, id, cnt, pol, swz); break;
            default: stage_rows<2, 0, true>(stg, stride, codes, dp, id, cnt, pol, swz);
        }
    }
    __device__ __forceinline__ uint32_t dist(int r) const {
        const uint4* row = (const uint4*)(stg + (size_t)r * stride);
        const int x = r & swz;
        uint32_t dot0 = 0, dot1 = 0, bb0 = 0, bb1 = 0;
        const int nch = NCH > 0 ? NCH : nchunks;
        if ((NCH == 0 || NCH == 8) && nch == 8) {  // 128-byte rows: fully unrolled, same order of sums
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint4 b = row[c ^ x];
                const uint4 a = qs[c];
                dot0 = __dp4a(a.x, b.x, dot0);
                bb0 = __dp4a(b.x, b.x, bb0);
                dot1 = __dp4a(a.y, b.y, dot1);
                bb1 = __dp4a(b.y, b.y, bb1);
                dot0 = __dp4a(a.z, b.z, dot0);
                bb0 = __dp4a(b.z, b.z, bb0);
                dot1 = __dp4a(a.w, b.w, dot1);
                bb1 = __dp4a(b.w, b.w, bb1);
            }
            return qq + (bb0 + bb1) - 2u * (dot0 + dot1);
        }
#pragma unroll 2
        for (int c = 0; c < nch; ++c) {
            const uint4 b = row[c ^ x];
            const uint4 a = qs[c];
            dot0 = __dp4a(a.x, b.x, dot0);
            bb0 = __dp4a(b.x, b.x, bb0);
            dot1 = __dp4a(a.y, b.y, dot1);
            bb1 = __dp4a(b.y, b.y, bb1);
            dot0 = __dp4a(a.z, b.z, dot0);
            bb0 = __dp4a(b.z, b.z, bb0);
            dot1 = __dp4a(a.w, b.w, dot1);
            bb1 = __dp4a(b.w, b.w, bb1);
        }
        return qq + (bb0 + bb1) - 2u * (dot0 + dot1);
    }
};
using CodeLaneEval = CodeLaneEvalT<0>;

// Quantised-path evaluator for wide code rows: TEAM lanes per candidate,
// lane tl holding the probe's chunks tl + TEAM * i in registers.
template <int TEAM>
struct CodeEval {
    const uint8_t* codes;
    int dp, nchunks, tl, cap_rows;
    unsigned char* stg;
    uint4 qc[kMaxChunks];
    uint64_t pol;
    // four lanes per row (a quarter of the copies of a row each): fewer rows
    // per lane than with TEAM lanes per row
    __device__ __forceinline__ void stage(const uint32_t* ids, int cnt) {
        stage_rows<4, 0, true>(stg, dp, codes, dp, [&](int r) { return ids[r]; }, cnt, pol);
    }
    __device__ __forceinline__ uint32_t dist(int r) {
        return team_sum_u32<TEAM>(code_partial_s<TEAM>((const uint4*)(stg + (size_t)r * dp), qc, tl,
                                                       nchunks));
    }
};

// Plain-path evaluator: FP32 squared L2 of the staged FP32 rows (returned as
// the bit pattern, which orders like the non-negative value).
template <int TEAM>
struct F32Eval {
    const float* x;
    int row_bytes, ngroups, tl, cap_rows;
    unsigned char* stg;
    const float* qf;
    __device__ __forceinline__ void stage(const uint32_t* ids, int cnt) {
        stage_rows<TEAM, 0, false>(stg, row_bytes, (const unsigned char*)x, row_bytes,
                                   [&](int r) { return ids[r]; }, cnt, 0);
    }
    __device__ __forceinline__ uint32_t dist(int r) {
        return __float_as_uint(team_sum_f32<TEAM>(
            f32_partial_s((const float4*)(stg + (size_t)r * row_bytes), qf, tl, TEAM, ngroups)));
    }
};

// ---- sorting / searching helpers -------------------------------------------
// First index j in [0, n) with (W[j] & ~1) >= key (W ascending).
__device__ __forceinline__ int lower_bound_w(const u64* W, int n, u64 key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((W[mid] & ~1ull) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
// Number of entries of W[0, n) (ascending by key with the flag cleared) below
// key: binary search on the distance word (32-bit loads and compares) in
// power-of-two steps from the largest one <= n (lo only grows; no upper
// bound to keep), then a step over the entries of equal distance, compared
// in full.
__device__ __forceinline__ int rank_in_w(const u64* W, int n, u64 key) {
    const uint32_t* W32 = (const uint32_t*)W;  // W32[2j + 1]: distance word of W[j]
    const uint32_t kh = key_hi(key);
    int lo = 0;
    if (n > 0)
        for (int step = 1 << (31 - __clz(n)); step; step >>= 1)
            if (lo + step <= n && W32[2 * (lo + step) - 1] < kh) lo += step;
    while (lo < n && W32[2 * lo + 1] == kh && (W[lo] & ~1ull) < key) ++lo;
    return lo;
}
// Number of entries of sorted S[0, n) strictly below key.
__device__ __forceinline__ int count_below(const u64* S, int n, u64 key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// In-place ascending bitonic sort of W[0, P), P a power of two, by one warp.
__device__ inline void warp_bitonic_sort(u64* W, int P) {
    const int lane = threadIdx.x & 31;
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncwarp();
            for (int t = lane; t < P / 2; t += 32) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = ((i & size) == 0);
                const u64 a = W[i], b = W[j];
                if ((a > b) == up) {
                    W[i] = b;
                    W[j] = a;
                }
            }
        }
    }
    __syncwarp();
}

// Adjacency of one layer: row(id) -> pointer to `stride` entries (kNone-padded).
struct Layer {
    const uint32_t* base;
    const int32_t* upper_base;  // null for layer 0
    int stride;                 // entries per row (multiple of 32, at most 128)
    int lc;                     // layer number
    __device__ __forceinline__ const uint32_t* row(uint32_t id) const {
        if (lc == 0) return base + (int64_t)id * stride;
        return base + ((int64_t)upper_base[id] + lc - 1) * stride;
    }
};

// Load one row: lane l gets entries [l * epl, l * epl + epl), one vector load.
__device__ __forceinline__ void load_row(const uint32_t* row, int epl, uint32_t (&e)[4]) {
    const int lane = threadIdx.x & 31;
    e[0] = e[1] = e[2] = e[3] = kNone;
    if (epl == 2) {
        const uint2 v = __ldg((const uint2*)row + lane);
        e[0] = v.x;
        e[1] = v.y;
    } else if (epl == 4) {
        const uint4 v = __ldg((const uint4*)row + lane);
        e[0] = v.x;
        e[1] = v.y;
        e[2] = v.z;
        e[3] = v.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < epl) e[j] = __ldg(row + lane * epl + j);
    }
}

// Per-warp shared memory used by the layer search.
struct BeamMem {
    u64* W;            // [ef_cap] result set, ascending
    uint32_t* H;       // [2 * hsets] visited hash: hsets sets of 8 bytes
    uint32_t* cand;    // [rmax] new neighbour ids of one expansion
    u64* surv;         // [rmax] survivors of one expansion (team evaluators only)
    uint32_t hsets;    // number of sets
    uint32_t id_mask;  // tag16: 2^B - 1, B >= bits of the largest id
    int tag_bits;      // tag16: B - log2(hsets), at most 15
    int tag16;         // 1: four 16-bit tags per set; 0: two 32-bit ids per set
    int ef_cap;        // entries of W
    int rmax;          // entries of cand and surv
    int* err;          // error word of the checked build
};

constexpr uint32_t kHashMul = 0x9E3779B1u;  // odd: id -> id * kHashMul is a bijection mod 2^B

// Empty visited hash (all ways kNone / 0xFFFF), warp-collective.
__device__ __forceinline__ void visited_clear(BeamMem& m) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < 2 * (int)m.hsets; i += 32) m.H[i] = kNone;
}

// Test-and-insert of id e: true if e was not found (it is then inserted,
// unless another lane overwrites the same way in the same step).
//   tag16: hv = e * kHashMul mod 2^B; the set is the top log2(hsets) bits of
//     hv, the tag its low tag_bits bits; (set, tag) gives hv and so e.  A
//     full set gives up the way picked by two bits of a second hash.
//   32-bit ids: the set is a multiply-high range reduction of e * kHashMul
//     (any number of sets); a full set gives up the way picked by a hash bit.
__device__ __forceinline__ bool visited_insert(const BeamMem& m, uint32_t e) {
    if (m.tag16) {
        const uint32_t hv = (e * kHashMul) & m.id_mask;
        const uint32_t set = hv >> m.tag_bits;
        const uint32_t tag = hv & ((1u << m.tag_bits) - 1u);
        if (!AQR_IN(m.err, set < m.hsets)) return false;
        const uint2 pr = ((const uint2*)m.H)[set];
        // a 16-bit half of v equal to the tag is a zero half of v ^ (tag, tag)
        const uint32_t vx = pr.x ^ (tag * 0x10001u), vy = pr.y ^ (tag * 0x10001u);
        if (((vx - 0x10001u) & ~vx & 0x80008000u) | ((vy - 0x10001u) & ~vy & 0x80008000u))
            return false;
        // ways fill in order and full sets only overwrite, so the empty ways
        // (0xFFFF) are a suffix: the first empty way is the number of full ones
        const uint32_t full = (pr.x != 0xFFFFFFFFu) + (pr.x < 0xFFFF0000u) +
                              (pr.y != 0xFFFFFFFFu) + (pr.y < 0xFFFF0000u);
        const uint32_t way = full < 4u ? full : (e * 0x85EBCA6Bu) >> 30;
        ((uint16_t*)m.H)[4 * set + way] = (uint16_t)tag;
        return true;
    }
    const uint32_t hv = e * kHashMul;
    const uint32_t p = __umulhi(hv, m.hsets);
    if (!AQR_IN(m.err, p < m.hsets)) return false;
    const uint2 pr = ((const uint2*)m.H)[p];
    if (pr.x == e || pr.y == e) return false;
    const uint32_t way = pr.x == kNone ? 0u : pr.y == kNone ? 1u : (hv >> 7) & 1u;
    m.H[2 * p + way] = e;
    return true;
}

// Merge s <= 32 survivors into W.  Lane i < s holds survivor i (distinct
// keys, flag clear, each below the worst of W when W is full); other lanes
// hold EMPTY.  Each survivor is ranked in W (a survivor equal to a W entry is
// a re-evaluated duplicate and is dropped); valid survivor i lands at
// pos_i = rank_i + (valid survivors with a smaller key).  The other output
// positions of [p0, new nW) take the W entries from p0 on in order, so the
// output position o takes W[o - (survivor positions below o)], counted with
// one bitmap word per 32 positions.  Returns the position of the smallest
// inserted key, or INT_MAX when nothing was inserted.
__device__ __forceinline__ int merge_survivors(BeamMem& m, int& nW, int ef_eff, u64 x, int s) {
    const int lane = threadIdx.x & 31;
    const int rw = lane < s && AQR_IN(m.err, nW <= m.ef_cap) ? rank_in_w(m.W, nW, x) : nW;
    const bool valid = lane < s && !(rw < nW && (m.W[rw] & ~1ull) == x);
    const uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
    if (!vmask) return 0x7FFFFFFF;
    int below_me = 0;
    for (int j = 0; j < s; ++j) {
        const u64 xj = shfl_u64(x, j);
        below_me += ((vmask >> j) & 1u) && xj < x;
    }
    const int pos = rw + below_me;
    const int p0 = (int)__reduce_min_sync(0xFFFFFFFFu, valid ? (uint32_t)pos : 0x7FFFFFFFu);
    const int nW2 = min(nW + __popc(vmask), ef_eff);
    const int rel = pos - p0;  // survivor's position relative to p0 (valid lanes)
    const uint32_t below = (1u << lane) - 1u;
    for (int t = (nW2 - 1 - p0) >> 5; t >= 0; --t) {
        // survivors in this chunk of 32 output positions, and before it
        const uint32_t bm =
            __reduce_or_sync(0xFFFFFFFFu, valid && (rel >> 5) == t ? 1u << (rel & 31) : 0u);
        const int pre = __popc(__ballot_sync(0xFFFFFFFFu, valid && rel < 32 * t));
        const int o = p0 + 32 * t + lane;
        const int j = o - pre - __popc(bm & below);
        const bool mv = o < nW2 && !((bm >> lane) & 1u) && j != o &&
                        AQR_IN(m.err, j >= 0 && j < nW && o < m.ef_cap);
        const u64 w = mv ? m.W[j] : 0ull;
        __syncwarp();
        if (mv) m.W[o] = w;
        __syncwarp();
    }
    if (valid && pos < ef_eff && AQR_IN(m.err, pos >= 0 && pos < m.ef_cap)) m.W[pos] = x;
    __syncwarp();
    nW = nW2;
    return p0;
}

struct BeamStats {  // per query (or insertion): 32 bits suffice
    uint32_t expansions = 0, evals = 0, adj = 0, l0_evals = 0;
};

// Greedy descent on one layer (ef = 1): move to the best neighbour by
// (distance, id) while it is strictly better.
template <int TEAM, class Eval>
__device__ u64 greedy_layer(const Layer& L, u64 ck, BeamMem& m, Eval& ev, int64_t max_steps,
                            BeamStats& st) {
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31, team = lane / TEAM;
    const int epl = L.stride >> 5;
    for (int64_t step = 0; step <= max_steps; ++step) {
        const uint32_t cur = key_id(ck);
        uint32_t ent[4];
        load_row(L.row(cur), epl, ent);
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= epl) break;
            const bool ok = ent[j] != kNone;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
            const int at = cnt + __popc(bal & ((1u << lane) - 1));
            if (ok && AQR_IN(m.err, at < m.rmax)) m.cand[at] = ent[j];
            cnt += __popc(bal);
        }
        __syncwarp();
        st.expansions += 1;
        st.adj += cnt;
        st.evals += cnt;
        u64 best = kEmpty;
        for (int base = 0; base < cnt; base += ev.cap_rows) {
            const int nr = min(ev.cap_rows, cnt - base);
            ev.stage(m.cand + base, nr);
            for (int b2 = 0; b2 < nr; b2 += NT) {
                const int i = b2 + team;
                const uint32_t dv = ev.dist(i < nr ? i : 0);
                if (i < nr && AQR_IN(m.err, base + i < m.rmax)) {
                    const u64 kk = make_key(dv, m.cand[base + i]);
                    best = kk < best ? kk : best;
                }
            }
            __syncwarp();
        }
        best = warp_min_u64(best);
        __syncwarp();
        if (best < ck) ck = best;
        else break;
    }
    return ck;
}

// ef-bounded layer search from the entry key `ek` (flag clear).  Leaves the
// ascending result set in m.W[0, nW) (expanded flags set) and returns nW.
// exp_seq (optional) receives the expansion order, up to cap_exp entries.
template <int TEAM, class Eval>
__device__ int beam_layer(const Layer& L, u64 ek, int ef_eff, int ef_cap, BeamMem& m, Eval& ev,
                          int64_t max_exp, BeamStats& st, uint32_t* exp_seq, int cap_exp,
                          int* n_exp_out, bool* overflow) {
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31, team = lane / TEAM, tl = lane & (TEAM - 1);
    for (int i = lane; i < ef_cap; i += 32)
        if (AQR_IN(m.err, i < m.ef_cap)) m.W[i] = kEmpty;
    visited_clear(m);
    __syncwarp();
    if (lane == 0) {
        m.W[0] = ek;
        visited_insert(m, key_id(ek));
    }
    __syncwarp();
    int nW = 1, cursor = 0, n_exp = 0;
    const int epl = L.stride >> 5;
    while (cursor < nW) {
        if (n_exp > max_exp) {  // each node is expanded at most once
            *overflow = true;
            break;
        }
        if (!AQR_IN(m.err, cursor >= 0 && cursor < m.ef_cap)) break;
        const u64 c_key = m.W[cursor];
        const uint32_t cid = key_id(c_key);
        __syncwarp();
        if (lane == 0) m.W[cursor] = c_key | 1ull;
        if (exp_seq && lane == 0 && n_exp < cap_exp) exp_seq[n_exp] = cid;
        ++n_exp;
        // neighbour row (one vector load per lane), visited filter, compaction
        uint32_t ent[4];
        load_row(L.row(cid), epl, ent);
        // t: the first unexpanded entry after the cursor.  Unless a better
        // neighbour arrives it is the next one expanded: its row is
        // prefetched into L2 now.
        int t_next = nW;
        for (int base = cursor + 1; base < nW; base += 32) {
            const int j = base + lane;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, j < nW && !(m.W[j] & 1ull));
            if (bal) {
                t_next = base + __ffs(bal) - 1;
                const uint32_t* pr = L.row(key_id(m.W[t_next]));
                if (lane * 32 < L.stride) prefetch_l2(pr + lane * 32);
                break;
            }
        }
        int ncand = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= epl) break;
            const uint32_t e = ent[j];
            bool ok = e != kNone;
            st.adj += __popc(__ballot_sync(0xFFFFFFFFu, ok));
            if (ok) ok = visited_insert(m, e);  // one 8-byte load per probe
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
            const int at = ncand + __popc(bal & ((1u << lane) - 1));
            if (ok && AQR_IN(m.err, at < m.rmax)) m.cand[at] = e;
            ncand += __popc(bal);
        }
        __syncwarp();
        st.evals += ncand;
        if (L.lc == 0) st.l0_evals += ncand;
        // smallest position of a key inserted by this expansion (INT_MAX: none)
        int p0min = 0x7FFFFFFF;
        if constexpr (TEAM == 1) {
            // one lane per candidate: merge the survivors of every round
            // (at most 32) straight from registers
            for (int base = 0; base < ncand; base += ev.cap_rows) {
                const int nr = min(ev.cap_rows, ncand - base);
                if (!AQR_IN(m.err, base + nr <= m.rmax && nr <= 32)) break;
                ev.stage(m.cand + base, nr);
                const int r = lane < nr ? lane : 0;
                const uint32_t dv = ev.dist(r);
                const u64 worst = nW == ef_eff ? (m.W[ef_eff - 1] & ~1ull) : kEmpty;
                const u64 kk = make_key(dv, m.cand[base + r]);
                const bool sv = lane < nr && kk < worst;
                const uint32_t smask = __ballot_sync(0xFFFFFFFFu, sv);
                __syncwarp();
                if (smask) {
                    // compact through the staging tile, dead until the next round
                    const int s = __popc(smask);
                    u64* tmp = (u64*)ev.stg;
                    if (sv) tmp[__popc(smask & ((1u << lane) - 1u))] = kk;
                    __syncwarp();
                    const u64 xk = lane < s ? tmp[lane] : kEmpty;
                    __syncwarp();
                    const int p0 = merge_survivors(m, nW, ef_eff, xk, s);
                    p0min = min(p0min, p0);
                }
            }
        } else {
            const u64 worst = nW == ef_eff ? (m.W[ef_eff - 1] & ~1ull) : kEmpty;
            // distances of the staged rows; survivors are the keys below the worst
            int s = 0;
            for (int base = 0; base < ncand; base += ev.cap_rows) {
                const int nr = min(ev.cap_rows, ncand - base);
                if (!AQR_IN(m.err, base + nr <= m.rmax)) break;
                ev.stage(m.cand + base, nr);
                for (int b2 = 0; b2 < nr; b2 += NT) {
                    const int i = b2 + team;
                    const uint32_t dv = ev.dist(i < nr ? i : 0);
                    const u64 kk = make_key(dv, m.cand[base + (i < nr ? i : 0)]);
                    const bool sv = (i < nr) && (tl == 0) && kk < worst;
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, sv);
                    const int at = s + __popc(bal & ((1u << lane) - 1));
                    if (sv && AQR_IN(m.err, at < m.rmax)) m.surv[at] = kk;
                    s += __popc(bal);
                }
                __syncwarp();
            }
            if (s > 0 && s <= 32) {
                p0min = merge_survivors(m, nW, ef_eff, lane < s ? m.surv[lane] : kEmpty, s);
            } else if (s > 0) {
                    // (a) drop survivors already in W, remember their rank in W
                    u64 sk[4];
                    int rw[4];
        #pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int i = lane + 32 * t;
                        sk[t] = kEmpty;
                        rw[t] = 0;
                        if (i < s) {
                            const u64 kk = m.surv[i];
                            const int p = lower_bound_w(m.W, nW, kk);
                            const bool dup = p < nW && (m.W[p] & ~1ull) == kk;
                            sk[t] = dup ? kEmpty : kk;
                            rw[t] = p;
                        }
                    }
                    __syncwarp();
        #pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (lane + 32 * t < s) m.surv[lane + 32 * t] = sk[t];
                    __syncwarp();
                    // (b) rank among survivors -> final position in the merged W
                    int pos[4];
                    int s2 = 0;
        #pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        pos[t] = -1;
                        if (sk[t] != kEmpty) {
                            int r = 0;
                            for (int j = 0; j < s; ++j) r += m.surv[j] < sk[t];
                            pos[t] = rw[t] + r;
                        }
                        s2 += __popc(__ballot_sync(0xFFFFFFFFu, sk[t] != kEmpty));
                    }
                    __syncwarp();
                    // (c) survivors sorted in place
        #pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (sk[t] != kEmpty) m.surv[pos[t] - rw[t]] = sk[t];
                    __syncwarp();
                    if (s2 > 0) {
                        int p0 = 0x7FFFFFFF;
        #pragma unroll
                        for (int t = 0; t < 4; ++t)
                            if (sk[t] != kEmpty) p0 = min(p0, pos[t]);
        #pragma unroll
                        for (int mm = 16; mm; mm >>= 1) p0 = min(p0, __shfl_xor_sync(0xFFFFFFFFu, p0, mm));
                        // (d) shift W[p0, nW) right, highest chunk first
                        const int span = nW - p0;
                        for (int t = (span + 31) / 32 - 1; t >= 0; --t) {
                            const int j = p0 + 32 * t + lane;
                            u64 w = 0;
                            int np = -1;
                            if (j < nW) {
                                w = m.W[j];
                                np = j + count_below(m.surv, s2, w & ~1ull);
                            }
                            __syncwarp();
                            if (np >= 0 && np < ef_eff) m.W[np] = w;
                            __syncwarp();
                        }
                        // (e) survivors into their slots
        #pragma unroll
                        for (int t = 0; t < 4; ++t)
                            if (sk[t] != kEmpty && pos[t] < ef_eff) m.W[pos[t]] = sk[t];
                        __syncwarp();
                        nW = min(nW + s2, ef_eff);
                        p0min = p0;
                    }
            }

        }
        // next cursor: the first unexpanded entry.  Entries before t are
        // expanded; a key inserted at p0min shifts only the entries at or
        // after p0min, so the first unexpanded is at min(t, p0min).
        cursor = min(t_next, p0min);
        __syncwarp();
    }
    st.expansions += n_exp;
    if (n_exp_out) *n_exp_out = n_exp;
    return nW;
}

// ---- several warps per query ----------------------------------------------
// A group of G warps (G = 2 or 4, consecutive warps of one block) searches
// one query.  The result set W and the visited hash are the group's (in
// shared memory); every warp has its own candidate list and staging tile.
// Per expansion:
//   (A) barrier; every warp reads the cursor and |W| the leader published;
//   each warp loads its slice of the expanded node's neighbour list (entries
//   [gw * S, gw * S + S), S = stride / G), filters it through the shared
//   hash (distinct ids in one list, so the warps insert distinct ids; two
//   inserts into one set may lose one of them, which only forgets), stages
//   and evaluates its candidates and writes the keys below the worst of W
//   to its survivor list;
//   (B) barrier; the leader (warp 0 of the group) marks the expanded entry,
//   merges all survivors into W and publishes the next cursor and |W|.
// W after an expansion is the ef smallest of W and the new neighbours in any
// insertion order, so the expansion order and W are those of one warp.
// Every warp of the group passes the same barriers: the loop's decisions
// are taken on the published values that all warps read after (A).
struct GroupSync {
    int* sc;    // shared scalars (GS_*)
    u64* surv;  // [G][smax] survivors of each warp
    int smax;   // survivor slots per warp
    int G;      // warps in the group
    int gw;     // this warp's index in the group
    int bar;    // named barrier id of the group (1..15)
};
enum {
    GS_CURSOR = 0,
    GS_NW,
    GS_SLOT,
    GS_KEY_LO,
    GS_KEY_HI,
    GS_NE,
    GS_ET,
    GS_SCOUNT,  // G survivor counts from here
    GS_NUM = GS_SCOUNT + 4
};

// Named barrier of the group: id 1 or 2 (at most two groups per block), an
// immediate so that the kernel reserves only those barriers.
__device__ __forceinline__ void group_bar(const GroupSync& g) {
    if (g.bar == 1)
        asm volatile("bar.sync 1, %0;\n" ::"r"(g.G * 32) : "memory");
    else
        asm volatile("bar.sync 2, %0;\n" ::"r"(g.G * 32) : "memory");
}

// Entries [first, first + cnt) of a row, cnt <= 128: lane l gets entries
// first + l + 32 j for j < ceil(cnt / 32) (kNone past cnt); coalesced.
__device__ __forceinline__ void load_row_slice(const uint32_t* row, int first, int cnt,
                                               uint32_t (&e)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = lane + 32 * j;
        e[j] = i < cnt ? __ldg(row + first + i) : kNone;
    }
}

// Group form of beam_layer (same arguments; m.W and m.H are the group's,
// m.cand the warp's own).  Returns |W| to every warp of the group.
template <int TEAM, class Eval>
__device__ int beam_layer_group(const Layer& L, u64 ek, int ef_eff, int ef_cap, BeamMem& m,
                                const GroupSync& g, Eval& ev, int64_t max_exp, BeamStats& st,
                                uint32_t* exp_seq, int cap_exp, int* n_exp_out, bool* overflow) {
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31, team = lane / TEAM, tl = lane & (TEAM - 1);
    const bool leader = g.gw == 0;
    for (int i = g.gw * 32 + lane; i < ef_cap; i += g.G * 32)
        if (AQR_IN(m.err, i < m.ef_cap)) m.W[i] = kEmpty;
    for (int i = g.gw * 32 + lane; i < 2 * (int)m.hsets; i += g.G * 32) m.H[i] = kNone;
    group_bar(g);
    if (leader && lane == 0) {
        m.W[0] = ek;
        visited_insert(m, key_id(ek));
        g.sc[GS_CURSOR] = 0;
        g.sc[GS_NW] = 1;
    }
    const int S = L.stride / g.G;  // neighbour-list entries per warp
    const int epl = (S + 31) >> 5;
    int n_exp = 0, nW = 1;
    for (;;) {
        group_bar(g);  // (A)
        const int cursor = g.sc[GS_CURSOR];
        nW = g.sc[GS_NW];
        if (cursor >= nW) break;
        if (n_exp > max_exp) {  // each node is expanded at most once
            *overflow = true;
            break;
        }
        if (!AQR_IN(m.err, cursor >= 0 && cursor < m.ef_cap)) break;
        const uint32_t cid = key_id(m.W[cursor]);
        if (leader && exp_seq && lane == 0 && n_exp < cap_exp) exp_seq[n_exp] = cid;
        ++n_exp;
        uint32_t ent[4];
        load_row_slice(L.row(cid), g.gw * S, S, ent);
        // leader: the first unexpanded entry after the cursor (next cursor
        // unless a better neighbour arrives); its row is prefetched into L2
        int t_next = nW;
        if (leader) {
            for (int base = cursor + 1; base < nW; base += 32) {
                const int j = base + lane;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, j < nW && !(m.W[j] & 1ull));
                if (bal) {
                    t_next = base + __ffs(bal) - 1;
                    const uint32_t* pr = L.row(key_id(m.W[t_next]));
                    if (lane * 32 < L.stride) prefetch_l2(pr + lane * 32);
                    break;
                }
            }
        }
        int ncand = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= epl) break;
            const uint32_t e = ent[j];
            bool ok = e != kNone;
            st.adj += __popc(__ballot_sync(0xFFFFFFFFu, ok));
            if (ok) ok = visited_insert(m, e);
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
            const int at = ncand + __popc(bal & ((1u << lane) - 1));
            if (ok && AQR_IN(m.err, at < m.rmax)) m.cand[at] = e;
            ncand += __popc(bal);
        }
        __syncwarp();
        st.evals += ncand;
        if (L.lc == 0) st.l0_evals += ncand;
        // evaluate this warp's candidates; survivors: keys below the worst
        const u64 worst = nW == ef_eff ? (m.W[ef_eff - 1] & ~1ull) : kEmpty;
        u64* sv_out = g.surv + g.gw * g.smax;
        int s = 0;
        for (int base = 0; base < ncand; base += ev.cap_rows) {
            const int nr = min(ev.cap_rows, ncand - base);
            if (!AQR_IN(m.err, base + nr <= m.rmax)) break;
            ev.stage(m.cand + base, nr);
            for (int b2 = 0; b2 < nr; b2 += NT) {
                const int i = b2 + team;
                const int r = i < nr ? i : 0;
                const uint32_t dv = ev.dist(r);
                const u64 kk = make_key(dv, m.cand[base + r]);
                const bool sv = i < nr && tl == 0 && kk < worst;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, sv);
                const int at = s + __popc(bal & ((1u << lane) - 1));
                if (sv && AQR_IN(m.err, at < g.smax)) sv_out[at] = kk;
                s += __popc(bal);
            }
            __syncwarp();
        }
        if (lane == 0) g.sc[GS_SCOUNT + g.gw] = min(s, g.smax);
        group_bar(g);  // (B)
        if (leader) {
            if (lane == 0) m.W[cursor] |= 1ull;
            __syncwarp();
            // survivors of all warps, 32 at a time (distinct ids); entry i
            // of their concatenation is warp w's entry i - (counts before w)
            const int c0n = g.sc[GS_SCOUNT];
            const int c1n = g.G > 1 ? g.sc[GS_SCOUNT + 1] : 0;
            const int c2n = g.G > 2 ? g.sc[GS_SCOUNT + 2] : 0;
            const int c3n = g.G > 3 ? g.sc[GS_SCOUNT + 3] : 0;
            const int e1 = c0n, e2 = e1 + c1n, e3 = e2 + c2n, tot = e3 + c3n;
            int p0min = 0x7FFFFFFF;
            for (int c0 = 0; c0 < tot; c0 += 32) {
                const int i = c0 + lane;
                u64 x = kEmpty;
                if (i < tot) {
                    const int w = (i >= e1) + (i >= e2) + (i >= e3);
                    const int off = i - (w == 0 ? 0 : w == 1 ? e1 : w == 2 ? e2 : e3);
                    x = g.surv[w * g.smax + off];
                }
                const int p0 = merge_survivors(m, nW, ef_eff, x, min(32, tot - c0));
                p0min = min(p0min, p0);
            }
            if (lane == 0) {
                g.sc[GS_CURSOR] = min(t_next, p0min);
                g.sc[GS_NW] = nW;
            }
        }
    }
    if (leader) st.expansions += n_exp;
    if (n_exp_out) *n_exp_out = n_exp;
    return nW;
}

}  // namespace dev
}  // namespace aqr
