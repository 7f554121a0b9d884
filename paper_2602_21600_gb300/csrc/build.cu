// GPU graph construction on codes (Alg. 1).
//
// Nodes are inserted in id order in batches: node 0 alone, then
// b = min(max(1, s / batch_div), batch_max) nodes starting at node s.
// Within a batch:
//   1. search: one warp per new node v searches the graph as it stood before
//      the batch (greedy ef = 1 above v's level, then ef_c on each of v's
//      layers), selects at most M_i neighbours per layer with the HNSW
//      heuristic (Malkov & Yashunin, Alg. 4: keep e iff it is strictly closer
//      to v than to every kept neighbour), writes v's own lists, and emits
//      one reverse-link request (target row, v) per selected neighbour;
//   2. link: requests are grouped by target row; one warp per target applies
//      its incoming sources in ascending id: append while the list has room
//      (2 M_i on layer 0, M_i above), otherwise re-select the list plus the
//      new source with the same heuristic.
// The result does not depend on thread scheduling: searches read only rows
// that no thread writes during the search phase, and each target's updates
// are applied in a fixed order.  With batch_max = 1 this is the sequential
// insertion of Malkov & Yashunin (their Alg. 1).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "aqr_internal.h"
#include "beam.cuh"

namespace aqr {

aqr_status init_index_shape(Ctx* c, DeviceIndex& ix, int64_t n, int d, int M_i);
aqr_status upload_index_arrays(Ctx* c, DeviceIndex& ix, const float* mn, const float* sc,
                               const uint8_t* codes, const float* x, const uint32_t* adj0,
                               const int64_t* ub, const uint32_t* up);
int search_team_width(int dp);
HashGeom search_hash_geom(int ef_cap, int ldx, int64_t n, int requested, int tag_req);
int search_stage_bytes(int dp, int ldx, bool lane_path);

namespace {

using namespace dev;

constexpr int kWarps = 4;
constexpr int kThreads = 128;

struct BuildArgs {
    const uint8_t* codes;
    int dp;
    uint32_t* adj0;
    uint32_t* upper;
    const int32_t* upper_base;
    const uint32_t* upper_owner;
    const int32_t* level;
    int R0, R1, R0p, R1p;
    int64_t n;
    int M;
    int ef_c;
    // batch
    int64_t s, e;
    uint32_t ep;
    int L;
    // requests
    unsigned long long* req;  // (slot << 32) | source
    unsigned int* req_count;
    unsigned int* cnt;        // per slot
    unsigned int* off;
    unsigned int* fill;
    unsigned int* touched;
    unsigned int* n_touched;
    unsigned int* cursor;
    unsigned int* inc;
    int* error;
};

constexpr int kStageBytes = 4096;  // per-warp candidate staging (cp.async)

__host__ __device__ inline int build_warp_bytes(int ef_cap, int hsets, int rmax, int M) {
    int b = ef_cap * 8 + hsets * 8 + rmax * 4 + rmax * 8 + kStageBytes + ((M * 4 + 15) & ~15);
    return (b + 15) & ~15;
}

// HNSW neighbour-selection heuristic over the sorted keys C[0, nC) (distance
// to the base node in the high word).  Writes the kept ids to sel and their
// keys to selk (optional); returns how many were kept (<= Mmax).
template <int TEAM>
__device__ int select_heuristic(const u64* C, int nC, int Mmax, const uint8_t* codes, int dp,
                                uint32_t* sel, u64* selk) {
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31, team = lane / TEAM, tl = lane & (TEAM - 1);
    const int nchunks = dp >> 4;
    int c = 0;
    for (int i = 0; i < nC && c < Mmax; ++i) {
        const u64 ke = C[i];
        const uint32_t e = key_id(ke);
        const uint32_t de = key_hi(ke);
        uint4 ec[kMaxChunks];
        load_chunks<TEAM>(codes + (int64_t)e * dp, ec, tl, nchunks);
        bool good = true;
        for (int base = 0; base < c; base += NT) {
            const int j = base + team;
            const uint32_t r = j < c ? sel[j] : e;
            const uint32_t drr = team_sum_u32<TEAM>(
                code_partial_g<TEAM>((const uint4*)(codes + (int64_t)r * dp), ec, tl, nchunks));
            const bool viol = j < c && tl == 0 && drr <= de;
            if (__any_sync(0xFFFFFFFFu, viol)) {
                good = false;
                break;
            }
        }
        if (good) {
            if (lane == 0) {
                sel[c] = e;
                if (selk) selk[c] = ke & ~1ull;
            }
            ++c;
        }
        __syncwarp();
    }
    return c;
}

template <int TEAM>
__global__ void __launch_bounds__(kThreads, 4) insert_search_kernel(BuildArgs a, int ef_cap,
                                                                    HashGeom hg, int rmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int tl = lane & (TEAM - 1);
    const int nchunks = a.dp >> 4;
    unsigned char* wb = smem + wib * build_warp_bytes(ef_cap, hg.sets, rmax, a.M);
    BeamMem m;
    m.W = (u64*)wb;
    m.H = (uint32_t*)(wb + ef_cap * 8);
    m.cand = m.H + 2 * hg.sets;
    m.surv = (u64*)(m.cand + rmax);
    m.hsets = (uint32_t)hg.sets;
    m.id_mask = hg.id_mask;
    m.tag_bits = hg.tag_bits;
    m.tag16 = hg.tag16;
    m.ef_cap = ef_cap;
    m.rmax = rmax;
    m.err = a.error;
    unsigned char* stg = (unsigned char*)(m.surv + rmax);
    uint32_t* sel = (uint32_t*)(stg + kStageBytes);

    const int64_t v64 = a.s + (int64_t)blockIdx.x * kWarps + wib;
    if (v64 >= a.e) return;
    const uint32_t v = (uint32_t)v64;
    const int lv = a.level[v];
    CodeEval<TEAM> ev;
    ev.codes = a.codes;
    ev.dp = a.dp;
    ev.nchunks = nchunks;
    ev.tl = tl;
    ev.cap_rows = kStageBytes / a.dp;
    ev.stg = stg;
    ev.pol = policy_evict_last();  // code rows are re-read by every insertion
    load_chunks<TEAM>(a.codes + (int64_t)v * a.dp, ev.qc, tl, nchunks);
    BeamStats st;
    if (lane == 0) m.cand[0] = a.ep;
    __syncwarp();
    ev.stage(m.cand, 1);
    u64 ck = make_key(ev.dist(0), a.ep);
    __syncwarp();
    for (int lc = a.L; lc > lv; --lc) {
        const Layer Lu{a.upper, a.upper_base, a.R1p, lc};
        ck = greedy_layer<TEAM>(Lu, ck, m, ev, a.n, st);
    }
    for (int lc = min(a.L, lv); lc >= 0; --lc) {
        const Layer Ly = lc == 0 ? Layer{a.adj0, nullptr, a.R0p, 0}
                                 : Layer{a.upper, a.upper_base, a.R1p, lc};
        bool overflow = false;
        const int nW = beam_layer<TEAM>(Ly, ck & ~1ull, a.ef_c, ef_cap, m, ev, a.n, st, nullptr,
                                        0, nullptr, &overflow);
        if (overflow && lane == 0) atomicExch(a.error, 1);
        const int c = select_heuristic<TEAM>(m.W, nW, a.M, a.codes, a.dp, sel, nullptr);
        // v's own list at layer lc
        uint32_t* row = lc == 0 ? a.adj0 + (int64_t)v * a.R0p
                                : a.upper + ((int64_t)a.upper_base[v] + lc - 1) * a.R1p;
        const int stride = lc == 0 ? a.R0p : a.R1p;
        for (int i = lane; i < stride; i += 32) row[i] = i < c ? sel[i] : kNone;
        // reverse-link requests
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(a.req_count, (unsigned)c);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        for (int i = lane; i < c; i += 32) {
            const uint32_t r = sel[i];
            const unsigned long long slot =
                lc == 0 ? r : (unsigned long long)a.n + a.upper_base[r] + lc - 1;
            a.req[base + i] = (slot << 32) | v;
        }
        ck = m.W[0] & ~1ull;
        __syncwarp();
    }
}

__global__ void count_kernel(BuildArgs a, unsigned int max_req) {
    const unsigned int nreq = min(*a.req_count, max_req);
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < nreq; t += gridDim.x * blockDim.x) {
        const unsigned int slot = (unsigned int)(a.req[t] >> 32);
        if (atomicAdd(a.cnt + slot, 1u) == 0u) a.touched[atomicAdd(a.n_touched, 1u)] = slot;
    }
}

__global__ void offset_kernel(BuildArgs a) {
    const unsigned int nt = *a.n_touched;
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const unsigned int slot = a.touched[t];
        a.off[slot] = atomicAdd(a.cursor, a.cnt[slot]);
        a.fill[slot] = 0;
    }
}

__global__ void scatter_kernel(BuildArgs a, unsigned int max_req) {
    const unsigned int nreq = min(*a.req_count, max_req);
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < nreq; t += gridDim.x * blockDim.x) {
        const unsigned long long r = a.req[t];
        const unsigned int slot = (unsigned int)(r >> 32);
        a.inc[a.off[slot] + atomicAdd(a.fill + slot, 1u)] = (unsigned int)r;
    }
}

// One warp per touched row: apply the incoming sources in ascending id.
template <int TEAM>
__global__ void __launch_bounds__(kThreads) link_kernel(BuildArgs a) {
    constexpr int NT = 32 / TEAM;
    __shared__ uint32_t s_lst[kWarps][128];
    __shared__ u64 s_key[kWarps][384];  // candidates [0, P) + selected keys [P, P + cap)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int team = lane / TEAM, tl = lane & (TEAM - 1);
    const int nchunks = a.dp >> 4;
    const unsigned int nt = *a.n_touched;
    uint32_t* lst = s_lst[wib];
    u64* K = s_key[wib];
    for (unsigned int t = blockIdx.x * kWarps + wib; t < nt; t += gridDim.x * kWarps) {
        const unsigned int slot = a.touched[t];
        uint32_t* row;
        uint32_t r;
        int cap, stride;
        if (slot < a.n) {
            r = slot;
            row = a.adj0 + (int64_t)r * a.R0p;
            cap = a.R0;
            stride = a.R0p;
        } else {
            const int64_t u = (int64_t)slot - a.n;
            r = a.upper_owner[u];
            row = a.upper + u * a.R1p;
            cap = a.R1;
            stride = a.R1p;
        }
        uint4 rc[kMaxChunks];
        load_chunks<TEAM>(a.codes + (int64_t)r * a.dp, rc, tl, nchunks);
        auto dist = [&](uint32_t u) -> uint32_t {
            return team_sum_u32<TEAM>(
                code_partial_g<TEAM>((const uint4*)(a.codes + (int64_t)u * a.dp), rc, tl, nchunks));
        };
        // current list and its distances to r (keys in K[0, c))
        int c = 0;
        for (int base = 0; base < stride; base += 32) {
            const uint32_t e = row[base + lane];
            const bool ok = e != kNone;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ok);
            if (ok) lst[c + __popc(bal & ((1u << lane) - 1))] = e;
            c += __popc(bal);
        }
        __syncwarp();
        for (int base = 0; base < c; base += NT) {
            const int i = base + team;
            const uint32_t u = i < c ? lst[i] : r;
            const uint32_t du = dist(u);
            if (i < c && tl == 0) K[i] = make_key(du, u);
        }
        __syncwarp();
        const unsigned int n_in = a.cnt[slot];
        const unsigned int* in = a.inc + a.off[slot];
        int64_t last = -1;
        for (unsigned int it = 0; it < n_in; ++it) {
            // next source: smallest id above the last one applied
            uint32_t best = kNone;
            for (unsigned int j = lane; j < n_in; j += 32) {
                const uint32_t s = in[j];
                if ((int64_t)s > last && s < best) best = s;
            }
#pragma unroll
            for (int mm = 16; mm; mm >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, mm));
            last = best;
            const uint32_t dv = dist(best);
            if (c < cap) {
                if (lane == 0) K[c] = make_key(dv, best);
                ++c;
                __syncwarp();
            } else {
                if (lane == 0) K[c] = make_key(dv, best);
                int P = 1;
                while (P < c + 1) P <<= 1;
                __syncwarp();
                for (int i = c + 1 + lane; i < P; i += 32) K[i] = kEmpty;
                warp_bitonic_sort(K, P);
                // re-select into lst, keys written back into K afterwards
                const int nc = select_heuristic<TEAM>(K, c + 1, cap, a.codes, a.dp, lst, K + P);
                __syncwarp();
                for (int i = lane; i < nc; i += 32) K[i] = K[P + i];
                c = nc;
                __syncwarp();
            }
        }
        for (int i = lane; i < stride; i += 32) row[i] = i < c ? key_id(K[i]) : kNone;
        if (lane == 0) a.cnt[slot] = 0;
        __syncwarp();
    }
}

}  // namespace
}  // namespace aqr

using namespace aqr;

static aqr_status build_graph_impl(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d,
                                   const float* min_host, const float* scale_host,
                                   const double* U_host, int32_t M_i, int32_t ef_c,
                                   int32_t batch_div, int32_t batch_max, double s_dist) {
    NvtxRange range("aqr.build_graph");
    if (!ctx) return AQR_ERR_INVALID_ARG;
    if (ctx->serve)
        return fail(ctx, AQR_ERR_BUSY, "aqr_build_graph: stop serving before replacing the index");
    if (!x_dev || !min_host || !scale_host || !U_host || ef_c < 1 || ef_c > 1024 ||
        batch_div < 1 || batch_max < 1)
        return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_build_graph: bad arguments");
    for (int j = 0; j < d; ++j)
        if (!(scale_host[j] > 0.0f) || !std::isfinite(min_host[j]))
            return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_build_graph: bad quantiser parameters");
    cudaSetDevice(ctx->device);
    DeviceIndex ix;
    IndexGuard guard(ix);  // device arrays released unless the index is committed
    aqr_status st = init_index_shape(ctx, ix, n, d, M_i);
    if (st != AQR_OK) return st;
    if (ix.R0p > 128) return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_build_graph: M_i > 64");
    // levels l = floor(-ln(U) / ln(M_i)), rows of the upper layers
    std::vector<int32_t> lv(n);
    std::vector<int64_t> ub(n);
    const double mL = 1.0 / std::log((double)M_i);
    int64_t rows = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(U_host[i] > 0.0 && U_host[i] <= 1.0))
            return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_build_graph: U must lie in (0, 1]");
        lv[i] = (int32_t)std::floor(-std::log(U_host[i]) * mL);
        if (lv[i] > 32) return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_build_graph: level above 32");
        ub[i] = lv[i] > 0 ? rows : -1;
        rows += lv[i];
    }
    if (n + rows >= 0xFFFFFFFFll) return fail(ctx, AQR_ERR_INVALID_ARG, "aqr_build_graph: too many rows");
    std::vector<uint32_t> owner(std::max<int64_t>(rows, 1));
    for (int64_t i = 0; i < n; ++i)
        for (int l = 0; l < lv[i]; ++l) owner[ub[i] + l] = (uint32_t)i;
    ix.n_upper = rows;
    ix.ef_c = ef_c;
    ix.s_dist = s_dist;
    st = upload_index_arrays(ctx, ix, min_host, scale_host, nullptr, nullptr, nullptr, ub.data(), nullptr);
    if (st != AQR_OK) return st;
    cudaStream_t s = ctx->own_stream;

    // batch schedule and the entry point / top level before each batch
    std::vector<int64_t> starts;
    for (int64_t p = 0; p < n;) {
        starts.push_back(p);
        int64_t b = p == 0 ? 1 : std::min<int64_t>(std::max<int64_t>(1, p / batch_div), batch_max);
        p = std::min(n, p + b);
    }
    starts.push_back(n);
    const int nb = (int)starts.size() - 1;
    std::vector<uint32_t> ep_b(nb);
    std::vector<int> L_b(nb);
    std::vector<int64_t> req_b(nb);
    uint32_t ep = kNoId;
    int L = -1;
    int64_t max_req = 1;
    for (int b = 0; b < nb; ++b) {
        ep_b[b] = ep;
        L_b[b] = L;
        int64_t rq = 0;
        for (int64_t v = starts[b]; v < starts[b + 1]; ++v) {
            if (ep != kNoId) rq += (int64_t)(std::min(L, lv[v]) + 1) * M_i;
        }
        req_b[b] = rq;
        max_req = std::max(max_req, rq);
        for (int64_t v = starts[b]; v < starts[b + 1]; ++v)
            if (lv[v] > L) {
                L = lv[v];
                ep = (uint32_t)v;
            }
    }
    ix.entry = ep;
    ix.max_level = L;

    int32_t* d_level = nullptr;
    uint32_t* d_owner = nullptr;
    unsigned long long* d_req = nullptr;
    unsigned int *d_cnt = nullptr, *d_off = nullptr, *d_fill = nullptr, *d_touched = nullptr,
                 *d_inc = nullptr, *d_scal = nullptr;
    const int64_t slots = n + rows;
    auto cleanup = [&]() {
        cudaFree(d_level);
        cudaFree(d_owner);
        cudaFree(d_req);
        cudaFree(d_cnt);
        cudaFree(d_off);
        cudaFree(d_fill);
        cudaFree(d_touched);
        cudaFree(d_inc);
        cudaFree(d_scal);
    };
    cudaError_t e = cudaMalloc(&d_level, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_owner, owner.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_req, max_req * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_cnt, slots * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_off, slots * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_fill, slots * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_touched, max_req * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_inc, max_req * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_scal, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_level, lv.data(), n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_owner, owner.data(), owner.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, slots * 4, s);
    // FP32 store and codes (Alg. 1)
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(ix.x, (size_t)ix.ldx * 4, x_dev, (size_t)d * 4, (size_t)d * 4, n,
                              cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_encode(x_dev, n, d, d, ix.qmin, ix.qscale, ix.codes, ix.dp, s);
    if (e != cudaSuccess) {
        cleanup();
        ix.release();
        return cuda_fail(ctx, e, "aqr_build_graph setup");
    }
    BuildArgs a{};
    a.codes = ix.codes;
    a.dp = ix.dp;
    a.adj0 = ix.adj0;
    a.upper = ix.upper;
    a.upper_base = ix.upper_base;
    a.upper_owner = d_owner;
    a.level = d_level;
    a.R0 = ix.R0;
    a.R1 = ix.R1;
    a.R0p = ix.R0p;
    a.R1p = ix.R1p;
    a.n = n;
    a.M = M_i;
    a.ef_c = ef_c;
    a.req = d_req;
    a.req_count = d_scal;
    a.n_touched = d_scal + 1;
    a.cursor = d_scal + 2;
    a.cnt = d_cnt;
    a.off = d_off;
    a.fill = d_fill;
    a.touched = d_touched;
    a.inc = d_inc;
    a.error = ctx->d_error;

    const int team = search_team_width(ix.dp);
    const int ef_cap = ef_class_cap(ef_c);
    const HashGeom hg = search_hash_geom(ef_cap, ix.ldx, ix.n, 0, 0);
    const int rmax = std::max(ix.R0p, ix.R1p);
    const int smem = kWarps * build_warp_bytes(ef_cap, hg.sets, rmax, M_i);
    auto ins = team == 4 ? insert_search_kernel<4> : team == 8 ? insert_search_kernel<8>
             : team == 16 ? insert_search_kernel<16> : insert_search_kernel<32>;
    auto lnk = team == 4 ? link_kernel<4> : team == 8 ? link_kernel<8>
             : team == 16 ? link_kernel<16> : link_kernel<32>;
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {
        if (ep_b[b] == kNoId) continue;  // first node: nothing to search
        a.s = starts[b];
        a.e = starts[b + 1];
        a.ep = ep_b[b];
        a.L = L_b[b];
        const unsigned int mr = (unsigned int)req_b[b];
        e = cudaMemsetAsync(d_scal, 0, 4 * sizeof(unsigned int), s);
        if (e != cudaSuccess) break;
        const int64_t nodes = a.e - a.s;
        {
            std::lock_guard<std::mutex> g(kernel_attr_mutex());  // from the set to the launch
            e = cudaFuncSetAttribute(ins, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) break;
            ins<<<(unsigned)((nodes + kWarps - 1) / kWarps), kThreads, smem, s>>>(a, ef_cap, hg, rmax);
        }
        const unsigned g = (unsigned)std::min<int64_t>((mr + 255) / 256, 4096);
        count_kernel<<<g, 256, 0, s>>>(a, mr);
        offset_kernel<<<g, 256, 0, s>>>(a);
        scatter_kernel<<<g, 256, 0, s>>>(a, mr);
        const unsigned gl = (unsigned)std::min<int64_t>((mr + kWarps - 1) / kWarps, 8192);
        lnk<<<gl, kThreads, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) {
        ix.release();
        return cuda_fail(ctx, e, "aqr_build_graph");
    }
    if (err) {
        ix.release();
        cudaMemset(ctx->d_error, 0, sizeof(int));
        return fail(ctx, AQR_ERR_INTERNAL, "aqr_build_graph: device-side bound exceeded");
    }
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    ctx->ix.release();
    guard.commit();
    ctx->ix = std::move(ix);
    ctx->has_index = true;
    ++ctx->config_gen;
    return AQR_OK;
}

// Host allocations (levels, batch schedule, per-node tables) become
// AQR_ERR_NO_MEMORY, not an exception through the C boundary.
extern "C" aqr_status aqr_build_graph(aqr_ctx* ctx, const float* x_dev, int64_t n, int32_t d,
                                      const float* min_host, const float* scale_host,
                                      const double* U_host, int32_t M_i, int32_t ef_c,
                                      int32_t batch_div, int32_t batch_max, double s_dist) {
    try {
        return build_graph_impl(ctx, x_dev, n, d, min_host, scale_host, U_host, M_i, ef_c,
                                batch_div, batch_max, s_dist);
    } catch (const std::bad_alloc&) {
        return fail(ctx, AQR_ERR_NO_MEMORY, "aqr_build_graph: out of host memory");
    }
}
