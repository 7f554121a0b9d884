// Persistent batched query kernel (Alg. 2): one warp per query; warps pull
// queries from a work counter until the launch's queries are exhausted.
//
// Per query:
//   encode the FP32 query to uint8 codes (Alg. 2), in shared memory for one
//     lane per candidate, in registers for teams of lanes per candidate
//   greedy descent with ef = 1 through layers L..1
//   layer-0 search with ef_eff = max(ef, k) on integer code distances
//     (Alg. 2), result set W sorted in shared memory, visited ids in a
//     set-associative hash in shared memory
//   C = W[0:N_c); Stage 2: asymmetric distances to the decoded codes
//     x~_j = code_j / scale_j + min_j, sort by (d^a, id) (Alg. 2)
//   early termination test on d^a_k, d^a_k+1 (Alg. 2)
//   Stage 3: exact FP32 distances for the first n_exact of A
//   merge with the rest of A, sort by (distance, id), top k
// Every candidate row (codes in Stages 1-2, FP32 vectors in Stage 3) is
// gathered into a per-warp shared staging buffer with cp.async before use.
//
// The plain comparison path (PLAIN = true) runs the same search with FP32
// distances on the FP32 vectors and returns the top k of W directly.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "aqr_internal.h"
#include "beam.cuh"

#include "search_common.cuh"

namespace aqr {
namespace {

using namespace dev;


// TEAM: lanes per candidate in Stages 2-3 (and in Stage 1 when LANE is
// false); LANE: Stage-1 code distances one lane per candidate.
// Register bound: 8 blocks per SM (64 registers) where shared memory allows
// that many; the team kernels of the quantised path (wide code rows, 4 to 5
// blocks by shared memory) get 5 blocks' worth (102 registers).
template <bool PLAIN, int TEAM, bool LANE, int NCH = 0>
__device__ __forceinline__ void search_body(const SearchArgs& a, const WarpLayout& wl) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NT = 32 / TEAM;  // teams per warp
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int tl = lane & (TEAM - 1);
    const int team = lane / TEAM;
    const int d = a.d;
    const int nchunks = a.dp >> 4;
    const int ngroups = a.ldx >> 2;
    const int xrow = a.ldx * 4;

    // Block area: dequantisation constants min_j and 1/scale_j.
    float* s_min = (float*)smem;
    float* s_inv = s_min + a.ldx;
    const int blk_bytes = PLAIN ? 0 : ((2 * a.ldx * 4 + 15) & ~15);
    if (!PLAIN) {
        for (int j = threadIdx.x; j < a.ldx; j += blockDim.x) {
            s_min[j] = j < d ? a.qmin[j] : 0.0f;
            s_inv[j] = j < d ? a.qinv[j] : 0.0f;
        }
    }
    __syncthreads();
    unsigned char* wbase = smem + blk_bytes + wib * wl.bytes();
    BeamMem m;
    m.W = (u64*)wbase;
    m.H = (uint32_t*)(wbase + wl.ef_cap * 8);
    m.cand = m.H + 2 * wl.hg.sets;
    m.surv = (u64*)(m.cand + wl.rmax);
    m.hsets = (uint32_t)wl.hg.sets;
    m.id_mask = wl.hg.id_mask;
    m.tag_bits = wl.hg.tag_bits;
    m.tag16 = wl.hg.tag16;
    m.ef_cap = wl.ef_cap;
    m.rmax = wl.rmax;
    m.err = a.error;
    unsigned char* stg = (unsigned char*)(m.surv + wl.surv);
    // FP32 query: its own area on the plain path; on the quantised path it
    // reuses the visited hash, which is dead after Stage 1.
    float* qf = PLAIN ? (float*)(stg + wl.stg) : (float*)m.H;
    uint4* qs = (uint4*)(stg + wl.stg);  // query codes (lane-per-candidate path)

    const Layer L0{a.adj0, nullptr, a.R0p, 0};
    // code rows stay in L2 across queries; FP32 rows of the re-rank do not
    const uint64_t pol_codes = policy_evict_last();
    const uint64_t pol_rows = policy_evict_first();

    for (;;) {
        unsigned int slot = 0;
        if (lane == 0) slot = atomicAdd(a.work, 1u);
        slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
        if ((int64_t)slot >= a.nq) break;
        const int64_t qrow = a.q_index ? a.q_index[slot] : (int64_t)slot;
        const int k = a.q_k ? a.q_k[qrow] : a.k;
        const int ef = a.q_ef ? a.q_ef[qrow] : a.ef;
        const int ef_eff = max(ef, k);
        int Nc = a.n_coarse > 0 ? a.n_coarse : (ef_eff + a.m_ef - 1) / a.m_ef;
        Nc = min(max(Nc, k), ef_eff);
        int Nr = a.n_rerank > 0 ? a.n_rerank : (int)(((int64_t)Nc * a.rerank_pct + 99) / 100);
        Nr = min(max(Nr, k), Nc);
        const float* qv = a.q + qrow * a.ldq;

        // ---- evaluators: query codes (registers or shared) / FP32 query
        CodeEval<TEAM> ce;
        CodeLaneEvalT<NCH> le;
        F32Eval<TEAM> fe;
        if constexpr (!PLAIN && LANE) {
            // lane c encodes chunk c (16 dimensions) into shared memory
            uint32_t qq = 0;
            if (lane < nchunks) {
                const uint4 w = encode_chunk(qv, a.qmin, a.qscale, lane, d);
                qs[lane] = w;
                qq = __dp4a(w.x, w.x, __dp4a(w.y, w.y, __dp4a(w.z, w.z, __dp4a(w.w, w.w, 0u))));
            }
            le.codes = a.codes;
            le.dp = a.dp;
            le.nchunks = nchunks;
            le.swz = (nchunks & 7) == 0 ? 7 : 0;
            le.stride = search_lane_stride(a.dp);
            le.cap_rows = min(32, wl.stg / le.stride);
            le.stg = stg;
            le.qs = qs;
            le.qq = __reduce_add_sync(0xFFFFFFFFu, qq);
            le.pol = pol_codes;
        } else if constexpr (!PLAIN) {
            ce.codes = a.codes;
            ce.dp = a.dp;
            ce.nchunks = nchunks;
            ce.tl = tl;
            ce.cap_rows = wl.stg / a.dp;
            ce.stg = stg;
            ce.pol = pol_codes;
#pragma unroll
            for (int i = 0; i < kMaxChunks; ++i) {
                const int c = tl + TEAM * i;
                ce.qc[i] = c < nchunks ? encode_chunk(qv, a.qmin, a.qscale, c, d)
                                       : make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
            for (int j = lane; j < a.ldx; j += 32) qf[j] = j < d ? qv[j] : 0.0f;
            fe.x = a.x;
            fe.row_bytes = xrow;
            fe.ngroups = ngroups;
            fe.tl = tl;
            fe.cap_rows = wl.stg / xrow;
            fe.stg = stg;
            fe.qf = qf;
        }
        __syncwarp();

        BeamStats st;
        int n_l0exp = 0;
        bool overflow = false;
        uint32_t* exp_seq = a.tr.exp_seq ? a.tr.exp_seq + qrow * a.tr.cap_exp : nullptr;
        int nW;
        u64 ck;
        {
            // entry point, greedy descent through the upper layers, layer 0
            uint32_t ep = a.entry;
            m.cand[0] = ep;
            __syncwarp();
            constexpr int BT = (!PLAIN && LANE) ? 1 : TEAM;  // lanes per candidate in Stage 1
            auto run = [&](auto& ev) {
                ev.stage(m.cand, 1);
                const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, ev.dist(0), 0);
                ck = make_key(d0, ep);
                __syncwarp();
                st.evals += 1;
                for (int lc = a.max_level; lc >= 1; --lc) {
                    const Layer Lu{a.upper, a.upper_base, a.R1p, lc};
                    ck = greedy_layer<BT>(Lu, ck, m, ev, a.n, st);
                }
                if (a.tr.l0_entry && lane == 0) a.tr.l0_entry[qrow] = key_id(ck);
                nW = beam_layer<BT>(L0, ck & ~1ull, ef_eff, wl.ef_cap, m, ev, a.n, st, exp_seq,
                                    a.tr.cap_exp, &n_l0exp, &overflow);
            };
            if constexpr (PLAIN) run(fe);
            else if constexpr (LANE) run(le);
            else run(ce);
        }
        if (overflow && lane == 0) atomicExch(a.error, 1);

        const int nc = min(Nc, nW);
        if (a.tr.exp_count && lane == 0) a.tr.exp_count[qrow] = n_l0exp;
        if (a.tr.c_count && lane == 0) a.tr.c_count[qrow] = nc;
        if (a.tr.c_ids)
            for (int i = lane; i < nc; i += 32) {
                const u64 kk = m.W[i];
                a.tr.c_ids[qrow * a.tr.cap_c + i] = key_id(kk);
                a.tr.c_dist[qrow * a.tr.cap_c + i] = (int32_t)key_hi(kk);
            }
        __syncwarp();

        int ne = 0, et = 0;
        int nout;
        if (PLAIN) {
            nout = nW;
        } else {
            // ---- Stage 2: asymmetric distances to the decoded candidates
            for (int j = lane; j < a.ldx; j += 32) qf[j] = j < d ? qv[j] : 0.0f;
            __syncwarp();
            const int st2 = stage2_stride(a.dp, TEAM);
            const int nw = (d + 3) >> 2;
            const int cap2 = wl.stg / st2;
            const int win2 = prefetch_window(cap2, a.dp);
            for (int base = 0; base < nc; base += cap2) {
                const int nr = min(cap2, nc - base);
                const u64* Wb = m.W + base;
                // rows [base, base + win2) prefetched once this round is issued
                const int pf = base ? min(nc, base - cap2 + win2) : 0;
                prefetch_rows_l2(a.codes, a.dp, m.W + pf, min(nc, base + win2) - pf);
                stage_rows<TEAM, 0, true>(stg, st2, a.codes, a.dp,
                                          [&](int r) { return key_id(Wb[r]); }, nr, pol_codes);
                for (int b2 = 0; b2 < nr; b2 += NT) {
                    const int i = b2 + team;
                    const int r = i < nr ? i : 0;
                    const uint32_t v = key_id(m.W[base + r]);
                    float acc = asym_partial_s<TEAM>((const uint32_t*)(stg + (size_t)r * st2), qf,
                                                     s_inv, s_min, tl, nw);
                    acc = team_sum_f32<TEAM>(acc);
                    __syncwarp();
                    if (i < nr && tl == 0)
                        m.W[base + i] = ((u64)__float_as_uint(acc) << 32) | ((u64)v << 1);
                }
                __syncwarp();
            }
            int P = 1;
            while (P < nc) P <<= 1;
            if (!AQR_IN(a.error, P <= wl.ef_cap)) P = 1;
            for (int i = nc + lane; i < P; i += 32) m.W[i] = kEmpty;
            warp_bitonic_sort(m.W, P);
            if (a.tr.a_ids)
                for (int i = lane; i < nc; i += 32) {
                    const u64 kk = m.W[i];
                    a.tr.a_ids[qrow * a.tr.cap_c + i] = key_id(kk);
                    a.tr.a_dist[qrow * a.tr.cap_c + i] = __uint_as_float(key_hi(kk));
                }
            // ---- early termination (Section 3.2)
            if (nc > k) {
                const float dk = __uint_as_float(key_hi(m.W[k - 1]));
                const float dk1 = __uint_as_float(key_hi(m.W[k]));
                const float gap = (dk1 - dk) / (dk + a.eps);
                const float ratio = dk1 / (dk + a.eps);
                et = (gap > a.tau_gap || ratio > a.tau_ratio) ? 1 : 0;
            }
            ne = et ? min(k, nc) : min(Nr, nc);
            __syncwarp();
            // ---- Stage 3: exact FP32 distances for the first ne entries
            const int cap3 = wl.stg / xrow;
            const int win3 = prefetch_window(cap3, xrow);
            for (int base = 0; base < ne; base += cap3) {
                const int nr = min(cap3, ne - base);
                const u64* Wb = m.W + base;
                const int pf = base ? min(ne, base - cap3 + win3) : 0;
                prefetch_rows_l2((const unsigned char*)a.x, xrow, m.W + pf, min(ne, base + win3) - pf);
                stage_rows<TEAM, 0, true>(stg, xrow, (const unsigned char*)a.x, xrow,
                                          [&](int r) { return key_id(Wb[r]); }, nr, pol_rows);
                for (int b2 = 0; b2 < nr; b2 += NT) {
                    const int i = b2 + team;
                    const int r = i < nr ? i : 0;
                    const uint32_t v = key_id(m.W[base + r]);
                    float acc = f32_partial_s((const float4*)(stg + (size_t)r * xrow), qf, tl, TEAM,
                                              ngroups);
                    acc = team_sum_f32<TEAM>(acc);
                    __syncwarp();
                    if (i < nr && tl == 0)
                        m.W[base + i] = ((u64)__float_as_uint(acc) << 32) | ((u64)v << 1) | 1ull;
                }
                __syncwarp();
            }
            // ---- assembly: exact head and asymmetric tail in one order
            warp_bitonic_sort(m.W, P);
            nout = nc;
        }
        // ---- top k
        for (int i = lane; i < a.k_stride; i += 32) {
            const int64_t o = qrow * a.k_stride + i;
            if (i < k && i < nout) {
                const u64 kk = m.W[i];
                a.ids[o] = key_id(kk);
                a.dists[o] = __uint_as_float(key_hi(kk));
                if (a.exact) a.exact[o] = PLAIN ? 1 : (uint8_t)(kk & 1ull);
            } else {
                a.ids[o] = -1;
                a.dists[o] = __int_as_float(0x7f800000);
                if (a.exact) a.exact[o] = 0;
            }
        }
        if (lane == 0) {
            if (a.tr.et) a.tr.et[qrow] = (uint8_t)et;
            if (a.tr.n_exact) a.tr.n_exact[qrow] = ne;
            unsigned long long* C = a.counters;
            atomicAdd(C + C_QUERIES, 1ull);
            atomicAdd(C + C_EXPANSIONS, (unsigned long long)st.expansions);
            atomicAdd(C + C_EVALS, (unsigned long long)st.evals);
            atomicAdd(C + C_ADJ, (unsigned long long)st.adj);
            atomicAdd(C + C_STAGE2, (unsigned long long)(PLAIN ? 0 : nc));
            atomicAdd(C + C_EXACT, (unsigned long long)ne);
            atomicAdd(C + C_ET, (unsigned long long)et);
            atomicAdd(C + C_EVALS_L0, (unsigned long long)st.l0_evals);
        }
        __syncwarp();
    }
}

// NCH: code-row chunks fixed at compile time on the lane path (0: any).
template <bool PLAIN, int TEAM, bool LANE, int NCH = 0>
__global__ void __launch_bounds__(kThreads, (PLAIN || LANE) ? 8 : 5)
    search_kernel(SearchArgs a, WarpLayout wl) {
    search_body<PLAIN, TEAM, LANE, NCH>(a, wl);
}

// The lane path in blocks of kWideWarps warps, registers capped so that
// kWideBlocks blocks fit an SM.  NCH as for search_kernel.
template <int TEAM, int NCH = 0>
__global__ void __maxnreg__(56) search_kernel_wide(SearchArgs a, WarpLayout wl) {
    search_body<false, TEAM, true, NCH>(a, wl);
}

template <class K>
cudaError_t launch_k(K kern, int wpb, bool plain, const SearchArgs& a, const WarpLayout& wl,
                     int num_sms, cudaStream_t s) {
    const int blk = plain ? 0 : ((2 * a.ldx * 4 + 15) & ~15);
    const int smem = blk + wpb * wl.bytes();
    std::lock_guard<std::mutex> g(kernel_attr_mutex());  // from the set to the launch
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = kernel_occupancy((const void*)kern, wpb * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (a.nq + wpb - 1) / wpb;
    int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, wpb * 32, smem, s>>>(a, wl);
    return cudaGetLastError();
}

template <bool PLAIN, int TEAM, bool LANE, int NCH = 0>
cudaError_t launch_t(const SearchArgs& a, const WarpLayout& wl, int num_sms, cudaStream_t s) {
    return launch_k(search_kernel<PLAIN, TEAM, LANE, NCH>, kWarps, PLAIN, a, wl, num_sms, s);
}
template <int TEAM, int NCH = 0>
cudaError_t launch_wide(const SearchArgs& a, const WarpLayout& wl, int num_sms, cudaStream_t s) {
    return launch_k(search_kernel_wide<TEAM, NCH>, kWideWarps, false, a, wl, num_sms, s);
}

}  // namespace

int ef_class_cap(int ef_eff) {
    const int caps[] = {64, 128, 256, 512, 1024};
    for (int c : caps)
        if (ef_eff <= c) return c;
    return 0;
}

// Lanes per candidate of the team evaluators: every lane holds at most
// kMaxChunks (4) 16-byte chunks of the probe, so 16 lanes cover rows up to
// 64 chunks (d <= 1024) and leave two candidates per warp step.
int search_team_width(int dp) {
    const int chunks = dp / 16;
    return chunks <= 4 ? 4 : chunks <= 8 ? 8 : chunks <= 64 ? 16 : 32;
}

// Visited hash of `requested` ids (0: 1024, 2048 or 4096 by ef class).  The
// area also holds the FP32 query after Stage 1 (at least 4 * ldx bytes) and
// has at least 32 sets.  tag_req 0 or 16: 16-bit tags, four per set, sets
// the largest power of two with 4 * sets <= ids, B = max(bits of n - 1,
// log2 sets), tag = the low B - log2(sets) bits of the B-bit hash; 0 falls
// back to 32-bit ids when that tag exceeds 15 bits, 16 adds sets until it
// fits.  tag_req 32 (or no fit within 8192 sets): two 32-bit ids per set.
HashGeom search_hash_geom(int ef_cap, int ldx, int64_t n, int requested, int tag_req) {
    const int ids = requested > 0 ? requested : (ef_cap <= 128 ? 1024 : ef_cap <= 256 ? 2048 : 4096);
    const int min_sets = std::max(32, (ldx * 4 + 7) / 8);
    int B = 1;
    while (B < 31 && (int64_t(1) << B) < n) ++B;
    HashGeom g{};
    if (tag_req != 32) {
        int S = 0;
        while ((4 << (S + 1)) <= ids) ++S;
        while ((1 << S) < min_sets) ++S;
        if (tag_req == 16) S = std::max(S, B - 15);
        const int Bp = std::max(B, S);
        if (Bp - S <= 15 && S <= 13) {
            g.sets = 1 << S;
            g.tag16 = 1;
            g.tag_bits = Bp - S;
            g.id_mask = (uint32_t)((int64_t(1) << Bp) - 1);
            return g;
        }
    }
    g.sets = std::max((ids + 63) / 64 * 32, (min_sets + 31) / 32 * 32);
    return g;
}

// Staging buffer per warp.  Quantised path with code rows up to 256 bytes:
// 32 padded code rows (one warp-width of candidates).  Otherwise 4 KB, and
// always room for at least two FP32 rows.
int search_stage_bytes(int dp, int ldx, bool lane_path) {
    if (lane_path) return 32 * search_lane_stride(dp);
    int b = 4096;
    while (b < 2 * ldx * 4) b <<= 1;
    return b;
}

cudaError_t launch_search(const SearchArgs& a, int ef_cap, bool plain, int num_sms,
                          cudaStream_t s) {
    const bool lane = !plain && a.dp <= 256 && a.kc.team_lanes != 2;
    const bool wide = lane && a.kc.warps_per_block == kWideWarps;
    // A batch of at most one query per SM is latency-bound: unless the
    // configuration says otherwise it runs groups of warps (below) with a
    // visited hash of 32 ids per result-set entry (4,096 to 16,384 ids),
    // which forgets almost nothing; the extra shared memory costs no
    // occupancy at that batch size.
    const bool small = !plain && a.kc.warps_per_query == 0 && a.nq <= num_sms;
    const int hash_req = (small && a.kc.hash_slots == 0)
                             ? std::min(16384, std::max(4096, 32 * ef_cap))
                             : a.kc.hash_slots;
    WarpLayout wl;
    wl.ef_cap = ef_cap;
    wl.hg = search_hash_geom(ef_cap, a.ldx, a.n, hash_req, a.kc.hash_tag_bits);
    wl.rmax = std::max(a.R0p, a.R1p);
    wl.surv = lane ? 0 : wl.rmax;
    if (wide && a.kc.tile_rows <= 0) {
        // the largest tile (at most 32 rows) with which kWideBlocks blocks fit an SM
        int dev = 0, sm_bytes = 0, reserved = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        const int blk = (2 * a.ldx * 4 + 15) & ~15;
        const int per_warp = ((sm_bytes / kWideBlocks - reserved - blk) / kWideWarps) & ~15;
        wl.stg = 0;
        wl.qf = a.dp;
        const int stride = search_lane_stride(a.dp);
        const int rows = std::min(32, (per_warp - wl.bytes()) / stride);
        wl.stg = std::max(1, rows) * stride;
    } else if (a.kc.tile_rows > 0) {
        const int rows = std::min(a.kc.tile_rows, 32);
        wl.stg = rows * (lane ? search_lane_stride(a.dp) : (plain ? a.ldx * 4 : a.dp));
    } else {
        wl.stg = search_stage_bytes(a.dp, a.ldx, lane);
    }
    // Stages 2-3 stage into the same buffer: it must hold one FP32 row
    while (wl.stg < a.ldx * 4) wl.stg += 512;
    wl.stg = (wl.stg + 15) & ~15;
    wl.qf = plain ? a.ldx * 4 : (lane ? a.dp : 0);
    // Several warps per query: Stage 1 one lane per candidate for code rows
    // up to 256 bytes (team_lanes and warps_per_block do not apply), teams of
    // lanes beyond; Stages 2-3 with the team width of the row size, as in the
    // one-warp kernels, so that the results are the same.
    // 0 = automatic: a batch of at most one query per SM runs groups of
    // warps (4 for team-path rows, 2 on the lane path), which lowers the
    // latency of each query; larger batches run one warp per query, which
    // gives more queries per second.
    int G = a.kc.warps_per_query;
    if (small) G = a.dp > 256 ? 4 : 2;
    if (!plain && (G == 2 || G == 4)) {
        const bool glane = a.dp <= 256;
        GroupLayout gl;
        gl.G = G;
        gl.ef_cap = ef_cap;
        gl.hg = wl.hg;
        gl.rmax = std::max(round_up(a.R0p / G, 32), a.R1p);  // a warp's slice, or an upper row
        gl.smax = round_up(std::max(a.R0p / G, 1), 32);
        // staging tile: 32 code rows on the lane path; on the team path 4 KB
        // (the group's warps stage fewer rows each, and a smaller tile lets
        // more groups stay resident)
        if (a.kc.tile_rows > 0)
            gl.stg = std::min(a.kc.tile_rows, 32) * (glane ? search_lane_stride(a.dp) : a.dp);
        else
            gl.stg = glane ? search_stage_bytes(a.dp, a.ldx, true) : 4096;
        while (gl.stg < a.ldx * 4) gl.stg += 512;  // Stages 2-3 need one FP32 row
        gl.stg = (gl.stg + 15) & ~15;
        gl.qf = glane ? a.dp : 0;
        return launch_group(a, gl, glane, search_team_width(a.dp), num_sms, s);
    }
    if (wide) {
        switch (search_team_width(a.dp)) {
            case 4: return launch_wide<4>(a, wl, num_sms, s);
            case 8:
                if (a.dp == 128) return launch_wide<8, 8>(a, wl, num_sms, s);
                return launch_wide<8>(a, wl, num_sms, s);
            default: return launch_wide<16>(a, wl, num_sms, s);
        }
    }
    switch (search_team_width(a.dp) | (plain ? 0x100 : 0) | (lane ? 0 : 0x200)) {
        // lane path: rows of 6, 8 and 16 chunks (d_pad = 96, 128, 256) get
        // kernels specialised for their width
        case 4: return launch_t<false, 4, true>(a, wl, num_sms, s);
        case 8:
            if (a.dp == 96) return launch_t<false, 8, true, 6>(a, wl, num_sms, s);
            if (a.dp == 128) return launch_t<false, 8, true, 8>(a, wl, num_sms, s);
            return launch_t<false, 8, true>(a, wl, num_sms, s);
        case 16:
            if (a.dp == 256) return launch_t<false, 16, true, 16>(a, wl, num_sms, s);
            return launch_t<false, 16, true>(a, wl, num_sms, s);
        case 0x204: return launch_t<false, 4, false>(a, wl, num_sms, s);
        case 0x208: return launch_t<false, 8, false>(a, wl, num_sms, s);
        case 0x210: return launch_t<false, 16, false>(a, wl, num_sms, s);
        case 0x220: return launch_t<false, 32, false>(a, wl, num_sms, s);
        case 0x304: return launch_t<true, 4, false>(a, wl, num_sms, s);
        case 0x308: return launch_t<true, 8, false>(a, wl, num_sms, s);
        case 0x310: return launch_t<true, 16, false>(a, wl, num_sms, s);
        default: return launch_t<true, 32, false>(a, wl, num_sms, s);
    }
}

}  // namespace aqr
