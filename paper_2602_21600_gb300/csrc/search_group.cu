// Batched query kernel with several warps per query (Alg. 2): the form of
// search.cu's kernel in which a group of G warps (2 or 4) searches one
// query together; see beam_layer_group for the Stage-1 protocol.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "aqr_internal.h"
#include "beam.cuh"
#include "search_common.cuh"

namespace aqr {
namespace {

using namespace dev;

// The query kernel with G warps per query.  Every step is the one-warp
// kernel's; the group splits the neighbour lists of Stage 1 (see
// beam_layer_group) and the rows of Stages 2 and 3 among its warps, and its
// leader (warp 0 of the group) takes the query from the work counter, runs
// the greedy descent, sorts, decides early termination and writes the
// results.  All warps of a group pass the same named barriers.
template <int TEAM, bool LANE, int G, int NCH = 0>
__device__ __forceinline__ void search_body_group(const SearchArgs& a, const GroupLayout& gl) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gw = wib % G, grp = wib / G;
    const bool leader = gw == 0;
    const int tl = lane & (TEAM - 1);
    const int d = a.d;
    const int nchunks = a.dp >> 4;

    float* s_min = (float*)smem;
    float* s_inv = s_min + a.ldx;
    const int blk_bytes = (2 * a.ldx * 4 + 15) & ~15;
    for (int j = threadIdx.x; j < a.ldx; j += blockDim.x) {
        s_min[j] = j < d ? a.qmin[j] : 0.0f;
        s_inv[j] = j < d ? a.qinv[j] : 0.0f;
    }
    __syncthreads();
    unsigned char* gbase = smem + blk_bytes + grp * gl.bytes();
    BeamMem m;
    m.W = (u64*)gbase;
    m.H = (uint32_t*)(gbase + gl.ef_cap * 8);
    GroupSync g;
    g.surv = (u64*)(m.H + 2 * gl.hg.sets);
    g.sc = (int*)(g.surv + G * gl.smax);
    g.smax = gl.smax;
    g.G = G;
    g.gw = gw;
    g.bar = 1 + grp;
    unsigned char* wb = gbase + gl.shared_bytes() + gw * gl.warp_bytes();
    m.cand = (uint32_t*)wb;
    m.surv = nullptr;
    m.hsets = (uint32_t)gl.hg.sets;
    m.id_mask = gl.hg.id_mask;
    m.tag_bits = gl.hg.tag_bits;
    m.tag16 = gl.hg.tag16;
    m.ef_cap = gl.ef_cap;
    m.rmax = gl.rmax;
    m.err = a.error;
    unsigned char* stg = wb + gl.rmax * 4;
    uint4* qs = (uint4*)(stg + gl.stg);
    float* qf = (float*)m.H;  // the group's FP32 query once Stage 1 is over

    const Layer L0{a.adj0, nullptr, a.R0p, 0};
    const uint64_t pol_codes = policy_evict_last();
    const uint64_t pol_rows = policy_evict_first();

    for (;;) {
        if (leader && lane == 0) g.sc[GS_SLOT] = (int)atomicAdd(a.work, 1u);
        group_bar(g);
        const unsigned int slot = (unsigned int)g.sc[GS_SLOT];
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

        // every warp encodes the query for its own evaluator
        CodeEval<TEAM> ce;
        CodeLaneEvalT<NCH> le;
        if constexpr (LANE) {
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
            le.cap_rows = min(32, gl.stg / le.stride);
            le.stg = stg;
            le.qs = qs;
            le.qq = __reduce_add_sync(0xFFFFFFFFu, qq);
            le.pol = pol_codes;
        } else {
            ce.codes = a.codes;
            ce.dp = a.dp;
            ce.nchunks = nchunks;
            ce.tl = tl;
            ce.cap_rows = gl.stg / a.dp;
            ce.stg = stg;
            ce.pol = pol_codes;
#pragma unroll
            for (int i = 0; i < kMaxChunks; ++i) {
                const int c = tl + TEAM * i;
                ce.qc[i] = c < nchunks ? encode_chunk(qv, a.qmin, a.qscale, c, d)
                                       : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncwarp();

        BeamStats st;
        int n_l0exp = 0;
        bool overflow = false;
        uint32_t* exp_seq = (a.tr.exp_seq && leader) ? a.tr.exp_seq + qrow * a.tr.cap_exp : nullptr;
        int nW = 0;
        constexpr int BT = LANE ? 1 : TEAM;
        auto run = [&](auto& ev) {
            // entry point and greedy descent: the leader alone
            if (leader) {
                const uint32_t ep = a.entry;
                m.cand[0] = ep;
                __syncwarp();
                ev.stage(m.cand, 1);
                const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, ev.dist(0), 0);
                u64 ck = make_key(d0, ep);
                __syncwarp();
                st.evals += 1;
                for (int lc = a.max_level; lc >= 1; --lc) {
                    const Layer Lu{a.upper, a.upper_base, a.R1p, lc};
                    ck = greedy_layer<BT>(Lu, ck, m, ev, a.n, st);
                }
                if (a.tr.l0_entry && lane == 0) a.tr.l0_entry[qrow] = key_id(ck);
                if (lane == 0) {
                    g.sc[GS_KEY_LO] = (int)(uint32_t)ck;
                    g.sc[GS_KEY_HI] = (int)(uint32_t)(ck >> 32);
                }
            }
            group_bar(g);
            const u64 ck = ((u64)(uint32_t)g.sc[GS_KEY_HI] << 32) | (uint32_t)g.sc[GS_KEY_LO];
            nW = beam_layer_group<BT>(L0, ck & ~1ull, ef_eff, gl.ef_cap, m, g, ev, a.n, st,
                                      exp_seq, a.tr.cap_exp, &n_l0exp, &overflow);
        };
        if constexpr (LANE) run(le);
        else run(ce);
        if (overflow && leader && lane == 0) atomicExch(a.error, 1);

        const int nc = min(Nc, nW);
        if (leader) {
            if (a.tr.exp_count && lane == 0) a.tr.exp_count[qrow] = n_l0exp;
            if (a.tr.c_count && lane == 0) a.tr.c_count[qrow] = nc;
            if (a.tr.c_ids)
                for (int i = lane; i < nc; i += 32) {
                    const u64 kk = m.W[i];
                    a.tr.c_ids[qrow * a.tr.cap_c + i] = key_id(kk);
                    a.tr.c_dist[qrow * a.tr.cap_c + i] = (int32_t)key_hi(kk);
                }
        }
        // the hash is dead after Stage 1: it takes the FP32 query
        for (int j = gw * 32 + lane; j < a.ldx; j += G * 32) qf[j] = j < d ? qv[j] : 0.0f;
        group_bar(g);
        // ---- Stage 2 on this warp's share of C
        const int per2 = (nc + G - 1) / G;
        stage2_rows<TEAM>(a.codes, a.d, a.dp, m.W, min(nc, gw * per2), min(nc, gw * per2 + per2), stg, gl.stg, qf,
                          s_min, s_inv, pol_codes);
        group_bar(g);
        int P = 1;
        while (P < nc) P <<= 1;
        if (!AQR_IN(a.error, P <= gl.ef_cap)) P = 1;
        if (leader) {
            for (int i = nc + lane; i < P; i += 32) m.W[i] = kEmpty;
            warp_bitonic_sort(m.W, P);
            if (a.tr.a_ids)
                for (int i = lane; i < nc; i += 32) {
                    const u64 kk = m.W[i];
                    a.tr.a_ids[qrow * a.tr.cap_c + i] = key_id(kk);
                    a.tr.a_dist[qrow * a.tr.cap_c + i] = __uint_as_float(key_hi(kk));
                }
            // early termination (Section 3.2)
            int et = 0;
            if (nc > k) {
                const float dk = __uint_as_float(key_hi(m.W[k - 1]));
                const float dk1 = __uint_as_float(key_hi(m.W[k]));
                const float gap = (dk1 - dk) / (dk + a.eps);
                const float ratio = dk1 / (dk + a.eps);
                et = (gap > a.tau_gap || ratio > a.tau_ratio) ? 1 : 0;
            }
            if (lane == 0) {
                g.sc[GS_ET] = et;
                g.sc[GS_NE] = et ? min(k, nc) : min(Nr, nc);
            }
        }
        group_bar(g);
        const int et = g.sc[GS_ET], ne = g.sc[GS_NE];
        // ---- Stage 3 on this warp's share of the first ne entries
        const int per3 = (ne + G - 1) / G;
        stage3_rows<TEAM>(a.x, a.ldx, m.W, min(ne, gw * per3), min(ne, gw * per3 + per3), stg, gl.stg, qf,
                          pol_rows);
        group_bar(g);
        if (leader) {
            warp_bitonic_sort(m.W, P);
            for (int i = lane; i < a.k_stride; i += 32) {
                const int64_t o = qrow * a.k_stride + i;
                if (i < k && i < nc) {
                    const u64 kk = m.W[i];
                    a.ids[o] = key_id(kk);
                    a.dists[o] = __uint_as_float(key_hi(kk));
                    if (a.exact) a.exact[o] = (uint8_t)(kk & 1ull);
                } else {
                    a.ids[o] = -1;
                    a.dists[o] = __int_as_float(0x7f800000);
                    if (a.exact) a.exact[o] = 0;
                }
            }
        }
        if (lane == 0) {
            unsigned long long* C = a.counters;
            if (leader) {
                if (a.tr.et) a.tr.et[qrow] = (uint8_t)et;
                if (a.tr.n_exact) a.tr.n_exact[qrow] = ne;
                atomicAdd(C + C_QUERIES, 1ull);
                atomicAdd(C + C_EXPANSIONS, (unsigned long long)st.expansions);
                atomicAdd(C + C_STAGE2, (unsigned long long)nc);
                atomicAdd(C + C_EXACT, (unsigned long long)ne);
                atomicAdd(C + C_ET, (unsigned long long)et);
            }
            atomicAdd(C + C_EVALS, (unsigned long long)st.evals);
            atomicAdd(C + C_ADJ, (unsigned long long)st.adj);
            atomicAdd(C + C_EVALS_L0, (unsigned long long)st.l0_evals);
        }
        __syncwarp();
    }
}

// NCH: code-row chunks fixed at compile time on the lane path (0: any).
template <int TEAM, bool LANE, int G, int NCH = 0>
__global__ void __launch_bounds__(kThreads, LANE ? 8 : 5)
    search_kernel_group(SearchArgs a, GroupLayout gl) {
    search_body_group<TEAM, LANE, G, NCH>(a, gl);
}

template <int TEAM, bool LANE, int G, int NCH = 0>
cudaError_t launch_group_t(const SearchArgs& a, const GroupLayout& gl, int num_sms, cudaStream_t s) {
    constexpr int per_block = kWarps / G;  // queries a block holds at once
    const int blk = (2 * a.ldx * 4 + 15) & ~15;
    const int smem = blk + per_block * gl.bytes();
    auto kern = search_kernel_group<TEAM, LANE, G, NCH>;
    std::lock_guard<std::mutex> lk(kernel_attr_mutex());  // from the set to the launch
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = kernel_occupancy((const void*)kern, kThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (a.nq + per_block - 1) / per_block;
    int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(a, gl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_group(const SearchArgs& a, const GroupLayout& gl, bool lane, int tw,
                         int num_sms, cudaStream_t s) {
    const int G = gl.G;
    if (lane) {
        // 128-byte code rows: kernels instantiated for that width
        if (a.dp == 128)
            return G == 2 ? launch_group_t<8, true, 2, 8>(a, gl, num_sms, s)
                          : launch_group_t<8, true, 4, 8>(a, gl, num_sms, s);
        if (G == 2) return tw == 4 ? launch_group_t<4, true, 2>(a, gl, num_sms, s)
                         : tw == 8 ? launch_group_t<8, true, 2>(a, gl, num_sms, s)
                                   : launch_group_t<16, true, 2>(a, gl, num_sms, s);
        return tw == 4 ? launch_group_t<4, true, 4>(a, gl, num_sms, s)
             : tw == 8 ? launch_group_t<8, true, 4>(a, gl, num_sms, s)
                       : launch_group_t<16, true, 4>(a, gl, num_sms, s);
    }
    if (G == 2) return tw == 16 ? launch_group_t<16, false, 2>(a, gl, num_sms, s)
                                : launch_group_t<32, false, 2>(a, gl, num_sms, s);
    return tw == 16 ? launch_group_t<16, false, 4>(a, gl, num_sms, s)
                    : launch_group_t<32, false, 4>(a, gl, num_sms, s);
}

}  // namespace aqr
