// Persistent batched query kernel (Alg. 2): one warp per query; warps pull
// queries from a work counter until the launch's queries are exhausted.
//
// Per query:
//   encode the FP32 query to uint8 codes held in registers (Alg. 2 line 4)
//   greedy descent with ef = 1 through layers L..1
//   layer-0 search with ef_eff = max(ef, k) on integer code distances
//     (Alg. 2 lines 6-7), result set W sorted in shared memory
//   C = W[0:N_c); Stage 2: asymmetric distances to the decoded codes
//     x~_j = code_j / scale_j + min_j, sort by (d^a, id) (Alg. 2 lines 9-13)
//   early termination test on d^a_k, d^a_k+1 (Alg. 2 lines 15-17)
//   Stage 3: exact FP32 distances for the first n_exact of A (lines 19-22)
//   merge with the rest of A, sort by (distance, id), top k (lines 23-24)
//
// The plain comparison path (PLAIN = true) runs the same search with FP32
// distances on the FP32 vectors and returns the top k of W directly.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "aqr_internal.h"
#include "beam.cuh"

namespace aqr {
namespace {

using namespace dev;

constexpr int kWarps = 4;  // warps per block
constexpr int kThreads = kWarps * 32;

// Per-warp shared memory bytes.
__host__ __device__ inline int warp_bytes(int ef_cap, int hsize, int rmax, bool plain, int ldx) {
    int b = ef_cap * 8 + hsize * 4 + rmax * 4 + rmax * 8;
    if (plain) b += ldx * 4;
    return (b + 15) & ~15;
}

template <bool PLAIN, int TEAM>
__global__ void __launch_bounds__(kThreads, 8) search_kernel(SearchArgs a, int ef_cap, int hbits,
                                                          int rmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NT = 32 / TEAM;  // teams per warp
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int tl = lane & (TEAM - 1);
    const int team = lane / TEAM;
    const int hsize = 1 << hbits;
    const int d = a.d;
    const int nchunks = a.dp >> 4;
    const int ngroups = a.ldx >> 2;

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
    unsigned char* wbase = smem + blk_bytes + wib * warp_bytes(ef_cap, hsize, rmax, PLAIN, a.ldx);
    BeamMem m;
    m.W = (u64*)wbase;
    m.H = (uint32_t*)(wbase + ef_cap * 8);
    m.cand = m.H + hsize;
    m.surv = (u64*)(m.cand + rmax);
    m.hbits = hbits;
    // FP32 query: its own area on the plain path; on the quantised path it
    // reuses the visited hash, which is dead after Stage 1.
    float* qf = PLAIN ? (float*)(m.surv + rmax) : (float*)m.H;

    const Layer L0{a.adj0, nullptr, a.R0p, 0};

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

        // ---- query codes in registers (quantised path) / FP32 copy (plain)
        uint4 qc[kMaxChunks];
#pragma unroll
        for (int i = 0; i < kMaxChunks; ++i) {
            int c = tl + TEAM * i;
            uint32_t w[4] = {0, 0, 0, 0};
            if (!PLAIN && c < nchunks) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    int j = c * 16 + t;
                    uint32_t code = j < d ? encode1(__ldg(qv + j), __ldg(a.qmin + j), __ldg(a.qscale + j)) : 0u;
                    w[t >> 2] |= code << (8 * (t & 3));
                }
            }
            qc[i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (PLAIN)
            for (int j = lane; j < a.ldx; j += 32) qf[j] = j < d ? qv[j] : 0.0f;
        __syncwarp();

        auto dist = [&](uint32_t v) -> uint32_t {
            if (PLAIN) {
                float s = f32_partial((const float4*)(a.x + (int64_t)v * a.ldx), qf, tl, TEAM, ngroups);
                return __float_as_uint(team_sum_f32<TEAM>(s));
            } else {
                uint32_t s = code_partial<TEAM>((const uint4*)(a.codes + (int64_t)v * a.dp), qc, tl, nchunks);
                return team_sum_u32<TEAM>(s);
            }
        };

        BeamStats st;
        // ---- greedy descent through the upper layers
        u64 ck = make_key(dist(a.entry), a.entry);
        st.evals += 1;
        for (int lc = a.max_level; lc >= 1; --lc) {
            const Layer Lu{a.upper, a.upper_base, a.R1p, lc};
            ck = greedy_layer<TEAM>(Lu, ck, m, dist, a.n, st);
        }
        if (a.tr.l0_entry && lane == 0) a.tr.l0_entry[qrow] = key_id(ck);

        // ---- layer-0 search
        int n_l0exp = 0;
        bool overflow = false;
        uint32_t* exp_seq = a.tr.exp_seq ? a.tr.exp_seq + qrow * a.tr.cap_exp : nullptr;
        const int nW = beam_layer<TEAM>(L0, ck & ~1ull, ef_eff, ef_cap, m, dist, a.n, st, exp_seq,
                                        a.tr.cap_exp, &n_l0exp, &overflow);
        if (overflow && lane == 0) atomicExch(a.error, 1);

        const int nc = min(Nc, nW);
        if (a.tr.exp_count && lane == 0) a.tr.exp_count[qrow] = n_l0exp;
        if (a.tr.c_count && lane == 0) a.tr.c_count[qrow] = nc;
        if (a.tr.c_ids)
            for (int i = lane; i < nc; i += 32) {
                u64 kk = m.W[i];
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
            for (int base = 0; base < nc; base += NT) {
                const int i = base + team;
                const uint32_t v = key_id(m.W[i < nc ? i : 0]);
                const uint4* row = (const uint4*)(a.codes + (int64_t)v * a.dp);
                float acc = 0.0f;
#pragma unroll
                for (int t = 0; t < kMaxChunks; ++t) {
                    int c = tl + TEAM * t;
                    if (c < nchunks) {
                        uint4 b = __ldg(row + c);
                        uint32_t wd[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            int j = c * 16 + u;
                            if (j < d) {
                                float code = (float)((wd[u >> 2] >> (8 * (u & 3))) & 0xFFu);
                                float xt = fmaf(code, s_inv[j], s_min[j]);
                                float df = qf[j] - xt;
                                acc = fmaf(df, df, acc);
                            }
                        }
                    }
                }
                acc = team_sum_f32<TEAM>(acc);
                __syncwarp();
                if (i < nc && tl == 0) m.W[i] = ((u64)__float_as_uint(acc) << 32) | ((u64)v << 1);
            }
            __syncwarp();
            int P = 1;
            while (P < nc) P <<= 1;
            for (int i = nc + lane; i < P; i += 32) m.W[i] = kEmpty;
            warp_bitonic_sort(m.W, P);
            if (a.tr.a_ids)
                for (int i = lane; i < nc; i += 32) {
                    u64 kk = m.W[i];
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
            for (int base = 0; base < ne; base += NT) {
                const int i = base + team;
                const uint32_t v = key_id(m.W[i < ne ? i : 0]);
                float acc = f32_partial((const float4*)(a.x + (int64_t)v * a.ldx), qf, tl, TEAM, ngroups);
                acc = team_sum_f32<TEAM>(acc);
                __syncwarp();
                if (i < ne && tl == 0)
                    m.W[i] = ((u64)__float_as_uint(acc) << 32) | ((u64)v << 1) | 1ull;
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
        }
        __syncwarp();
    }
}

template <bool PLAIN, int TEAM>
cudaError_t launch_t(const SearchArgs& a, int ef_cap, int hbits, int rmax, int num_sms,
                     cudaStream_t s) {
    const int blk = PLAIN ? 0 : ((2 * a.ldx * 4 + 15) & ~15);
    const int smem = blk + kWarps * warp_bytes(ef_cap, 1 << hbits, rmax, PLAIN, a.ldx);
    auto kern = search_kernel<PLAIN, TEAM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (a.nq + kWarps - 1) / kWarps;
    int64_t grid = std::min<int64_t>((int64_t)per_sm * num_sms, want);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(a, ef_cap, hbits, rmax);
    return cudaGetLastError();
}

}  // namespace

int ef_class_cap(int ef_eff) {
    const int caps[] = {64, 128, 256, 512, 1024};
    for (int c : caps)
        if (ef_eff <= c) return c;
    return 0;
}

int search_team_width(int dp) {
    const int chunks = dp / 16;
    return chunks <= 4 ? 4 : chunks <= 8 ? 8 : chunks <= 16 ? 16 : 32;
}

int search_hbits(int ef_cap, int ldx) {
    int hb = ef_cap <= 64 ? 10 : ef_cap <= 256 ? 11 : 12;
    while ((1 << hb) < ldx) ++hb;
    return hb;
}

cudaError_t launch_search(const SearchArgs& a, int ef_cap, bool plain, int num_sms,
                          cudaStream_t s) {
    const int hbits = search_hbits(ef_cap, a.ldx);
    const int rmax = std::max(a.R0p, a.R1p);
    switch (search_team_width(a.dp) | (plain ? 0x100 : 0)) {
        case 4: return launch_t<false, 4>(a, ef_cap, hbits, rmax, num_sms, s);
        case 8: return launch_t<false, 8>(a, ef_cap, hbits, rmax, num_sms, s);
        case 16: return launch_t<false, 16>(a, ef_cap, hbits, rmax, num_sms, s);
        case 32: return launch_t<false, 32>(a, ef_cap, hbits, rmax, num_sms, s);
        case 0x104: return launch_t<true, 4>(a, ef_cap, hbits, rmax, num_sms, s);
        case 0x108: return launch_t<true, 8>(a, ef_cap, hbits, rmax, num_sms, s);
        case 0x110: return launch_t<true, 16>(a, ef_cap, hbits, rmax, num_sms, s);
        default: return launch_t<true, 32>(a, ef_cap, hbits, rmax, num_sms, s);
    }
}

}  // namespace aqr
