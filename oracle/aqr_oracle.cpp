// AQR-HNSW CPU oracle: plain, slow, obviously correct.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code,
// header, table or helper with the CUDA library; both read the same seeded
// inputs and nothing else.
//
// Arithmetic: FP64 for real-valued quantities, int64 for code distances,
// except the encode step, which the method defines on FP32 parameters and
// which is emulated here in IEEE FP32 with contraction disabled
// (compile with -ffp-contract=off).
//
// Ordering: every candidate set is ordered lexicographically by
// (distance, id).  The paper leaves tie-breaking open; this total order makes
// every result unique.
//
// What is pinned, and how (tests/test_oracle_*.py):
//   encode           round-trip bound, hand-computed codes, identity case
//   training         closed forms on hand-made sets, direct sort percentiles
//   int distance     brute-force sum of squared code differences
//   search           ef >= n gives brute-force top N_c; ef = 1 is greedy
//   full pipeline    ef >= n, rerank everything, no early exit = exact top-k
//   early exit       hand-made candidate lists around both thresholds
//   graph build      degree, self-loop, duplicate and level invariants;
//                    batch size 1 equals the sequential textbook insertion
// Parity unpinned: absolute codes for a given data set (the paper gives no
// worked example and no value of P_max) and the sampled density (RNG choice);
// both are pinned only by their closed forms on small inputs.

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>
#include <utility>
#include <vector>

#if FLT_EVAL_METHOD != 0
#error "the FP32 encode emulation needs float arithmetic without excess precision"
#endif

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;

int n_threads(int requested) {
    if (requested > 0) return requested;
    unsigned h = std::thread::hardware_concurrency();
    return h == 0 ? 1 : (int)h;
}

template <class F>
void parallel_for(int64_t n, int threads, F f) {
    threads = (int)std::min<int64_t>(threads, std::max<int64_t>(n, 1));
    if (threads <= 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= n) break;
                f(i);
            }
        });
    for (auto& th : pool) th.join();
}

// Squared L2 in FP64 between float vectors (Section 3.1 density, Alg. 2
// exact distance).
double l2_f64(const float* a, const float* b, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)a[j] - (double)b[j];
        s += t * t;
    }
    return s;
}

// Integer squared L2 between two code vectors (Alg. 2, quantised distance,
// without the constant factor s_dist).
int64_t l2_codes(const uint8_t* a, const uint8_t* b, int d) {
    int64_t s = 0;
    for (int j = 0; j < d; ++j) {
        int64_t t = (int64_t)a[j] - (int64_t)b[j];
        s += t * t;
    }
    return s;
}

// Hyndman-Fan type 7 percentile of a sorted column: h = (n-1) p,
// linear interpolation between the two order statistics around h.
double percentile7(const std::vector<double>& v, double p) {
    int64_t n = (int64_t)v.size();
    if (n == 1) return v[0];
    double h = (double)(n - 1) * p;
    int64_t lo = (int64_t)std::floor(h);
    if (lo < 0) lo = 0;
    if (lo >= n - 1) return v[n - 1];
    double frac = h - (double)lo;
    return v[lo] + frac * (v[lo + 1] - v[lo]);
}

using Key = std::pair<int64_t, uint32_t>;  // (distance, id)

// One HNSW graph: layer-0 lists and per-node upper lists (layers 1..level).
struct Graph {
    int64_t n = 0;
    int d = 0;
    int M = 0;    // M_i: selection size and upper-layer capacity
    int cap0 = 0; // 2 M_i: layer-0 capacity
    const uint8_t* codes = nullptr;
    std::vector<int> level;
    std::vector<std::vector<uint32_t>> l0;
    std::vector<std::vector<std::vector<uint32_t>>> up;  // up[v][lc-1]
    uint32_t entry = kNone;
    int max_level = -1;

    const std::vector<uint32_t>& nbrs(uint32_t v, int lc) const {
        return lc == 0 ? l0[v] : up[v][lc - 1];
    }
    std::vector<uint32_t>& nbrs(uint32_t v, int lc) {
        return lc == 0 ? l0[v] : up[v][lc - 1];
    }
    const uint8_t* code(uint32_t v) const { return codes + (int64_t)v * d; }
};

// Read-only view of an index given as flat arrays (the index file layout).
struct FlatIndex {
    int64_t n;
    int d;
    int R0, R1;
    const uint8_t* codes;
    const float* x;
    const uint32_t* adj0;       // n x R0, unused slots = kNone
    const int64_t* upper_base;  // n, -1 when the node has no upper layer
    const uint32_t* upper;      // rows x R1
    uint32_t entry;
    int max_level;
    const float* minv;
    const float* scale;

    void nbrs(uint32_t v, int lc, std::vector<uint32_t>& out) const {
        out.clear();
        const uint32_t* row;
        int cap;
        if (lc == 0) {
            row = adj0 + (int64_t)v * R0;
            cap = R0;
        } else {
            row = upper + (upper_base[v] + (lc - 1)) * (int64_t)R1;
            cap = R1;
        }
        for (int i = 0; i < cap; ++i)
            if (row[i] != kNone) out.push_back(row[i]);
    }
    const uint8_t* code(uint32_t v) const { return codes + (int64_t)v * d; }
};

struct SearchTrace {
    std::vector<uint32_t> expanded;  // expansion order (textbook pop order)
    int64_t evals = 0;               // distance evaluations
};

// HNSW SEARCH-LAYER (Malkov & Yashunin, Alg. 2), on code distances, with
// the total order (distance, id): a candidate set C (min-heap), a result
// set W (max-heap) bounded by ef, and a visited set.  Returns W ascending.
template <class NbrFn>
std::vector<Key> search_layer(const uint8_t* qc, int d, Key ep, int ef,
                              const std::function<const uint8_t*(uint32_t)>& code_of,
                              NbrFn nbrs_of, std::vector<uint8_t>& visited,
                              std::vector<uint32_t>& touched, SearchTrace* tr) {
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> C;
    std::priority_queue<Key> W;
    visited[ep.second] = 1;
    touched.push_back(ep.second);
    C.push(ep);
    W.push(ep);
    std::vector<uint32_t> nb;
    while (!C.empty()) {
        Key c = C.top();
        C.pop();
        Key f = W.top();
        if (c > f) break;
        if (tr) tr->expanded.push_back(c.second);
        nbrs_of(c.second, nb);
        for (uint32_t e : nb) {
            if (visited[e]) continue;
            visited[e] = 1;
            touched.push_back(e);
            Key ek{l2_codes(qc, code_of(e), d), e};
            if (tr) tr->evals++;
            f = W.top();
            if ((int)W.size() < ef || ek < f) {
                C.push(ek);
                W.push(ek);
                if ((int)W.size() > ef) W.pop();
            }
        }
    }
    std::vector<Key> out;
    while (!W.empty()) {
        out.push_back(W.top());
        W.pop();
    }
    std::reverse(out.begin(), out.end());
    for (uint32_t t : touched) visited[t] = 0;
    touched.clear();
    return out;
}

// SELECT-NEIGHBORS-HEURISTIC (Malkov & Yashunin, Alg. 4) without candidate
// extension or kept pruned connections.  cand is ascending by (d(base,e), e);
// e is kept iff it is strictly closer to the base than to every kept r.
std::vector<uint32_t> select_heuristic(const Graph& g, const std::vector<Key>& cand, int M) {
    std::vector<uint32_t> R;
    for (const Key& e : cand) {
        if ((int)R.size() >= M) break;
        bool good = true;
        for (uint32_t r : R) {
            if (l2_codes(g.code(e.second), g.code(r), g.d) <= e.first) {
                good = false;
                break;
            }
        }
        if (good) R.push_back(e.second);
    }
    return R;
}

}  // namespace

extern "C" {

// ----------------------------------------------------------------------------
// Section 3.1, Stage 1: local density rho_i = 1 / (mean of squared L2 to the
// k nearest other points + eps), eps = 1e-6, brute force in FP64.  ids lists
// the points whose density is computed (all points, or the sample).
int oracle_density(const float* x, int64_t n, int32_t d, const int64_t* ids, int64_t m,
                   int32_t kd, int32_t nthreads, double* rho_out) {
    if (!x || !ids || !rho_out || n < 2 || d <= 0 || kd <= 0 || kd > n - 1) return 1;
    parallel_for(m, n_threads(nthreads), [&](int64_t t) {
        int64_t i = ids[t];
        const float* xi = x + i * d;
        std::vector<std::pair<double, int64_t>> best;  // max-heap of kd smallest
        best.reserve(kd + 1);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            std::pair<double, int64_t> e{l2_f64(xi, x + j * d, d), j};
            if ((int)best.size() < kd) {
                best.push_back(e);
                std::push_heap(best.begin(), best.end());
            } else if (e < best.front()) {
                std::pop_heap(best.begin(), best.end());
                best.back() = e;
                std::push_heap(best.begin(), best.end());
            }
        }
        double s = 0.0;
        std::sort(best.begin(), best.end());
        for (auto& b : best) s += b.first;
        rho_out[t] = 1.0 / (s / (double)kd + 1e-6);
    });
    return 0;
}

// ----------------------------------------------------------------------------
// Alg. 1: density, heterogeneity delta, adaptive percentiles,
// per-dimension range and scale, density weights, s_dist (Eq. 1), eta,
// M_i and ef_construction.
//
// sample: ids whose density is computed when n > 10,000 (the paper's
// threshold); when n <= 10,000 every point's density is computed and the
// sample is ignored.  Unsampled points take the sample mean density.
//
// scalars_out: [delta, rho_bar, w, s_dist, eta, M_i, ef_c, P_l, P_h,
//               rho_min, rho_max]
int oracle_train(const float* x, int64_t n, int32_t d, const int64_t* sample, int64_t n_s,
                 double p_max, int32_t M0, int32_t ef0, int32_t nthreads, float* min_out,
                 float* max_out, float* scale_out, double* scalars_out) {
    if (!x || n < 11 || d <= 0 || !min_out || !max_out || !scale_out || !scalars_out) return 1;
    const double eps = 1e-6;
    const int kd = 10;
    std::vector<int64_t> ids;
    if (n > 10000) {
        if (!sample || n_s <= 0) return 1;
        ids.assign(sample, sample + n_s);
    } else {
        ids.resize(n);
        for (int64_t i = 0; i < n; ++i) ids[i] = i;
    }
    int64_t m = (int64_t)ids.size();
    std::vector<double> rho(m);
    if (oracle_density(x, n, d, ids.data(), m, kd, nthreads, rho.data())) return 1;

    double rmax = rho[0], rmin = rho[0], rsum = 0.0;
    for (double r : rho) {
        rmax = std::max(rmax, r);
        rmin = std::min(rmin, r);
        rsum += r;
    }
    double rho_bar = rsum / (double)m;
    // Alg. 1.
    double delta = (rmax - rmin) / (rmax + eps);
    // Alg. 1 (fractions in [0, 1]).
    double P_l = delta * p_max;
    double P_h = 1.0 - delta * p_max;

    // Alg. 1: per-dimension percentile range and scale.
    std::vector<double> col(n);
    for (int j = 0; j < d; ++j) {
        for (int64_t i = 0; i < n; ++i) col[i] = (double)x[i * d + j];
        std::sort(col.begin(), col.end());
        float lo = (float)percentile7(col, P_l);
        float hi = (float)percentile7(col, P_h);
        min_out[j] = lo;
        max_out[j] = hi;
        scale_out[j] = (float)(255.0 / ((double)hi - (double)lo + eps));
    }

    // Alg. 1: w_j = (1/n) sum_i rho_i, unsampled points at rho_bar.
    double w_sum = rsum + (double)(n - m) * rho_bar;
    double w = w_sum / (double)n;
    std::vector<double> wj(d, w);

    // Eq. 1.
    double num = 0.0, den = 0.0;
    for (int j = 0; j < d; ++j) {
        double r = (double)max_out[j] - (double)min_out[j];
        num += r * r * wj[j];
        den += 255.0 * 255.0 * wj[j];
    }
    double s_dist = std::sqrt(num / den);

    // Section 3.1 dimension heterogeneity: eta = sigma_w / mean_w, with the
    // mean and deviations taken relative to w_1 (shifted two-pass form, exact
    // when all w_j are equal).
    double shift = 0.0;
    for (int j = 0; j < d; ++j) shift += wj[j] - wj[0];
    double wbar = wj[0] + shift / (double)d;
    double var = 0.0;
    for (int j = 0; j < d; ++j) var += (wj[j] - wbar) * (wj[j] - wbar);
    double eta = std::sqrt(var / (double)d) / wbar;

    // Alg. 1.
    int M_i = (int)std::floor((double)M0 * (1.0 + delta * (1.0 + eta)));
    int ef_c = (int)std::floor((double)ef0 * (1.0 / (1.0 + delta * eta)));

    double* s = scalars_out;
    s[0] = delta;
    s[1] = rho_bar;
    s[2] = w;
    s[3] = s_dist;
    s[4] = eta;
    s[5] = M_i;
    s[6] = ef_c;
    s[7] = P_l;
    s[8] = P_h;
    s[9] = rmin;
    s[10] = rmax;
    return 0;
}

// ----------------------------------------------------------------------------
// Alg. 1 / Alg. 2 / Section 3.3: shift by min_j, multiply by
// scale_j, clip to [0, 255], round to nearest (ties to even).  Emulated in
// IEEE FP32, two roundings, no fused multiply-add.
int oracle_encode(const float* x, int64_t n, int32_t d, const float* minv, const float* scale,
                  uint8_t* codes) {
    if (!x || !minv || !scale || !codes || n < 0 || d <= 0) return 1;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j) {
            float diff = x[i * d + j] - minv[j];
            float t = diff * scale[j];
            if (!(t >= 0.0f)) t = 0.0f;  // also maps NaN to 0
            if (t > 255.0f) t = 255.0f;
            codes[i * d + j] = (uint8_t)std::nearbyint(t);
        }
    return 0;
}

// HNSW level draw: l = floor(-ln(U) * mL), mL = 1 / ln(M_i); U in (0, 1].
int oracle_levels(const double* U, int64_t n, int32_t M_i, int32_t* levels) {
    if (!U || !levels || M_i < 2) return 1;
    double mL = 1.0 / std::log((double)M_i);
    for (int64_t i = 0; i < n; ++i) levels[i] = (int32_t)std::floor(-std::log(U[i]) * mL);
    return 0;
}

// Insertion batches: node 0 alone, then [s, s + b) with
// b = min(max(1, s / batch_div), batch_max).  Returns the number of batches;
// starts (if non-null, size >= count + 1) receives the batch boundaries.
int64_t oracle_batch_schedule(int64_t n, int32_t batch_div, int32_t batch_max, int64_t* starts) {
    int64_t cnt = 0, s = 0;
    while (s < n) {
        if (starts) starts[cnt] = s;
        int64_t b = s == 0 ? 1 : std::min<int64_t>(std::max<int64_t>(1, s / batch_div), batch_max);
        s = std::min(n, s + b);
        ++cnt;
    }
    if (starts) starts[cnt] = n;
    return cnt;
}

// ----------------------------------------------------------------------------
// Alg. 1: HNSW construction on the codes with M_i and
// ef_construction, insertion in id order, processed in batches: every node
// of a batch searches the graph as it stood before the batch (so a batch's
// searches are independent), then the batch's links are applied node by
// node in id order.  With batch_max = 1 this is the sequential insertion of
// Malkov & Yashunin (Alg. 1 there), with
//   selection by the heuristic (their Alg. 4) to at most M_i neighbours,
//   layer-0 capacity 2 M_i and upper-layer capacity M_i,
//   a full list re-selected by the same heuristic when a link overflows it,
//   the entry point replaced only by a node of strictly higher level.
//
// Outputs: adj0 [n x 2M_i] (kNone-padded), upper_base [n] (-1 or the first
// row of the node's layers 1..level), upper [rows x M_i], entry_level[2].
int oracle_build(const uint8_t* codes, int64_t n, int32_t d, const int32_t* levels, int32_t M_i,
                 int32_t ef_c, int32_t batch_div, int32_t batch_max, int32_t nthreads,
                 uint32_t* adj0, int64_t* upper_base, uint32_t* upper, int32_t* entry_level) {
    if (!codes || !levels || n < 1 || d <= 0 || M_i < 2 || ef_c < 1 || batch_div < 1 ||
        batch_max < 1 || !adj0 || !upper_base || !entry_level)
        return 1;
    Graph g;
    g.n = n;
    g.d = d;
    g.M = M_i;
    g.cap0 = 2 * M_i;
    g.codes = codes;
    g.level.assign(levels, levels + n);
    g.l0.assign(n, {});
    g.up.resize(n);
    for (int64_t v = 0; v < n; ++v) g.up[v].assign(std::max(0, g.level[v]), {});

    std::vector<int64_t> starts(oracle_batch_schedule(n, batch_div, batch_max, nullptr) + 1);
    int64_t nb = oracle_batch_schedule(n, batch_div, batch_max, starts.data());
    const int T = n_threads(nthreads);
    std::function<const uint8_t*(uint32_t)> code_of = [&](uint32_t v) { return g.code(v); };

    for (int64_t b = 0; b < nb; ++b) {
        int64_t s = starts[b], e = starts[b + 1];
        // results[v - s][lc] = selected neighbours at layer lc
        std::vector<std::vector<std::vector<uint32_t>>> sel(e - s);
        if (g.entry != kNone) {
            const uint32_t ep = g.entry;
            const int L = g.max_level;
            parallel_for(e - s, T, [&](int64_t t) {
                uint32_t v = (uint32_t)(s + t);
                std::vector<uint8_t> visited(n, 0);
                std::vector<uint32_t> touched;
                auto nbrs_of = [&](uint32_t u, int lc, std::vector<uint32_t>& out) {
                    out = g.nbrs(u, lc);
                };
                const uint8_t* qc = g.code(v);
                Key cur{l2_codes(qc, g.code(ep), d), ep};
                int lv = g.level[v];
                for (int lc = L; lc > lv; --lc) {
                    auto W = search_layer(qc, d, cur, 1, code_of,
                                          [&](uint32_t u, std::vector<uint32_t>& o) { nbrs_of(u, lc, o); },
                                          visited, touched, nullptr);
                    cur = W[0];
                }
                sel[t].assign(std::min(L, lv) + 1, {});
                for (int lc = std::min(L, lv); lc >= 0; --lc) {
                    auto W = search_layer(qc, d, cur, ef_c, code_of,
                                          [&](uint32_t u, std::vector<uint32_t>& o) { nbrs_of(u, lc, o); },
                                          visited, touched, nullptr);
                    sel[t][lc] = select_heuristic(g, W, M_i);
                    cur = W[0];
                }
            });
        }
        // Links, node by node in id order.
        for (int64_t v = s; v < e; ++v) {
            auto& sv = sel[v - s];
            for (int lc = 0; lc < (int)sv.size(); ++lc) {
                g.nbrs((uint32_t)v, lc) = sv[lc];
                int cap = lc == 0 ? g.cap0 : g.M;
                for (uint32_t r : sv[lc]) {
                    auto& lst = g.nbrs(r, lc);
                    if ((int)lst.size() < cap) {
                        lst.push_back((uint32_t)v);
                    } else {
                        std::vector<Key> cand;
                        for (uint32_t u : lst) cand.push_back({l2_codes(g.code(r), g.code(u), d), u});
                        cand.push_back({l2_codes(g.code(r), g.code((uint32_t)v), d), (uint32_t)v});
                        std::sort(cand.begin(), cand.end());
                        lst = select_heuristic(g, cand, cap);
                    }
                }
            }
        }
        // Entry point: the first node (in id order) of strictly higher level.
        for (int64_t v = s; v < e; ++v)
            if (g.level[v] > g.max_level) {
                g.max_level = g.level[v];
                g.entry = (uint32_t)v;
            }
    }

    // Flatten.
    const int R0 = g.cap0, R1 = g.M;
    int64_t row = 0;
    for (int64_t v = 0; v < n; ++v) {
        uint32_t* r0 = adj0 + v * R0;
        for (int i = 0; i < R0; ++i) r0[i] = i < (int)g.l0[v].size() ? g.l0[v][i] : kNone;
        if (g.level[v] > 0) {
            if (!upper) return 1;
            upper_base[v] = row;
            for (int lc = 1; lc <= g.level[v]; ++lc, ++row) {
                const auto& lst = g.up[v][lc - 1];
                uint32_t* r1 = upper + row * R1;
                for (int i = 0; i < R1; ++i) r1[i] = i < (int)lst.size() ? lst[i] : kNone;
            }
        } else {
            upper_base[v] = -1;
        }
    }
    entry_level[0] = (int32_t)g.entry;
    entry_level[1] = g.max_level;
    return 0;
}

// ----------------------------------------------------------------------------
// Alg. 2: quantise the query, greedy descent (ef = 1) through layers L..1,
// SEARCH-LAYER on layer 0 with ef_eff = max(ef, k), C = first N_c of W,
// asymmetric distances to the decoded candidates (Stage 2), sort by (d^a, id),
// early-termination test when |A| > k, exact distances for the first
// n_exact entries (Stage 3), union with the rest of A, sort, top k.
//
// Counts: N_c = n_coarse, or ceil(ef_eff / m_ef), clamped to [k, ef_eff];
//         N_rerank = n_rerank, or ceil(N_c * rerank_pct / 100), clamped to [k, N_c].
// Outputs per query: ids/dists/exact flags [k] (padding -1 / +inf / 0).
// Optional traces (null to skip): the layer-0 entry point, C ids and integer
// distances [cap_c], |C|, the A list [cap_c], the early-exit flag, n_exact,
// the layer-0 expansion sequence [cap_exp] and its length, the number of
// layer-0 distance evaluations.
struct OracleSearchParams {
    int32_t k, ef, m_ef, rerank_pct, n_coarse, n_rerank;
    double tau_gap, tau_ratio, eps;
};

int oracle_search(int64_t n, int32_t d, int32_t R0, int32_t R1, const uint8_t* codes,
                  const float* x, const uint32_t* adj0, const int64_t* upper_base,
                  const uint32_t* upper, uint32_t entry, int32_t max_level, const float* minv,
                  const float* scale, const float* q, int64_t nq, const OracleSearchParams* P,
                  int32_t nthreads, int64_t* ids_out, double* dists_out, uint8_t* exact_out,
                  uint32_t* l0_entry, uint32_t* c_ids, int64_t* c_dist, int32_t* c_count,
                  uint32_t* a_ids, double* a_dist, uint8_t* et_flag, int32_t* n_exact_out,
                  int32_t cap_c, uint32_t* exp_seq, int32_t* exp_count, int32_t cap_exp,
                  int64_t* evals_out) {
    if (!P || !codes || !x || !adj0 || !q || !ids_out || !dists_out || n < 1 || d <= 0) return 1;
    const int k = P->k;
    if (k < 1 || P->ef < 1 || P->m_ef < 1 || P->rerank_pct < 0) return 1;
    FlatIndex ix{n, d, R0, R1, codes, x, adj0, upper_base, upper, entry, max_level, minv, scale};
    const int ef_eff = std::max(P->ef, k);
    int Nc = P->n_coarse > 0 ? P->n_coarse : (ef_eff + P->m_ef - 1) / P->m_ef;
    Nc = std::min(std::max(Nc, k), ef_eff);
    int Nr = P->n_rerank > 0 ? P->n_rerank : (int)(((int64_t)Nc * P->rerank_pct + 99) / 100);
    Nr = std::min(std::max(Nr, k), Nc);
    if ((c_ids || a_ids) && cap_c < Nc) return 1;
    std::function<const uint8_t*(uint32_t)> code_of = [&](uint32_t v) { return ix.code(v); };

    parallel_for(nq, n_threads(nthreads), [&](int64_t qi) {
        const float* qv = q + qi * d;
        std::vector<uint8_t> qc(d);
        oracle_encode(qv, 1, d, minv, scale, qc.data());
        std::vector<uint8_t> visited(n, 0);
        std::vector<uint32_t> touched;
        Key cur{l2_codes(qc.data(), ix.code(entry), d), entry};
        for (int lc = max_level; lc >= 1; --lc) {
            auto W = search_layer(qc.data(), d, cur, 1, code_of,
                                  [&](uint32_t u, std::vector<uint32_t>& o) { ix.nbrs(u, lc, o); },
                                  visited, touched, nullptr);
            cur = W[0];
        }
        if (l0_entry) l0_entry[qi] = cur.second;
        SearchTrace tr;
        auto W = search_layer(qc.data(), d, cur, ef_eff, code_of,
                              [&](uint32_t u, std::vector<uint32_t>& o) { ix.nbrs(u, 0, o); },
                              visited, touched, &tr);
        int nc = std::min<int>(Nc, (int)W.size());
        if (c_ids)
            for (int i = 0; i < nc; ++i) {
                c_ids[qi * cap_c + i] = W[i].second;
                c_dist[qi * cap_c + i] = W[i].first;
            }
        if (c_count) c_count[qi] = nc;
        if (exp_seq) {
            int m = std::min<int>(cap_exp, (int)tr.expanded.size());
            for (int i = 0; i < m; ++i) exp_seq[qi * cap_exp + i] = tr.expanded[i];
        }
        if (exp_count) exp_count[qi] = (int32_t)tr.expanded.size();
        if (evals_out) evals_out[qi] = tr.evals;

        // Stage 2: decode x~ = code / scale_j + min_j and take the squared
        // distance to the full-precision query.
        std::vector<std::pair<double, uint32_t>> A(nc);
        for (int i = 0; i < nc; ++i) {
            const uint8_t* c = ix.code(W[i].second);
            double s = 0.0;
            for (int j = 0; j < d; ++j) {
                double xt = (double)c[j] / (double)scale[j] + (double)minv[j];
                double t = (double)qv[j] - xt;
                s += t * t;
            }
            A[i] = {s, W[i].second};
        }
        std::sort(A.begin(), A.end());
        if (a_ids)
            for (int i = 0; i < nc; ++i) {
                a_ids[qi * cap_c + i] = A[i].second;
                a_dist[qi * cap_c + i] = A[i].first;
            }
        // Early termination (Section 3.2).
        bool et = false;
        if (nc > k) {
            double dk = A[k - 1].first, dk1 = A[k].first;
            double gap = (dk1 - dk) / (dk + P->eps);
            double ratio = dk1 / (dk + P->eps);
            et = gap > P->tau_gap || ratio > P->tau_ratio;
        }
        int ne = et ? std::min(k, nc) : std::min(Nr, nc);
        if (et_flag) et_flag[qi] = et ? 1 : 0;
        if (n_exact_out) n_exact_out[qi] = ne;
        // Stage 3 and assembly.
        struct R {
            double dist;
            uint32_t id;
            uint8_t exact;
        };
        std::vector<R> res;
        for (int i = 0; i < nc; ++i) {
            if (i < ne)
                res.push_back({l2_f64(qv, x + (int64_t)A[i].second * d, d), A[i].second, 1});
            else
                res.push_back({A[i].first, A[i].second, 0});
        }
        std::sort(res.begin(), res.end(), [](const R& a, const R& b) {
            return a.dist != b.dist ? a.dist < b.dist : a.id < b.id;
        });
        for (int i = 0; i < k; ++i) {
            if (i < (int)res.size()) {
                ids_out[qi * k + i] = res[i].id;
                dists_out[qi * k + i] = res[i].dist;
                if (exact_out) exact_out[qi * k + i] = res[i].exact;
            } else {
                ids_out[qi * k + i] = -1;
                dists_out[qi * k + i] = HUGE_VAL;
                if (exact_out) exact_out[qi * k + i] = 0;
            }
        }
    });
    return 0;
}

// Distances of given (query, base id) pairs, one by one, in the oracle's
// arithmetic: exact FP64 squared L2 (Alg. 2), asymmetric FP64
// distance to the decoded code (Alg. 2) and the integer code distance
// of the encoded query (Alg. 2 without s_dist).  Any output may be null.
int oracle_pair_dists(const float* x, const uint8_t* codes, int32_t d, const float* minv,
                      const float* scale, const float* q, const int64_t* qi, const int64_t* ids,
                      int64_t m, double* exact_out, double* asym_out, int64_t* code_out) {
    if (!q || !qi || !ids || d <= 0) return 1;
    std::vector<uint8_t> qc(d);
    for (int64_t t = 0; t < m; ++t) {
        const float* qv = q + qi[t] * d;
        if (exact_out) exact_out[t] = l2_f64(qv, x + ids[t] * d, d);
        if (asym_out || code_out) {
            const uint8_t* c = codes + ids[t] * d;
            if (asym_out) {
                double s = 0.0;
                for (int j = 0; j < d; ++j) {
                    double xt = (double)c[j] / (double)scale[j] + (double)minv[j];
                    double u = (double)qv[j] - xt;
                    s += u * u;
                }
                asym_out[t] = s;
            }
            if (code_out) {
                oracle_encode(qv, 1, d, minv, scale, qc.data());
                code_out[t] = l2_codes(qc.data(), c, d);
            }
        }
    }
    return 0;
}

// Brute-force exact k nearest neighbours by FP64 squared L2, ties by id.
int oracle_bruteforce(const float* x, int64_t n, int32_t d, const float* q, int64_t nq, int32_t k,
                      int32_t nthreads, int64_t* ids, double* dists) {
    if (!x || !q || !ids || !dists || k < 1 || d <= 0) return 1;
    parallel_for(nq, n_threads(nthreads), [&](int64_t qi) {
        std::vector<std::pair<double, int64_t>> all(n);
        for (int64_t j = 0; j < n; ++j) all[j] = {l2_f64(q + qi * d, x + j * d, d), j};
        int m = (int)std::min<int64_t>(k, n);
        std::partial_sort(all.begin(), all.begin() + m, all.end());
        for (int i = 0; i < k; ++i) {
            ids[qi * k + i] = i < m ? all[i].second : -1;
            dists[qi * k + i] = i < m ? all[i].first : HUGE_VAL;
        }
    });
    return 0;
}

// Brute-force top-k by integer code distance (ties by id): the exact answer
// layer-0 search must return when its beam covers a connected graph.
int oracle_bruteforce_codes(const uint8_t* codes, int64_t n, int32_t d, const uint8_t* qc,
                            int64_t nq, int32_t k, int64_t* ids, int64_t* dists) {
    if (!codes || !qc || !ids || !dists || k < 1) return 1;
    for (int64_t qi = 0; qi < nq; ++qi) {
        std::vector<Key> all(n);
        for (int64_t j = 0; j < n; ++j)
            all[j] = {l2_codes(qc + qi * d, codes + j * d, d), (uint32_t)j};
        int m = (int)std::min<int64_t>(k, n);
        std::partial_sort(all.begin(), all.begin() + m, all.end());
        for (int i = 0; i < k; ++i) {
            ids[qi * k + i] = i < m ? (int64_t)all[i].second : -1;
            dists[qi * k + i] = i < m ? all[i].first : -1;
        }
    }
    return 0;
}

// Top-k of the union of per-shard result lists (database sharding; the
// paper has none): every (distance, id + offset of its shard) with id >= 0,
// sorted by distance then global id like the final ranking of Alg. 2, the
// first k, padded with id -1 / +inf.  dists, ids: [S, n, kin] row-major.
int oracle_merge_topk(const float* dists, const int64_t* ids, int32_t S, int64_t n, int32_t kin,
                      const int64_t* offsets, int32_t k, int64_t* ids_out, double* dists_out) {
    if (!dists || !ids || !ids_out || !dists_out || S < 1 || kin < 1 || k < 1) return 1;
    for (int64_t q = 0; q < n; ++q) {
        std::vector<std::pair<double, int64_t>> all;
        for (int32_t s = 0; s < S; ++s)
            for (int32_t j = 0; j < kin; ++j) {
                const int64_t at = ((int64_t)s * n + q) * kin + j;
                if (ids[at] >= 0) all.push_back({(double)dists[at], ids[at] + (offsets ? offsets[s] : 0)});
            }
        std::sort(all.begin(), all.end());
        for (int32_t t = 0; t < k; ++t) {
            const bool have = t < (int32_t)all.size();
            ids_out[q * k + t] = have ? all[t].second : -1;
            dists_out[q * k + t] = have ? all[t].first : HUGE_VAL;
        }
    }
    return 0;
}

// ----------------------------------------------------------------------------
// Index file writer (format "AQRIDX01", little-endian):
//   char magic[8]; u32 version=1; u32 d; u64 n; u32 M_i; u32 R0; u32 R1;
//   u32 entry; i32 max_level; u32 ef_c; u64 n_upper_rows;
//   f64 s_dist; f64 delta; f64 eta;                       (80-byte header)
//   f32 min[d]; f32 scale[d]; u8 codes[n*d]; f32 x[n*d];
//   u32 adj0[n*R0]; i64 upper_base[n]; u32 upper[n_upper_rows*R1];
//   u64 FNV-1a-64 of every preceding byte.
int oracle_write_index(const char* path, int64_t n, int32_t d, int32_t M_i, int32_t R0, int32_t R1,
                       uint32_t entry, int32_t max_level, int32_t ef_c, int64_t n_upper,
                       double s_dist, double delta, double eta, const float* minv,
                       const float* scale, const uint8_t* codes, const float* x,
                       const uint32_t* adj0, const int64_t* upper_base, const uint32_t* upper) {
    FILE* f = std::fopen(path, "wb");
    if (!f) return 1;
    uint64_t h = 1469598103934665603ull;
    bool ok = true;
    auto put = [&](const void* p, size_t bytes) {
        const uint8_t* b = (const uint8_t*)p;
        for (size_t i = 0; i < bytes; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
        if (bytes && std::fwrite(p, 1, bytes, f) != bytes) ok = false;
    };
    const char magic[8] = {'A', 'Q', 'R', 'I', 'D', 'X', '0', '1'};
    uint32_t version = 1, ud = (uint32_t)d, um = (uint32_t)M_i, ur0 = (uint32_t)R0,
             ur1 = (uint32_t)R1, uef = (uint32_t)ef_c;
    uint64_t un = (uint64_t)n, uup = (uint64_t)n_upper;
    put(magic, 8);
    put(&version, 4);
    put(&ud, 4);
    put(&un, 8);
    put(&um, 4);
    put(&ur0, 4);
    put(&ur1, 4);
    put(&entry, 4);
    put(&max_level, 4);
    put(&uef, 4);
    put(&uup, 8);
    put(&s_dist, 8);
    put(&delta, 8);
    put(&eta, 8);
    put(minv, 4 * (size_t)d);
    put(scale, 4 * (size_t)d);
    put(codes, (size_t)n * d);
    put(x, 4 * (size_t)n * d);
    put(adj0, 4 * (size_t)n * R0);
    put(upper_base, 8 * (size_t)n);
    if (n_upper) put(upper, 4 * (size_t)n_upper * R1);
    uint64_t hh = h;
    if (std::fwrite(&hh, 1, 8, f) != 8) ok = false;
    std::fclose(f);
    return ok ? 0 : 1;
}

}  // extern "C"
