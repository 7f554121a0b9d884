"""Full-size checks on the benchmark's workload (1M x 128, 10,000 queries) in
the launch configuration the benchmark times (k = 10, ef = 96, N_c = ef/2,
every candidate of C re-ranked, one lane per candidate, 1024-id visited hash
of 16-bit tags, 32-row tile).

The oracle cannot build a 1M graph in test time, so it checks what it can
compute one by one, from the seeded inputs only: the quantiser parameters
(its own FP64 training on the same 1M set), sampled code rows, and, for
sampled queries, every distance the GPU reports (integer code distances of
C, asymmetric distances of A, exact or asymmetric distances of the result),
the early-termination decision on those distances, and recall against its
brute-force top-10.  It also searches the GPU-built graph itself (exported)
for sampled queries: the layer-0 expansion sequence, C, A, the early-exit
decision and the result must match the full batch's trace.  Properties that
hold at any size are checked on the whole graph.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import TOL, _close, check_stage1, check_stages_2_3, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K, EF, M_EF, RERANK = 10, 96, 2, 100
KCFG = dict(hash_slots=1024, tile_rows=32, team_lanes=1)


@pytest.fixture(scope="module")
def full():
    from paper_2602_21600_gb300 import Context
    w = synth.workload("gmm1m_d128_int")
    ctx = Context(0)
    xd = torch.from_numpy(w["x"]).cuda()
    P_g = ctx.train(xd, w["sample"], M0=w["M0"], ef0=w["ef0"])
    ctx.build_graph(xd, P_g["min"], P_g["scale"], w["U"], P_g["M_i"], P_g["ef_c"],
                    s_dist=P_g["s_dist"])
    del xd
    yield w, ctx, P_g
    ctx.close()


def test_training_equals_oracle_at_full_size(full):
    w, ctx, P_g = full
    P_o = oracle.train(w["x"], w["sample"], M0=w["M0"], ef0=w["ef0"])
    for key in ("min", "max", "scale"):
        np.testing.assert_array_equal(P_g[key], P_o[key])
    for key in ("delta", "rho_bar", "eta", "M_i", "ef_c", "P_l", "P_h"):
        assert P_g[key] == P_o[key], key


def test_graph_properties_and_codes_at_full_size(full):
    w, ctx, P_g = full
    g = ctx.export_graph()
    n = w["x"].shape[0]
    M = P_g["M_i"]
    adj = g["adj0"].astype(np.int64)
    none = np.int64(oracle.NONE)
    valid = adj != none
    # packed rows, ids in range, no self loops, no duplicates, degree >= 1
    assert np.all(valid[:, :-1] | ~valid[:, 1:])
    assert np.all(adj[valid] < n)
    assert not np.any(adj == np.arange(n)[:, None])
    srt = np.sort(np.where(valid, adj, -1 - np.arange(adj.shape[1])[None, :]), axis=1)
    assert not np.any(srt[:, 1:] == srt[:, :-1])
    assert np.all(valid.sum(1) >= 1) and adj.shape[1] == 2 * M
    # upper layers: entries reach their layer
    lv = oracle.levels(w["U"], M)
    assert g["max_level"] == lv.max() and lv[g["entry"]] == lv.max()
    ub = g["upper_base"]
    np.testing.assert_array_equal(ub >= 0, lv > 0)
    for v in np.nonzero(lv > 0)[0][:20000]:
        for lc in range(1, lv[v] + 1):
            r = g["upper"][ub[v] + lc - 1]
            r = r[r != oracle.NONE].astype(np.int64)
            assert np.all(lv[r] >= lc) and v not in r and len(set(r.tolist())) == len(r) <= M
    # sampled code rows: bit-exact against the oracle's encode
    rows = np.random.default_rng(1).choice(n, 4000, replace=False)
    np.testing.assert_array_equal(g["codes"][rows], oracle.encode(w["x"][rows], P_g["min"], P_g["scale"]))


def test_sampled_queries_at_full_size(full):
    w, ctx, P_g = full
    ctx.set_params(m_ef=M_EF, rerank_pct=RERANK)
    ctx.set_kernel_config(EF, K, **KCFG)
    qd = torch.from_numpy(w["q"]).cuda()
    t = ctx.search_trace(qd, K, EF, cap_exp=1)
    torch.cuda.synchronize()
    t = {k: v.cpu().numpy() for k, v in t.items()}
    ctx.set_kernel_config(EF, K)
    codes = ctx.export_graph()["codes"]
    x, q = w["x"], w["q"]
    S = np.random.default_rng(2).choice(len(q), 120, replace=False)
    tau_gap, tau_ratio, eps = float(np.float32(0.010)), float(np.float32(1.008)), 1e-6
    Nc = -(-EF // M_EF)
    hits = 0
    gt, _ = oracle.bruteforce(x, q[S], K)
    for row, i in enumerate(S):
        nc = int(t["c_count"][i])
        assert nc == Nc
        cid = t["c_ids"][i, :nc].astype(np.int64)
        cd = t["c_dist"][i, :nc].astype(np.int64)
        assert np.all((cid >= 0) & (cid < x.shape[0])) and len(set(cid.tolist())) == nc
        # Stage 1: integer code distances, one by one, bit-exact; C ascending by (d, id)
        ex, asy, code = oracle.pair_dists(x, codes, P_g["min"], P_g["scale"], q, np.full(nc, i), cid)
        np.testing.assert_array_equal(cd, code)
        assert np.all((cd[1:] > cd[:-1]) | ((cd[1:] == cd[:-1]) & (cid[1:] > cid[:-1])))
        # Stage 2: asymmetric distances within the tolerance, A ordered by them
        aid = t["a_ids"][i, :nc].astype(np.int64)
        assert sorted(aid.tolist()) == sorted(cid.tolist())
        ref_a = dict(zip(cid.tolist(), asy.tolist()))
        ra = np.array([ref_a[v] for v in aid.tolist()])
        assert np.all(_close(t["a_dist"][i, :nc], ra, TOL))
        assert np.all(ra[:-1] <= ra[1:] * (1 + 2 * TOL))
        # early termination on the oracle's values at the GPU's positions
        dk, dk1 = ra[K - 1], ra[K]
        gap, ratio = (dk1 - dk) / (dk + eps), dk1 / (dk + eps)
        et = int(gap > tau_gap or ratio > tau_ratio)
        if et != int(t["et"][i]):
            assert abs(gap - tau_gap) <= 4e-5 * max(1, gap) + 4e-5 * ratio or \
                abs(ratio - tau_ratio) <= 4e-5 * ratio
        ne = K if t["et"][i] else nc
        assert int(t["n_exact"][i]) == ne
        # result: distances exact or asymmetric as flagged, (distance, id) order
        ids = t["ids"][i].astype(np.int64)
        dd = t["dists"][i].astype(np.float64)
        fl = t["exact"][i]
        assert len(set(ids.tolist())) == K and np.all(ids >= 0)
        ref_e = dict(zip(cid.tolist(), ex.tolist()))
        for p in range(K):
            ref = ref_e[ids[p]] if fl[p] else ref_a[ids[p]]
            assert _close(dd[p], ref, TOL), (i, p)
        assert np.all(dd[1:] >= dd[:-1])
        hits += len(set(ids.tolist()) & set(gt[row].tolist()))
    assert hits / (K * len(S)) >= 0.95


def test_oracle_search_of_the_full_size_graph(full):
    w, ctx, P_g = full
    ctx.set_params(m_ef=M_EF, rerank_pct=RERANK)
    ctx.set_kernel_config(EF, K, **KCFG)
    qd = torch.from_numpy(w["q"]).cuda()
    t = to_np(ctx.search_trace(qd, K, EF, cap_exp=1024))
    torch.cuda.synchronize()
    ctx.set_kernel_config(EF, K)
    idx = dict(P_g)
    idx.update(ctx.export_graph())
    idx["x"] = w["x"]
    S = np.sort(np.random.default_rng(3).choice(len(w["q"]), 200, replace=False))
    o = oracle.search(idx, w["q"][S], k=K, ef=EF, m_ef=M_EF, rerank_pct=RERANK, trace=True,
                      cap_exp=1024)
    g = {key: v[S] for key, v in t.items()}
    assert int(g["exp_count"].max()) <= 1024
    check_stage1(g, o, len(S))
    amb = check_stages_2_3(idx, w["q"][S], g, o, K, EF, m_ef=M_EF, rerank_pct=RERANK)
    assert amb["et"] <= len(S) // 8 and amb["final"] <= len(S) // 4
