"""Pins for the oracle's search path (Section 3.2, Alg. 2) and its graph build.

Special cases that reduce to brute force: with ef >= n on a connected
layer-0 graph, Stage 1 returns the exact top N_c by integer code distance;
with every candidate re-ranked and early exit off the pipeline returns the
exact top-k by FP64 L2.  Early exit is pinned on hand-made lists; the
greedy descent against an independent Python walk; the layer-0 beam at
intermediate ef against the textbook SEARCH-LAYER written out in Python;
the build against a plain Python re-statement of the textbook insertion on
tiny inputs.
"""

import collections
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

NONE = oracle.NONE


@pytest.fixture(scope="module")
def small():
    w = synth.workload("gmm10k_d128", n=1500, nq=40)
    idx = oracle.make_index(w["x"], w["U"], w["sample"], M0=8, ef0=60)
    return w, idx


def _reachable(adj0, entry):
    seen = {entry}
    dq = collections.deque([entry])
    while dq:
        u = dq.popleft()
        for v in adj0[u]:
            if v != NONE and v not in seen:
                seen.add(int(v))
                dq.append(int(v))
    return seen


def test_graph_invariants(small):
    w, idx = small
    n = idx["codes"].shape[0]
    M = idx["M_i"]
    adj0, ub, up, lv = idx["adj0"], idx["upper_base"], idx["upper"], idx["levels"]
    assert adj0.shape == (n, 2 * M)
    for v in range(n):
        row = adj0[v][adj0[v] != NONE]
        assert np.all(adj0[v][len(row):] == NONE)  # packed at the front
        assert v not in row
        assert len(set(row.tolist())) == len(row)
        assert 1 <= len(row) <= 2 * M or n == 1
        if lv[v] > 0:
            for lc in range(1, lv[v] + 1):
                r = up[ub[v] + lc - 1]
                r = r[r != NONE]
                assert v not in r and len(set(r.tolist())) == len(r) and len(r) <= M
                assert np.all(lv[r] >= lc)
        else:
            assert ub[v] == -1
    assert lv[idx["entry"]] == idx["max_level"] == lv.max()
    assert idx["entry"] == int(np.argmax(lv))  # first node of the top level
    assert len(_reachable(adj0, idx["entry"])) == n


def test_stage1_exact_when_beam_covers_graph(small):
    w, idx = small
    n = idx["codes"].shape[0]
    q = w["q"][:8]
    r = oracle.search(idx, q, k=10, ef=n, trace=True)
    qc = oracle.encode(q, idx["min"], idx["scale"])
    nc = int(r["c_count"][0])
    assert nc == (n + 2) // 3
    bf_ids, bf_d = oracle.bruteforce_codes(idx["codes"], qc, nc)
    np.testing.assert_array_equal(r["c_ids"][:, :nc], bf_ids)
    np.testing.assert_array_equal(r["c_dist"][:, :nc], bf_d)
    # every node reachable -> every node expanded exactly once
    assert np.all(r["exp_count"] == n)


def test_int_distance_is_sum_of_squared_code_differences(small):
    w, idx = small
    qc = oracle.encode(w["q"][:3], idx["min"], idx["scale"])
    ids, dd = oracle.bruteforce_codes(idx["codes"], qc, 5)
    c = idx["codes"].astype(np.int64)
    for i in range(3):
        ref = ((c - qc[i].astype(np.int64)) ** 2).sum(1)
        order = np.lexsort((np.arange(len(ref)), ref))[:5]
        np.testing.assert_array_equal(ids[i], order)
        np.testing.assert_array_equal(dd[i], ref[order])


def test_bruteforce_matches_numpy(small):
    w, idx = small
    q = w["q"][:7]
    ids, dd = oracle.bruteforce(idx["x"], q, 12)
    x = idx["x"].astype(np.float64)
    for i in range(len(q)):
        ref = ((x - q[i].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((np.arange(len(ref)), ref))[:12]
        np.testing.assert_array_equal(ids[i], order)
        np.testing.assert_allclose(dd[i], ref[order], rtol=1e-14)


def test_full_rerank_without_early_exit_is_exact(small):
    w, idx = small
    n = idx["codes"].shape[0]
    q = w["q"][:6]
    r = oracle.search(idx, q, k=10, ef=n, n_coarse=n, n_rerank=n, tau_gap=np.inf,
                      tau_ratio=np.inf)
    gt, gd = oracle.bruteforce(idx["x"], q, 10)
    np.testing.assert_array_equal(r["ids"], gt)
    np.testing.assert_allclose(r["dists"], gd, rtol=0, atol=0)
    assert np.all(r["exact"] == 1)


def test_rerank_all_of_C_is_sorted_exact_distances(small):
    w, idx = small
    q = w["q"][:10]
    r = oracle.search(idx, q, k=10, ef=64, n_rerank=64, tau_gap=np.inf, tau_ratio=np.inf,
                      trace=True)
    x = idx["x"].astype(np.float64)
    for i in range(len(q)):
        c = r["c_ids"][i, : r["c_count"][i]].astype(np.int64)
        de = ((x[c] - q[i].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((c, de))[:10]
        np.testing.assert_array_equal(r["ids"][i], c[order])
        # numpy sums in a different order: agree to a few ulps
        np.testing.assert_allclose(r["dists"][i], de[order], rtol=1e-14)


def test_assembly_mixes_exact_and_asymmetric_distances(small):
    # Partial re-rank (Alg. 2, Stage 3 and the final assembly): the first
    # n_exact entries of the sorted asymmetric list A get exact FP64
    # distances, the rest keep their asymmetric ones, and the top k of the
    # union by (distance, id) is returned with a flag for the exact ones.
    # n_exact follows the early-exit test on A (k = 10, N_c = 32, N_rerank =
    # ceil(0.4 * 32) = 13).
    w, idx = small
    k, tg, tr, eps = 10, 0.010, 1.008, 1e-6
    r = oracle.search(idx, w["q"], k=k, ef=64, m_ef=2, rerank_pct=40, tau_gap=tg, tau_ratio=tr,
                      eps=eps, trace=True)
    x = idx["x"].astype(np.float64)
    n_et = 0
    for i in range(len(w["q"])):
        nc = int(r["c_count"][i])
        a_ids = r["a_ids"][i, :nc].astype(np.int64)
        a_d = r["a_dist"][i, :nc].astype(np.float64)
        et = 0
        if nc > k:
            dk, dk1 = a_d[k - 1], a_d[k]
            et = int((dk1 - dk) / (dk + eps) > tg or dk1 / (dk + eps) > tr)
        assert int(r["et"][i]) == et
        ne = min(k, nc) if et else min(13, nc)
        assert int(r["n_exact"][i]) == ne
        n_et += et
        de = ((x[a_ids[:ne]] - w["q"][i].astype(np.float64)) ** 2).sum(1)
        dist = np.concatenate([de, a_d[ne:]])
        order = np.lexsort((a_ids, dist))[:k]
        np.testing.assert_array_equal(r["ids"][i], a_ids[order])
        np.testing.assert_allclose(r["dists"][i], dist[order], rtol=1e-14)
        np.testing.assert_array_equal(r["exact"][i], (order < ne).astype(r["exact"].dtype))
    assert 0 < n_et < len(w["q"])  # both branches taken


def test_stage2_asymmetric_distance_by_decode(small):
    w, idx = small
    q = w["q"][:5]
    r = oracle.search(idx, q, k=10, ef=64, trace=True)
    codes = idx["codes"].astype(np.float64)
    dec = codes / idx["scale"].astype(np.float64) + idx["min"].astype(np.float64)
    for i in range(len(q)):
        nc = r["c_count"][i]
        a = r["a_ids"][i, :nc].astype(np.int64)
        assert set(a.tolist()) == set(r["c_ids"][i, :nc].tolist())
        da = ((dec[a] - q[i].astype(np.float64)) ** 2).sum(1)
        np.testing.assert_allclose(r["a_dist"][i, :nc], da, rtol=1e-12)
        assert np.all(np.diff(r["a_dist"][i, :nc]) >= 0)


def test_pair_dists_hand_made():
    # Alg. 2's three distances on a case small enough to work out by hand.
    # d = 2, min = (0, 10), scale = (2, 0.5): codes decode as code / scale +
    # min, i.e. x~ = (c0 / 2, 10 + 2 c1).  Base point x = (3, 14) encodes to
    # rne((3 - 0) * 2) = 6 and rne((14 - 10) * 0.5) = 2, which decode to
    # (3, 14) exactly.  Query q = (0, 10) encodes to codes (0, 0).
    x = np.array([[3.0, 14.0], [1.0, 11.0]], np.float32)
    minv = np.array([0.0, 10.0], np.float32)
    scale = np.array([2.0, 0.5], np.float32)
    codes = oracle.encode(x, minv, scale)
    np.testing.assert_array_equal(codes, [[6, 2], [2, 0]])
    q = np.array([[0.0, 10.0], [3.0, 14.0]], np.float32)
    ex, asy, cd = oracle.pair_dists(x, codes, minv, scale, q, np.array([0, 0, 1, 1]),
                                    np.array([0, 1, 0, 1]))
    # exact: |(3, 4)|^2 = 25, |(1, 1)|^2 = 2, 0, |(2, 3)|^2 = 13
    np.testing.assert_array_equal(ex, [25.0, 2.0, 0.0, 13.0])
    # asymmetric: x1 = (1, 11) has codes (2, 0) -> x~1 = (1, 10), so
    # |q0 - x~1|^2 = 1 and |q1 - x~1|^2 = 4 + 16 = 20
    np.testing.assert_array_equal(asy, [25.0, 1.0, 0.0, 20.0])
    # code distance: q0 -> (0, 0), q1 -> (6, 2): 36 + 4, 4, 0, 16 + 4
    np.testing.assert_array_equal(cd, [40, 4, 0, 20])


def test_pair_dists_against_independent_routines(small):
    # exact: the brute-force routine's own distances for its own ids (that
    # routine is pinned against numpy); code distance: the brute force over
    # codes of the encoded queries; asymmetric: the decode definition
    # x~_j = code_j / scale_j + min_j written out in numpy, and the triangle
    # inequality with the quantisation error, | sqrt(d^a) - sqrt(d^e) | <=
    # |x - x~| <= sqrt(sum_j (1 / (2 scale_j))^2) for x inside the training
    # range, plus the distance to that range outside it (a swapped scale or
    # min breaks the bound).
    w, idx = small
    q = w["q"][:8]
    x = idx["x"]
    gt, gd = oracle.bruteforce(x, q, 15)
    qi = np.repeat(np.arange(len(q)), 15)
    ex, asy, cd = oracle.pair_dists(x, idx["codes"], idx["min"], idx["scale"], q, qi,
                                    gt.reshape(-1))
    np.testing.assert_array_equal(ex, gd.reshape(-1))
    qc = oracle.encode(q, idx["min"], idx["scale"])
    cid, cdd = oracle.bruteforce_codes(idx["codes"], qc, 15)
    _, _, cd2 = oracle.pair_dists(x, idx["codes"], idx["min"], idx["scale"], q, qi,
                                  cid.reshape(-1))
    np.testing.assert_array_equal(cd2, cdd.reshape(-1))
    dec = idx["codes"].astype(np.float64) / idx["scale"].astype(np.float64) + \
        idx["min"].astype(np.float64)
    ids = gt.reshape(-1)
    da = ((dec[ids] - q[qi].astype(np.float64)) ** 2).sum(1)
    np.testing.assert_allclose(asy, da, rtol=1e-12)
    lo, hi = idx["min"].astype(np.float64), idx["max"].astype(np.float64)
    half = 0.5 / idx["scale"].astype(np.float64)
    xb = x[ids].astype(np.float64)
    out = np.maximum(0.0, np.maximum(lo - xb, xb - hi))
    bound = np.sqrt(((half + out) ** 2).sum(1))
    gap = np.abs(np.sqrt(asy) - np.sqrt(ex))
    assert np.all(gap <= bound * (1 + 1e-5) + 1e-6)
    assert np.all(gap > 0)  # decoding is not the identity on this data
    # a base point against itself: exact 0, code distance 0
    self_ids = np.arange(0, x.shape[0], 97)
    ex0, asy0, cd0 = oracle.pair_dists(x, idx["codes"], idx["min"], idx["scale"], x[self_ids],
                                       np.arange(len(self_ids)), self_ids)
    assert np.all(ex0 == 0) and np.all(cd0 == 0)
    xs = x[self_ids].astype(np.float64)
    out0 = np.maximum(0.0, np.maximum(lo - xs, xs - hi))
    np.testing.assert_allclose(np.sqrt(asy0), np.sqrt(((dec[self_ids] - xs) ** 2).sum(1)),
                               rtol=1e-12)
    assert np.all(np.sqrt(asy0) <= np.sqrt(((half + out0) ** 2).sum(1)) * (1 + 1e-5) + 1e-6)


def test_greedy_descent_matches_python_walk(small):
    # ef = 1 on layer 0 is a greedy walk: from the entry, move to the best
    # neighbour by (distance, id) while it is strictly better.
    w, idx = small
    qc = oracle.encode(w["q"], idx["min"], idx["scale"]).astype(np.int64)
    codes = idx["codes"].astype(np.int64)
    r = oracle.search(idx, w["q"], k=1, ef=1, trace=True)
    ub, up = idx["upper_base"], idx["upper"]
    for i in range(len(qc)):
        def dist(v):
            return int(((codes[v] - qc[i]) ** 2).sum())

        def walk(cur, rows):
            path = [cur]
            while True:
                best = (dist(cur), cur)
                for v in rows(cur):
                    if v != NONE:
                        best = min(best, (dist(int(v)), int(v)))
                if best[1] == cur:
                    return path
                cur = best[1]
                path.append(cur)

        cur = idx["entry"]
        for lc in range(idx["max_level"], 0, -1):
            cur = walk(cur, lambda u, lc=lc: up[ub[u] + lc - 1])[-1]
        assert r["l0_entry"][i] == cur
        path = walk(cur, lambda u: idx["adj0"][u])
        assert r["exp_count"][i] == len(path)
        np.testing.assert_array_equal(r["exp_seq"][i, : len(path)], path)
        assert r["ids"][i, 0] == path[-1]


@pytest.mark.parametrize("ef", [8, 24, 60])
def test_layer0_beam_matches_textbook_search_layer(small, ef):
    # The layer-0 beam from the oracle's entry point against the textbook
    # SEARCH-LAYER written out in Python (a candidate list and a result list
    # of at most ef, both by (distance, id); stop when the best candidate is
    # worse than the worst result): the same expansions in the same order and
    # the same final result set (m_ef = 1 makes C the whole of W).
    w, idx = small
    qc = oracle.encode(w["q"], idx["min"], idx["scale"]).astype(np.int64)
    codes = idx["codes"].astype(np.int64)
    adj0 = idx["adj0"]
    r = oracle.search(idx, w["q"], k=1, ef=ef, m_ef=1, trace=True)
    for i in range(len(qc)):
        def dist(v):
            return int(((codes[v] - qc[i]) ** 2).sum())

        ep = int(r["l0_entry"][i])
        visited = {ep}
        cand = [(dist(ep), ep)]
        W = [(dist(ep), ep)]
        order = []
        while cand:
            c = min(cand)
            cand.remove(c)
            if c > max(W):
                break
            order.append(c[1])
            for e in adj0[c[1]]:
                e = int(e)
                if e == NONE or e in visited:
                    continue
                visited.add(e)
                ek = (dist(e), e)
                if len(W) < ef or ek < max(W):
                    cand.append(ek)
                    W.append(ek)
                    if len(W) > ef:
                        W.remove(max(W))
        W.sort()
        n_c = int(r["c_count"][i])
        assert n_c == len(W)
        got = list(zip(r["c_dist"][i, :n_c].tolist(), r["c_ids"][i, :n_c].tolist()))
        assert got == W
        assert int(r["exp_count"][i]) == len(order)
        np.testing.assert_array_equal(r["exp_seq"][i, : len(order)], order)


def _line_index(xs, R0=None):
    """1-D index with identity quantiser (min 0, scale 1), complete layer 0."""
    xs = np.asarray(xs, np.float32)
    n = len(xs)
    R0 = R0 or max(n - 1, 1)
    adj0 = np.full((n, R0), NONE, np.uint32)
    for v in range(n):
        nb = [u for u in range(n) if u != v]
        adj0[v, : len(nb)] = nb
    return dict(codes=np.rint(xs).astype(np.uint8)[:, None], x=xs[:, None], adj0=adj0,
                upper_base=np.full(n, -1, np.int64), upper=np.zeros((0, 1), np.uint32), entry=0,
                max_level=0, min=np.zeros(1, np.float32), scale=np.ones(1, np.float32))


@pytest.mark.parametrize("pts,k,tau_gap,tau_ratio,et,n_exact", [
    # A = 0, 1, 4, 9, 16 (q = 0): d_k=1, d_k+1=4 -> ratio ~4 -> exit, rerank k
    ([0, 1, 2, 3, 4], 2, 0.010, 1.008, 1, 2),
    # thresholds above the separation -> no exit, rerank N_rerank (=3 here)
    ([0, 1, 2, 3, 4], 2, 10.0, 10.0, 0, 3),
    # |A| = k -> no test, n_exact = min(N_rerank, |A|)
    ([0, 1], 2, 0.0, 0.0, 0, 2),
    # A = 0, 40000, 40401: gap = 0.010025, ratio = 1.010025 (to 1e-6)
    # ratio exit only: gap not > 0.02, ratio > 1.008
    ([0, 200, 201], 2, 0.02, 1.008, 1, 2),
    # gap exit only (tau_ratio out of reach)
    ([0, 200, 201], 2, 0.005, 5.0, 1, 2),
    # neither: gap <= 0.02 and ratio <= 1.02 -> rerank N_rerank = 3
    ([0, 200, 201], 2, 0.02, 1.02, 0, 3),
])
def test_early_exit_hand_made(pts, k, tau_gap, tau_ratio, et, n_exact):
    idx = _line_index(pts)
    n = len(pts)
    r = oracle.search(idx, np.zeros((1, 1), np.float32), k=k, ef=n, n_coarse=n,
                      n_rerank=min(3, n), tau_gap=tau_gap, tau_ratio=tau_ratio, trace=True)
    assert int(r["et"][0]) == et
    assert int(r["n_exact"][0]) == n_exact


def test_gap_ratio_identity():
    # gap = ratio - d_k / (d_k + eps): with tau_gap >= tau_ratio - 1 the
    # ratio test decides every case the gap test does.
    rng = np.random.default_rng(7)
    dk = rng.uniform(1e-3, 1e4, 1000)
    dk1 = dk * rng.uniform(1.0, 1.05, 1000)
    eps = 1e-6
    gap = (dk1 - dk) / (dk + eps)
    ratio = dk1 / (dk + eps)
    np.testing.assert_allclose(gap, ratio - dk / (dk + eps), rtol=1e-9, atol=1e-15)


def test_padding_when_graph_smaller_than_k():
    idx = _line_index([5, 9, 1])
    r = oracle.search(idx, np.array([[4.0]], np.float32), k=5, ef=8)
    assert list(r["ids"][0]) == [0, 2, 1, -1, -1]
    assert list(r["dists"][0][:3]) == [1.0, 9.0, 25.0]
    assert np.all(np.isinf(r["dists"][0][3:]))


# --- graph build: textbook sequential insertion re-stated in Python ---------

def _py_build(codes, lv, M, ef_c, starts):
    codes = codes.astype(np.int64)
    n = len(codes)

    def d(a, b):
        return int(((codes[a] - codes[b]) ** 2).sum())

    nb = [[[] for _ in range(lv[v] + 1)] for v in range(n)]

    def search(q, ep, ef, lc):
        vis = {ep}
        cand = [(d(q, ep), ep)]
        W = [(d(q, ep), ep)]
        while cand:
            cand.sort()
            c = cand.pop(0)
            if c > max(W):
                break
            for e in nb[c[1]][lc]:
                if e in vis:
                    continue
                vis.add(e)
                ek = (d(q, e), e)
                if len(W) < ef or ek < max(W):
                    cand.append(ek)
                    W.append(ek)
                    if len(W) > ef:
                        W.remove(max(W))
        return sorted(W)

    def heuristic(base_cands, Mx):
        R = []
        for de, e in base_cands:
            if len(R) >= Mx:
                break
            if all(d(e, r) > de for r in R):
                R.append(e)
        return R

    entry, L = None, -1
    for b in range(len(starts) - 1):
        s, e = starts[b], starts[b + 1]
        sel = {}
        if entry is not None:
            for v in range(s, e):
                cur = (d(v, entry), entry)
                for lc in range(L, lv[v], -1):
                    cur = search(v, cur[1], 1, lc)[0]
                sel[v] = {}
                for lc in range(min(L, lv[v]), -1, -1):
                    W = search(v, cur[1], ef_c, lc)
                    sel[v][lc] = heuristic(W, M)
                    cur = W[0]
        for v in range(s, e):
            for lc, R in sorted(sel.get(v, {}).items()):
                nb[v][lc] = list(R)
                cap = 2 * M if lc == 0 else M
                for r in R:
                    if len(nb[r][lc]) < cap:
                        nb[r][lc].append(v)
                    else:
                        cands = sorted([(d(r, u), u) for u in nb[r][lc]] + [(d(r, v), v)])
                        nb[r][lc] = heuristic(cands, cap)
        for v in range(s, e):
            if lv[v] > L:
                L, entry = lv[v], v
    return nb, entry, L


@pytest.mark.parametrize("batch_div,batch_max", [(1, 1), (4, 16)])
def test_build_matches_python_restatement(batch_div, batch_max):
    rng = np.random.default_rng(11)
    n, d, M, ef_c = 160, 6, 4, 12
    codes = rng.integers(0, 256, (n, d)).astype(np.uint8)
    codes[5] = codes[4]  # a duplicate vector: distance-0 ties
    lv = oracle.levels(synth.level_uniforms(n, 3), M)
    g = oracle.build_graph(codes, lv, M, ef_c, batch_div, batch_max, nthreads=2)
    starts = oracle.batch_schedule(n, batch_div, batch_max)
    nb, entry, L = _py_build(codes, lv, M, ef_c, list(starts))
    assert g["entry"] == entry and g["max_level"] == L
    for v in range(n):
        row = g["adj0"][v]
        assert list(row[row != NONE]) == nb[v][0]
        for lc in range(1, lv[v] + 1):
            r = g["upper"][g["upper_base"][v] + lc - 1]
            assert list(r[r != NONE]) == nb[v][lc]


def test_build_is_deterministic_across_thread_counts():
    w = synth.workload("gmm10k_d128", n=600, nq=1)
    P = oracle.train(w["x"], M0=8, ef0=40)
    codes = oracle.encode(w["x"], P["min"], P["scale"])
    lv = oracle.levels(w["U"], P["M_i"])
    a = oracle.build_graph(codes, lv, P["M_i"], P["ef_c"], nthreads=1)
    b = oracle.build_graph(codes, lv, P["M_i"], P["ef_c"], nthreads=5)
    for key in ("adj0", "upper_base", "upper"):
        np.testing.assert_array_equal(a[key], b[key])


def test_recall_sanity(small):
    w, idx = small
    gt, _ = oracle.bruteforce(idx["x"], w["q"], 10)
    r = oracle.search(idx, w["q"], k=10, ef=256)
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(r["ids"], gt)])
    assert rec >= 0.95


def test_index_file_round_trip(small):
    w, idx = small
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "i.aqr")
        oracle.write_index(path, idx)
        raw = open(path, "rb").read()
    assert raw[:8] == b"AQRIDX01"
    hdr = np.frombuffer(raw[8:80], dtype=np.uint8)
    version, d = np.frombuffer(hdr[:8].tobytes(), np.uint32)
    n = int(np.frombuffer(hdr[8:16].tobytes(), np.uint64)[0])
    assert version == 1 and d == 128 and n == idx["codes"].shape[0]
    h = 1469598103934665603
    for byte in raw[:-8]:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    assert h == int(np.frombuffer(raw[-8:], np.uint64)[0])
    rows = idx["upper"].shape[0]
    M = idx["M_i"]
    size = 80 + 8 * d + n * d + 4 * n * d + 4 * n * 2 * M + 8 * n + 4 * rows * M + 8
    assert len(raw) == size
