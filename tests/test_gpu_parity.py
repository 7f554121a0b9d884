"""CUDA query path against the oracle, through the C ABI (libaqr.so).

Small indexes built by the oracle (several tiles of candidates, ragged
dimension counts, several HNSW levels) are loaded from the index file;
every ef class of the kernel and several k are exercised.
"""

import os
import tempfile

import numpy as np
import pytest

import oracle
import synth
from parity import TOL, check_stage1, check_stages_2_3, derived_counts, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_21600_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _make(name, n, nq, M0, ef0, d=None, int_data=False):
    w = synth.workload(name, n=n, nq=nq)
    x, q = w["x"], w["q"]
    if d is not None:
        x, q = x[:, :d].copy(), q[:, :d].copy()
    P = oracle.train(x, w["sample"] if n > 10000 else None, M0=M0, ef0=ef0)
    idx = oracle.make_index(x, w["U"], None, params=P)
    return w, x, q, idx


@pytest.fixture(scope="module")
def idx128():
    return _make("gmm10k_d128", 3000, 48, M0=8, ef0=60)


@pytest.fixture(scope="module")
def idx37():
    # ragged: 37 dimensions -> 48-byte code rows, 40-float rows
    return _make("gmm10k_d128", 1500, 32, M0=6, ef0=40, d=37)


def _load(ctx, idx):
    with tempfile.TemporaryDirectory() as td:
        p = os.path.join(td, "idx.aqr")
        oracle.write_index(p, idx)
        ctx.load_graph(p)


def _run_parity(ctx, idx, q, k, ef, **params):
    ctx.set_params(**params)
    qd = torch.from_numpy(q).cuda()
    g = to_np(ctx.search_trace(qd, k, ef))
    torch.cuda.synchronize()
    ef_eff, Nc, Nr = derived_counts(k, ef, params.get("m_ef", 3), params.get("rerank_pct", 40),
                                    params.get("n_coarse", 0), params.get("n_rerank", 0))
    o = oracle.search(idx, q, k=k, ef=ef, trace=True, cap_exp=4096,
                      tau_gap=params.get("tau_gap", np.float32(0.010)),
                      tau_ratio=params.get("tau_ratio", np.float32(1.008)),
                      m_ef=params.get("m_ef", 3), rerank_pct=params.get("rerank_pct", 40),
                      n_coarse=params.get("n_coarse", 0), n_rerank=params.get("n_rerank", 0))
    check_stage1(g, o, len(q))
    amb = check_stages_2_3(idx, q, g, o, k, ef, tau_gap=float(np.float32(params.get("tau_gap", 0.010))),
                           tau_ratio=float(np.float32(params.get("tau_ratio", 1.008))),
                           m_ef=params.get("m_ef", 3), rerank_pct=params.get("rerank_pct", 40),
                           n_coarse=params.get("n_coarse", 0), n_rerank=params.get("n_rerank", 0))
    return g, o, amb


@pytest.mark.parametrize("wpq", [0, 1])  # automatic (groups for this small batch), one warp
@pytest.mark.parametrize("k,ef", [(10, 16), (10, 64), (1, 1), (10, 100), (32, 200), (10, 300),
                                  (50, 600), (5, 1000)])
def test_search_parity_d128(ctx, idx128, k, ef, wpq):
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_kernel_config(ef, k, warps_per_query=wpq)
    g, o, amb = _run_parity(ctx, idx, q, k, ef)
    ctx.set_kernel_config(ef, k)
    # the tolerance band is rare: most queries agree on every decision
    assert amb["et"] <= len(q) // 8 and amb["final"] <= len(q) // 4


@pytest.mark.parametrize("k,ef", [(10, 32), (7, 130)])
def test_search_parity_ragged_d37(ctx, idx37, k, ef):
    w, x, q, idx = idx37
    _load(ctx, idx)
    _run_parity(ctx, idx, q, k, ef)


def test_search_parity_param_variants(ctx, idx128):
    w, x, q, idx = idx128
    _load(ctx, idx)
    # explicit N_c / N_rerank, early exit off, then always on
    _run_parity(ctx, idx, q, 10, 128, n_coarse=40, n_rerank=25, tau_gap=1e30, tau_ratio=1e30)
    _run_parity(ctx, idx, q, 10, 128, tau_gap=-1.0, tau_ratio=-1.0)
    _run_parity(ctx, idx, q, 10, 90, m_ef=2, rerank_pct=70)


@pytest.mark.parametrize("target", [0.87, 0.92, 0.96, 0.98])
def test_search_parity_table3_presets(ctx, idx128, target):
    # each Table 3 preset at its own search depth ef = N_c * m_ef
    from paper_2602_21600_gb300.aqr import params_for_recall
    w, x, q, idx = idx128
    _load(ctx, idx)
    p, ef = params_for_recall(target)
    _run_parity(ctx, idx, q, 10, ef, m_ef=p["m_ef"], n_coarse=p["n_coarse"],
                n_rerank=p["n_rerank"], tau_gap=np.float32(p["tau_gap"]),
                tau_ratio=np.float32(p["tau_ratio"]))


def _reachable0(adj0, entry):
    seen = np.zeros(adj0.shape[0], bool)
    seen[entry] = True
    front = [entry]
    while front:
        nxt = adj0[front].reshape(-1)
        nxt = nxt[nxt != oracle.NONE].astype(np.int64)
        nxt = nxt[~seen[nxt]]
        seen[nxt] = True
        front = np.unique(nxt).tolist()
    return seen


def _assert_exact_topk(ids, dd, x, q, k, tol=TOL):
    """ids/dd (CUDA, FP32) against the FP64 brute force: every returned
    distance within tol of the FP64 distance of its id, the i-th distance
    within tol of the i-th true one, and the ids equal wherever the true
    distances around position i are separated by more than 2 tol (FP32
    rounding may swap near-ties only)."""
    gt, gd = oracle.bruteforce(x, q, k + 1)
    ex, _, _ = oracle.pair_dists(x, np.zeros_like(x, np.uint8), np.zeros(x.shape[1], np.float32),
                                 np.ones(x.shape[1], np.float32), q,
                                 np.repeat(np.arange(len(q)), k), ids.reshape(-1))
    ex = ex.reshape(len(q), k)
    np.testing.assert_allclose(dd, ex, rtol=tol)
    np.testing.assert_allclose(ex, gd[:, :k], rtol=2 * tol)
    n_tie = 0
    for i in range(len(q)):
        g = gd[i]
        for j in range(k):
            lo = g[j - 1] if j > 0 else -np.inf
            hi = g[j + 1]
            if g[j] - lo > 2 * tol * g[j] and hi - g[j] > 2 * tol * g[j]:
                assert ids[i, j] == gt[i, j], (i, j)
            else:
                n_tie += 1
    return n_tie


def test_exact_when_beam_covers_graph(ctx):
    # Section 3.2 with the beam as wide as the graph: ef >= n on a connected
    # layer-0 graph visits every node, so C is the whole set; with N_c =
    # N_rerank = n and early exit off every candidate gets its exact
    # distance, and the result is the brute-force top k (by FP32 distance
    # here, FP64 in the brute force).  n = 1000 stays inside the largest ef
    # class (1024).
    w, x, q, idx = _make("gmm10k_d128", 1000, 40, M0=8, ef0=60)
    n = x.shape[0]
    assert _reachable0(idx["adj0"], idx["entry"]).all()  # the premise: one component
    _load(ctx, idx)
    ctx.set_params(n_coarse=1024, n_rerank=1024, tau_gap=1e30, tau_ratio=1e30)
    qd = torch.from_numpy(q).cuda()
    for k, ef in [(10, 1024), (100, 1000), (1, 1000)]:
        t = ctx.search_trace(qd, k, ef)
        g = to_np(t)
        assert np.all(g["c_count"] == n) and np.all(g["n_exact"] == n) and np.all(g["et"] == 0)
        assert np.all(g["exact"] == 1)
        _assert_exact_topk(g["ids"], g["dists"], x, q, k)
        # the oracle's own search takes the same path to the same ids
        o = oracle.search(idx, q, k=k, ef=ef, n_coarse=1024, n_rerank=1024, tau_gap=np.inf,
                          tau_ratio=np.inf)
        gt, _ = oracle.bruteforce(x, q, k)
        np.testing.assert_array_equal(o["ids"], gt)
    # the plain FP32 path at ef >= n: W is the whole graph by FP32 distance
    ids, dd = ctx.search_plain(qd, 10, 1024)
    _assert_exact_topk(ids.cpu().numpy(), dd.cpu().numpy(), x, q, 10)
    ctx.set_params()


def test_search_edge_cases(ctx, idx128):
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    # n = 0 is a no-op
    e = torch.empty((0, 128), dtype=torch.float32, device="cuda")
    ids, dd = ctx.search(e, 10, 64)
    assert ids.shape == (0, 10)
    # one query, k = ef_eff = 1024 (largest class)
    qd = torch.from_numpy(q[:1]).cuda()
    ids, dd = ctx.search(qd, 1024, 1)
    ids = ids.cpu().numpy()[0]
    assert len(set(ids.tolist())) == 1024 and np.all(ids >= 0)
    # out-of-range arguments are rejected with status codes, nothing launched
    from paper_2602_21600_gb300.aqr import AqrError
    for k, ef in [(0, 10), (10, 0), (10, 2000), (2000, 10)]:
        with pytest.raises(AqrError):
            ctx.search(qd, k, ef)
    # queries far outside the training range clip to codes 0 / 255
    qx = torch.full((2, 128), 1e6, device="cuda")
    qx[1] = -1e6
    ids, dd = ctx.search(qx, 5, 32)
    assert np.all(ids.cpu().numpy() >= 0)


def test_encode_bit_exact(ctx):
    rng = np.random.default_rng(3)
    for n, d in [(1000, 128), (257, 37), (3, 960), (0, 16)]:
        x = rng.normal(50, 40, (n, d)).astype(np.float32)
        if n > 4:
            x[0, 0] = np.nan
            x[1, :3] = [np.inf, -np.inf, 1e30]
            # exact .5 ties after scaling
            x[2, :] = 0.5
        mn = rng.uniform(-10, 10, d).astype(np.float32)
        sc = rng.uniform(0.5, 3, d).astype(np.float32)
        if n > 4:
            mn[:] = 0.0
            sc[: d // 2] = 1.0
        ldc = (d + 15) // 16 * 16
        out = ctx.quantize(torch.from_numpy(x).cuda(), torch.from_numpy(mn).cuda(),
                           torch.from_numpy(sc).cuda(), ldc=ldc).cpu().numpy()
        ref = oracle.encode(x, mn, sc) if n else np.zeros((0, d), np.uint8)
        np.testing.assert_array_equal(out[:, :d], ref)
        assert np.all(out[:, d:] == 0)


def test_bruteforce_knn(ctx):
    rng = np.random.default_rng(4)
    # integer data: FP32 sums exact -> ids and distances equal the FP64 oracle
    x = rng.integers(0, 256, (5000, 128)).astype(np.float32)
    q = rng.integers(0, 256, (130, 128)).astype(np.float32)
    ids, dd = ctx.knn(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), 10)
    gt, gd = oracle.bruteforce(x, q, 10)
    np.testing.assert_array_equal(ids.cpu().numpy(), gt)
    np.testing.assert_array_equal(dd.cpu().numpy().astype(np.float64), gd)
    # self exclusion
    sid = torch.arange(130, dtype=torch.int64, device="cuda")
    ids2, _ = ctx.knn(torch.from_numpy(x).cuda(), torch.from_numpy(x[:130]).cuda(), 5, sid)
    ids2 = ids2.cpu().numpy()
    assert all(i not in row for i, row in enumerate(ids2))
    # the largest k (128), k = 100, and more neighbours asked than points exist
    for k, nb in ((128, 5000), (100, 3000), (100, 60)):
        ids, dd = ctx.knn(torch.from_numpy(x[:nb]).cuda(), torch.from_numpy(q).cuda(), k)
        gt, gd = oracle.bruteforce(x[:nb], q, k)
        np.testing.assert_array_equal(ids.cpu().numpy(), gt)
        np.testing.assert_array_equal(dd.cpu().numpy().astype(np.float64), gd)
    with pytest.raises(Exception):
        ctx.knn(torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda(), 129)


def test_train_matches_oracle(ctx):
    # SIFT-like integer data: every FP32 distance is exact -> identical parameters
    w = synth.workload("gmm1m_d128_int", n=4000, nq=1)
    x = w["x"]
    P_o = oracle.train(x, M0=16, ef0=200)
    P_g = ctx.train(torch.from_numpy(x).cuda(), None, M0=16, ef0=200)
    for key in ("min", "max", "scale"):
        np.testing.assert_array_equal(P_g[key], P_o[key])
    for key in ("delta", "rho_bar", "w", "s_dist", "eta", "M_i", "ef_c", "P_l", "P_h"):
        assert P_g[key] == P_o[key], key
    # float data: FP32 distance sums -> agreement to FP32 rounding
    w = synth.workload("gmm10k_d128", n=2500, nq=1)
    P_o = oracle.train(w["x"], M0=16, ef0=100)
    P_g = ctx.train(torch.from_numpy(w["x"]).cuda(), None, M0=16, ef0=100)
    assert P_g["delta"] == pytest.approx(P_o["delta"], rel=1e-5)
    np.testing.assert_allclose(P_g["min"], P_o["min"], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(P_g["scale"], P_o["scale"], rtol=1e-5)
    assert P_g["M_i"] == P_o["M_i"] and P_g["ef_c"] == P_o["ef_c"]


def test_train_sampled(ctx):
    # above 10,000 points only the sample's densities are computed
    w = synth.workload("gmm1m_d128_int", n=12000, nq=1)
    P_o = oracle.train(w["x"], w["sample"][:300], M0=16, ef0=200)
    P_g = ctx.train(torch.from_numpy(w["x"]).cuda(), w["sample"][:300], M0=16, ef0=200)
    for key in ("min", "max", "scale"):
        np.testing.assert_array_equal(P_g[key], P_o[key])
    assert P_g["delta"] == P_o["delta"] and P_g["rho_bar"] == P_o["rho_bar"]


@pytest.mark.parametrize("n,d,M0,ef0,div,bmax", [(2500, 128, 8, 60, 32, 16384),
                                                   (1200, 37, 6, 40, 4, 64),
                                                   (300, 20, 5, 16, 1, 1)])
def test_gpu_build_matches_oracle(ctx, n, d, M0, ef0, div, bmax):
    w = synth.workload("gmm10k_d128", n=n, nq=1)
    x = w["x"][:, :d].copy()
    P = oracle.train(x, M0=M0, ef0=ef0)
    codes = oracle.encode(x, P["min"], P["scale"])
    lv = oracle.levels(w["U"], P["M_i"])
    g_o = oracle.build_graph(codes, lv, P["M_i"], P["ef_c"], div, bmax)
    ctx.build_graph(torch.from_numpy(x).cuda(), P["min"], P["scale"], w["U"], P["M_i"],
                    P["ef_c"], div, bmax)
    g_g = ctx.export_graph()
    np.testing.assert_array_equal(g_g["codes"], codes)
    assert g_g["entry"] == g_o["entry"] and g_g["max_level"] == g_o["max_level"]
    np.testing.assert_array_equal(g_g["upper_base"], g_o["upper_base"])
    np.testing.assert_array_equal(g_g["adj0"], g_o["adj0"])
    np.testing.assert_array_equal(g_g["upper"], g_o["upper"])


def test_mixed_batch_equals_uniform_calls(ctx, idx128):
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    rng = np.random.default_rng(9)
    nq = len(q)
    ks = rng.choice([1, 10, 33], nq).astype(np.int32)
    efs = rng.choice([16, 64, 128, 256, 512, 1000], nq).astype(np.int32)
    qd = torch.from_numpy(q).cuda()
    for rep in range(2):  # second call replays the captured graph
        ids, dd = ctx.search_mixed(qd, ks, efs, k_stride=40)
        ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
        for (k, ef) in set(zip(ks.tolist(), efs.tolist())):
            sel = np.where((ks == k) & (efs == ef))[0]
            ui, ud = ctx.search(qd[sel], int(k), int(ef))
            np.testing.assert_array_equal(ids[sel, :k], ui.cpu().numpy())
            np.testing.assert_array_equal(dd[sel, :k], ud.cpu().numpy())
            assert np.all(ids[sel, k:] == -1)


def test_host_path_equals_device_path(ctx, idx128):
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    ids_h, dd_h = ctx.search_host(torch.from_numpy(q).pin_memory(), 10, 64)
    ids_d, dd_d = ctx.search(torch.from_numpy(q).cuda(), 10, 64)
    np.testing.assert_array_equal(ids_h.numpy(), ids_d.cpu().numpy())
    np.testing.assert_array_equal(dd_h.numpy(), dd_d.cpu().numpy())


def test_plain_f32_path(ctx, idx37):
    w, x, q, idx = idx37
    _load(ctx, idx)
    qd = torch.from_numpy(q).cuda()
    ids, dd = ctx.search_plain(qd, 10, 1024)
    gt, gd = oracle.bruteforce(x, q, 10)
    ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids, gt)])
    assert rec >= 0.99
    # distances are FP32 squared L2 of the returned ids
    ex, _, _ = oracle.pair_dists(x, idx["codes"], idx["min"], idx["scale"], q,
                                 np.repeat(np.arange(len(q)), 10), ids.reshape(-1))
    np.testing.assert_allclose(dd.reshape(-1), ex, rtol=TOL)


def test_stats_counters(ctx, idx128):
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    g = to_np(ctx.search_trace(qd, 10, 64))
    s = ctx.stats()
    assert s["queries"] == len(q) and s["device_errors"] == 0
    assert s["expansions"] >= g["exp_count"].sum()
    assert s["stage2_evals"] == g["c_count"].sum()
    assert s["exact_evals"] == g["n_exact"].sum()
    assert s["early_exits"] == g["et"].sum()


def test_bad_index_files(ctx, idx37):
    from paper_2602_21600_gb300.aqr import AQR_ERR_BAD_FILE, AqrError
    w, x, q, idx = idx37
    with tempfile.TemporaryDirectory() as td:
        p = os.path.join(td, "idx.aqr")
        oracle.write_index(p, idx)
        raw = open(p, "rb").read()
        # huge_n: the header claims 2^31 - 16 points; the file is refused by
        # its size before anything of that size is allocated
        huge_n = raw[:16] + (0x7FFFFFF0).to_bytes(8, "little") + raw[24:]
        for name, blob in [("short", raw[:100]), ("magic", b"XXXXXXXX" + raw[8:]),
                           ("flip", raw[:5000] + bytes([raw[5000] ^ 1]) + raw[5001:]),
                           ("huge_n", huge_n)]:
            bp = os.path.join(td, name)
            open(bp, "wb").write(blob)
            with pytest.raises(AqrError) as ei:
                ctx.load_graph(bp)
            assert ei.value.status == AQR_ERR_BAD_FILE
        with pytest.raises(AqrError):
            ctx.load_graph(os.path.join(td, "missing"))
        # a layer-0 row naming one node twice (valid checksum)
        bad = dict(idx)
        adj = idx["adj0"].copy()
        r = int(np.nonzero((adj != oracle.NONE).sum(1) >= 2)[0][0])
        adj[r, 1] = adj[r, 0]
        bad["adj0"] = adj
        bp = os.path.join(td, "dup")
        oracle.write_index(bp, bad)
        with pytest.raises(AqrError) as ei:
            ctx.load_graph(bp)
        assert ei.value.status == AQR_ERR_BAD_FILE


def test_binding_refuses_bad_arguments_before_launch(ctx, idx128):
    # host tensors, wrong dtypes, wrong query width, short result buffers and
    # short per-query lists are refused in Python; the context stays usable
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    n, d = qd.shape
    with pytest.raises(ValueError, match="CUDA tensor"):
        ctx.search(torch.from_numpy(q), 10, 64)
    with pytest.raises(TypeError, match="dtype"):
        ctx.search(qd.double(), 10, 64)
    with pytest.raises(ValueError, match="columns"):
        ctx.search(qd[:, : d - 1].contiguous(), 10, 64)
    with pytest.raises(ValueError, match="contiguous"):
        ctx.search(torch.zeros((d, n), device="cuda").t(), 10, 64)
    with pytest.raises(ValueError, match="shape"):
        ctx.search(qd, 10, 64, torch.empty((n, 5), dtype=torch.int64, device="cuda"),
                   torch.empty((n, 5), device="cuda"))
    with pytest.raises(ValueError, match="host"):
        ctx.search_host(qd, 10, 64)
    with pytest.raises(ValueError, match="entries"):
        ctx.search_mixed(qd, np.full(n - 1, 10, np.int32), np.full(n, 64, np.int32))
    with pytest.raises(ValueError, match="columns"):
        ctx.knn(qd, qd[:, :8].contiguous(), 5)
    with pytest.raises(ValueError, match="CUDA tensor"):
        ctx.quantize(torch.from_numpy(x), torch.zeros(d, device="cuda"),
                     torch.ones(d, device="cuda"))
    ids, dd = ctx.search(qd, 10, 64)  # still usable
    assert ids.shape == (n, 10)


def test_no_index_is_an_error():
    from paper_2602_21600_gb300 import Context
    from paper_2602_21600_gb300.aqr import AQR_ERR_NO_INDEX, AqrError
    c = Context(0)
    with pytest.raises(AqrError) as ei:
        c.search(torch.zeros((1, 8), device="cuda"), 1, 1)
    assert ei.value.status == AQR_ERR_NO_INDEX
    c.close()


def test_kernel_configs_do_not_change_results(ctx, idx128):
    # hash size, neighbour tile and lanes per candidate change speed only
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    ref_i, ref_d = ctx.search(qd, 10, 100)
    ref_i, ref_d = ref_i.cpu().numpy(), ref_d.cpu().numpy()
    # hash: 16-bit quotient tags and 32-bit ids, from 32 sets (heavy
    # forgetting) to more sets than the search visits
    for hs in (64, 384, 512, 8192):
        for tile in (1, 7, 32):
            for team in (1, 2):
                for tag in (16, 32):
                    ctx.set_kernel_config(100, 10, hash_slots=hs, tile_rows=tile, team_lanes=team,
                                          hash_tag_bits=tag, warps_per_query=1)
                    ids, dd = ctx.search(qd, 10, 100)
                    np.testing.assert_array_equal(ids.cpu().numpy(), ref_i)
                    np.testing.assert_array_equal(dd.cpu().numpy(), ref_d)
    # blocks of 11 warps (56 registers, three blocks per SM): the tile that
    # fits, and explicit tiles
    for hs in (0, 64, 1024):
        for tile in (0, 1, 13, 32):
            ctx.set_kernel_config(100, 10, hash_slots=hs, tile_rows=tile, team_lanes=1,
                                  warps_per_block=11, warps_per_query=1)
            ids, dd = ctx.search(qd, 10, 100)
            np.testing.assert_array_equal(ids.cpu().numpy(), ref_i)
            np.testing.assert_array_equal(dd.cpu().numpy(), ref_d)
    chosen = ctx.autotune(qd, 10, 100)
    assert chosen["team_lanes"] in (1, 2) and chosen["warps_per_block"] in (0, 4, 11)
    ids, dd = ctx.search(qd, 10, 100)
    np.testing.assert_array_equal(ids.cpu().numpy(), ref_i)
    ctx.set_kernel_config(100, 10)


def _recall(ids, gt, k):
    return float(np.mean([len(set(a[:k].tolist()) & set(b[:k].tolist())) / k
                          for a, b in zip(ids, gt)]))


def test_autotune_recall_picks_a_setting_that_reaches_the_target(ctx, idx128):
    # the library's autotuner of shortlist policy, ef and kernel: its sweep
    # recalls are those of plain searches with the same settings, the winner
    # reaches the target and is left set on the context
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    gt, _ = oracle.bruteforce(x, q, 12)
    efs = [10, 16, 24, 32, 64, 128]
    r = ctx.autotune_recall(qd, 10, gt, 0.95, efs)
    assert r["reached"] and r["recall"] >= 0.95 and r["ef"] in efs and r["ms"] > 0
    assert (r["m_ef"], r["rerank_pct"]) in [(3, 40), (3, 100), (2, 40), (2, 100), (1, 40),
                                            (1, 100)]
    ids, _ = ctx.search(qd, 10, r["ef"])  # the context is left at the winner
    assert abs(_recall(ids.cpu().numpy(), gt, 10) - r["recall"]) < 1e-12
    for row in r["sweep"][:4]:
        ctx.set_params(m_ef=row["m_ef"], rerank_pct=row["rerank_pct"])
        ids, _ = ctx.search(qd, 10, row["ef"])
        assert abs(_recall(ids.cpu().numpy(), gt, 10) - row["recall"]) < 1e-5
    # a target nobody reaches: the best recall found, reached = False
    ctx.set_params()
    r2 = ctx.autotune_recall(qd, 10, gt, 1.0, [10, 12])
    best = max(row["recall"] for row in r2["sweep"])
    assert not r2["reached"] or r2["recall"] == 1.0
    if not r2["reached"]:
        assert abs(r2["recall"] - best) < 1e-5  # the sweep table is rounded to 5 digits
    from paper_2602_21600_gb300.aqr import AqrError
    with pytest.raises(AqrError):
        ctx.autotune_recall(qd, 10, gt, 0.9, [64, 32])  # not ascending
    ctx.set_params()
    for ef in efs:
        ctx.set_kernel_config(ef, 10)


# --- the other workload shapes at sizes the oracle finishes in seconds -------

@pytest.fixture(scope="module")
def idx_wide():
    # GIST-like: 960 dimensions, cluster spreads 100x apart (team path, two
    # 16-byte chunks per lane, 960-float rows)
    return _make("gmm1m_d960_spread", 1200, 16, M0=8, ef0=40)


@pytest.fixture(scope="module")
def idx_sphere768():
    # unit-norm embeddings, 768 dimensions (team path, 48 chunks)
    return _make("sphere1m_d768", 1500, 24, M0=8, ef0=40)


@pytest.fixture(scope="module")
def idx_sphere96():
    # unit-norm, 96 dimensions: 6 chunks per code row (lane path, odd stride)
    return _make("sphere10m_d96", 3000, 40, M0=8, ef0=60)


@pytest.mark.parametrize("k,ef", [(100, 256), (10, 64)])
def test_search_parity_wide_d960(ctx, idx_wide, k, ef):
    w, x, q, idx = idx_wide
    _load(ctx, idx)
    _run_parity(ctx, idx, q, k, ef)


@pytest.mark.parametrize("k,ef", [(10, 128), (1, 32), (100, 512)])
def test_search_parity_sphere_d768(ctx, idx_sphere768, k, ef):
    w, x, q, idx = idx_sphere768
    _load(ctx, idx)
    _run_parity(ctx, idx, q, k, ef)


@pytest.mark.parametrize("k,ef", [(10, 64), (10, 16), (20, 200)])
def test_search_parity_sphere_d96(ctx, idx_sphere96, k, ef):
    w, x, q, idx = idx_sphere96
    _load(ctx, idx)
    _run_parity(ctx, idx, q, k, ef)


@pytest.fixture(scope="module")
def idx_d256():
    # 256 dimensions: 16 chunks per code row, the widest rows of the lane
    # path (swizzled tile, copy loop instantiated for 16 chunks)
    return _make("sphere1m_d768", 2000, 32, M0=8, ef0=40, d=256)


@pytest.fixture(scope="module")
def idx_d200():
    # 200 dimensions: 208-byte code rows, 13 chunks (odd stride, generic copy loop)
    return _make("sphere1m_d768", 2000, 32, M0=8, ef0=40, d=200)


@pytest.mark.parametrize("which", ["idx_d256", "idx_d200"])
@pytest.mark.parametrize("k,ef", [(10, 64), (5, 200)])
def test_search_parity_lane_path_wide_rows(ctx, request, which, k, ef):
    w, x, q, idx = request.getfixturevalue(which)
    _load(ctx, idx)
    _run_parity(ctx, idx, q, k, ef)
    # tiles of 1, 7 and 32 rows and both lane modes give the same bits
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    ref_i, ref_d = ctx.search(qd, k, ef)
    for tile in (1, 7, 32):
        for team in (1, 2):
            ctx.set_kernel_config(ef, k, tile_rows=tile, team_lanes=team, warps_per_query=1)
            ids, dd = ctx.search(qd, k, ef)
            np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
            np.testing.assert_array_equal(dd.cpu().numpy(), ref_d.cpu().numpy())
    ctx.set_kernel_config(ef, k)


# --- several warps per query ----------------------------------------------

@pytest.mark.parametrize("G", [2, 4])
@pytest.mark.parametrize("which,k,ef", [("idx128", 10, 64), ("idx128", 32, 200),
                                        ("idx128", 5, 1000), ("idx128", 1, 1),
                                        ("idx37", 7, 130), ("idx_wide", 100, 256),
                                        ("idx_sphere96", 10, 16), ("idx_d200", 5, 200),
                                        ("idx_d256", 10, 64)])
def test_group_search_parity(ctx, request, G, which, k, ef):
    # a group of G warps per query: the same expansion sequence, C and stage
    # values as the oracle, and bit for bit the results of one warp per query
    w, x, q, idx = request.getfixturevalue(which)
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    ctx.set_kernel_config(ef, k, warps_per_query=1)  # one warp per query, forced
    ref_i, ref_d = ctx.search(qd, k, ef)
    st1 = ctx.stats()
    _run_parity(ctx, idx, q, k, ef)
    ctx.set_kernel_config(ef, k, warps_per_query=G)
    try:
        ids, dd = ctx.search(qd, k, ef)
        stG = ctx.stats()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
        np.testing.assert_array_equal(dd.cpu().numpy(), ref_d.cpu().numpy())
        # the group expands the same nodes; only hash re-evaluations may differ
        assert stG["expansions"] == st1["expansions"]
        assert stG["queries"] == st1["queries"] == len(q)
        _run_parity(ctx, idx, q, k, ef)
        # hash and tile extremes inside the group form
        for hs, tile in ((64, 1), (8192, 32), (512, 7)):
            ctx.set_kernel_config(ef, k, hash_slots=hs, tile_rows=tile, warps_per_query=G)
            ids, dd = ctx.search(qd, k, ef)
            np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
            np.testing.assert_array_equal(dd.cpu().numpy(), ref_d.cpu().numpy())
    finally:
        ctx.set_kernel_config(ef, k)


def test_group_mixed_batch_and_odd_batch_sizes(ctx, idx128):
    # mixed ef classes with groups of 2 and 4 in one CUDA graph, and batches
    # that do not fill the last group of a block
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    rng = np.random.default_rng(4)
    ks = rng.choice([1, 10, 33], len(q)).astype(np.int32)
    efs = rng.choice([16, 64, 200, 700], len(q)).astype(np.int32)
    for ef in (64, 200, 700, 16):
        ctx.set_kernel_config(ef, 1, warps_per_query=1)
    ref = [t.cpu().numpy() for t in ctx.search_mixed(qd, ks, efs, k_stride=40)]
    for ef, G in ((64, 2), (200, 4), (700, 2), (16, 4)):
        ctx.set_kernel_config(ef, 1, warps_per_query=G)
    try:
        got = [t.cpu().numpy() for t in ctx.search_mixed(qd, ks, efs, k_stride=40)]
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)
        for n in (1, 3, 5, 7):
            r_i, r_d = ctx.search(qd[:n], 10, 200)
            ctx.set_kernel_config(200, 10, warps_per_query=1)
            u_i, u_d = ctx.search(qd[:n], 10, 200)
            ctx.set_kernel_config(200, 10, warps_per_query=4)
            np.testing.assert_array_equal(r_i.cpu().numpy(), u_i.cpu().numpy())
            np.testing.assert_array_equal(r_d.cpu().numpy(), u_d.cpu().numpy())
    finally:
        for ef in (64, 200, 700, 16):
            ctx.set_kernel_config(ef, 1)


def test_mixed_graph_follows_parameters_and_index(ctx, idx128):
    # the cached launch graph of a mixed batch is replayed only while the
    # index, the search parameters and the kernel configurations are those
    # it was captured with
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    qd = torch.from_numpy(q).cuda()
    n = len(q)
    ks = np.array([1, 10, 5, 10] * n, np.int32)[:n]
    efs = np.array([16, 64, 128, 300] * n, np.int32)[:n]
    ids = torch.empty((n, 10), dtype=torch.int64, device="cuda")
    dd = torch.empty((n, 10), device="cuda")

    def check():
        ctx.search_mixed(qd, ks, efs, k_stride=10, ids=ids, dists=dd)  # same buffers
        torch.cuda.synchronize()
        for i in range(n):
            ui, ud = ctx.search(qd[i:i + 1], int(ks[i]), int(efs[i]))
            np.testing.assert_array_equal(ids.cpu().numpy()[i, : ks[i]], ui.cpu().numpy()[0])
            np.testing.assert_array_equal(dd.cpu().numpy()[i, : ks[i]], ud.cpu().numpy()[0])

    check()
    ctx.set_params(m_ef=1, rerank_pct=100)  # other parameters
    check()
    ctx.set_kernel_config(64, 10, hash_slots=256, tile_rows=7)  # other configuration
    check()
    ctx.set_kernel_config(64, 10)
    # another index of the same width: the replay must not use the old one
    _, _, _, idx_b = _make("gmm10k_d128", 2500, 8, M0=6, ef0=40)
    _load(ctx, idx_b)
    check()
    _load(ctx, idx)
    ctx.set_params()


def test_searches_on_two_streams_may_overlap(ctx, idx128):
    # each launch has its own work counter: two searches of one context in
    # flight on different streams each answer all of their queries
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.set_params()
    q1 = torch.from_numpy(q[:24]).cuda()
    q2 = torch.from_numpy(q[24:]).cuda()
    r1 = [t.cpu().numpy() for t in ctx.search(q1, 10, 200)]
    r2 = [t.cpu().numpy() for t in ctx.search(q2, 10, 64)]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        o1 = ctx.search(q1, 10, 200, stream=s1)
        o2 = ctx.search(q2, 10, 64, stream=s2)
        torch.cuda.synchronize()
        for got, ref in ((o1, r1), (o2, r2)):
            np.testing.assert_array_equal(got[0].cpu().numpy(), ref[0])
            np.testing.assert_array_equal(got[1].cpu().numpy(), ref[1])


def test_host_path_follows_index_width(ctx, idx37, idx128):
    # the host path's device buffers are sized for the index's d: after an
    # index of another width they are sized again, not overrun
    for w, x, q, idx in (idx37, idx128, idx37):
        _load(ctx, idx)
        ctx.set_params()
        ih, dh = ctx.search_host(torch.from_numpy(q[:16]).contiguous(), 10, 64)
        di, dd = ctx.search(torch.from_numpy(q[:16]).cuda(), 10, 64)
        np.testing.assert_array_equal(ih.numpy(), di.cpu().numpy())
        np.testing.assert_array_equal(dh.numpy(), dd.cpu().numpy())


def test_index_replacement_refused_while_serving(ctx, idx128):
    from paper_2602_21600_gb300.aqr import AQR_ERR_BUSY, AqrError
    w, x, q, idx = idx128
    _load(ctx, idx)
    ctx.serve_start(max_batch=8, n_streams=1)
    try:
        with pytest.raises(AqrError) as ei:
            _load(ctx, idx)
        assert ei.value.status == AQR_ERR_BUSY
        with pytest.raises(AqrError) as ei:
            ctx.build_graph(torch.from_numpy(x).cuda(), np.zeros(x.shape[1], np.float32),
                            np.ones(x.shape[1], np.float32), w["U"][: len(x)], 8, 40)
        assert ei.value.status == AQR_ERR_BUSY
        # parameters may change while serving; results stay those of a search
        ctx.set_params(m_ef=2)
        t = ctx.submit(q[0], 10, 64)
        got = ctx.poll(t, 10, timeout_us=5_000_000)
        assert got is not None
        ui, ud = ctx.search(torch.from_numpy(q[:1]).cuda(), 10, 64)
        np.testing.assert_array_equal(got[0], ui.cpu().numpy()[0])
    finally:
        ctx.serve_stop()
    _load(ctx, idx)  # allowed again
    ctx.set_params()


def test_mixed_batch_wide_rows(ctx, idx_wide):
    w, x, q, idx = idx_wide
    _load(ctx, idx)
    ctx.set_params()
    ks = np.array([1, 10, 100, 10] * 4, np.int32)[: len(q)]
    efs = np.array([32, 128, 256, 600] * 4, np.int32)[: len(q)]
    qd = torch.from_numpy(q).cuda()
    ids, dd = ctx.search_mixed(qd, ks, efs, k_stride=100)
    for i in range(len(q)):
        ui, ud = ctx.search(qd[i:i + 1], int(ks[i]), int(efs[i]))
        np.testing.assert_array_equal(ids.cpu().numpy()[i, : ks[i]], ui.cpu().numpy()[0])
        np.testing.assert_array_equal(dd.cpu().numpy()[i, : ks[i]], ud.cpu().numpy()[0])


@pytest.mark.parametrize("name,n,d,M0,ef0,sched", [
    ("gmm1m_d960_spread", 700, 960, 8, 30, oracle.BATCHED),
    ("sphere10m_d96", 2000, 96, 8, 40, oracle.BATCHED),
    ("gmm1m_d960_spread", 400, 960, 8, 30, oracle.SEQUENTIAL),
    ("sphere10m_d96", 600, 96, 8, 40, oracle.SEQUENTIAL)])
def test_gpu_build_matches_oracle_other_shapes(ctx, name, n, d, M0, ef0, sched):
    # both sides run the same insertion schedule: the GPU builder's batched
    # reading, or the sequential insertion of Alg. 1
    w = synth.workload(name, n=n, nq=1)
    x = w["x"]
    P = oracle.train(x, M0=M0, ef0=ef0)
    codes = oracle.encode(x, P["min"], P["scale"])
    lv = oracle.levels(w["U"], P["M_i"])
    g_o = oracle.build_graph(codes, lv, P["M_i"], P["ef_c"], *sched)
    ctx.build_graph(torch.from_numpy(x).cuda(), P["min"], P["scale"], w["U"], P["M_i"], P["ef_c"],
                    *sched)
    g_g = ctx.export_graph()
    np.testing.assert_array_equal(g_g["codes"], codes)
    assert g_g["entry"] == g_o["entry"] and g_g["max_level"] == g_o["max_level"]
    np.testing.assert_array_equal(g_g["adj0"], g_o["adj0"])
    np.testing.assert_array_equal(g_g["upper"], g_o["upper"])
