"""aqr_merge_topk against the oracle's merge (bit for bit: the merge only
selects and orders), on random shard lists with padding and cross-shard
distance ties, and on real shards: three contexts on one GPU, each holding
its own GPU-trained, GPU-built index over one third of the base set."""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _random_lists(rng, S, n, k):
    ids = np.full((S, n, k), -1, np.int64)
    dd = np.full((S, n, k), np.inf, np.float32)
    for s in range(S):
        for q in range(n):
            m = int(rng.integers(0, k + 1))          # valid entries, padding after them
            d = rng.choice(np.arange(8, dtype=np.float32), m)  # few values: many ties
            i = rng.choice(5000, m, replace=False)
            o = np.lexsort((i, d))
            ids[s, q, :m] = i[o]
            dd[s, q, :m] = d[o]
    return ids, dd


@pytest.mark.parametrize("S,k", [(1, 10), (2, 1), (5, 10), (32, 100), (3, 1024)])
def test_merge_equals_oracle_on_random_lists(S, k):
    from paper_2602_21600_gb300 import Context
    rng = np.random.default_rng(S * 1000 + k)
    n = 200 if k < 1000 else 20
    ids, dd = _random_lists(rng, S, n, k)
    off = np.cumsum(rng.integers(0, 2000, S)).astype(np.int64)
    ctx = Context(0)
    gi, gd = ctx.merge_topk(torch.from_numpy(dd).cuda(), torch.from_numpy(ids).cuda(), off)
    torch.cuda.synchronize()
    oi, od = oracle.merge_topk(dd, ids, off)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_array_equal(gd.cpu().numpy(), od.astype(np.float32))
    ctx.close()


def test_merge_rejects_bad_arguments():
    from paper_2602_21600_gb300 import Context
    from paper_2602_21600_gb300.aqr import AQR_ERR_INVALID_ARG, AqrError
    ctx = Context(0)
    for S in (33,):
        with pytest.raises(AqrError) as ei:
            ctx.merge_topk(torch.zeros((S, 4, 2), device="cuda"),
                           torch.zeros((S, 4, 2), dtype=torch.int64, device="cuda"))
        assert ei.value.status == AQR_ERR_INVALID_ARG
    with pytest.raises(AqrError) as ei:
        ctx.merge_topk(torch.zeros((2, 4, 2), device="cuda"),
                       torch.zeros((2, 4, 2), dtype=torch.int64, device="cuda"), [0, -5])
    assert ei.value.status == AQR_ERR_INVALID_ARG
    ctx.close()


def test_three_shards_on_one_gpu():
    from paper_2602_21600_gb300 import Context
    from paper_2602_21600_gb300.shard import shard_offsets, shard_range
    w = synth.workload("gmm10k_d128", nq=200)
    x, q, k, ef, S = w["x"], w["q"], 10, 64, 3
    qd = torch.from_numpy(q).cuda()
    ctxs, lists_i, lists_d = [], [], []
    for r in range(S):
        lo, hi = shard_range(len(x), r, S)
        ctx = Context(0)
        xd = torch.from_numpy(x[lo:hi]).cuda()
        P = ctx.train(xd, None, M0=w["M0"], ef0=w["ef0"])
        ctx.build_graph(xd, P["min"], P["scale"], w["U"][lo:hi], P["M_i"], P["ef_c"],
                        s_dist=P["s_dist"])
        ctx.set_params()
        i, d = ctx.search(qd, k, ef)
        ctxs.append(ctx)
        lists_i.append(i)
        lists_d.append(d)
    gi = torch.stack(lists_i)
    gd = torch.stack(lists_d)
    off = shard_offsets(len(x), S)
    mi, md = ctxs[0].merge_topk(gd, gi, off)
    torch.cuda.synchronize()
    oi, od = oracle.merge_topk(gd.cpu().numpy(), gi.cpu().numpy(), off)
    np.testing.assert_array_equal(mi.cpu().numpy(), oi)
    np.testing.assert_array_equal(md.cpu().numpy(), od.astype(np.float32))
    # the sharded search finds the global neighbours
    gt, _ = oracle.bruteforce(x, q, k)
    m = mi.cpu().numpy()
    hits = sum(len(set(m[j].tolist()) & set(gt[j].tolist())) for j in range(len(q)))
    assert hits / (k * len(q)) >= 0.9
    for c in ctxs:
        c.close()
