"""The two further dataset shapes of Table 1, as synthetic stand-ins:
60,000 x 784 8-bit images with blank background (Fashion-MNIST shape) and
100,000 x 300 signed embeddings (GloVe-300D shape), 10,000 queries each
(the query counts of Section 4.5, Figure 4).  Both take the team path of the
query kernel (code rows wider than 256 bytes).

Per workload: GPU training against the oracle's FP64 training (equal up to
FP32 rounding of the density sums: squared distances of 784 pixels exceed
2^24); with the oracle's parameters, GPU codes equal the oracle's encode;
the GPU builds the graph, and the oracle searches that graph (exported) for
sampled queries: expansion sequence and C bit for bit, Stages 2-3 within the
tolerance; recall@10 against the oracle's brute force.
"""

import numpy as np
import pytest

import oracle
import synth
from parity import check_stage1, check_stages_2_3, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 10


@pytest.fixture(scope="module", params=[("pix60k_d784_int", 64), ("emb100k_d300", 96)],
                ids=lambda p: p[0])
def built(request):
    from paper_2602_21600_gb300 import Context
    name, ef = request.param
    w = synth.workload(name)
    ctx = Context(0)
    xd = torch.from_numpy(w["x"]).cuda()
    P_g = ctx.train(xd, w["sample"], M0=w["M0"], ef0=w["ef0"])
    P_o = oracle.train(w["x"], w["sample"], M0=w["M0"], ef0=w["ef0"])
    ctx.build_graph(xd, P_o["min"], P_o["scale"], w["U"], P_o["M_i"], P_o["ef_c"],
                    s_dist=P_o["s_dist"])
    del xd
    yield w, ef, ctx, P_g, P_o
    ctx.close()


def test_training_within_fp32_rounding(built):
    w, ef, ctx, P_g, P_o = built
    assert P_g["delta"] == pytest.approx(P_o["delta"], rel=1e-4)
    np.testing.assert_allclose(P_g["min"], P_o["min"], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(P_g["scale"], P_o["scale"], rtol=1e-4)
    assert P_g["M_i"] == P_o["M_i"] and P_g["ef_c"] == P_o["ef_c"]


def test_codes_and_graph_invariants(built):
    w, ef, ctx, P_g, P_o = built
    g = ctx.export_graph()
    rows = np.random.default_rng(1).choice(w["n"], 3000, replace=False)
    np.testing.assert_array_equal(g["codes"][rows],
                                  oracle.encode(w["x"][rows], P_o["min"], P_o["scale"]))
    adj = g["adj0"].astype(np.int64)
    valid = adj != np.int64(oracle.NONE)
    assert np.all(valid[:, :-1] | ~valid[:, 1:]) and np.all(adj[valid] < w["n"])
    assert not np.any(adj == np.arange(w["n"])[:, None])
    assert np.all(valid.sum(1) >= 1)


def test_oracle_search_of_the_gpu_graph(built):
    w, ef, ctx, P_g, P_o = built
    ctx.set_params()
    qd = torch.from_numpy(w["q"]).cuda()
    t = to_np(ctx.search_trace(qd, K, ef, cap_exp=2048))
    torch.cuda.synchronize()
    idx = dict(P_o)
    idx.update(ctx.export_graph())
    idx["x"] = w["x"]
    S = np.sort(np.random.default_rng(4).choice(len(w["q"]), 150, replace=False))
    o = oracle.search(idx, w["q"][S], k=K, ef=ef, trace=True, cap_exp=2048)
    g = {key: v[S] for key, v in t.items()}
    check_stage1(g, o, len(S))
    amb = check_stages_2_3(idx, w["q"][S], g, o, K, ef)
    assert amb["et"] <= len(S) // 8 and amb["final"] <= len(S) // 4
    gt, _ = oracle.bruteforce(w["x"], w["q"][S], K)
    hits = sum(len(set(g["ids"][i].tolist()) & set(gt[i].tolist())) for i in range(len(S)))
    recall = hits / (K * len(S))
    print(f"{w['name']}: recall@10 {recall:.3f} at ef {ef}")
    assert recall >= 0.85
