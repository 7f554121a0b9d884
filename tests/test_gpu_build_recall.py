"""Recall contract of the batched GPU graph build against Alg. 1.

Alg. 1 inserts the nodes one at a time, each searching the graph of all
earlier nodes.  The GPU builder's default is the batched reading (node 0
alone, then batches of min(max(1, s / 32), 16384) nodes that search the
graph as it stood before their batch), which is not bit-identical to the
sequential insertion.  The contract: on the same data, quantiser and level
draws, the batched graph's recall@k at equal ef is at least the sequential
graph's minus DELTA, at every ef of the sweep.  The sequential graph is
built by the same GPU builder with batch size 1, which is bit-identical to
the oracle's sequential insertion (test_gpu_build_matches_oracle).

DELTA = 0.005 (half a percentage point of recall@k): with 1,000 queries,
recall@10 is a mean over 10,000 hits, whose sampling error is about 0.001,
and the batched schedule hides at most 1/32 of the graph from a node.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DELTA = 0.005


def _recall(ids, gt, k):
    return float(np.mean([len(set(a[:k].tolist()) & set(b[:k].tolist())) / k
                          for a, b in zip(ids, gt)]))


@pytest.mark.parametrize("name,n,k,efs", [
    ("gmm1m_d128_int", 100_000, 10, [16, 32, 64, 128]),     # the metric's law, M0 16
    ("gmm1m_d960_spread", 50_000, 100, [128, 256, 1024]),   # 100x spread, M0 32
])
def test_batched_build_recall_within_delta_of_sequential(name, n, k, efs):
    from paper_2602_21600_gb300 import Context
    ctx = Context(0)
    w = synth.workload(name, n=n, nq=1000)
    xd = torch.from_numpy(w["x"]).cuda()
    qd = torch.from_numpy(w["q"]).cuda()
    P = ctx.train(xd, w["sample"] if n > 10000 else None, M0=w["M0"], ef0=w["ef0"])
    gt, _ = ctx.knn(xd, qd, k)
    gt = gt.cpu().numpy()
    ctx.set_params(m_ef=1, rerank_pct=100)
    rec = {}
    for label, sched in [("batched", (32, 16384)), ("sequential", (1, 1))]:
        ctx.build_graph(xd, P["min"], P["scale"], w["U"], P["M_i"], P["ef_c"], *sched)
        rec[label] = [_recall(ctx.search(qd, k, ef)[0].cpu().numpy(), gt, k) for ef in efs]
    ctx.close()
    for ef, rb, rs in zip(efs, rec["batched"], rec["sequential"]):
        assert rb >= rs - DELTA, (name, ef, rb, rs)
