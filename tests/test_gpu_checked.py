"""The bounds-checked build (libaqr_checked.so, compiled with -DAQR_CHECKED).

Every shared-memory index of the layer search (result set W, candidate and
survivor lists, visited-hash sets, the sort range of Stages 2-3) is checked
before use; a violation would record its source line in the context's error
word and skip the access.  On the parity workloads -- one lane per candidate,
team evaluators for wide rows, the plain path, mixed ef, kernel
configurations from a heavily forgetting hash to a large one, and the GPU
graph build -- the checked build must report no violation and return
exactly what the normal build returns.
"""

import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _make(name, n, nq, M0, ef0, d=None):
    w = synth.workload(name, n=n, nq=nq)
    x, q = w["x"], w["q"]
    if d is not None:
        x, q = x[:, :d].copy(), q[:, :d].copy()
    P = oracle.train(x, None, M0=M0, ef0=ef0)
    idx = oracle.make_index(x, w["U"], None, params=P)
    return w, x, q, idx


@pytest.fixture(scope="module")
def pair():
    from paper_2602_21600_gb300 import Context
    cn, cc = Context(0), Context(0, checked=True)
    yield cn, cc
    cn.close()
    cc.close()


def _load_both(pair, idx):
    with tempfile.TemporaryDirectory() as td:
        p = os.path.join(td, "i.aqr")
        oracle.write_index(p, idx)
        for c in pair:
            c.load_graph(p)


def _same(pair, fn):
    outs = []
    for c in pair:
        r = fn(c)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in r])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)
    assert pair[1].stats()["device_errors"] == 0


@pytest.mark.parametrize("case", ["d128", "d37", "d960", "d96"])
def test_checked_build_matches_and_stays_in_bounds(pair, case):
    name, n, nq, M0, ef0, d = {"d128": ("gmm10k_d128", 3000, 48, 8, 60, None),
                               "d37": ("gmm10k_d128", 1500, 32, 6, 40, 37),
                               "d960": ("gmm1m_d960_spread", 1200, 16, 8, 40, None),
                               "d96": ("sphere10m_d96", 3000, 40, 8, 60, None)}[case]
    w, x, q, idx = _make(name, n, nq, M0, ef0, d)
    _load_both(pair, idx)
    qd = torch.from_numpy(q).cuda()
    for c in pair:
        c.set_params()
    for k, ef in ((10, 16), (10, 100), (32, 200), (5, 1000), (1, 1)):
        _same(pair, lambda c: c.search(qd, k, ef))
        _same(pair, lambda c: c.search_plain(qd, k, ef))
    # kernel configurations: a hash of 32 sets (heavy forgetting) to one
    # larger than the search visits, narrow and full tiles, both evaluators
    for hs, tile, team in ((64, 1, 1), (64, 7, 2), (8192, 32, 1), (512, 32, 2)):
        for c in pair:
            c.set_kernel_config(100, 10, hash_slots=hs, tile_rows=tile, team_lanes=team,
                                warps_per_query=1)
        _same(pair, lambda c: c.search(qd, 10, 100))
    # blocks of 11 warps, and two or four warps per query (group form)
    for hs, tile, wpb, g in ((0, 0, 11, 1), (64, 1, 11, 1), (0, 0, 0, 2), (64, 7, 0, 4),
                             (8192, 32, 0, 2)):
        for c in pair:
            c.set_kernel_config(100, 10, hash_slots=hs, tile_rows=tile, team_lanes=1,
                                warps_per_block=wpb, warps_per_query=g)
        _same(pair, lambda c: c.search(qd, 10, 100))
        for c in pair:
            c.set_kernel_config(1000, 5, hash_slots=hs, tile_rows=tile, warps_per_query=g)
        _same(pair, lambda c: c.search(qd, 5, 1000))
    for c in pair:
        c.set_kernel_config(100, 10)
        c.set_kernel_config(1000, 5)
    rng = np.random.default_rng(3)
    ks = rng.choice([1, 10, 33], len(q)).astype(np.int32)
    efs = rng.choice([16, 64, 200, 700], len(q)).astype(np.int32)
    _same(pair, lambda c: c.search_mixed(qd, ks, efs))


def test_checked_gpu_build(pair):
    w = synth.workload("gmm10k_d128", n=2500, nq=1)
    x = w["x"]
    P = oracle.train(x, M0=8, ef0=60)
    graphs = []
    for c in pair:
        c.build_graph(torch.from_numpy(x).cuda(), P["min"], P["scale"], w["U"], P["M_i"],
                      P["ef_c"], 32, 16384)
        graphs.append(c.export_graph())
    for key in ("adj0", "upper_base", "upper", "codes"):
        np.testing.assert_array_equal(graphs[0][key], graphs[1][key])
    assert pair[1].stats()["device_errors"] == 0
