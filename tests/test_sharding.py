"""Database sharding on CPU: the oracle's top-k merge, pinned against the
brute force it must reproduce (the union of exact per-shard top-k lists
holds the global top-k), the shard split, and the exchange step between
gloo ranks (world size 2) feeding that merge."""

import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shard_lists(x, q, k, world):
    from paper_2602_21600_gb300.shard import shard_range
    ids, dd = [], []
    for r in range(world):
        lo, hi = shard_range(len(x), r, world)
        i, d = oracle.bruteforce(x[lo:hi], q, k)
        ids.append(i)
        dd.append(d.astype(np.float32))
    return np.stack(ids), np.stack(dd)


def test_shard_ranges_cover_the_set():
    from paper_2602_21600_gb300.shard import shard_offsets, shard_range
    for n, world in [(10, 3), (7, 7), (5, 8), (1000, 4)]:
        got = [shard_range(n, r, world) for r in range(world)]
        assert got[0][0] == 0 and got[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
        assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1
        assert shard_offsets(n, world) == [l for l, _ in got]
    with pytest.raises(ValueError):
        shard_range(10, 3, 3)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_merge_of_exact_shard_lists_is_global_bruteforce(world):
    from paper_2602_21600_gb300.shard import shard_offsets
    w = synth.workload("gmm10k_d128", n=3000, nq=40)
    x, q, k = w["x"], w["q"], 10
    ids, dd = _shard_lists(x, q, k, world)
    mi, md = oracle.merge_topk(dd, ids, shard_offsets(len(x), world))
    gi, gd = oracle.bruteforce(x, q, k)
    np.testing.assert_array_equal(mi, gi)
    np.testing.assert_array_equal(md, gd.astype(np.float32).astype(np.float64))


def test_merge_pads_and_breaks_ties_by_global_id():
    # shard 1 holds 2 points (k = 4 pads it); shard 0 and 1 share a point
    x0 = np.array([[0.0, 0.0], [3.0, 0.0], [5.0, 0.0]], np.float32)
    x1 = np.array([[1.0, 0.0], [5.0, 0.0]], np.float32)
    q = np.array([[4.0, 0.0]], np.float32)
    i0, d0 = oracle.bruteforce(x0, q, 4)
    i1, d1 = oracle.bruteforce(x1, q, 4)
    assert i1[0, 2] == -1 and i0[0, 3] == -1
    mi, md = oracle.merge_topk(np.stack([d0, d1]), np.stack([i0, i1]), [0, 3], k=4)
    # distances: id 1 (x=3): 1, id 2 (x=5): 1, id 4 (x=5): 1, then id 3 (x=1): 9
    assert mi[0].tolist() == [1, 2, 4, 3]
    assert md[0].tolist() == [1.0, 1.0, 1.0, 9.0]
    mi, md = oracle.merge_topk(np.stack([d0, d1]), np.stack([i0, i1]), [0, 3], k=7)
    assert mi[0].tolist() == [1, 2, 4, 3, 0, -1, -1] and np.isinf(md[0, 5:]).all()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2602_21600_gb300.shard import gather_lists, shard_offsets, shard_range
    w = synth.workload("gmm10k_d128", n=2000, nq=16)
    lo, hi = shard_range(len(w["x"]), rank, world)
    i, d = oracle.bruteforce(w["x"][lo:hi], w["q"], 10)
    gi, gd = gather_lists(torch.from_numpy(i), torch.from_numpy(d.astype(np.float32)))
    mi, md = oracle.merge_topk(gd.numpy(), gi.numpy(), shard_offsets(len(w["x"]), world))
    out[rank] = (tuple(gi.shape), mi.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_between_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        [p.start() for p in procs]
        [p.join(120) for p in procs]
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    w = synth.workload("gmm10k_d128", n=2000, nq=16)
    gt, _ = oracle.bruteforce(w["x"], w["q"], 10)
    for r in range(world):
        shape, merged = res[r]
        assert shape == (2, 16, 10)
        np.testing.assert_array_equal(np.array(merged), gt)
