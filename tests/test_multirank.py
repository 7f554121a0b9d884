"""The benchmark's multi-process path on CPU ranks (gloo, world size 2): the
job time is the slowest rank's, the job throughput counts every rank's
queries, and every rank draws its own query batch (weak scaling with
replicated index)."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    import bench
    import synth
    ms = bench.max_over_ranks(1.0 + rank, "cpu")  # rank r took 1 + r ms
    w = synth.workload("gmm10k_d128", n=64, nq=8, seed_query=4321 + rank)
    out[rank] = (ms, bench.job_qps(1000, world, ms), float(w["q"].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
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
    for r in range(world):
        ms, qps, qsum = res[r]
        assert ms == 2.0                      # the slowest rank
        assert qps == pytest.approx(2 * 1000 / 2e-3)
    assert res[0][2] != res[1][2]             # each rank has its own queries


def test_single_process_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_qps(10_000, 1, 2.0) == pytest.approx(5e6)


def test_traffic_record_matches_only_its_launch(tmp_path, monkeypatch):
    # roofline.traffic comes from the committed ncu record only for the
    # launch it was taken on and while the kernel sources hash to it
    import json
    import sys
    import types
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(traffic=None)
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "search_kernel_traffic.json")))
    launch = dict(rec["launch"])
    kcs = launch.pop("kernel_configs")
    assert len(kcs) >= 1
    for kc in kcs:  # every listed equivalent configuration matches
        got = bench.kernel_traffic(args, dict(launch, kernel_config=kc))
        assert got in (rec["dram_bytes_per_launch"], None)  # None once the sources change
    launch["kernel_config"] = kcs[0]
    for key, other in (("workload", "gmm1m_d960_spread"), ("queries", 1000), ("ef", 1024),
                       ("m_ef", 3), ("kernel_config", {"hash_slots": 512, "tile_rows": 24,
                                                        "team_lanes": 1, "hash_tag_bits": 0})):
        assert bench.kernel_traffic(args, dict(launch, **{key: other})) is None
    # a record whose source hash no longer matches gives None
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    for f in rec["kernel_sources"]:
        (root / f).parent.mkdir(parents=True, exist_ok=True)
        (root / f).write_text("changed")
    (root / "profiles" / "search_kernel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic(args, launch) is None
    # an explicit --traffic wins
    assert bench.kernel_traffic(types.SimpleNamespace(traffic=123), launch) == 123
