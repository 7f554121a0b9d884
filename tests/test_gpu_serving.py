"""Serving with continuous batching (aqr_serve_start / aqr_submit / aqr_poll).

Requests of mixed k and ef arrive while earlier micro-batches are on the
GPU; every result must be identical to the same query answered alone (a
single uniform aqr_search call), since no state crosses queries.
"""

import os
import tempfile
import threading
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    from paper_2602_21600_gb300 import Context
    w = synth.workload("gmm10k_d128", n=4000, nq=400)
    idx = oracle.make_index(w["x"], w["U"], None, M0=8, ef0=60)
    ctx = Context(0)
    with tempfile.TemporaryDirectory() as td:
        p = os.path.join(td, "s.aqr")
        oracle.write_index(p, idx)
        ctx.load_graph(p)
    yield ctx, w["q"]
    ctx.close()


def _alone(ctx, q, k, ef):
    ids, dd = ctx.search(torch.from_numpy(q[None]).cuda(), k, ef)
    return ids.cpu().numpy()[0], dd.cpu().numpy()[0]


def test_results_identical_alone_and_in_the_mix(served):
    ctx, q = served
    rng = np.random.default_rng(1)
    ks = rng.choice([1, 10, 100], len(q))
    efs = rng.choice([32, 128, 512], len(q))
    ctx.serve_start(max_batch=64, n_streams=4, batch_wait_us=20)
    tickets = []
    # three submitter threads with staggered arrivals
    lock = threading.Lock()

    def submitter(part):
        for i in part:
            t = ctx.submit(q[i], int(ks[i]), int(efs[i]))
            with lock:
                tickets.append((i, t))
            if i % 7 == 0:
                time.sleep(0.0005)

    parts = [range(j, len(q), 3) for j in range(3)]
    th = [threading.Thread(target=submitter, args=(p,)) for p in parts]
    [t.start() for t in th]
    [t.join() for t in th]
    res = {}
    batches = []
    for i, t in tickets:
        r = ctx.poll(t, int(ks[i]), timeout_us=10_000_000)
        assert r is not None, "request did not complete"
        res[i] = r
        batches.append(r[2]["batch_size"])
    ctx.serve_stop()
    assert len(res) == len(q)
    assert max(batches) > 1  # requests were batched together
    for i in range(len(q)):
        ids, dd = _alone(ctx, q[i], int(ks[i]), int(efs[i]))
        np.testing.assert_array_equal(res[i][0], ids)
        np.testing.assert_array_equal(res[i][1], dd)
        assert res[i][2]["latency_us"] >= res[i][2]["queue_us"] >= 0


def test_cancel_and_not_ready(served):
    ctx, q = served
    # a huge batching window keeps requests pending long enough to cancel
    ctx.serve_start(max_batch=4, n_streams=1, batch_wait_us=200_000)
    ts = [ctx.submit(q[i], 10, 512) for i in range(40)]
    cancelled = sum(1 for t in ts[::-1] if ctx.cancel(t) == 0)
    assert cancelled >= 1
    done = 0
    for t in ts:
        try:
            r = ctx.poll(t, 10, timeout_us=20_000_000)
            done += r is not None
        except Exception:
            pass  # cancelled tickets are unknown now
    ctx.serve_stop()
    assert done + cancelled == len(ts)


def test_admission_refuses_what_can_never_fit(served):
    from paper_2602_21600_gb300.aqr import AQR_ERR_NO_MEMORY, AqrError
    ctx, q = served
    ctx.serve_start(max_batch=8, n_streams=2, hbm_budget=4096)
    with pytest.raises(AqrError) as ei:
        ctx.submit(q[0], 10, 1000)
    assert ei.value.status == AQR_ERR_NO_MEMORY
    ctx.serve_stop()


def test_budget_limits_work_in_flight(served):
    # a budget of two requests: everything still completes, two at a time
    ctx, q = served
    from paper_2602_21600_gb300 import aqr as A
    one = 128 * 4 + 128 + 128 * 12 + 64 * 8 + 1024 * 4
    ctx.serve_start(max_batch=64, n_streams=4, hbm_budget=2 * one, batch_wait_us=0)
    ts = [ctx.submit(q[i], 10, 32) for i in range(30)]
    out = [ctx.poll(t, 10, timeout_us=20_000_000) for t in ts]
    ctx.serve_stop()
    assert all(o is not None for o in out)
    assert max(o[2]["batch_size"] for o in out) <= 2
    assert A.AQR_OK == 0


def test_open_loop_replay_matches_uniform_calls(served):
    # Poisson arrivals at 50,000 requests/s from the native replay loop;
    # each request must get the answer of a uniform batch with its (k, ef)
    ctx, q = served
    rng = np.random.default_rng(3)
    n = len(q)
    ks = rng.choice([1, 10, 100], n).astype(np.int32)
    efs = rng.choice([32, 128, 512], n).astype(np.int32)
    arrival = np.cumsum(rng.exponential(1e6 / 50_000, n))
    ctx.serve_start(max_batch=64, n_streams=4, batch_wait_us=20)
    ids, dd, lat, batch = ctx.serve_replay(q, ks, efs, arrival, k_stride=100)
    ctx.serve_stop()
    assert np.all(lat > 0) and batch.max() > 1
    qd = torch.from_numpy(q).cuda()
    for kk in (1, 10, 100):
        for ee in (32, 128, 512):
            sel = np.nonzero((ks == kk) & (efs == ee))[0]
            if len(sel) == 0:
                continue
            ri, rd = ctx.search(qd[torch.from_numpy(sel).cuda()].contiguous(), kk, ee)
            np.testing.assert_array_equal(ids[sel, :kk], ri.cpu().numpy())
            np.testing.assert_array_equal(dd[sel, :kk], rd.cpu().numpy())
            assert np.all(ids[sel, kk:] == -1)


def test_replay_rejects_bad_schedules(served):
    from paper_2602_21600_gb300.aqr import AQR_ERR_INVALID_ARG, AqrError
    ctx, q = served
    ctx.serve_start(max_batch=16, n_streams=2)
    with pytest.raises(AqrError) as ei:   # arrivals must not go backwards
        ctx.serve_replay(q[:3], [1, 1, 1], [16, 16, 16], [0.0, 5.0, 2.0])
    assert ei.value.status == AQR_ERR_INVALID_ARG
    with pytest.raises(AqrError) as ei:   # k beyond the row width
        ctx.serve_replay(q[:2], [5, 50], [16, 64], [0.0, 1.0], k_stride=10)
    assert ei.value.status == AQR_ERR_INVALID_ARG
    ctx.serve_stop()


def test_scheduler_host_exception_fails_submit_and_poll(served):
    # Failure injected on the host: the scheduler thread throws the
    # exception it would throw when host memory runs out.  Afterwards no
    # request may wait for ever: submits are refused, and every request
    # still queued or on the GPU completes with an error.  Serving can then
    # be stopped and started again on the same context.
    from paper_2602_21600_gb300.aqr import AQR_ERR_CUDA, AqrError
    ctx, q = served
    ctx.serve_start(max_batch=16, n_streams=2, batch_wait_us=20)
    tickets = [ctx.submit(q[i], 10, 128) for i in range(40)]
    ctx.serve_inject_host_fault()
    deadline = time.time() + 10
    while True:
        try:
            t = ctx.submit(q[0], 10, 64)
            tickets.append(t)
        except AqrError as e:
            assert e.status == AQR_ERR_CUDA
            break
        assert time.time() < deadline, "submit still accepted after the scheduler stopped"
        time.sleep(0.001)
    n_ok = n_err = 0
    for t in tickets:
        try:
            r = ctx.poll(t, 10, timeout_us=2_000_000)
            assert r is not None, "request left waiting after the scheduler stopped"
            n_ok += 1
        except AqrError as e:
            assert e.status == AQR_ERR_CUDA
            n_err += 1
    assert n_err >= 1 and n_ok + n_err == len(tickets)
    ctx.serve_stop()
    # a new service on the same context answers again, as a search alone does
    ctx.serve_start(max_batch=16, n_streams=2, batch_wait_us=20)
    t = ctx.submit(q[3], 10, 64)
    ids, dd, _ = ctx.poll(t, 10, timeout_us=5_000_000)
    a_ids, a_dd = _alone(ctx, q[3], 10, 64)
    np.testing.assert_array_equal(ids, a_ids)
    np.testing.assert_array_equal(dd, a_dd)
    ctx.serve_stop()
