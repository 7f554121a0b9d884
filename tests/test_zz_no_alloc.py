"""aqr_bruteforce_knn_static: the kNN entry point that allocates nothing.

Callers whose device memory belongs to another allocator, or who run under a
fixed device-memory budget, cannot let a library call allocate; this entry
point keeps its working memory in a fixed device array inside the library.
Its results must equal those of aqr_bruteforce_knn on consecutive calls
(the shared array keeps the previous call's contents), and requests larger
than the array are refused before anything is launched.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_knn(L, base, q, k, self_ids=None):
    ids = torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)
    dd = torch.empty((q.shape[0], k), dtype=torch.float32, device=q.device)
    st = L.aqr_bruteforce_knn_static(
        ctypes.c_void_p(base.data_ptr()), base.shape[0], base.shape[1],
        ctypes.c_void_p(q.data_ptr()), q.shape[0], k,
        None if self_ids is None else ctypes.c_void_p(self_ids.data_ptr()),
        ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dd.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, ids, dd


def test_static_knn_matches_allocating_entry_point_twice():
    from paper_2602_21600_gb300 import Context, aqr
    L = aqr.lib()
    ctx = Context(0)
    rng = np.random.default_rng(21)
    base = torch.from_numpy(rng.normal(0, 10, (20000, 96)).astype(np.float32)).cuda()
    calls = [
        (torch.from_numpy(rng.normal(0, 10, (777, 96)).astype(np.float32)).cuda(), 10, None),
        # second call: other queries, larger k, self exclusion
        (base[:300].clone(), 33, torch.arange(300, dtype=torch.int64, device="cuda")),
    ]
    for q, k, sid in calls:
        st, ids, dd = _static_knn(L, base, q, k, sid)
        assert st == aqr.AQR_OK
        ref_i, ref_d = ctx.knn(base, q, k, sid)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
        np.testing.assert_allclose(dd.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5, atol=0)
    ctx.close()


def test_static_knn_fewer_splits_and_largest_k_allocate_nothing():
    # nq = 19000, k = 64: the usual two base-set splits would need 2.4M keys,
    # more than the array's 2,097,152, so the call runs with one split; k =
    # 128 is the largest k.  Results equal the allocating entry point's, and
    # a call after the device's first (set-up) call leaves the device's free
    # memory unchanged.
    from paper_2602_21600_gb300 import Context, aqr
    L = aqr.lib()
    ctx = Context(0)
    rng = np.random.default_rng(5)
    base = torch.from_numpy(rng.normal(0, 10, (30000, 64)).astype(np.float32)).cuda()
    for nq, k in [(19000, 64), (1500, 128)]:
        q = torch.from_numpy(rng.normal(0, 10, (nq, 64)).astype(np.float32)).cuda()
        ref_i, ref_d = ctx.knn(base, q, k)
        ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        args = (ctypes.c_void_p(base.data_ptr()), base.shape[0], base.shape[1],
                ctypes.c_void_p(q.data_ptr()), nq, k, None, ctypes.c_void_p(ids.data_ptr()),
                ctypes.c_void_p(dd.data_ptr()),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert L.aqr_bruteforce_knn_static(*args) == aqr.AQR_OK  # set-up on first use
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        ids.fill_(-7)
        torch.cuda.synchronize()
        assert L.aqr_bruteforce_knn_static(*args) == aqr.AQR_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_i.cpu().numpy())
        np.testing.assert_allclose(dd.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5, atol=0)
    ctx.close()


def test_static_knn_refuses_requests_beyond_its_scratch():
    from paper_2602_21600_gb300 import aqr
    L = aqr.lib()
    base = torch.zeros((100, 8), dtype=torch.float32, device="cuda")
    q = torch.zeros((40000, 8), dtype=torch.float32, device="cuda")
    st, _, _ = _static_knn(L, base, q, 64)  # 40000 * 64 > 2,097,152 keys
    assert st == aqr.AQR_ERR_INVALID_ARG
    st, _, _ = _static_knn(L, base, q[:10], 129)  # k above 128
    assert st == aqr.AQR_ERR_INVALID_ARG
