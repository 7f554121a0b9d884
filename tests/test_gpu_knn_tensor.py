"""Brute-force kNN on the tensor cores (knn_mma.cu) against the CUDA-core kernel.

For integer-valued sets of magnitude <= 256 whose largest query and base
squared norms sum below 2^24, the tensor-core distances (BF16 operands,
FP32 accumulation) are exact, so ids and distances must equal the CUDA-core
kernel's bit for bit (that kernel is what aqr_bruteforce_knn_static always
runs) and the FP64 brute force of the oracle.  Other sets must fall back to
the CUDA cores, which the context's stats report.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2602_21600_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _cuda_core_knn(base, q, k, self_ids=None):
    from paper_2602_21600_gb300 import aqr
    ids = torch.empty((q.shape[0], k), dtype=torch.int64, device="cuda")
    dd = torch.empty((q.shape[0], k), dtype=torch.float32, device="cuda")
    st = aqr.lib().aqr_bruteforce_knn_static(
        ctypes.c_void_p(base.data_ptr()), base.shape[0], base.shape[1],
        ctypes.c_void_p(q.data_ptr()), q.shape[0], k,
        None if self_ids is None else ctypes.c_void_p(self_ids.data_ptr()),
        ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dd.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dd.cpu().numpy()


def _run(ctx, x, q, k, self_ids=None):
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    qd = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    sd = None if self_ids is None else torch.from_numpy(self_ids).cuda()
    ids, dd = ctx.knn(xd, qd, k, sd)
    torch.cuda.synchronize()
    tensor = ctx.stats()["knn_tensor"]
    ri, rd = _cuda_core_knn(xd, qd, k, sd)
    return ids.cpu().numpy(), dd.cpu().numpy(), ri, rd, tensor


@pytest.mark.parametrize("n,nq,d,k", [(20000, 300, 128, 10), (3001, 129, 37, 32),
                                      (1000, 1, 128, 1), (517, 260, 256, 8)])
def test_tensor_knn_equals_cuda_cores_on_integer_sift_like_data(ctx, n, nq, d, k):
    # the 1M x 128 law (non-negative integers <= 255), ragged sizes and d
    w = synth.workload("gmm1m_d128_int", n=n, nq=nq)
    x, q = w["x"], w["q"]
    if d < 128:
        x, q = x[:, :d].copy(), q[:, :d].copy()
    if d > 128:  # 256 dims: two copies of the columns, values halved to keep the norms < 2^23
        x = np.floor(np.concatenate([x, x[:, ::-1]], 1) / 2)
        q = np.floor(np.concatenate([q, q[:, ::-1]], 1) / 2)
    ids, dd, ri, rd, tensor = _run(ctx, x, q, k)
    assert tensor == 1
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(dd, rd)
    gi, gd = oracle.bruteforce(x, q, k)  # FP64, ties by id: the same lists
    np.testing.assert_array_equal(ids, gi)
    np.testing.assert_array_equal(dd.astype(np.float64), gd)


def test_tensor_knn_self_exclusion_and_signed_values(ctx):
    rng = np.random.default_rng(8)
    x = rng.integers(-256, 257, (5000, 64)).astype(np.float32)  # |v| <= 256, norms < 2^23
    x[7] = x[3]  # a duplicate: a tie broken by id
    sid = np.arange(0, 5000, 37, dtype=np.int64)
    ids, dd, ri, rd, tensor = _run(ctx, x, x[sid], 10, sid)
    assert tensor == 1
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(dd, rd)
    assert not np.any(ids == sid[:, None])


@pytest.mark.parametrize("case", ["float", "too_large", "norms", "k33", "d272", "d256_k16"])
def test_tensor_knn_falls_back_where_it_would_not_be_exact(ctx, case):
    rng = np.random.default_rng(9)
    x = rng.integers(0, 256, (3000, 128)).astype(np.float32)
    k = 10
    if case == "float":
        x = x + 0.5
    elif case == "too_large":
        x[5, 3] = 257.0
    elif case == "norms":  # 256 dims of 255: |q|^2 + |x|^2 above 2^24
        x = np.full((3000, 256), 255.0, np.float32)
        x[:, 0] = np.arange(3000) % 200
    elif case == "k33":
        k = 33
    elif case == "d272":
        x = rng.integers(0, 16, (3000, 272)).astype(np.float32)
    elif case == "d256_k16":  # exact data, but four 16-deep lists per query exceed shared memory
        x = rng.integers(0, 16, (3000, 256)).astype(np.float32)
        k = 16
    q = x[:50] + 1.0
    ids, dd, ri, rd, tensor = _run(ctx, x, q, k)
    assert tensor == 0
    np.testing.assert_array_equal(ids, ri)
    np.testing.assert_array_equal(dd, rd)


def test_training_density_runs_on_the_tensor_cores(ctx):
    # the density kNN of Alg. 1 on the integer law: tensor path, and the
    # trained parameters still equal the oracle's bit for bit
    w = synth.workload("gmm1m_d128_int", n=12000, nq=1)
    P_o = oracle.train(w["x"], w["sample"][:300], M0=16, ef0=200)
    P_g = ctx.train(torch.from_numpy(w["x"]).cuda(), w["sample"][:300], M0=16, ef0=200)
    torch.cuda.synchronize()
    assert ctx.stats()["knn_tensor"] == 1
    for key in ("min", "max", "scale"):
        np.testing.assert_array_equal(P_g[key], P_o[key])
    assert P_g["delta"] == P_o["delta"] and P_g["rho_bar"] == P_o["rho_bar"]
