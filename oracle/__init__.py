"""CPU oracle for the AQR-HNSW query path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The C++ source
(``aqr_oracle.cpp``) is compiled with g++ into ``oracle/_build/`` on first
use (or by ``build()``); it shares no code with the CUDA library.

Every function here is argument marshalling around one C function; the
arithmetic and its citations live in the C++ file.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aqr_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF

# Insertion schedules of the graph build, as (batch_div, batch_max).
# SEQUENTIAL is Alg. 1 as written: nodes are inserted one at a time in id
# order, each searching the graph built from all earlier nodes.  It is the
# default of every build here.  BATCHED is the reading the GPU builder runs
# by default (node 0 alone, then batches of min(max(1, s / 32), 16384) nodes
# that search the graph as it stood before their batch); the oracle builds
# it only when asked, so that the GPU build can be checked bit for bit.
SEQUENTIAL = (1, 1)
BATCHED = (32, 16384)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP contraction off) if missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
            "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class SearchParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("ef", C.c_int32), ("m_ef", C.c_int32),
                ("rerank_pct", C.c_int32), ("n_coarse", C.c_int32), ("n_rerank", C.c_int32),
                ("tau_gap", C.c_double), ("tau_ratio", C.c_double), ("eps", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.oracle_batch_schedule.restype = C.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def density(x, ids, kd=10, nthreads=0):
    """rho_i = 1 / (mean squared L2 to the kd nearest other points + 1e-6)."""
    x = _f32(x)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.empty(len(ids), dtype=np.float64)
    rc = lib().oracle_density(_p(x), C.c_int64(x.shape[0]), C.c_int32(x.shape[1]), _p(ids),
                              C.c_int64(len(ids)), C.c_int32(kd), C.c_int32(nthreads), _p(out))
    if rc:
        raise ValueError("oracle_density: invalid arguments")
    return out


def train(x, sample=None, p_max=0.01, M0=16, ef0=200, nthreads=0):
    """Quantiser training and graph parameters (Alg. 1)."""
    x = _f32(x)
    n, d = x.shape
    smp = None if sample is None else np.ascontiguousarray(sample, dtype=np.int64)
    mn = np.empty(d, np.float32)
    mx = np.empty(d, np.float32)
    sc = np.empty(d, np.float32)
    s = np.empty(11, np.float64)
    rc = lib().oracle_train(_p(x), C.c_int64(n), C.c_int32(d), _p(smp),
                            C.c_int64(0 if smp is None else len(smp)), C.c_double(p_max),
                            C.c_int32(M0), C.c_int32(ef0), C.c_int32(nthreads),
                            _p(mn), _p(mx), _p(sc), _p(s))
    if rc:
        raise ValueError("oracle_train: invalid arguments")
    return dict(min=mn, max=mx, scale=sc, delta=s[0], rho_bar=s[1], w=s[2], s_dist=s[3],
                eta=s[4], M_i=int(s[5]), ef_c=int(s[6]), P_l=s[7], P_h=s[8],
                rho_min=s[9], rho_max=s[10])


def encode(x, minv, scale):
    x = _f32(x)
    if x.ndim == 1:
        x = x[None]
    n, d = x.shape
    out = np.empty((n, d), np.uint8)
    rc = lib().oracle_encode(_p(x), C.c_int64(n), C.c_int32(d), _p(_f32(minv)), _p(_f32(scale)),
                             _p(out))
    if rc:
        raise ValueError("oracle_encode: invalid arguments")
    return out


def levels(U, M_i):
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty(len(U), np.int32)
    if lib().oracle_levels(_p(U), C.c_int64(len(U)), C.c_int32(M_i), _p(out)):
        raise ValueError("oracle_levels: invalid arguments")
    return out


def batch_schedule(n, batch_div=BATCHED[0], batch_max=BATCHED[1]):
    L = lib()
    cnt = L.oracle_batch_schedule(C.c_int64(n), C.c_int32(batch_div), C.c_int32(batch_max), None)
    st = np.empty(cnt + 1, np.int64)
    L.oracle_batch_schedule(C.c_int64(n), C.c_int32(batch_div), C.c_int32(batch_max), _p(st))
    return st


def build_graph(codes, lv, M_i, ef_c, batch_div=SEQUENTIAL[0], batch_max=SEQUENTIAL[1],
                nthreads=0):
    """HNSW construction on codes (Alg. 1).  Returns a dict with
    adj0 [n, 2M_i], upper_base [n], upper [rows, M_i], entry, max_level.
    The default is the sequential insertion of Alg. 1; pass ``*BATCHED``
    for the batched reading of the GPU builder."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    lv = np.ascontiguousarray(lv, dtype=np.int32)
    n, d = codes.shape
    rows = int(lv.clip(min=0).sum())
    adj0 = np.empty((n, 2 * M_i), np.uint32)
    ub = np.empty(n, np.int64)
    up = np.empty((max(rows, 1), M_i), np.uint32)
    el = np.empty(2, np.int32)
    rc = lib().oracle_build(_p(codes), C.c_int64(n), C.c_int32(d), _p(lv), C.c_int32(M_i),
                            C.c_int32(ef_c), C.c_int32(batch_div), C.c_int32(batch_max),
                            C.c_int32(nthreads), _p(adj0), _p(ub), _p(up), _p(el))
    if rc:
        raise ValueError("oracle_build: invalid arguments")
    return dict(adj0=adj0, upper_base=ub, upper=up[:rows], entry=int(el[0]),
                max_level=int(el[1]), M_i=M_i, ef_c=ef_c, levels=lv)


def search(index, q, k=10, ef=64, m_ef=3, rerank_pct=40, n_coarse=0, n_rerank=0,
           tau_gap=0.010, tau_ratio=1.008, eps=1e-6, trace=False, cap_exp=4096, nthreads=0):
    """Alg. 2 over a flat index dict (codes, x, adj0, upper_base, upper,
    entry, max_level, min, scale).  Returns ids, dists, exact flags and,
    with trace=True, the stage traces."""
    q = _f32(q)
    if q.ndim == 1:
        q = q[None]
    nq, d = q.shape
    codes = np.ascontiguousarray(index["codes"], np.uint8)
    x = _f32(index["x"])
    adj0 = np.ascontiguousarray(index["adj0"], np.uint32)
    ub = np.ascontiguousarray(index["upper_base"], np.int64)
    up = np.ascontiguousarray(index["upper"], np.uint32)
    if up.size == 0:
        up = np.full((1, max(1, adj0.shape[1] // 2)), NONE, np.uint32)
    n = codes.shape[0]
    P = SearchParams(k, ef, m_ef, rerank_pct, n_coarse, n_rerank, tau_gap, tau_ratio, eps)
    ids = np.empty((nq, k), np.int64)
    dists = np.empty((nq, k), np.float64)
    exact = np.empty((nq, k), np.uint8)
    ef_eff = max(ef, k)
    cap_c = ef_eff
    tr = {}
    if trace:
        tr = dict(l0_entry=np.empty(nq, np.uint32), c_ids=np.full((nq, cap_c), NONE, np.uint32),
                  c_dist=np.full((nq, cap_c), -1, np.int64), c_count=np.empty(nq, np.int32),
                  a_ids=np.full((nq, cap_c), NONE, np.uint32),
                  a_dist=np.full((nq, cap_c), np.inf, np.float64), et=np.empty(nq, np.uint8),
                  n_exact=np.empty(nq, np.int32), exp_seq=np.full((nq, cap_exp), NONE, np.uint32),
                  exp_count=np.empty(nq, np.int32), evals=np.empty(nq, np.int64))
    g = tr.get
    rc = lib().oracle_search(
        C.c_int64(n), C.c_int32(d), C.c_int32(adj0.shape[1]), C.c_int32(up.shape[1]),
        _p(codes), _p(x), _p(adj0), _p(ub), _p(up), C.c_uint32(index["entry"]),
        C.c_int32(index["max_level"]), _p(_f32(index["min"])), _p(_f32(index["scale"])),
        _p(q), C.c_int64(nq), C.byref(P), C.c_int32(nthreads), _p(ids), _p(dists), _p(exact),
        _p(g("l0_entry")), _p(g("c_ids")), _p(g("c_dist")), _p(g("c_count")), _p(g("a_ids")),
        _p(g("a_dist")), _p(g("et")), _p(g("n_exact")), C.c_int32(cap_c), _p(g("exp_seq")),
        _p(g("exp_count")), C.c_int32(cap_exp), _p(g("evals")))
    if rc:
        raise ValueError("oracle_search: invalid arguments")
    out = dict(ids=ids, dists=dists, exact=exact)
    out.update(tr)
    return out


def pair_dists(x, codes, minv, scale, q, qi, ids):
    """Exact, asymmetric and integer code distances of (q[qi[t]], base ids[t]) pairs."""
    x = _f32(x)
    q = _f32(q)
    codes = np.ascontiguousarray(codes, np.uint8)
    qi = np.ascontiguousarray(qi, np.int64)
    ids = np.ascontiguousarray(ids, np.int64)
    m = len(ids)
    ex = np.empty(m, np.float64)
    asy = np.empty(m, np.float64)
    cd = np.empty(m, np.int64)
    rc = lib().oracle_pair_dists(_p(x), _p(codes), C.c_int32(x.shape[1]), _p(_f32(minv)),
                                 _p(_f32(scale)), _p(q), _p(qi), _p(ids), C.c_int64(m), _p(ex),
                                 _p(asy), _p(cd))
    if rc:
        raise ValueError("oracle_pair_dists: invalid arguments")
    return ex, asy, cd


def bruteforce(x, q, k, nthreads=0):
    x = _f32(x)
    q = _f32(q)
    if q.ndim == 1:
        q = q[None]
    ids = np.empty((q.shape[0], k), np.int64)
    dd = np.empty((q.shape[0], k), np.float64)
    rc = lib().oracle_bruteforce(_p(x), C.c_int64(x.shape[0]), C.c_int32(x.shape[1]), _p(q),
                                 C.c_int64(q.shape[0]), C.c_int32(k), C.c_int32(nthreads),
                                 _p(ids), _p(dd))
    if rc:
        raise ValueError("oracle_bruteforce: invalid arguments")
    return ids, dd


def bruteforce_codes(codes, qc, k):
    codes = np.ascontiguousarray(codes, np.uint8)
    qc = np.ascontiguousarray(qc, np.uint8)
    if qc.ndim == 1:
        qc = qc[None]
    ids = np.empty((qc.shape[0], k), np.int64)
    dd = np.empty((qc.shape[0], k), np.int64)
    rc = lib().oracle_bruteforce_codes(_p(codes), C.c_int64(codes.shape[0]),
                                       C.c_int32(codes.shape[1]), _p(qc), C.c_int64(qc.shape[0]),
                                       C.c_int32(k), _p(ids), _p(dd))
    if rc:
        raise ValueError("oracle_bruteforce_codes: invalid arguments")
    return ids, dd


def make_index(x, U, sample=None, M0=16, ef0=100, p_max=0.01, batch_div=SEQUENTIAL[0],
               batch_max=SEQUENTIAL[1], nthreads=0, params=None):
    """Train (or take ``params``), encode and build (sequential insertion,
    Alg. 1, unless a batch schedule is given): the full index dict."""
    P = params if params is not None else train(x, sample, p_max, M0, ef0, nthreads)
    codes = encode(x, P["min"], P["scale"])
    lv = levels(U, P["M_i"])
    g = build_graph(codes, lv, P["M_i"], P["ef_c"], batch_div, batch_max, nthreads)
    idx = dict(P)
    idx.update(g)
    idx.update(codes=codes, x=_f32(x))
    return idx


def write_index(path, idx):
    """Write an index dict in the library's file format (AQRIDX01)."""
    x = _f32(idx["x"])
    n, d = x.shape
    adj0 = np.ascontiguousarray(idx["adj0"], np.uint32)
    up = np.ascontiguousarray(idx["upper"], np.uint32)
    ub = np.ascontiguousarray(idx["upper_base"], np.int64)
    M_i = int(idx["M_i"])
    rc = lib().oracle_write_index(
        path.encode(), C.c_int64(n), C.c_int32(d), C.c_int32(M_i), C.c_int32(adj0.shape[1]),
        C.c_int32(M_i), C.c_uint32(idx["entry"]), C.c_int32(idx["max_level"]),
        C.c_int32(idx["ef_c"]), C.c_int64(up.shape[0]), C.c_double(idx.get("s_dist", 0.0)),
        C.c_double(idx.get("delta", 0.0)), C.c_double(idx.get("eta", 0.0)),
        _p(_f32(idx["min"])), _p(_f32(idx["scale"])),
        _p(np.ascontiguousarray(idx["codes"], np.uint8)), _p(x), _p(adj0), _p(ub),
        _p(up if up.size else None))
    if rc:
        raise OSError(f"oracle_write_index: cannot write {path}")


def merge_topk(dists, ids, id_offsets=None, k=None):
    """Top-k of the union of per-shard lists dists/ids [S, n, kin] by
    (distance, global id); returns ids int64 [n, k], dists float64 [n, k]."""
    d32 = np.ascontiguousarray(dists, np.float32)
    i64 = np.ascontiguousarray(ids, np.int64)
    S, n, kin = i64.shape
    k = kin if k is None else k
    off = None if id_offsets is None else np.ascontiguousarray(id_offsets, np.int64)
    out_i = np.empty((n, k), np.int64)
    out_d = np.empty((n, k), np.float64)
    rc = lib().oracle_merge_topk(_p(d32), _p(i64), C.c_int32(S), C.c_int64(n), C.c_int32(kin),
                                 _p(off), C.c_int32(k), _p(out_i), _p(out_d))
    if rc:
        raise ValueError("oracle_merge_topk: invalid arguments")
    return out_i, out_d
