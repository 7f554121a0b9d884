"""Thin ctypes binding of libaqr.so (include/aqr.h).

Every ``aqr_*`` function of the C ABI is exposed under the same name with
the same arguments (pointers as ints, streams as ints).  ``Context`` wraps
them for torch tensors: it only checks shapes/dtypes and passes pointers;
every step of the query path runs in the library's CUDA kernels.  There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None


class AqrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


STATUS = {0: "AQR_OK", 1: "AQR_ERR_INVALID_ARG", 2: "AQR_ERR_NO_MEMORY", 3: "AQR_ERR_NO_INDEX",
          4: "AQR_ERR_CUDA", 5: "AQR_ERR_TIMEOUT", 6: "AQR_ERR_BAD_FILE", 7: "AQR_ERR_BUSY",
          8: "AQR_ERR_NOT_READY", 9: "AQR_ERR_INTERNAL"}
AQR_OK, AQR_ERR_INVALID_ARG, AQR_ERR_NO_MEMORY, AQR_ERR_NO_INDEX, AQR_ERR_CUDA = 0, 1, 2, 3, 4
AQR_ERR_TIMEOUT, AQR_ERR_BAD_FILE, AQR_ERR_BUSY, AQR_ERR_NOT_READY, AQR_ERR_INTERNAL = 5, 6, 7, 8, 9


class aqr_search_params(C.Structure):
    _fields_ = [("m_ef", C.c_int32), ("rerank_pct", C.c_int32), ("n_coarse", C.c_int32),
                ("n_rerank", C.c_int32), ("tau_gap", C.c_float), ("tau_ratio", C.c_float),
                ("eps", C.c_float)]


class aqr_kernel_config(C.Structure):
    _fields_ = [("hash_slots", C.c_int32), ("tile_rows", C.c_int32), ("team_lanes", C.c_int32),
                ("hash_tag_bits", C.c_int32), ("warps_per_block", C.c_int32),
                ("warps_per_query", C.c_int32)]


class aqr_tune_result(C.Structure):
    _fields_ = [("params", aqr_search_params), ("ef", C.c_int32),
                ("kernel", aqr_kernel_config), ("recall", C.c_double), ("ms", C.c_double),
                ("reached", C.c_int32)]


class aqr_index_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("d_pad", C.c_int32), ("M_i", C.c_int32),
                ("R0", C.c_int32), ("R1", C.c_int32), ("ef_c", C.c_int32),
                ("max_level", C.c_int32), ("entry", C.c_uint32), ("n_upper", C.c_int64),
                ("s_dist", C.c_double), ("device_bytes", C.c_int64)]


class aqr_stats(C.Structure):
    _fields_ = [("queries", C.c_int64), ("expansions", C.c_int64), ("dist_evals", C.c_int64),
                ("adj_entries", C.c_int64), ("stage2_evals", C.c_int64),
                ("exact_evals", C.c_int64), ("early_exits", C.c_int64),
                ("algo_bytes", C.c_int64), ("device_errors", C.c_int32),
                ("l0_evals", C.c_int64), ("knn_tensor", C.c_int32)]


class aqr_trace(C.Structure):
    _fields_ = [("l0_entry", C.c_void_p), ("c_ids", C.c_void_p), ("c_dist", C.c_void_p),
                ("c_count", C.c_void_p), ("a_ids", C.c_void_p), ("a_dist", C.c_void_p),
                ("et", C.c_void_p), ("n_exact", C.c_void_p), ("exp_seq", C.c_void_p),
                ("exp_count", C.c_void_p), ("cap_c", C.c_int32), ("cap_exp", C.c_int32)]


class aqr_serve_config(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("n_streams", C.c_int32), ("hbm_budget", C.c_int64),
                ("max_pending", C.c_int32), ("batch_wait_us", C.c_int32)]


class aqr_request_stats(C.Structure):
    _fields_ = [("queue_us", C.c_double), ("latency_us", C.c_double), ("batch_size", C.c_int32)]


P = C.c_void_p
I32, I64, U32, U64, F32, F64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float, C.c_double
ST = C.c_int

# name -> (restype, argtypes); the C ABI of include/aqr.h.
SIGNATURES = {
    "aqr_create": (ST, [C.POINTER(P), I32]),
    "aqr_destroy": (ST, [P]),
    "aqr_status_string": (C.c_char_p, [ST]),
    "aqr_last_error": (C.c_char_p, [P]),
    "aqr_default_search_params": (ST, [C.POINTER(aqr_search_params)]),
    "aqr_set_search_params": (ST, [P, C.POINTER(aqr_search_params)]),
    "aqr_merge_topk": (ST, [P, P, P, I32, I64, I32, P, P, P, P]),
    "aqr_search_params_for_recall": (ST, [C.c_double, C.POINTER(aqr_search_params),
                                          C.POINTER(I32)]),
    "aqr_quantize": (ST, [P, P, I64, I32, I64, P, P, P, I64, P]),
    "aqr_train_quantizer": (ST, [P, P, I64, I32, P, I64, F64, I32, I32, P, P, P, P]),
    "aqr_load_graph": (ST, [P, C.c_char_p]),
    "aqr_build_graph": (ST, [P, P, I64, I32, P, P, P, I32, I32, I32, I32, F64]),
    "aqr_index_info_get": (ST, [P, C.POINTER(aqr_index_info)]),
    "aqr_export_graph": (ST, [P, P, P, P, P, P]),
    "aqr_search": (ST, [P, P, I64, I32, I32, P, P, P]),
    "aqr_search_trace": (ST, [P, P, I64, I32, I32, P, P, P, C.POINTER(aqr_trace), P]),
    "aqr_search_mixed": (ST, [P, P, I64, P, P, I32, P, P, P]),
    "aqr_search_host": (ST, [P, P, I64, I32, I32, P, P]),
    "aqr_search_plain_f32": (ST, [P, P, I64, I32, I32, P, P, P]),
    "aqr_get_stats": (ST, [P, C.POINTER(aqr_stats)]),
    "aqr_set_kernel_config": (ST, [P, I32, I32, C.POINTER(aqr_kernel_config)]),
    "aqr_autotune": (ST, [P, P, I64, I32, I32, C.POINTER(aqr_kernel_config)]),
    "aqr_autotune_recall": (ST, [P, P, I64, I32, P, I32, C.c_double, P, I32,
                                 C.POINTER(aqr_tune_result), P]),
    "aqr_bruteforce_knn": (ST, [P, P, I64, I32, P, I64, I32, P, P, P, P]),
    "aqr_bruteforce_knn_static": (ST, [P, I64, I32, P, I64, I32, P, P, P, P]),
    "aqr_serve_start": (ST, [P, C.POINTER(aqr_serve_config)]),
    "aqr_submit": (ST, [P, P, I32, I32, C.POINTER(U64)]),
    "aqr_poll": (ST, [P, U64, P, P, C.POINTER(aqr_request_stats), I64]),
    "aqr_cancel": (ST, [P, U64]),
    "aqr_serve_stop": (ST, [P]),
    "aqr_serve_inject_host_fault": (ST, [P]),
    "aqr_serve_replay": (ST, [P, P, I64, P, P, P, I32, P, P, P, I64]),
}


def library_path() -> str:
    return _build.LIB


_lib_checked = None


def lib(build_if_missing: bool = True, checked: bool = False):
    """Load libaqr.so, or libaqr_checked.so (the bounds-checked build), compiling
    it first if it is missing or stale."""
    global _lib, _lib_checked
    with _lock:
        if (_lib_checked if checked else _lib) is None:
            path = _build.LIB_CHECKED if checked else _build.LIB
            if build_if_missing:
                _build.build_library(checked=checked)
            if not os.path.exists(path):
                raise RuntimeError(f"{os.path.basename(path)} is not built; run __graft_entry__.build()")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            if checked:
                _lib_checked = L
            else:
                _lib = L
    return _lib_checked if checked else _lib


def __getattr__(name):
    # aqr_xxx at module level resolves to the C function of the same name
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


def params_for_recall(target_recall: float):
    """Table 3 preset for a target recall: (search-parameter dict for
    Context.set_params, the layer-0 search depth ef = N_c * m_ef)."""
    p = aqr_search_params()
    ef = I32()
    st = lib().aqr_search_params_for_recall(float(target_recall), C.byref(p), C.byref(ef))
    if st != 0:
        raise AqrError(st, f"no preset for target recall {target_recall!r}")
    return {f: getattr(p, f) for f, _ in aqr_search_params._fields_}, ef.value


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_tensor(t, dtype, name, cuda, ndim=None, shape=None, device=None, rows=False):
    """Checks that the library can take t's data pointer: on the GPU (cuda)
    or in host memory, of dtype, of ndim dimensions or exactly `shape`, and
    dense (rows: only the last dimension dense, the call takes a row
    stride).  Raises ValueError / TypeError before anything is launched."""
    global _torch
    if _torch is None:
        import torch as _t
        _torch = _t
    if not isinstance(t, _torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is needed, not {type(t).__name__}")
    if t.is_cuda != cuda:
        raise ValueError(f"{name}: a CUDA tensor is needed (no CPU fallback exists)" if cuda
                         else f"{name}: a host (CPU) tensor is needed")
    if cuda and device is not None and t.get_device() != device:
        raise ValueError(f"{name}: tensor on cuda:{t.get_device()}, context on cuda:{device}")
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if shape is not None:
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    elif ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name}: {t.dim()} dimensions, expected {ndim}")
    if rows:
        if t.numel() and t.stride(-1) != 1:
            raise ValueError(f"{name}: the last dimension must be dense")
    elif not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is needed")
    return C.c_void_p(t.data_ptr())


_torch = None


def _check_len(a, n, name):
    if len(a) != n:
        raise ValueError(f"{name}: {len(a)} entries, expected {n}")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, checked: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("AQR needs a CUDA device; no CPU fallback exists")
        self.L = lib(checked=checked)
        self.device = device
        self._d = None  # dimension of the loaded or built index
        h = C.c_void_p()
        st = self.L.aqr_create(C.byref(h), device)
        if st != AQR_OK:
            raise AqrError(st, "aqr_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.aqr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != AQR_OK:
            raise AqrError(st, self.L.aqr_last_error(self.h).decode(errors="replace"))

    # -- argument checks (before any pointer reaches the library) ---------
    def _dev(self, t, dtype, name, **kw):
        return _check_tensor(t, dtype, name, True, device=self.device, **kw)

    def _queries(self, q, name="q", cuda=True):
        """FP32 queries [n, d]; d must be the index's once one is loaded."""
        import torch
        p = _check_tensor(q, torch.float32, name, cuda, ndim=2,
                          device=self.device if cuda else None)
        if self._d is not None and q.shape[1] != self._d:
            raise ValueError(f"{name}: {q.shape[1]} columns, the index has d = {self._d}")
        return p

    def _results(self, ids, dists, n, k, device, cuda=True):
        """Result buffers [n, k] (int64 ids, float32 distances), allocated if
        not given."""
        import torch
        if ids is None and dists is None:
            if cuda:
                return self._out(n, k, device)
            return (torch.empty((n, k), dtype=torch.int64),
                    torch.empty((n, k), dtype=torch.float32))
        if ids is None or dists is None:
            raise ValueError("give both ids and dists, or neither")
        dev = self.device if cuda else None
        _check_tensor(ids, torch.int64, "ids", cuda, shape=(n, k), device=dev)
        _check_tensor(dists, torch.float32, "dists", cuda, shape=(n, k), device=dev)
        return ids, dists

    # -- parameters -----------------------------------------------------
    def set_params(self, **kw):
        p = aqr_search_params()
        self.L.aqr_default_search_params(C.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        self._check(self.L.aqr_set_search_params(self.h, C.byref(p)))
        return p

    # -- quantiser --------------------------------------------------------
    def quantize(self, x, minv, scale, out=None, ldc=None, stream=None):
        import torch
        self._dev(x, torch.float32, "x", ndim=2, rows=True)
        n, d = x.shape
        ldc = ldc or d
        if ldc < d:
            raise ValueError(f"ldc = {ldc} is below d = {d}")
        self._dev(minv, torch.float32, "minv", shape=(d,))
        self._dev(scale, torch.float32, "scale", shape=(d,))
        if out is None:
            out = torch.empty((n, ldc), dtype=torch.uint8, device=x.device)
        self._dev(out, torch.uint8, "out", shape=(n, ldc))
        ldx = x.stride(0) if n > 0 else d  # empty tensors report stride 0
        self._check(self.L.aqr_quantize(self.h, _ptr(x), n, d, ldx, _ptr(minv), _ptr(scale),
                                        _ptr(out), ldc, _stream(stream)))
        return out

    def train(self, x, sample=None, p_max=0.01, M0=16, ef0=200):
        import numpy as np
        import torch
        self._dev(x, torch.float32, "x", ndim=2)
        n, d = x.shape
        mn = np.empty(d, np.float32)
        mx = np.empty(d, np.float32)
        sc = np.empty(d, np.float32)
        s = np.empty(11, np.float64)
        smp = None if sample is None else np.ascontiguousarray(sample, np.int64)
        self._check(self.L.aqr_train_quantizer(
            self.h, _ptr(x), n, d, None if smp is None else smp.ctypes.data_as(P),
            0 if smp is None else len(smp), p_max, M0, ef0, mn.ctypes.data_as(P),
            mx.ctypes.data_as(P), sc.ctypes.data_as(P), s.ctypes.data_as(P)))
        return dict(min=mn, max=mx, scale=sc, delta=s[0], rho_bar=s[1], w=s[2], s_dist=s[3],
                    eta=s[4], M_i=int(s[5]), ef_c=int(s[6]), P_l=s[7], P_h=s[8],
                    rho_min=s[9], rho_max=s[10])

    # -- index ------------------------------------------------------------
    def load_graph(self, path: str):
        self._check(self.L.aqr_load_graph(self.h, path.encode()))
        self._d = self.info()["d"]

    def build_graph(self, x, minv, scale, U, M_i, ef_c, batch_div=32, batch_max=16384,
                    s_dist=0.0):
        import numpy as np
        import torch
        self._dev(x, torch.float32, "x", ndim=2)
        n, d = x.shape
        mn = np.ascontiguousarray(minv, np.float32).reshape(-1)
        sc = np.ascontiguousarray(scale, np.float32).reshape(-1)
        U = np.ascontiguousarray(U, np.float64).reshape(-1)
        _check_len(mn, d, "minv")
        _check_len(sc, d, "scale")
        _check_len(U, n, "U")
        self._check(self.L.aqr_build_graph(self.h, _ptr(x), n, d, mn.ctypes.data_as(P),
                                           sc.ctypes.data_as(P), U.ctypes.data_as(P), M_i, ef_c,
                                           batch_div, batch_max, s_dist))
        self._d = d

    def info(self):
        i = aqr_index_info()
        self._check(self.L.aqr_index_info_get(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in aqr_index_info._fields_}

    def export_graph(self):
        import numpy as np
        inf = self.info()
        n, R0, R1, rows = inf["n"], inf["R0"], inf["R1"], inf["n_upper"]
        adj0 = np.empty((n, R0), np.uint32)
        ub = np.empty(n, np.int64)
        up = np.empty((max(rows, 1), R1), np.uint32)
        codes = np.empty((n, inf["d"]), np.uint8)
        el = np.empty(2, np.int32)
        self._check(self.L.aqr_export_graph(self.h, adj0.ctypes.data_as(P), ub.ctypes.data_as(P),
                                            up.ctypes.data_as(P), codes.ctypes.data_as(P),
                                            el.ctypes.data_as(P)))
        return dict(adj0=adj0, upper_base=ub, upper=up[:rows], codes=codes, entry=int(el[0]),
                    max_level=int(el[1]))

    # -- search -----------------------------------------------------------
    def _out(self, n, k, device):
        import torch
        return (torch.empty((n, k), dtype=torch.int64, device=device),
                torch.empty((n, k), dtype=torch.float32, device=device))

    def search(self, q, k, ef, ids=None, dists=None, stream=None):
        self._queries(q)
        n = q.shape[0]
        ids, dists = self._results(ids, dists, n, k, q.device)
        self._check(self.L.aqr_search(self.h, _ptr(q), n, k, ef, _ptr(ids), _ptr(dists),
                                      _stream(stream)))
        return ids, dists

    def search_trace(self, q, k, ef, cap_exp=4096, stream=None):
        import torch
        self._queries(q)
        n = q.shape[0]
        dev = q.device
        ids, dists = self._out(n, k, dev)
        exact = torch.empty((n, k), dtype=torch.uint8, device=dev)
        cap_c = max(k, ef)
        t = dict(l0_entry=torch.full((n,), -1, dtype=torch.int32, device=dev),
                 c_ids=torch.full((n, cap_c), -1, dtype=torch.int32, device=dev),
                 c_dist=torch.full((n, cap_c), -1, dtype=torch.int32, device=dev),
                 c_count=torch.zeros(n, dtype=torch.int32, device=dev),
                 a_ids=torch.full((n, cap_c), -1, dtype=torch.int32, device=dev),
                 a_dist=torch.full((n, cap_c), float("inf"), dtype=torch.float32, device=dev),
                 et=torch.zeros(n, dtype=torch.uint8, device=dev),
                 n_exact=torch.zeros(n, dtype=torch.int32, device=dev),
                 exp_seq=torch.full((n, cap_exp), -1, dtype=torch.int32, device=dev),
                 exp_count=torch.zeros(n, dtype=torch.int32, device=dev))
        tr = aqr_trace(*[t[f].data_ptr() for f, _ in aqr_trace._fields_[:10]], cap_c, cap_exp)
        self._check(self.L.aqr_search_trace(self.h, _ptr(q), n, k, ef, _ptr(ids), _ptr(dists),
                                            _ptr(exact), C.byref(tr), _stream(stream)))
        t.update(ids=ids, dists=dists, exact=exact)
        return t

    def search_mixed(self, q, k_list, ef_list, k_stride=None, stream=None, ids=None, dists=None):
        import numpy as np
        self._queries(q)
        n = q.shape[0]
        kk = np.ascontiguousarray(k_list, np.int32).reshape(-1)
        ee = np.ascontiguousarray(ef_list, np.int32).reshape(-1)
        _check_len(kk, n, "k_list")
        _check_len(ee, n, "ef_list")
        k_stride = k_stride or (int(kk.max()) if n else 1)
        ids, dists = self._results(ids, dists, n, k_stride, q.device)
        self._check(self.L.aqr_search_mixed(self.h, _ptr(q), n, kk.ctypes.data_as(P),
                                            ee.ctypes.data_as(P), k_stride, _ptr(ids),
                                            _ptr(dists), _stream(stream)))
        return ids, dists

    def search_host(self, q_host, k, ef, ids_host=None, dists_host=None):
        """q_host, ids_host, dists_host: CPU tensors (pinned for best speed)."""
        self._queries(q_host, "q_host", cuda=False)
        n = q_host.shape[0]
        ids_host, dists_host = self._results(ids_host, dists_host, n, k, None, cuda=False)
        self._check(self.L.aqr_search_host(self.h, _ptr(q_host), n, k, ef, _ptr(ids_host),
                                           _ptr(dists_host)))
        return ids_host, dists_host

    def search_plain(self, q, k, ef, ids=None, dists=None, stream=None):
        self._queries(q)
        n = q.shape[0]
        ids, dists = self._results(ids, dists, n, k, q.device)
        self._check(self.L.aqr_search_plain_f32(self.h, _ptr(q), n, k, ef, _ptr(ids),
                                                _ptr(dists), _stream(stream)))
        return ids, dists

    def set_kernel_config(self, ef, k, hash_slots=0, tile_rows=0, team_lanes=0, hash_tag_bits=0,
                          warps_per_block=0, warps_per_query=0):
        cfg = aqr_kernel_config(hash_slots, tile_rows, team_lanes, hash_tag_bits, warps_per_block,
                                warps_per_query)
        self._check(self.L.aqr_set_kernel_config(self.h, ef, k, C.byref(cfg)))

    def autotune(self, q, k, ef):
        """Time the kernel configurations on batch q; keep and return the fastest."""
        cfg = aqr_kernel_config()
        self._queries(q)
        self._check(self.L.aqr_autotune(self.h, _ptr(q), q.shape[0], k, ef, C.byref(cfg)))
        return dict(hash_slots=cfg.hash_slots, tile_rows=cfg.tile_rows, team_lanes=cfg.team_lanes,
                    hash_tag_bits=cfg.hash_tag_bits, warps_per_block=cfg.warps_per_block,
                    warps_per_query=cfg.warps_per_query)

    def autotune_recall(self, q, k, gt_ids, target_recall, ef_list):
        """Shortlist policy, search depth and kernel configuration for a
        target recall@k on the sample q (device) with true neighbours gt_ids
        [n, >= k] (host).  Leaves the context set to the winner; returns it
        with the recall sweep (policies m_ef 3, 2, 1 x rerank 40%, 100%)."""
        import numpy as np
        self._queries(q)
        n = q.shape[0]
        gt = np.ascontiguousarray(gt_ids, np.int64)
        if gt.ndim != 2 or gt.shape[0] != n or gt.shape[1] < k:
            raise ValueError(f"gt_ids: shape {gt.shape}, expected [{n}, >= {k}]")
        efs = np.ascontiguousarray(ef_list, np.int32).reshape(-1)
        sweep = np.empty(6 * max(len(efs), 1), np.float64)
        r = aqr_tune_result()
        self._check(self.L.aqr_autotune_recall(self.h, _ptr(q), n, k, gt.ctypes.data_as(P),
                                               gt.shape[1], float(target_recall),
                                               efs.ctypes.data_as(P), len(efs), C.byref(r),
                                               sweep.ctypes.data_as(P)))
        kc = r.kernel
        pols = [(3, 40), (3, 100), (2, 40), (2, 100), (1, 40), (1, 100)]
        table = [dict(m_ef=m, rerank_pct=pc, ef=int(e), recall=round(float(sweep[i * len(efs) + j]), 5))
                 for i, (m, pc) in enumerate(pols) for j, e in enumerate(efs)
                 if sweep[i * len(efs) + j] >= 0]
        return dict(m_ef=r.params.m_ef, rerank_pct=r.params.rerank_pct, ef=r.ef,
                    recall=r.recall, ms=r.ms, reached=bool(r.reached),
                    kernel=dict(hash_slots=kc.hash_slots, tile_rows=kc.tile_rows,
                                team_lanes=kc.team_lanes, hash_tag_bits=kc.hash_tag_bits,
                                warps_per_block=kc.warps_per_block,
                                warps_per_query=kc.warps_per_query),
                    sweep=table)

    def stats(self):
        s = aqr_stats()
        self._check(self.L.aqr_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in aqr_stats._fields_}

    def merge_topk(self, dists, ids, id_offsets=None, stream=None):
        """Merge per-shard results dists/ids [S, n, k] into the top k by
        (distance, global id); id_offsets [S] are added to shard s's ids."""
        import numpy as np
        import torch
        S, n, k = ids.shape
        off = None if id_offsets is None else np.ascontiguousarray(id_offsets, np.int64)
        if off is not None and off.shape != (S,):
            raise ValueError("id_offsets needs one entry per shard")
        dists, ids = dists.contiguous(), ids.contiguous()
        self._dev(ids, torch.int64, "ids", ndim=3)
        self._dev(dists, torch.float32, "dists", shape=(S, n, k))
        out_i, out_d = self._out(n, k, ids.device)
        self._check(self.L.aqr_merge_topk(self.h, _ptr(dists), _ptr(ids), S, n, k,
                                          None if off is None else off.ctypes.data_as(P),
                                          _ptr(out_i), _ptr(out_d), _stream(stream)))
        return out_i, out_d

    def knn(self, base, q, k, self_ids=None, stream=None):
        import torch
        self._dev(base, torch.float32, "base", ndim=2)
        n, d = base.shape
        self._dev(q, torch.float32, "q", ndim=2)
        if q.shape[1] != d:
            raise ValueError(f"q: {q.shape[1]} columns, base has {d}")
        nq = q.shape[0]
        if self_ids is not None:
            self._dev(self_ids, torch.int64, "self_ids", shape=(nq,))
        ids, dists = self._out(nq, k, q.device)
        self._check(self.L.aqr_bruteforce_knn(self.h, _ptr(base), n, d, _ptr(q), nq, k,
                                              _ptr(self_ids), _ptr(ids), _ptr(dists),
                                              _stream(stream)))
        return ids, dists

    # -- serving ----------------------------------------------------------
    def serve_start(self, max_batch=256, n_streams=4, hbm_budget=0, max_pending=1 << 20,
                    batch_wait_us=50):
        cfg = aqr_serve_config(max_batch, n_streams, hbm_budget, max_pending, batch_wait_us)
        self._check(self.L.aqr_serve_start(self.h, C.byref(cfg)))

    def serve_replay(self, q_np, ks, efs, arrival_us, k_stride=None, timeout_us=60_000_000):
        """Submit request i at arrival_us[i] (open loop, native thread of the
        caller); returns ids [n, k_stride], dists, latency_us [n], batch [n]."""
        import numpy as np
        q = np.ascontiguousarray(q_np, np.float32)
        kk = np.ascontiguousarray(ks, np.int32).reshape(-1)
        ee = np.ascontiguousarray(efs, np.int32).reshape(-1)
        at = np.ascontiguousarray(arrival_us, np.float64).reshape(-1)
        if q.ndim != 2 or (self._d is not None and q.shape[1] != self._d):
            raise ValueError(f"q: shape {q.shape}, expected [n, {self._d}]")
        n = q.shape[0]
        _check_len(kk, n, "ks")
        _check_len(ee, n, "efs")
        _check_len(at, n, "arrival_us")
        k_stride = k_stride or (int(kk.max()) if n else 1)
        ids = np.empty((n, k_stride), np.int64)
        dd = np.empty((n, k_stride), np.float32)
        st = (aqr_request_stats * max(n, 1))()
        self._check(self.L.aqr_serve_replay(self.h, q.ctypes.data_as(P), n, kk.ctypes.data_as(P),
                                            ee.ctypes.data_as(P), at.ctypes.data_as(P), k_stride,
                                            ids.ctypes.data_as(P), dd.ctypes.data_as(P), st,
                                            timeout_us))
        lat = np.array([st[i].latency_us for i in range(n)])
        batch = np.array([st[i].batch_size for i in range(n)])
        return ids, dd, lat, batch

    def submit(self, q_np, k, ef):
        import numpy as np
        q = np.ascontiguousarray(q_np, np.float32).reshape(-1)
        if self._d is not None and q.size != self._d:
            raise ValueError(f"q: {q.size} values, the index has d = {self._d}")
        t = U64()
        self._check(self.L.aqr_submit(self.h, q.ctypes.data_as(P), k, ef, C.byref(t)))
        return t.value

    def poll(self, ticket, k, timeout_us=0):
        """Returns (ids, dists, stats) or None if not ready."""
        import numpy as np
        ids = np.empty(k, np.int64)
        dd = np.empty(k, np.float32)
        st = aqr_request_stats()
        r = self.L.aqr_poll(self.h, ticket, ids.ctypes.data_as(P), dd.ctypes.data_as(P),
                            C.byref(st), timeout_us)
        if r == AQR_ERR_NOT_READY:
            return None
        self._check(r)
        return ids, dd, dict(queue_us=st.queue_us, latency_us=st.latency_us,
                             batch_size=st.batch_size)

    def cancel(self, ticket):
        return self.L.aqr_cancel(self.h, ticket)

    def serve_stop(self):
        self._check(self.L.aqr_serve_stop(self.h))

    def serve_inject_host_fault(self):
        """Test hook: the scheduler thread throws a host exception at its
        next pass (the out-of-host-memory path); no GPU fault."""
        self._check(self.L.aqr_serve_inject_host_fault(self.h))
