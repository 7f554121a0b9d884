"""Element-by-element comparison of the CUDA query path with the oracle.

Bit-exact parts (integer arithmetic, identical decisions): the layer-0 entry
point after the greedy descent, the layer-0 expansion sequence, the Stage-1
candidate list C with its integer distances.

Floating-point parts: Stage-2 (asymmetric) and Stage-3 (exact) distances
are FP32 on the GPU and FP64 in the oracle; each must agree within TOL
relative.  Where FP32 rounding may flip a decision -- the order of two
candidates whose distances tie within the tolerance, the early-termination
test within the tolerance of its threshold -- the GPU's branch is accepted
if it is one the oracle's values allow, and the rest of the pipeline is
then checked by applying the oracle's arithmetic to the GPU's branch.
"""

from __future__ import annotations

import numpy as np

import oracle

TOL = 1e-5  # relative, for FP32 distances against FP64


def _close(a, b, tol=TOL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) <= tol * np.maximum(np.abs(b), 1e-30) + 1e-30


def derived_counts(k, ef, m_ef=3, rerank_pct=40, n_coarse=0, n_rerank=0):
    ef_eff = max(ef, k)
    Nc = n_coarse if n_coarse > 0 else -(-ef_eff // m_ef)
    Nc = min(max(Nc, k), ef_eff)
    Nr = n_rerank if n_rerank > 0 else -(-(Nc * rerank_pct) // 100)
    Nr = min(max(Nr, k), Nc)
    return ef_eff, Nc, Nr


def check_stage1(g, o, nq):
    """GPU trace g and oracle trace o agree bit for bit on Stage 1."""
    np.testing.assert_array_equal(g["l0_entry"].astype(np.int64), o["l0_entry"].astype(np.int64))
    np.testing.assert_array_equal(g["exp_count"], o["exp_count"])
    cap = min(g["exp_seq"].shape[1], o["exp_seq"].shape[1])
    for i in range(nq):
        m = min(int(o["exp_count"][i]), cap)
        np.testing.assert_array_equal(g["exp_seq"][i, :m].astype(np.int64),
                                      o["exp_seq"][i, :m].astype(np.int64), err_msg=f"query {i}")
    np.testing.assert_array_equal(g["c_count"], o["c_count"])
    for i in range(nq):
        nc = int(o["c_count"][i])
        np.testing.assert_array_equal(g["c_ids"][i, :nc].astype(np.int64),
                                      o["c_ids"][i, :nc].astype(np.int64), err_msg=f"query {i}")
        np.testing.assert_array_equal(g["c_dist"][i, :nc].astype(np.int64),
                                      o["c_dist"][i, :nc], err_msg=f"query {i}")


def check_stages_2_3(idx, q, g, o, k, ef, tau_gap=0.010, tau_ratio=1.008, eps=1e-6, m_ef=3,
                     rerank_pct=40, n_coarse=0, n_rerank=0, tol=TOL):
    """Stage 2, early termination, Stage 3 and assembly.  Returns counts of
    the tolerance-band cases that were accepted on the GPU's branch."""
    nq = len(q)
    _, Nc, Nr = derived_counts(k, ef, m_ef, rerank_pct, n_coarse, n_rerank)
    amb = dict(order=0, et=0, final=0)
    for i in range(nq):
        nc = int(o["c_count"][i])
        oid = o["a_ids"][i, :nc].astype(np.int64)
        od = dict(zip(oid.tolist(), o["a_dist"][i, :nc].tolist()))
        gid = g["a_ids"][i, :nc].astype(np.int64)
        gd = g["a_dist"][i, :nc].astype(np.float64)
        assert sorted(gid.tolist()) == sorted(oid.tolist()), f"query {i}: A differs from C"
        ref = np.array([od[v] for v in gid.tolist()])
        assert np.all(_close(gd, ref, tol)), f"query {i}: asymmetric distance off"
        # GPU order must be ascending in the oracle's distances up to the tolerance
        if nc > 1:
            assert np.all(ref[:-1] <= ref[1:] * (1 + 2 * tol) + 1e-30), f"query {i}: A order"
        if not np.array_equal(gid, oid):
            amb["order"] += 1
        # early termination on the oracle's values at the GPU's positions
        et_g = int(g["et"][i])
        if nc > k:
            dk, dk1 = ref[k - 1], ref[k]
            gap = (dk1 - dk) / (dk + eps)
            ratio = dk1 / (dk + eps)
            et_o = int(gap > tau_gap or ratio > tau_ratio)
            if et_g != et_o:
                near = (abs(gap - tau_gap) <= 4 * tol * max(1.0, abs(gap)) + 4 * tol * ratio or
                        abs(ratio - tau_ratio) <= 4 * tol * max(1.0, ratio))
                assert near, f"query {i}: early exit {et_g} vs {et_o} (gap {gap}, ratio {ratio})"
                amb["et"] += 1
        else:
            assert et_g == 0
        ne = min(k, nc) if et_g else min(Nr, nc)
        assert int(g["n_exact"][i]) == ne, f"query {i}: n_exact"
        # assembly on the GPU's branch with the oracle's arithmetic
        ex, asy, _ = oracle.pair_dists(idx["x"], idx["codes"], idx["min"], idx["scale"], q,
                                       np.full(nc, i), gid)
        fin = [(ex[j] if j < ne else asy[j], int(gid[j]), 1 if j < ne else 0) for j in range(nc)]
        fin.sort()
        gi = g["ids"][i].astype(np.int64)
        gdist = g["dists"][i].astype(np.float64)
        gex = g["exact"][i]
        kk = min(k, nc)
        assert len(set(gi[:kk].tolist())) == kk
        for p in range(kk):
            e_d, e_id, e_ex = fin[p]
            assert _close(gdist[p], e_d, tol), f"query {i} pos {p}: {gdist[p]} vs {e_d}"
            if gi[p] != e_id:
                tied = [f for f in fin if _close(f[0], e_d, 2 * tol)]
                assert int(gi[p]) in [t[1] for t in tied], f"query {i} pos {p}: id"
                amb["final"] += 1
            else:
                assert int(gex[p]) == e_ex
        assert np.all(gi[kk:] == -1) and np.all(np.isinf(gdist[kk:]))
    return amb


def to_np(t):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in t.items()}
