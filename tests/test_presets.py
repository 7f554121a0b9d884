"""Table 3 presets (Section 4.4): the library's recall-target presets equal
the table, copied into tests/golden/table3_presets.txt with its citation.
Host-only calls: runs without a GPU."""

import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table3_presets.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        band, coarse, rerank, gap, ratio, mult = line.split()
        rows.append(dict(band=band, coarse=int(coarse), rerank=int(rerank), gap=float(gap),
                         ratio=float(ratio), mult=int(mult)))
    return rows


# one target inside each band, and the band edges (a band's upper edge
# belongs to the next row)
@pytest.mark.parametrize("target,row", [(0.5, 0), (0.87, 0), (0.8999, 0), (0.90, 1), (0.93, 1),
                                        (0.95, 2), (0.96, 2), (0.97, 3), (0.99, 3), (1.0, 3)])
def test_preset_equals_table3(target, row):
    from paper_2602_21600_gb300.aqr import params_for_recall
    r = _rows()[row]
    p, ef = params_for_recall(target)
    assert p["n_coarse"] == r["coarse"] and p["n_rerank"] == r["rerank"]
    assert p["m_ef"] == r["mult"]
    assert p["tau_gap"] == np.float32(r["gap"]) and p["tau_ratio"] == np.float32(r["ratio"])
    # search depth ef = N_c * m_ef (Section 3.2, Stage 1)
    assert ef == r["coarse"] * r["mult"]
    assert math.isclose(p["eps"], 1e-6, rel_tol=1e-6)


def test_table3_rows_are_monotone():
    # a higher recall target asks for no less work at every step
    rows = _rows()
    assert len(rows) == 4
    for a, b in zip(rows, rows[1:]):
        assert b["coarse"] > a["coarse"] and b["rerank"] > a["rerank"] and b["mult"] >= a["mult"]
        assert b["gap"] < a["gap"] and b["ratio"] < a["ratio"]


@pytest.mark.parametrize("target", [0.0, -0.5, 1.01, float("nan")])
def test_preset_rejects_targets_outside_0_1(target):
    from paper_2602_21600_gb300.aqr import AQR_ERR_INVALID_ARG, AqrError, params_for_recall
    with pytest.raises(AqrError) as ei:
        params_for_recall(target)
    assert ei.value.status == AQR_ERR_INVALID_ARG
