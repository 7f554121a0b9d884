"""Pins for the oracle's quantiser: encode and training (Section 3.1, Alg. 1).

Each check compares the oracle with something other than itself: values
derived by hand (tests/golden/encode_cases.txt), a library routine the step
reduces to (numpy percentiles, a numpy brute-force kNN), closed forms, and
the round-trip bound of an 8-bit uniform quantiser.
"""

import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _encode_cases():
    rows = []
    for line in open(os.path.join(GOLDEN, "encode_cases.txt")):
        line = line.split("#")[0].strip()
        if line:
            x, mn, sc, code = line.split()
            rows.append((float(x), float(mn), float(sc), int(code)))
    return rows


def test_encode_hand_cases():
    for x, mn, sc, code in _encode_cases():
        got = oracle.encode(np.array([[x]], np.float32), np.array([mn], np.float32),
                            np.array([sc], np.float32))
        assert int(got[0, 0]) == code, (x, mn, sc)


def test_encode_round_trip_bound():
    # For x inside [min_j, max_j] the decode code/scale + min is within half
    # a quantisation step of x; outside, within half a step of the clip bound.
    rng = np.random.default_rng(0)
    d = 37
    mn = rng.uniform(-5, 5, d).astype(np.float32)
    width = rng.uniform(0.5, 300, d)
    sc = (255.0 / (width + 1e-6)).astype(np.float32)
    mx = mn.astype(np.float64) + width
    x = (mn + rng.uniform(-0.2, 1.2, (500, d)) * width).astype(np.float32)
    codes = oracle.encode(x, mn, sc).astype(np.float64)
    dec = codes / sc.astype(np.float64) + mn.astype(np.float64)
    clipped = np.clip(x.astype(np.float64), mn.astype(np.float64), mx)
    step = 1.0 / sc.astype(np.float64)
    err = np.abs(dec - clipped)
    # FP32 evaluation of (x - min) * scale adds a few ulps of the code value.
    slack = 1e-4 * step
    assert np.all(err <= step / 2 + slack)


def test_encode_identity_on_full_range_integers():
    # Integer data spanning exactly [0, 255] in every dimension, with no
    # percentile trimming (P_max = 0): min = 0, max = 255, scale =
    # 255 / (255 + 1e-6), and every code equals the data value.
    rng = np.random.default_rng(1)
    n, d = 400, 6
    x = rng.integers(0, 256, (n, d)).astype(np.float32)
    x[0] = 0
    x[1] = 255
    P = oracle.train(x, p_max=0.0, M0=16, ef0=100)
    assert np.all(P["min"] == 0) and np.all(P["max"] == 255)
    np.testing.assert_array_equal(P["scale"], np.float32(255.0 / (255.0 + 1e-6)))
    codes = oracle.encode(x, P["min"], P["scale"])
    np.testing.assert_array_equal(codes, x.astype(np.uint8))


def _knn_density(x, ids, kd=10):
    # Plain numpy brute force: squared L2 to every other point, kd smallest.
    x = x.astype(np.float64)
    out = []
    for i in ids:
        dd = ((x - x[i]) ** 2).sum(1)
        dd[i] = np.inf
        out.append(1.0 / (np.sort(dd)[:kd].mean() + 1e-6))
    return np.array(out)


def test_density_matches_numpy_bruteforce():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(300, 5)).astype(np.float32) * rng.uniform(0.1, 3, (300, 1)).astype(np.float32)
    ids = np.arange(0, 300, 7)
    got = oracle.density(x, ids)
    np.testing.assert_allclose(got, _knn_density(x, ids), rtol=1e-12)


def test_density_on_a_line_by_hand():
    # 12 points at 0..11 on a line: point 0's 10 nearest others are 1..10,
    # mean squared distance (1+4+...+100)/10 = 38.5.
    x = np.arange(12, dtype=np.float32)[:, None]
    rho = oracle.density(x, np.array([0, 5]))
    assert rho[0] == pytest.approx(1.0 / (38.5 + 1e-6), rel=1e-15)
    # Point 5: others at distances 1,1,2,2,3,3,4,4,5,5 (6 is at 6, dropped).
    assert rho[1] == pytest.approx(1.0 / ((2 * (1 + 4 + 9 + 16 + 25)) / 10 + 1e-6), rel=1e-15)


def test_train_closed_forms_small():
    rng = np.random.default_rng(3)
    n, d = 800, 9
    # two clusters of very different spread -> large delta
    x = np.concatenate([rng.normal(0, 0.2, (400, d)), rng.normal(20, 5.0, (400, d))]).astype(np.float32)
    p_max, M0, ef0 = 0.05, 16, 200
    P = oracle.train(x, p_max=p_max, M0=M0, ef0=ef0)
    rho = _knn_density(x, np.arange(n))
    delta = (rho.max() - rho.min()) / (rho.max() + 1e-6)
    assert P["delta"] == pytest.approx(delta, rel=1e-12)
    assert 0.0 <= P["delta"] <= 1.0
    assert P["P_l"] == pytest.approx(delta * p_max, rel=1e-12)
    assert P["P_h"] == pytest.approx(1 - delta * p_max, rel=1e-12)
    lo = np.percentile(x.astype(np.float64), 100 * P["P_l"], axis=0, method="linear")
    hi = np.percentile(x.astype(np.float64), 100 * P["P_h"], axis=0, method="linear")
    np.testing.assert_array_equal(P["min"], lo.astype(np.float32))
    np.testing.assert_array_equal(P["max"], hi.astype(np.float32))
    sc = (255.0 / (hi.astype(np.float32).astype(np.float64) - lo.astype(np.float32).astype(np.float64) + 1e-6)).astype(np.float32)
    np.testing.assert_array_equal(P["scale"], sc)
    # The weights w_j = mean density do not depend on j, so eta = 0 and
    # s_dist reduces to the RMS range over 255.
    assert P["eta"] == 0.0
    rng_ = P["max"].astype(np.float64) - P["min"].astype(np.float64)
    assert P["s_dist"] == pytest.approx(math.sqrt((rng_ ** 2).sum() / (d * 255.0 ** 2)), rel=1e-12)
    assert P["w"] == pytest.approx(rho.mean(), rel=1e-12)
    assert P["M_i"] == math.floor(M0 * (1 + delta))
    assert P["ef_c"] == ef0


def test_train_uniform_density_gives_delta_near_zero():
    # A regular grid has equal density everywhere except at the border;
    # on a ring every point has the same neighbourhood -> delta = 0 exactly.
    t = np.arange(64) * (2 * np.pi / 64)
    x = np.stack([np.cos(t), np.sin(t)], 1).astype(np.float32) * 10
    P = oracle.train(x, p_max=0.01, M0=16, ef0=100)
    assert P["delta"] < 1e-5
    assert P["M_i"] == 16


def test_train_uses_sample_above_ten_thousand():
    rng = np.random.default_rng(4)
    n, d = 10_050, 3
    x = rng.normal(size=(n, d)).astype(np.float32)
    x[: n // 2] *= 0.1
    sample = np.sort(rng.choice(n, 500, replace=False))
    P = oracle.train(x, sample, p_max=0.01, M0=8, ef0=50)
    rho = _knn_density(x, sample)
    assert P["rho_bar"] == pytest.approx(rho.mean(), rel=1e-12)
    assert P["delta"] == pytest.approx((rho.max() - rho.min()) / (rho.max() + 1e-6), rel=1e-12)
    # unsampled points take rho_bar, so the weight equals rho_bar
    assert P["w"] == pytest.approx(rho.mean(), rel=1e-12)


def test_levels_distribution_and_boundaries():
    M = 16
    # exact boundaries: U just above 1/M -> level 0, just below -> 1
    U = np.array([1.0, 1.0 / M * (1 + 1e-12), 1.0 / M * (1 - 1e-12), 1.0 / M ** 2 * (1 - 1e-12)])
    np.testing.assert_array_equal(oracle.levels(U, M), [0, 0, 1, 2])
    # P(level >= l) = M^-l
    rng = np.random.default_rng(5)
    lv = oracle.levels(1.0 - rng.random(400_000), M)
    for l in (1, 2, 3):
        frac = (lv >= l).mean()
        assert frac == pytest.approx(M ** -l, rel=0.1 if l < 3 else 0.3)


def test_batch_schedule_by_hand():
    # div 4, max 3: node 0 alone; then b = min(max(1, s // 4), 3)
    st = oracle.batch_schedule(30, 4, 3)
    assert list(st) == [0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 15, 18, 21, 24, 27, 30]
    assert list(oracle.batch_schedule(5, 4, 1)) == [0, 1, 2, 3, 4, 5]
