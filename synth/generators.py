"""Gaussian-mixture vector sets, level draws and density samples.

Every stream is numpy's PCG64 seeded with a fixed integer, so the same call
gives the same bytes on x86 and Arm.  The mixture laws stand in for the
shapes of the paper's benchmark sets (Section 4.1, Table 1): SIFT-like
non-negative integer descriptors, GIST-like wide vectors with very uneven
cluster spreads, Fashion-MNIST-like 8-bit images with blank background,
GloVe-like signed word embeddings, and unit-norm embeddings.  No record of any public dataset
is reproduced; all values are drawn here.

Seeds: mixture parameters and base vectors 1234, queries 4321, HNSW level
uniforms 7, density sample 11 (the defaults of ``workload``).
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Mixture:
    """Parameters of an isotropic Gaussian mixture with uniform weights.

    kind: "box" (means U[lo,hi]^d, per-component sigma given), "pixel"
    (box means with a random share of the dimensions set to 0), "gauss"
    (means N(0, mean_sd^2 I)) or "sphere" (means N(0,I) normalised, fixed
    sigma, samples renormalised).
    """

    kind: str
    means: np.ndarray  # [n_comp, d] float32
    sigmas: np.ndarray  # [n_comp] float32
    clip: tuple | None = None  # (lo, hi) clip after sampling
    integer: bool = False  # round to integers after clipping
    unit_norm: bool = False  # renormalise every sample to unit L2 norm


def make_mixture(
    n_comp: int,
    d: int,
    seed: int,
    *,
    kind: str = "box",
    mean_lo: float = 0.0,
    mean_hi: float = 100.0,
    sigma_lo: float = 2.0,
    sigma_hi: float = 10.0,
    sigma_log_spread: float | None = None,
    sphere_sigma: float = 0.05,
    blank_frac: float = 0.5,
    mean_sd: float = 0.4,
    clip: tuple | None = None,
    integer: bool = False,
) -> Mixture:
    """Draw mixture parameters from PCG64(seed).

    box: means ~ U[mean_lo, mean_hi]^d; sigma_c ~ U[sigma_lo, sigma_hi], or,
    when ``sigma_log_spread`` = s is given, sigma_c = s**u with u ~ U[0,1]
    (so sigmas span a factor s between dense and sparse clusters).
    pixel: box means, then each mean coordinate is set to 0 with probability
    blank_frac (a background shared by the component's samples); sigma_c ~
    U[sigma_lo, sigma_hi].
    gauss: means ~ N(0, mean_sd^2 I); sigma_c ~ U[sigma_lo, sigma_hi].
    sphere: means ~ N(0, I) normalised to unit length, sigma = sphere_sigma.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "box":
        means = rng.uniform(mean_lo, mean_hi, size=(n_comp, d)).astype(np.float32)
        if sigma_log_spread is None:
            sig = rng.uniform(sigma_lo, sigma_hi, size=n_comp)
        else:
            sig = np.power(float(sigma_log_spread), rng.uniform(0.0, 1.0, size=n_comp))
        return Mixture("box", means, sig.astype(np.float32), clip, integer, False)
    if kind == "pixel":
        means = rng.uniform(mean_lo, mean_hi, size=(n_comp, d))
        means[rng.random((n_comp, d)) < blank_frac] = 0.0
        sig = rng.uniform(sigma_lo, sigma_hi, size=n_comp)
        return Mixture("pixel", means.astype(np.float32), sig.astype(np.float32), clip, integer,
                       False)
    if kind == "gauss":
        means = rng.normal(0.0, mean_sd, size=(n_comp, d))
        sig = rng.uniform(sigma_lo, sigma_hi, size=n_comp)
        return Mixture("gauss", means.astype(np.float32), sig.astype(np.float32), clip, integer,
                       False)
    if kind == "sphere":
        m = rng.standard_normal((n_comp, d))
        m /= np.linalg.norm(m, axis=1, keepdims=True)
        sig = np.full(n_comp, sphere_sigma, dtype=np.float32)
        return Mixture("sphere", m.astype(np.float32), sig, None, False, True)
    raise ValueError(f"unknown mixture kind {kind!r}")


def sample_mixture(mix: Mixture, n: int, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """Draw n float32 vectors [n, d] from ``mix`` with PCG64(seed).

    Component ids are uniform; each sample is mean + sigma * N(0, I), then
    clipped / rounded / renormalised as the mixture says.  Generated in
    chunks so that large sets do not need float64 temporaries.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_comp, d = mix.means.shape
    out = np.empty((n, d), dtype=np.float32)
    comp = rng.integers(0, n_comp, size=n)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        c = comp[s:e]
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        v = mix.means[c] + z * mix.sigmas[c][:, None]
        if mix.clip is not None:
            np.clip(v, mix.clip[0], mix.clip[1], out=v)
        if mix.integer:
            np.rint(v, out=v)
        if mix.unit_norm:
            v /= np.linalg.norm(v, axis=1, keepdims=True)
        out[s:e] = v
    return out


def level_uniforms(n: int, seed: int = 7) -> np.ndarray:
    """n float64 draws from U(0, 1] (never 0), one per base vector, in id order.

    HNSW assigns each inserted element a random top layer; the draw itself is
    made here and passed to both implementations as an input.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    return 1.0 - rng.random(n)  # random() is in [0, 1)


def density_sample(n: int, n_s: int = 5000, seed: int = 11) -> np.ndarray:
    """min(n_s, n) distinct ids drawn without replacement, sorted ascending (int64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = min(n_s, n)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


# Named workloads.  Sizes and laws follow the five synthetic configurations
# the query path is measured on; "small" variants keep the same law with
# fewer points so that CPU tests finish quickly.
WORKLOADS = {
    # 10,000 x 128 float32, 32 components, means U[0,100], sigma U[2,10].
    "gmm10k_d128": dict(n=10_000, d=128, n_comp=32, nq=100, mix=dict(kind="box"),
                        M0=16, ef0=100, k=10, ef=64),
    # 1,000,000 x 128, 256 components, clipped to [0,255] and rounded (SIFT-like).
    "gmm1m_d128_int": dict(n=1_000_000, d=128, n_comp=256, nq=10_000,
                           mix=dict(kind="box", clip=(0.0, 255.0), integer=True),
                           M0=16, ef0=200, k=10, ef=64),
    # 1,000,000 x 960, 512 components, sigma spread 100x (GIST-like shape).
    "gmm1m_d960_spread": dict(n=1_000_000, d=960, n_comp=512, nq=1_000,
                              mix=dict(kind="box", sigma_log_spread=100.0),
                              M0=32, ef0=200, k=100, ef=256),
    # 1,000,000 x 768 unit-norm embeddings, 1,024 components (serving load).
    "sphere1m_d768": dict(n=1_000_000, d=768, n_comp=1024, nq=10_000,
                          mix=dict(kind="sphere"), M0=16, ef0=200, k=10, ef=128),
    # 60,000 x 784 8-bit images (Fashion-MNIST shape, Table 1): 500
    # prototype images with half of each blank, sigma U[10, 25], clipped to
    # [0,255] and rounded.
    "pix60k_d784_int": dict(n=60_000, d=784, n_comp=500, nq=10_000,
                            mix=dict(kind="pixel", mean_hi=255.0, sigma_lo=10.0, sigma_hi=25.0,
                                     clip=(0.0, 255.0), integer=True),
                            M0=16, ef0=200, k=10, ef=64),
    # 100,000 x 300 signed embeddings (GloVe-300D shape, Table 1): 1,000
    # components, means N(0, 0.4^2), sigma U[0.15, 0.35].
    "emb100k_d300": dict(n=100_000, d=300, n_comp=1000, nq=10_000,
                         mix=dict(kind="gauss", sigma_lo=0.15, sigma_hi=0.35),
                         M0=16, ef0=200, k=10, ef=64),
    # 10,000,000 x 96 unit-norm, 4,096 components.
    "sphere10m_d96": dict(n=10_000_000, d=96, n_comp=4096, nq=100_000,
                          mix=dict(kind="sphere"), M0=16, ef0=200, k=10, ef=64),
}


def workload(name: str, *, n: int | None = None, nq: int | None = None,
             seed_data: int = 1234, seed_query: int = 4321, seed_levels: int = 7,
             seed_sample: int = 11) -> dict:
    """Materialise a named workload (optionally with fewer points / queries).

    Returns dict(x, q, U, sample, and the workload's scalar parameters).
    """
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = n
    if nq is not None:
        w["nq"] = nq
    mix = make_mixture(w["n_comp"], w["d"], seed_data, **w["mix"])
    w["x"] = sample_mixture(mix, w["n"], seed_data + 1)
    w["q"] = sample_mixture(mix, w["nq"], seed_query)
    w["U"] = level_uniforms(w["n"], seed_levels)
    w["sample"] = density_sample(w["n"], 5000, seed_sample)
    w["name"] = name
    return w
