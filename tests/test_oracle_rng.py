"""Pins for the oracle's seeded weights (Alg. 3: A_wj, zeta_w ~ U(-1,1)).

The generator is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  Its
sequential form is pinned by the published seed-0 outputs; the counter form
used to draw A and zeta is pinned against the sequential form; the uniform
law is pinned statistically."""
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
GAMMA = 0x9E3779B97F4A7C15  # the SplitMix64 increment, from the same paper


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        s, n, h = line.split()
        rows.append((int(s), int(n), int(h, 16)))
    return rows


def test_splitmix64_published_vectors(orc):
    rows = _golden()
    assert rows
    for seed, n, expect in rows:
        assert orc.splitmix64_seq(seed, n)[n - 1] == expect


def test_counter_form_is_position_in_the_sequence(orc):
    for seed in (0, 12345, 2**63 + 7, W.SEED_BASE):
        seq = orc.splitmix64_seq(seed, 64)
        for idx in range(64):
            assert orc.uniform(seed, 0, idx) == (seq[idx] >> 11) * 2.0**-53


def test_stream_offset_is_2_pow_40_positions(orc):
    # Output n of the generator seeded s is output 1 of the generator seeded
    # s + (n - 1) * GAMMA; stream t starts 2^40 * t positions later.
    seed = 987654321
    for idx in (0, 1, 77, 10**6):
        n = (1 << 40) + idx + 1
        shifted = (seed + (n - 1) * GAMMA) % (1 << 64)
        first = orc.splitmix64_seq(shifted, 1)[0]
        assert orc.uniform(seed, 1, idx) == (first >> 11) * 2.0**-53


def test_weights_are_affine_images_of_the_counter_draws(orc):
    cfg = W.config("burgers1d", nx=16, M=7)
    p = orc.problem(cfg)
    A, z = orc.weights(p)
    d = 16
    for w in range(7):
        for j in range(d):
            assert A[w, j] == 2.0 * orc.uniform(cfg["seed"], 0, w * d + j) - 1.0
        assert z[w] == 2.0 * orc.uniform(cfg["seed"], 1, w) - 1.0


def test_weights_are_uniform_on_minus1_1(orc):
    cfg = W.config("diffreact2d", nx=64, ny=64, M=100)
    A, z = orc.weights(orc.problem(cfg))
    a = A.ravel()
    n = a.size
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 4.0 * np.sqrt(1.0 / 3.0 / n)
    assert abs(a.var() - 1.0 / 3.0) < 4.0 * np.sqrt(4.0 / 45.0 / n)
    # rows are uncorrelated
    c = np.corrcoef(A[:10])
    off = c[~np.eye(10, dtype=bool)]
    assert np.abs(off).max() < 5.0 / np.sqrt(A.shape[1])
    assert z.min() >= -1.0 and z.max() < 1.0
