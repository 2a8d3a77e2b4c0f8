"""Pins of the oracle's 8-bit log depth codec (ImLoc Sec. 3.3 "Data
Compression": depth clipped to [0.25 m, 128 m] and quantized in log space with
256 levels; Sec. 4.3 "Depth Quantization": under 1.4 % relative error).

Reading (the paper does not spell out the level placement or the marker of a
pixel without depth): code 0 = no depth, codes 1..255 are 255 log-uniform
levels from 0.25 m to 128 m, encoding rounds to the nearest level in log space
with ties upward.  Half a level step bounds the relative error of an
in-range depth: 512^(1/508) - 1 = 1.2357 %.
"""
import numpy as np

import oracle

BOUND = 512.0 ** (1.0 / 508.0) - 1.0


def test_levels_and_special_values():
    dec = oracle.depth_decode_log8(np.arange(256, dtype=np.uint8))
    assert dec[0] == 0.0
    assert dec[1] == 0.25 and dec[255] == 128.0
    # log-uniform: a constant ratio 512^(1/254) between neighbouring levels
    np.testing.assert_allclose(dec[2:] / dec[1:-1], 512.0 ** (1.0 / 254.0), rtol=1e-13)
    d = np.array([0.0, -1.0, np.nan, np.inf, -np.inf, 0.01, 0.25, 128.0, 1e6, 1e-30], np.float32)
    assert list(oracle.depth_encode_log8(d)) == [0, 0, 0, 0, 0, 1, 1, 255, 255, 1]


def test_every_level_encodes_to_itself():
    lv = oracle.depth_decode_log8(np.arange(1, 256, dtype=np.uint8)).astype(np.float32)
    assert (oracle.depth_encode_log8(lv) == np.arange(1, 256)).all()


def test_nearest_level_in_log_space_by_brute_force():
    rng = np.random.default_rng(0)
    d = np.exp(rng.uniform(np.log(0.25), np.log(128.0), 20000)).astype(np.float32)
    codes = oracle.depth_encode_log8(d)
    levels = oracle.depth_decode_log8(np.arange(1, 256, dtype=np.uint8))
    dist = np.abs(np.log(d.astype(np.float64))[:, None] - np.log(levels)[None, :])
    assert (codes == 1 + np.argmin(dist, axis=1)).all()


def test_relative_error_bound_and_the_papers_claim():
    d = np.exp(np.linspace(np.log(0.25), np.log(128.0), 2_000_001)).astype(np.float32)
    d = d[(d >= 0.25) & (d <= 128.0)]
    err = np.abs(oracle.depth_decode_log8(oracle.depth_encode_log8(d)) - d) / d
    assert err.max() <= BOUND * (1 + 1e-6)
    assert err.max() >= 0.999 * BOUND  # reached next to a level midpoint
    assert BOUND < 0.014               # "less than 1.4% relative quantization error" (Sec. 4.3)


def test_clipping_and_monotonicity():
    d = np.sort(np.exp(np.random.default_rng(1).uniform(np.log(0.01), np.log(1000.0), 50000))).astype(np.float32)
    c = oracle.depth_encode_log8(d).astype(int)
    assert (np.diff(c) >= 0).all()
    assert (c[d <= 0.25] == 1).all() and (c[d >= 128.0] == 255).all()
    assert set(np.unique(c)) == set(range(1, 256))


def test_midpoints_round_up():
    """The float32 values on either side of the log-space midpoint between
    codes c and c+1 encode to c and c+1."""
    for c in range(1, 255):
        mid = 0.25 * 512.0 ** ((c - 0.5) / 254.0)
        f = np.float32(mid)
        if float(f) >= mid:
            up, dn = f, np.nextafter(f, np.float32(0))
        else:
            dn, up = f, np.nextafter(f, np.float32(np.inf))
        got = oracle.depth_encode_log8(np.array([dn, up], np.float32))
        assert list(got) == [c, c + 1], c
