"""The arithmetic behind the tensor-core scoring kernel's FP32-accurate
projection, checked on the CPU in numpy (no GPU, no CUDA code involved).

A FP32 value v is split into three pieces p0 + p1 + p2, each rounded to the
MMA input format (bf16, round to nearest even; or TF32, round to nearest with
ties away from zero), every difference being exact in FP32.  The projection
a . b of a pose row a and a record b (4-vectors) is then the sum of six piece
products (a0 b0, a0 b1, a1 b0, a0 b2, a1 b1, a2 b0) per component; each
piece product is exact in FP32, and the dropped products a1 b2, a2 b1, a2 b2
bound the error.  These are the facts the kernel's 1e-5 score tolerance
rests on (the same bar as the FP32 kernel)."""
import numpy as np
import pytest


def bf16(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def tf32(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def split3(v, rnd):
    v = np.asarray(v, np.float32)
    p0 = rnd(v)
    r1 = (v - p0).astype(np.float32)
    p1 = rnd(r1)
    r2 = (r1 - p1).astype(np.float32)
    p2 = rnd(r2)
    return p0, p1, p2, r1, r2


def sample(rng, n):
    # pose-row coefficients ~ f * R + c * R (|.| up to ~2e3) and world coordinates up to ~50 m,
    # with a spread of exponents
    a = (rng.normal(size=(n, 4)) * np.exp(rng.uniform(-3, 7.5, size=(n, 4)))).astype(np.float32)
    b = (rng.normal(size=(n, 4)) * np.exp(rng.uniform(-3, 4, size=(n, 4)))).astype(np.float32)
    b[:, 3] = 1.0
    return a, b


@pytest.mark.parametrize("rnd,bits", [(bf16, 8), (tf32, 11)])
def test_pieces_are_exact_and_fit_the_format(rnd, bits):
    rng = np.random.default_rng(0)
    v = (rng.normal(size=200000) * np.exp(rng.uniform(-20, 20, size=200000))).astype(np.float32)
    p0, p1, p2, r1, r2 = split3(v, rnd)
    v64 = v.astype(np.float64)
    # the differences are exact in FP32
    assert np.array_equal(r1.astype(np.float64), v64 - p0.astype(np.float64))
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - p1.astype(np.float64))
    # every piece has at most `bits` significant bits (it is representable in the MMA format)
    for p in (p0, p1, p2):
        m, _ = np.frexp(p.astype(np.float64))
        scaled = np.ldexp(m, bits)
        assert np.array_equal(scaled, np.round(scaled))
    # three pieces reproduce v to far below one FP32 ulp
    rem = np.abs(v64 - (p0.astype(np.float64) + p1 + p2))
    bound = 2.0 ** (-3 * bits - 1) * np.abs(v64) * 4
    assert np.all(rem <= bound)


@pytest.mark.parametrize("rnd,rel", [(bf16, 2.0 ** -22), (tf32, 2.0 ** -30)])
def test_six_piece_products_give_the_fp32_projection(rnd, rel):
    rng = np.random.default_rng(1)
    a, b = sample(rng, 100000)
    a0, a1, a2, _, _ = split3(a, rnd)
    b0, b1, b2, _, _ = split3(b, rnd)
    terms = [(a0, b0), (a0, b1), (a1, b0), (a0, b2), (a1, b1), (a2, b0)]
    # each piece product is exact in FP32
    for x, y in terms:
        assert np.array_equal((x * y).astype(np.float64), x.astype(np.float64) * y.astype(np.float64))
    approx = sum(x.astype(np.float64) * y.astype(np.float64) for x, y in terms).sum(axis=1)
    exact = (a.astype(np.float64) * b.astype(np.float64)).sum(axis=1)
    scale = np.abs(a.astype(np.float64) * b.astype(np.float64)).sum(axis=1)
    assert np.all(np.abs(approx - exact) <= rel * scale)
    # dropping any of the six terms costs more than FP32 rounding (2^-24 of the scale) somewhere
    for skip in range(6):
        partial = sum(x.astype(np.float64) * y.astype(np.float64) for i, (x, y) in enumerate(terms) if i != skip)
        assert np.max(np.abs(partial.sum(axis=1) - exact) / scale) > 2.0 ** -24
