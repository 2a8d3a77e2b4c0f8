"""The blocked float32 depth layouts (4x4 blocks, imloc_depth_tile4_async;
overlapping 8x4 blocks every 7 x 3 pixels, imloc_depth_halo_async) and the
lift of views stored in them, through the C ABI.

The layout is a storage choice of the map store: a lift of blocked views
must give exactly the outputs of the row-major float32 lift (the same depth
values reach the same arithmetic), and so the oracle's result within the
lift parity bar.  The re-layout itself is checked element by element
against its definition, with image sizes that are not multiples of the
block sizes.
"""
import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import lifted_to_host, matches_to_device, torch, views_to_device

pytestmark = pytest.mark.gpu


def blocked_reference(d, pitch_elems):
    """The layout's definition written out on the CPU (pixels beyond the image are 0)."""
    H, W = d.shape
    out = np.zeros(((H + 3) // 4, pitch_elems), np.float32)
    for y in range(((H + 3) // 4) * 4):
        for x in range(((W + 3) // 4) * 4):
            out[y // 4, (x // 4) * 16 + (y % 4) * 4 + x % 4] = d[y, x] if (y < H and x < W) else 0.0
    return out


@pytest.mark.parametrize("shape", [(7, 10), (16, 16), (33, 17)])
def test_relayout_matches_the_definition(shape):
    t = torch()
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    d = rng.uniform(0.5, 40.0, size=shape).astype(np.float32)
    got = imloc.depth_tile4(t.from_numpy(d).cuda())
    t.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), blocked_reference(d, got.shape[1]))


def test_relayout_rejects_bad_pitches():
    lib = imloc.load()
    t = torch()
    d = t.zeros((8, 10), dtype=t.float32, device="cuda")
    o = t.zeros((2, 64), dtype=t.float32, device="cuda")
    import ctypes as C
    s = C.c_void_p(t.cuda.current_stream().cuda_stream)
    assert lib.imloc_depth_tile4_async(C.c_void_p(d.data_ptr()), 10, 8, 10, C.c_void_p(o.data_ptr()), 40, s) == -1
    assert lib.imloc_depth_tile4_async(C.c_void_p(d.data_ptr()), 10, 8, 10, C.c_void_p(o.data_ptr()), 36, s) == -1
    assert lib.imloc_depth_tile4_async(C.c_void_p(d.data_ptr()), 10, 8, 10, C.c_void_p(o.data_ptr()), 48, s) == 0
    t.cuda.synchronize()


def test_lift_of_blocked_views_equals_row_major_and_the_oracle():
    t = torch()
    ctx = imloc.Context(0, 1 << 30)
    q = synth.config2(3)
    views = views_to_device(q["views"])
    m = matches_to_device(q["matches"])
    ref = lifted_to_host(ctx.lift(views, m))
    tiled = [imloc.tile4_view(v) for v in views]
    got = lifted_to_host(ctx.lift(tiled, m))
    t.cuda.synchronize()
    assert got["n"] == ref["n"] > 40000
    for k in ("x", "y", "X", "Y", "Z", "w", "src"):
        np.testing.assert_array_equal(got[k], ref[k])
    orc = oracle.lift(q["views"], q["matches"])
    np.testing.assert_array_equal(got["src"].astype(np.int64), orc["src"])
    # a batch mixing row-major, blocked and 8-bit views
    mixed = [views[0], tiled[1]] + [dict(v, depth=imloc.depth_encode_log8(v["depth"])) for v in views[2:4]] + tiled[4:]
    ref2 = lifted_to_host(ctx.lift([views[0], views[1]] + mixed[2:4] + views[4:], m))
    got2 = lifted_to_host(ctx.lift(mixed, m))
    t.cuda.synchronize()
    for k in ("x", "y", "X", "Y", "Z", "w", "src"):
        np.testing.assert_array_equal(got2[k], ref2[k])
    assert ctx.device_error() == 0
    ctx.close()


def halo_reference(d, pitch_elems):
    """The overlapping-block layout's definition written out on the CPU:
    block (bx, by) holds pixels 7 bx .. 7 bx + 7, 3 by .. 3 by + 3 (0 beyond the image)."""
    H, W = d.shape
    nby, nbx = (H - 1) // 3 + 1, (W - 1) // 7 + 1
    out = np.zeros((nby, pitch_elems), np.float32)
    for by in range(nby):
        for bx in range(nbx):
            for ly in range(4):
                for lx in range(8):
                    x, y = 7 * bx + lx, 3 * by + ly
                    out[by, bx * 32 + ly * 8 + lx] = d[y, x] if (y < H and x < W) else 0.0
    return out


@pytest.mark.parametrize("shape", [(2, 2), (7, 10), (16, 16), (33, 17), (40, 71)])
def test_halo_relayout_matches_the_definition(shape):
    t = torch()
    rng = np.random.default_rng(shape[0] * 100 + shape[1] + 7)
    d = rng.uniform(0.5, 40.0, size=shape).astype(np.float32)
    got = imloc.depth_halo(t.from_numpy(d).cuda())
    t.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), halo_reference(d, got.shape[1]))


def test_halo_footprints_lie_in_one_block():
    """Every bilinear footprint (top-left pixel i <= W-2, j <= H-2) and every
    lookup pixel reads block (i // 7, j // 3) at local offsets <= (7, 3): the
    four taps are one 128-byte block."""
    W, H = 1024, 768
    i = np.arange(W - 1)
    j = np.arange(H - 1)
    assert np.all(i - 7 * (i // 7) + 1 <= 7) and np.all(j - 3 * (j // 3) + 1 <= 3)
    assert (W - 1) // 7 + 1 == 147 and (H - 1) // 3 + 1 == 256
    x = np.arange(W)
    y = np.arange(H)
    assert np.all(x // 7 < 147) and np.all(y // 3 < 256)


def test_halo_relayout_rejects_bad_pitches():
    lib = imloc.load()
    t = torch()
    d = t.zeros((8, 10), dtype=t.float32, device="cuda")
    o = t.zeros((3, 128), dtype=t.float32, device="cuda")
    import ctypes as C
    s = C.c_void_p(t.cuda.current_stream().cuda_stream)
    # width 10: 2 blocks per row, so the pitch must be a multiple of 32 and >= 64
    assert lib.imloc_depth_halo_async(C.c_void_p(d.data_ptr()), 10, 8, 10, C.c_void_p(o.data_ptr()), 48, s) == -1
    assert lib.imloc_depth_halo_async(C.c_void_p(d.data_ptr()), 10, 8, 10, C.c_void_p(o.data_ptr()), 32, s) == -1
    assert lib.imloc_depth_halo_async(C.c_void_p(d.data_ptr()), 10, 8, 9, C.c_void_p(o.data_ptr()), 64, s) == -1
    assert lib.imloc_depth_halo_async(C.c_void_p(d.data_ptr()), 10, 8, 10, C.c_void_p(o.data_ptr()), 64, s) == 0
    t.cuda.synchronize()


def test_lift_of_halo_views_equals_row_major_and_the_oracle():
    t = torch()
    ctx = imloc.Context(0, 1 << 30)
    q = synth.config2(5)
    views = views_to_device(q["views"])
    m = matches_to_device(q["matches"])
    ref = lifted_to_host(ctx.lift(views, m))
    halo = [imloc.halo_view(v) for v in views]
    got = lifted_to_host(ctx.lift(halo, m))
    t.cuda.synchronize()
    assert got["n"] == ref["n"] > 40000
    for k in ("x", "y", "X", "Y", "Z", "w", "src"):
        np.testing.assert_array_equal(got[k], ref[k])
    orc = oracle.lift(q["views"], q["matches"])
    np.testing.assert_array_equal(got["src"].astype(np.int64), orc["src"])
    # ragged small views (sizes not multiples of 7 or 3), with taps at every border
    rng = np.random.default_rng(9)
    for (H, W) in ((5, 9), (11, 23)):
        depth = rng.uniform(1.0, 20.0, size=(H, W)).astype(np.float32)
        depth[rng.uniform(size=(H, W)) < 0.1] = 0.0
        view = dict(q["views"][0], depth=depth, width=W, height=H)
        n = 4000
        u = np.concatenate([rng.uniform(0.0, W, n), np.repeat(np.arange(W) + 0.5, 4)]).astype(np.float32)
        v = np.concatenate([rng.uniform(0.0, H, n), np.tile(np.array([0.2, 0.7, H - 0.7, H - 0.2]), W)]).astype(np.float32)
        nn = len(u)
        mm = {"q_u": rng.uniform(0, 640, nn).astype(np.float32), "q_v": rng.uniform(0, 480, nn).astype(np.float32),
              "db_u": u, "db_v": v, "conf": np.ones(nn, np.float32),
              "seg_off": np.array([0, nn // 2, nn], np.int64), "seg_view": np.array([0, 0], np.int32),
              "seg_dir": np.array([0, 1], np.int32)}
        dv = views_to_device([view])
        r1 = lifted_to_host(ctx.lift(dv, matches_to_device(mm)))
        r2 = lifted_to_host(ctx.lift([imloc.halo_view(dv[0])], matches_to_device(mm)))
        t.cuda.synchronize()
        assert r1["n"] == r2["n"] > 0
        for k in ("x", "y", "X", "Y", "Z", "w", "src"):
            np.testing.assert_array_equal(r2[k], r1[k])
        np.testing.assert_array_equal(r2["src"].astype(np.int64), oracle.lift([view], mm)["src"])
    assert ctx.device_error() == 0
    ctx.close()
