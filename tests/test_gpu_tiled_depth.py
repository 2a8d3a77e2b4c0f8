"""The 4x4-blocked float32 depth layout (imloc_depth_tile4_async) and the
lift of views stored in it, through the C ABI.

The layout is a storage choice of the map store: a lift of blocked views
must give exactly the outputs of the row-major float32 lift (the same depth
values reach the same arithmetic), and so the oracle's result within the
lift parity bar.  The re-layout itself is checked element by element
against its definition, with image sizes that are not multiples of 4.
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
