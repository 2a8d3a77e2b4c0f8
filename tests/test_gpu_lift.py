"""GPU lift kernel (through the C ABI) against the FP64 oracle.

Bar: kept/dropped decisions and source indices bit-exact (the threshold and
depth-validity decisions are taken in float32 on both sides); x, y, w are
copies and must be identical; world points agree to the float32 rounding of
the kernel's arithmetic: |dX| <= 2e-6 (|X_w| + 2 |C|), C the camera centre
(about 8 float32 roundings of magnitude |X_c| + |C| along the chain
bilinear -> back-projection -> rotation -> translation).
"""
import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import check_lift, lifted_to_host, matches_to_device, torch, views_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = imloc.Context(0, 1 << 30)
    yield c
    c.close()


def test_lift_config2_full_size(ctx):
    q = synth.config2(0)
    out = ctx.lift(views_to_device(q["views"]), matches_to_device(q["matches"]))
    torch().cuda.synchronize()
    g = lifted_to_host(out)
    ref = oracle.lift(q["views"], q["matches"])
    assert 40000 < g["n"] < 50000
    check_lift(g, ref, q["views"], q["matches"])
    assert ctx.device_error() == 0


@pytest.mark.parametrize("seed,n_views,per_pair", [(1, 1, 7), (2, 3, 1023), (3, 4, 2049), (4, 2, 5000)])
def test_lift_ragged_sizes(ctx, seed, n_views, per_pair):
    rng = np.random.default_rng(seed)
    q = synth.localization_query(rng, n_views=n_views, matches_per_pair=per_pair, width=320, height=240, f=260.0)
    out = ctx.lift(views_to_device(q["views"]), matches_to_device(q["matches"]))
    g = lifted_to_host(out)
    check_lift(g, oracle.lift(q["views"], q["matches"]), q["views"], q["matches"])


def test_lift_edge_values(ctx):
    """Filters at their exact boundaries: confidence == 0.05f, border taps,
    NaN / inf / zero / negative depth, NaN coordinates, empty segments."""
    H, W = 6, 9
    depth = np.full((H, W), 5.0, np.float32)
    depth[2, 3] = 0.0
    depth[4, 7] = np.nan
    depth[0, 8] = np.inf
    depth[5, 0] = -2.0
    view = dict(depth=depth, fx=100.0, fy=90.0, cx=4.5, cy=3.0, R=np.eye(3), t=np.array([0.1, -0.2, 0.3]))
    c05 = np.float32(0.05)
    above = np.nextafter(c05, np.float32(1))
    pts = []
    for dirn in (0, 1):
        for u in (-0.1, 0.0, 0.49, 0.5, 3.5, 4.0, 8.49, 8.5, 8.99, 9.0, np.nan):
            for v in (0.5, 2.5, 5.49, 5.5):
                for c in (c05, above, 0.9):
                    pts.append((dirn, u, v, c))
    n = len(pts)
    dirs = np.array([p[0] for p in pts])
    order = np.argsort(dirs, kind="stable")
    pts = [pts[i] for i in order]
    n0 = int(np.sum(dirs == 0))
    m = dict(q_u=np.arange(n, dtype=np.float32), q_v=np.ones(n, np.float32),
             db_u=np.array([p[1] for p in pts], np.float32), db_v=np.array([p[2] for p in pts], np.float32),
             conf=np.array([p[3] for p in pts], np.float32),
             seg_off=np.array([0, 0, n0, n0, n], np.int64), seg_view=np.array([0, 0, 0, 0], np.int32),
             seg_dir=np.array([1, 0, 0, 1], np.int32))
    out = ctx.lift(views_to_device([view]), matches_to_device(m))
    g = lifted_to_host(out)
    ref = oracle.lift([view], m)
    assert 0 < g["n"] < n
    check_lift(g, ref, [view], m)


def test_lift_empty_and_all_filtered(ctx):
    depth = np.ones((4, 4), np.float32)
    view = dict(depth=depth, fx=10.0, fy=10.0, cx=2.0, cy=2.0, R=np.eye(3), t=np.zeros(3))
    t = torch()
    for n in (0, 5):
        m = dict(q_u=np.zeros(n, np.float32), q_v=np.zeros(n, np.float32), db_u=np.ones(n, np.float32),
                 db_v=np.ones(n, np.float32), conf=np.zeros(n, np.float32),
                 seg_off=np.array([0, n], np.int64), seg_view=np.array([0], np.int32), seg_dir=np.array([1], np.int32))
        md = matches_to_device(m)
        out = imloc.alloc_corr(max(n, 1))
        out["count"].fill_(-1)
        ctx.lift(views_to_device([view]), md, out=out)
        assert int(out["count"].item()) == 0


def test_lift_batch_offsets(ctx):
    """Several queries (one empty) in one launch: per-query offsets and
    contents equal the single-query lifts."""
    rng = np.random.default_rng(9)
    qs = [synth.localization_query(rng, n_views=k, matches_per_pair=p, width=256, height=200, f=220.0)
          for k, p in ((2, 3001), (1, 5), (3, 777))]
    views, qb = [], [0]
    cat = {k: [] for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    seg_off, seg_view, seg_dir = [0], [], []
    order = [0, None, 1, 2]  # None: an empty query
    for item in order:
        if item is None:
            qb.append(qb[-1])
            continue
        q = qs[item]
        m = q["matches"]
        base_v = len(views)
        views += q["views"]
        for k in cat:
            cat[k].append(m[k])
        for s in range(len(m["seg_view"])):
            seg_off.append(qb[-1] + int(m["seg_off"][s + 1]))
            seg_view.append(base_v + int(m["seg_view"][s]))
            seg_dir.append(int(m["seg_dir"][s]))
        qb.append(qb[-1] + int(m["seg_off"][-1]))
    big = {k: np.concatenate(v) for k, v in cat.items()}
    big.update(seg_off=np.array(seg_off, np.int64), seg_view=np.array(seg_view, np.int32),
               seg_dir=np.array(seg_dir, np.int32))
    out, offs = ctx.lift_batch(qb, views_to_device(views), matches_to_device(big))
    total = int(out["count"].item())
    offs = offs.cpu().numpy()
    assert offs[0] == 0 and offs[-1] == total
    g_all = lifted_to_host(out, total)
    qi = 0
    for pos, item in enumerate(order):
        a, b = offs[pos], offs[pos + 1]
        if item is None:
            assert a == b
            continue
        q = qs[item]
        ref = oracle.lift(q["views"], q["matches"])
        g = {k: v[a:b] for k, v in g_all.items() if k != "n"}
        g["n"] = b - a
        check_lift(g, ref, q["views"], q["matches"], src_base=qb[pos])


def test_lift_many_small_segments(ctx):
    """Tiles that touch more than 8 segments (here ~200 per tile of 1,024
    matches: every view's segment cut into runs of 5) take the kernel's
    per-match segment search instead of the staged tile table; the result
    is the oracle's either way, and the same as the coarse segmentation."""
    q = synth.localization_query(np.random.default_rng(9), n_views=4, matches_per_pair=3001, width=320, height=240,
                                 f=260.0)
    m = dict(q["matches"])
    so, sv, sd = np.asarray(m["seg_off"]), np.asarray(m["seg_view"]), np.asarray(m["seg_dir"])
    off, view, dirn = [], [], []
    for s in range(len(sv)):
        for b in range(int(so[s]), int(so[s + 1]), 5):
            off.append(b); view.append(int(sv[s])); dirn.append(int(sd[s]))
    fine = dict(m, seg_off=np.array(off + [int(so[-1])], np.int64), seg_view=np.array(view, np.int32),
                seg_dir=np.array(dirn, np.int32))
    assert len(view) > 2000
    views = views_to_device(q["views"])
    g = lifted_to_host(ctx.lift(views, matches_to_device(fine)))
    check_lift(g, oracle.lift(q["views"], fine), q["views"], fine)
    coarse = lifted_to_host(ctx.lift(views, matches_to_device(m)))
    for k in ("x", "y", "X", "Y", "Z", "w", "src"):
        np.testing.assert_array_equal(g[k], coarse[k])
