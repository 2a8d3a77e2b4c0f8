"""8-bit log depth codec (ImLoc Sec. 3.3 "Data Compression", Sec. 4.3
"Depth Quantization") through the C ABI against the FP64 oracle.

Bar: codes bit-exact (the encoder decides each code by exact comparisons with
the level midpoints, the oracle by rounding its FP64 log-space position:
they differ only within ~1e-14 of a midpoint, where no float32 lies);
decoded depths equal the oracle's FP64 levels rounded to float32; the lift of
views stored as codes equals the oracle lift of the decoded float32 maps with
the same bar as the float32 lift (indices bit-exact, world points to the
float32 rounding of the kernel's arithmetic).
"""
import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import lifted_to_host, matches_to_device, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = imloc.Context(0, 1 << 30)
    yield c
    c.close()


def special_depths():
    vals = [0.0, -0.0, -1.0, np.nan, np.inf, -np.inf, 1e-45, 1e-30, 0.01, 0.2499999, 0.25, 128.0, 128.00002, 1e6]
    lv = oracle.depth_decode_log8(np.arange(1, 256, dtype=np.uint8))
    vals += list(lv.astype(np.float32))
    for c in range(1, 255):
        mid = 0.25 * 512.0 ** ((c - 0.5) / 254.0)
        f = np.float32(mid)
        vals += [np.nextafter(f, np.float32(0)), f, np.nextafter(f, np.float32(np.inf))]
    return np.array(vals, np.float32)


def test_encode_bit_exact_with_pitch():
    t = torch()
    rng = np.random.default_rng(3)
    H, W = 768, 1024
    d = np.exp(rng.uniform(np.log(0.05), np.log(300.0), (H, W))).astype(np.float32)
    d[rng.random((H, W)) < 0.05] = 0.0
    sp = special_depths()
    d.ravel()[: sp.size] = sp
    # pitched layouts on both sides
    dev = t.zeros((H, W + 37), dtype=t.float32, device="cuda")[:, :W]
    dev.copy_(t.from_numpy(d))
    codes = t.full((H, W + 11), 77, dtype=t.uint8, device="cuda")[:, :W]
    imloc.depth_encode_log8(dev, out=codes)
    t.cuda.synchronize()
    got = codes.cpu().numpy()
    np.testing.assert_array_equal(got, oracle.depth_encode_log8(d))


def test_decode_is_the_oracle_level_in_float32():
    t = torch()
    codes = np.tile(np.arange(256, dtype=np.uint8), (3, 5))
    out = imloc.depth_decode_log8(t.from_numpy(codes).cuda())
    t.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.depth_decode_log8(codes).astype(np.float32))


def encode_views(views):
    """device uint8 code maps of the views (GPU encoder) and the oracle-decoded float32 maps"""
    t = torch()
    dev, host = [], []
    for v in views:
        codes = imloc.depth_encode_log8(t.from_numpy(np.ascontiguousarray(v["depth"], np.float32)).cuda())
        d = dict(v)
        d["depth"] = codes
        dev.append(d)
        h = dict(v)
        h["depth"] = oracle.depth_decode_log8(oracle.depth_encode_log8(v["depth"])).astype(np.float32)
        host.append(h)
    return dev, host


def check(g, ref, views, matches):
    assert g["n"] == len(ref["src"])
    np.testing.assert_array_equal(g["src"].astype(np.int64), ref["src"])
    np.testing.assert_array_equal(g["x"].astype(np.float64), ref["x"])
    np.testing.assert_array_equal(g["w"].astype(np.float64), ref["w"])
    if g["n"] == 0:
        return
    seg_of = np.searchsorted(np.asarray(matches["seg_off"])[1:], ref["src"], side="right")
    vid = np.asarray(matches["seg_view"])[seg_of]
    C = np.stack([-np.asarray(views[v]["R"]).T @ np.asarray(views[v]["t"]) for v in range(len(views))])[vid]
    err = np.linalg.norm(g["Xw"] - ref["X"], axis=1)
    bound = 2e-6 * (np.linalg.norm(ref["X"], axis=1) + 2 * np.linalg.norm(C, axis=1))
    assert np.all(err <= bound), float(np.max(err / bound))


def test_lift_of_log8_views_config2_full_size(ctx):
    q = synth.config2(0)
    dev, host = encode_views(q["views"])
    out = ctx.lift(dev, matches_to_device(q["matches"]))
    torch().cuda.synchronize()
    g = lifted_to_host(out)
    ref = oracle.lift(host, q["matches"])
    assert 40000 < g["n"] < 50000
    check(g, ref, host, q["matches"])
    # the quantized depths move the lifted points by at most the codec's bound (1.24 %) of the depth
    ref32 = oracle.lift(q["views"], q["matches"])
    common = np.intersect1d(ref["src"], ref32["src"])
    assert len(common) > 0.99 * len(ref32["src"])
    assert ctx.device_error() == 0


def test_batch_with_mixed_formats(ctx):
    rng = np.random.default_rng(11)
    qs = [synth.localization_query(rng, n_views=3, matches_per_pair=1500, width=320, height=240, f=260.0) for _ in range(2)]
    t = torch()
    dev_views, host_views = [], []
    for i, q in enumerate(qs):
        if i == 0:
            for v in q["views"]:
                d = dict(v)
                d["depth"] = t.from_numpy(np.ascontiguousarray(v["depth"], np.float32)).cuda()
                dev_views.append(d)
            host_views.append(q["views"])
        else:
            dv, hv = encode_views(q["views"])
            dev_views += dv
            host_views.append(hv)
    # concatenated batch: query 1's segments index views 3..5
    cat = {k: np.concatenate([q["matches"][k] for q in qs]).astype(np.float32) for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    n0 = len(qs[0]["matches"]["q_u"])
    seg_off = np.concatenate([qs[0]["matches"]["seg_off"][:-1], n0 + np.asarray(qs[1]["matches"]["seg_off"])])
    seg_view = np.concatenate([qs[0]["matches"]["seg_view"], 3 + np.asarray(qs[1]["matches"]["seg_view"])])
    seg_dir = np.concatenate([qs[0]["matches"]["seg_dir"], qs[1]["matches"]["seg_dir"]])
    m = {k: t.from_numpy(v).cuda() for k, v in cat.items()}
    m.update(seg_off=seg_off, seg_view=seg_view, seg_dir=seg_dir)
    qb = np.array([0, n0, len(cat["q_u"])], np.int64)
    out, offs = ctx.lift_batch(qb, dev_views, m)
    t.cuda.synchronize()
    offs = offs.cpu().numpy()
    g = lifted_to_host(out, int(offs[-1]))
    for i, q in enumerate(qs):
        ref = oracle.lift(host_views[i], q["matches"])
        sl = slice(int(offs[i]), int(offs[i + 1]))
        gi = {k: (v[sl] if hasattr(v, "__len__") and len(v) == g["n"] else v) for k, v in g.items()}
        gi["n"] = int(offs[i + 1] - offs[i])
        gi["src"] = g["src"][sl] - (0 if i == 0 else n0)
        check(gi, ref, host_views[i], q["matches"])
