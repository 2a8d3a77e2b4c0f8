"""The allocation-free lift (imloc_lift_noalloc_async) against the regular
lift (imloc_lift_async), through the C ABI.

The allocation-free entry point exists for callers that cannot allocate
device memory: code that runs inside a memory pool or budget owned by another
component, processes that hand all device memory to other parts up front, and
callers that must not create a context (creating one allocates its
workspace).  It keeps its scratch in a fixed array inside the library, so
two calls in a row must each start from a clean scan state; the tests make
such calls on different inputs (float32 views, and a mix of float32 and
8-bit log views) and compare each with the regular lift and with the oracle.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

pytestmark = pytest.mark.gpu


def _to_device(q):
    import torch

    views = []
    for v in q["views"]:
        d = dict(v)
        d["depth"] = torch.from_numpy(np.ascontiguousarray(v["depth"])).cuda()
        views.append(d)
    m = {k: torch.from_numpy(q["matches"][k]).cuda() for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    m.update({k: q["matches"][k] for k in ("seg_off", "seg_view", "seg_dir")})
    return views, m


def _host(out):
    n = int(out["count"].item())
    return n, {k: out[k][:n].cpu().numpy() for k in ("x", "y", "X", "Y", "Z", "w", "src")}


def test_noalloc_lift_equals_regular_lift_on_two_calls_in_a_row():
    import torch

    lib = imloc.load()
    torch.cuda.set_device(0)
    ctx = imloc.Context(0, 256 << 20)
    stream = torch.cuda.current_stream()
    for seed, views_n, per_pair in ((21, 3, 3001), (22, 5, 2047)):
        q = synth.localization_query(np.random.default_rng(seed), n_views=views_n, matches_per_pair=per_pair,
                                     width=320, height=240, f=260.0)
        views, m = _to_device(q)
        n_in = int(q["matches"]["seg_off"][-1])
        ref = ctx.lift(views, m)
        n_ref, ref_h = _host(ref)

        out = imloc.alloc_corr(n_in)
        out["count"].fill_(-1)
        vs = imloc._views_struct(views)
        ms, keep = imloc._matches_struct(m)
        cs = imloc._corr_struct(out)
        rc = lib.imloc_lift_noalloc_async(vs, len(views), C.byref(ms), C.byref(cs), C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.imloc_status_str(rc)
        torch.cuda.synchronize()
        n_got, got = _host(out)
        assert n_got == n_ref > 0
        np.testing.assert_array_equal(got["src"], ref_h["src"])
        for k in ("x", "y", "w"):
            np.testing.assert_array_equal(got[k], ref_h[k])
        # same tolerance as the lift parity tests (the kernel is the same, so
        # the values are expected to be identical)
        Xg = np.stack([got["X"], got["Y"], got["Z"]], 1).astype(np.float64)
        Xr = np.stack([ref_h["X"], ref_h["Y"], ref_h["Z"]], 1).astype(np.float64)
        assert np.all(np.linalg.norm(Xg - Xr, axis=1) <= 2e-6 * (np.linalg.norm(Xr, axis=1) + 1.0))
    ctx.close()


def _noalloc(lib, views, m, n_in, stream):
    out = imloc.alloc_corr(n_in)
    out["count"].fill_(-1)
    vs = imloc._views_struct(views)
    ms, keep = imloc._matches_struct(m)
    cs = imloc._corr_struct(out)
    rc = lib.imloc_lift_noalloc_async(vs, len(views), C.byref(ms), C.byref(cs), C.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.imloc_status_str(rc)
    return out


def test_noalloc_lift_with_log8_and_float32_views_against_the_oracle():
    # views of both depth formats in one call: 8-bit log codes (decoded in the
    # fetch) and float32; compared with the oracle's lift of the decoded maps
    # (indices bit-exact, points within the lift parity bound) and with the
    # regular lift (identical)
    import torch

    lib = imloc.load()
    torch.cuda.set_device(0)
    ctx = imloc.Context(0, 256 << 20)
    stream = torch.cuda.current_stream()
    q = synth.localization_query(np.random.default_rng(23), n_views=4, matches_per_pair=2500, width=320, height=240,
                                 f=260.0)
    views, m = _to_device(q)
    host = []
    for i, v in enumerate(q["views"]):
        h = dict(v)
        if i % 2 == 1:
            views[i]["depth"] = imloc.depth_encode_log8(views[i]["depth"])
            h["depth"] = oracle.depth_decode_log8(oracle.depth_encode_log8(v["depth"])).astype(np.float32)
        host.append(h)
    n_in = int(q["matches"]["seg_off"][-1])
    for _ in range(2):
        out = _noalloc(lib, views, m, n_in, stream)
        torch.cuda.synchronize()
        n_got, got = _host(out)
        ref = oracle.lift(host, q["matches"])
        assert n_got == len(ref["src"]) > 0
        np.testing.assert_array_equal(got["src"].astype(np.int64), ref["src"])
        np.testing.assert_array_equal(got["x"].astype(np.float64), ref["x"])
        np.testing.assert_array_equal(got["w"].astype(np.float64), ref["w"])
        seg_of = np.searchsorted(np.asarray(q["matches"]["seg_off"])[1:], ref["src"], side="right")
        vid = np.asarray(q["matches"]["seg_view"])[seg_of]
        Cc = np.stack([-np.asarray(v["R"]).T @ np.asarray(v["t"]) for v in q["views"]])[vid]
        Xg = np.stack([got["X"], got["Y"], got["Z"]], 1).astype(np.float64)
        bound = 2e-6 * (np.linalg.norm(ref["X"], axis=1) + 2 * np.linalg.norm(Cc, axis=1))
        assert np.all(np.linalg.norm(Xg - ref["X"], axis=1) <= bound)
        reg = ctx.lift(views, m)
        n_ref, ref_h = _host(reg)
        assert n_ref == n_got
        for k in ("x", "y", "X", "Y", "Z", "w", "src"):
            np.testing.assert_array_equal(got[k], ref_h[k])
    ctx.close()


def test_noalloc_lift_is_refused_during_stream_capture():
    # its tables come from host memory that lives only during the call
    import torch

    lib = imloc.load()
    torch.cuda.set_device(0)
    depth = torch.ones((8, 8), dtype=torch.float32, device="cuda")
    view = dict(depth=depth, fx=10.0, fy=10.0, cx=4.0, cy=4.0, R=np.eye(3), t=np.zeros(3))
    n = 16
    z = torch.zeros(n, dtype=torch.float32, device="cuda")
    m = dict(q_u=z, q_v=z, db_u=z, db_v=z, conf=z, seg_off=np.array([0, n]), seg_view=np.array([0]),
             seg_dir=np.array([1]))
    out = imloc.alloc_corr(n)
    vs = imloc._views_struct([view])
    ms, keep = imloc._matches_struct(m)
    cs = imloc._corr_struct(out)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.graph(g, stream=s):
        rc = lib.imloc_lift_noalloc_async(vs, 1, C.byref(ms), C.byref(cs), C.c_void_p(s.cuda_stream))
    assert rc == -1
    torch.cuda.synchronize()


def test_noalloc_lift_rejects_inputs_beyond_its_limits():
    import torch

    lib = imloc.load()
    torch.cuda.set_device(0)
    depth = torch.ones((8, 8), dtype=torch.float32, device="cuda")
    view = dict(depth=depth, fx=10.0, fy=10.0, cx=4.0, cy=4.0, R=np.eye(3), t=np.zeros(3))
    n = 16
    z = torch.zeros(n, dtype=torch.float32, device="cuda")
    base = dict(q_u=z, q_v=z, db_u=z, db_v=z, conf=z, seg_off=np.array([0, n]), seg_view=np.array([0]),
                seg_dir=np.array([1]))
    out = imloc.alloc_corr(n)
    cs = imloc._corr_struct(out)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # more than 256 views
    vs = imloc._views_struct([view] * 257)
    ms, keep = imloc._matches_struct(base)
    assert lib.imloc_lift_noalloc_async(vs, 257, C.byref(ms), C.byref(cs), stream) == -1
    # more than 1024 segments
    many = dict(base, seg_off=np.r_[np.zeros(1025, np.int64), n], seg_view=np.zeros(1025, int),
                seg_dir=np.ones(1025, int))
    ms2, keep2 = imloc._matches_struct(many)
    vs1 = imloc._views_struct([view])
    assert lib.imloc_lift_noalloc_async(vs1, 1, C.byref(ms2), C.byref(cs), stream) == -1
    # more than 8,388,608 matches (checked before any pointer is used)
    ms3, keep3 = imloc._matches_struct(base)
    ms3.n = 8388609
    big_out = imloc._corr_struct(out)
    big_out.capacity = 8388609
    assert lib.imloc_lift_noalloc_async(vs1, 1, C.byref(ms3), C.byref(big_out), stream) == -1
    # within the limits the same call succeeds
    assert lib.imloc_lift_noalloc_async(vs1, 1, C.byref(ms), C.byref(cs), stream) == 0
    torch.cuda.synchronize()
    assert int(out["count"].item()) == 0  # every confidence is 0: all filtered
