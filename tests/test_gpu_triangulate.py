"""Dense triangulation of a mapping depth map (ImLoc Sec. 3.3 "Depth
Estimation by Dense Matching") through the C ABI against the FP64 oracle.

Bar: inlier counts and kept/dropped decisions identical, except at pixels
where an oracle angle (FP64, at any hypothesis) lies within 0.005 degrees of
the 2-degree threshold or a hypothesis comes from rays less than 0.06 degrees
apart (the kernel decides in FP32); refined depths within 2e-4 relative (FP32 angular
residuals of ~1e-7 rad against a minimum that can be shallow).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import torch

pytestmark = pytest.mark.gpu


def rays(cam, x, y):
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    k = np.stack([(x - cam["cx"]) / cam["fx"], (y - cam["cy"]) / cam["fy"], np.ones_like(x)], -1)
    return -R.T @ t, k @ R  # centre, directions (..., 3)


def borderline(m, thr_deg=2.0, band_deg=0.005, min_sin=1e-3):
    """pixels whose decisions the FP32 kernel may legitimately take differently"""
    S, H, W = m["u"].shape
    jj, ii = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    C0, d0 = rays(m["ref"], ii, jj)
    used = m["conf"] >= np.float32(0.05)
    cs, dss = [], []
    for s in range(S):
        C, d = rays(m["srcs"][s], m["u"][s].astype(np.float64), m["v"][s].astype(np.float64))
        cs.append(C)
        dss.append(d)
    thr = math.radians(thr_deg)
    band = math.radians(band_deg)
    bad = np.zeros((H, W), bool)
    for s in range(S):
        n = np.cross(d0, dss[s])
        wx = np.cross(C0 - cs[s], dss[s])
        nn = np.einsum("...i,...i", n, n)
        sin2 = nn / (np.einsum("...i,...i", d0, d0) * np.einsum("...i,...i", dss[s], dss[s]))
        with np.errstate(divide="ignore", invalid="ignore"):
            z = -np.einsum("...i,...i", wx, n) / nn
        valid = used[s] & (z > 0) & np.isfinite(z)
        bad |= used[s] & (sin2 < min_sin ** 2)
        for k in range(S):
            a = C0 + z[..., None] * d0 - cs[k]
            c = np.cross(a, dss[k])
            th = np.arctan2(np.sqrt(np.einsum("...i,...i", c, c)), np.einsum("...i,...i", a, dss[k]))
            bad |= valid & used[k] & (np.abs(th - thr) < band)
    return bad


def run_gpu(m, **kw):
    t = torch()
    u, v, c = (t.from_numpy(np.ascontiguousarray(m[k])).cuda() for k in ("u", "v", "conf"))
    depth, inl = imloc.triangulate_depth(m["ref"], m["srcs"], u, v, c, opts=imloc.triangulate_opts(**kw))
    t.cuda.synchronize()
    return depth.cpu().numpy().astype(np.float64), inl.cpu().numpy().astype(np.int64)


def compare(m, gd, gi, od, oi, max_excused=0.03, tol=2e-4):
    ex = borderline(m)
    assert ex.mean() < max_excused, ex.mean()
    ok = ~ex
    mism = ok & (gi != oi)
    assert not mism.any(), (int(mism.sum()), np.argwhere(mism)[:5])
    kept_g, kept_o = gd > 0, od > 0
    assert (kept_g[ok] == kept_o[ok]).all()
    both = ok & kept_g & kept_o
    if both.any():
        rel = np.abs(gd[both] - od[both]) / od[both]
        assert rel.max() <= tol, (float(rel.max()), float(np.percentile(rel, 99.9)))
    return both.sum()


def test_mapping_image_full_size():
    m = synth.mapping_image(np.random.default_rng(5), n_src=8, width=560, height=560, f=480.0)
    gd, gi = run_gpu(m)
    od, oi = oracle.triangulate_depth(m["ref"], m["srcs"], m["u"], m["v"], m["conf"])
    n = compare(m, gd, gi, od, oi)
    assert n > 0.3 * 560 * 560
    # sanity: the kept depths are near the true surface
    gt = m["depth_gt"]
    kept = gd > 0
    assert np.median(np.abs(gd[kept] - gt[kept]) / gt[kept]) < 0.02


@pytest.mark.parametrize("seed,n_src,w,h", [(6, 3, 37, 23), (7, 16, 61, 45), (8, 1, 16, 9), (9, 9, 100, 1)])
def test_ragged_sizes_and_source_counts(seed, n_src, w, h):
    m = synth.mapping_image(np.random.default_rng(seed), n_src=n_src, width=w, height=h, f=0.9 * max(w, h))
    gd, gi = run_gpu(m)
    od, oi = oracle.triangulate_depth(m["ref"], m["srcs"], m["u"], m["v"], m["conf"])
    compare(m, gd, gi, od, oi, max_excused=0.1)
    if n_src <= 3:
        assert (gd == 0).all()  # never more than 3 inliers


def test_no_usable_match_gives_no_depth():
    m = synth.mapping_image(np.random.default_rng(10), n_src=4, width=40, height=30, f=40.0)
    m["conf"][:] = np.float32(0.0499)
    gd, gi = run_gpu(m)
    assert (gd == 0).all() and (gi == 0).all()
