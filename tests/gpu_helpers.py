"""Shared helpers of the GPU tests: move seeded inputs to the device, compare
poses.  Imports the CUDA binding and (for expected values) the oracle."""
import math

import numpy as np

from paper_2601_04185_gb300 import imloc


def torch():
    import torch as t

    return t


def views_to_device(views):
    t = torch()
    out = []
    for v in views:
        d = dict(v)
        d["depth"] = t.from_numpy(np.ascontiguousarray(v["depth"], dtype=np.float32)).cuda()
        out.append(d)
    return out


def matches_to_device(m):
    t = torch()
    d = {k: t.from_numpy(np.ascontiguousarray(m[k], dtype=np.float32)).cuda() for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    d.update({k: m[k] for k in ("seg_off", "seg_view", "seg_dir")})
    return d


def lifted_to_host(out, n=None):
    if n is None:
        n = int(out["count"].item())
    g = {k: out[k][:n].cpu().numpy() for k in ("x", "y", "X", "Y", "Z", "w", "src")}
    g["Xw"] = np.stack([g["X"], g["Y"], g["Z"]], 1).astype(np.float64)
    g["n"] = n
    return g


def check_lift(g, ref, views, matches, src_base=0):
    """Lifted correspondences g (lifted_to_host) against the oracle's lift:
    kept matches and source indices bit-exact, x, y, w identical, world points
    within 2e-6 (|X_w| + 2 |C|), C the centre of the point's database camera."""
    assert g["n"] == len(ref["src"])
    np.testing.assert_array_equal(g["src"].astype(np.int64) - src_base, ref["src"])
    np.testing.assert_array_equal(g["x"].astype(np.float64), ref["x"])
    np.testing.assert_array_equal(g["y"].astype(np.float64), ref["y"])
    np.testing.assert_array_equal(g["w"].astype(np.float64), ref["w"])
    if g["n"] == 0:
        return
    seg_of = np.searchsorted(np.asarray(matches["seg_off"])[1:], ref["src"], side="right")
    vid = np.asarray(matches["seg_view"])[seg_of]
    C = np.stack([-np.asarray(views[v]["R"]).T @ np.asarray(views[v]["t"]) for v in range(len(views))])[vid]
    err = np.linalg.norm(g["Xw"] - ref["X"], axis=1)
    bound = 2e-6 * (np.linalg.norm(ref["X"], axis=1) + 2 * np.linalg.norm(C, axis=1))
    assert np.all(err <= bound), float(np.max(err / bound))


def rot_deg(Ra, Rb):
    """Angle between two rotations from the chord |Ra - Rb|_F = 2 sqrt(2) sin(angle / 2):
    exact for rotations and 0 for identical matrices."""
    chord = np.linalg.norm(np.asarray(Ra, np.float64) - np.asarray(Rb, np.float64))
    return math.degrees(2.0 * math.asin(min(1.0, chord / (2.0 * math.sqrt(2.0)))))


def centre(R, t):
    return -np.asarray(R).T @ np.asarray(t)


def pose_close(Ra, ta, Rb, tb, deg=0.05, mm=5.0):
    return rot_deg(Ra, Rb) <= deg and np.linalg.norm(centre(Ra, ta) - centre(Rb, tb)) <= mm * 1e-3


def residuals(x, y, X, K, R, t):
    """Per-point reprojection distance (pixels) and depth, float64 (test-side tolerance bookkeeping)."""
    fx, fy, cx, cy = K
    Xc = np.asarray(X, np.float64) @ np.asarray(R, np.float64).T + np.asarray(t, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * Xc[:, 0] / Xc[:, 2] + cx
        v = fy * Xc[:, 1] / Xc[:, 2] + cy
    return np.hypot(u - x, v - y), Xc[:, 2]


def ctx():
    return imloc.Context(0, 1 << 30)
