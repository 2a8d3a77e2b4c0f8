"""Pins of the oracle's dense triangulation (ImLoc Sec. 3.3 "Depth Estimation
by Dense Matching": one depth hypothesis per match along the known reference
ray, the hypothesis with the most inliers at a 2-degree angular threshold,
refinement of the confidence-weighted squared angular errors of its inliers,
kept with more than 3 inliers)."""
import math

import numpy as np
from scipy.optimize import minimize_scalar

import oracle
from paper_2601_04185_gb300 import synth


def ray(cam, x, y):
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    k = np.array([(x - cam["cx"]) / cam["fx"], (y - cam["cy"]) / cam["fy"], 1.0])
    return -R.T @ t, R.T @ k


def test_angle_exact_for_constructed_angles():
    for th in (1e-9, 1e-5, 0.01, 0.5, 1.5, 3.0):
        a = np.array([2.0, 0.0, 0.0])
        b = np.array([math.cos(th), math.sin(th), 0.0]) * 7.0
        assert abs(oracle.angle(a, b) - th) <= 1e-15 + 1e-14 * th
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = rng.normal(size=3), rng.normal(size=3)
        ref = math.acos(np.clip(a @ b / np.linalg.norm(a) / np.linalg.norm(b), -1, 1))
        assert abs(oracle.angle(a, b) - ref) < 1e-9


def test_closest_depth_is_the_least_squares_solution():
    rng = np.random.default_rng(1)
    for _ in range(200):
        C0, d0, C1, d1 = (rng.normal(size=3) for _ in range(4))
        z, l = np.linalg.lstsq(np.stack([d0, -d1], 1), C1 - C0, rcond=None)[0]
        assert abs(oracle.closest_depth(C0, d0, C1, d1) - z) <= 1e-9 * max(1.0, abs(z))
    d = np.array([0.0, 0.0, 1.0])
    assert oracle.closest_depth(np.zeros(3), d, np.ones(3), 2 * d) == 0.0  # parallel


def test_noise_free_pixels_recover_the_true_depth():
    m = synth.mapping_image(np.random.default_rng(2), n_src=6, width=96, height=80, f=90.0, inlier_prob=1.0,
                            pixel_noise=0.0)
    depth, inl = oracle.triangulate_depth(m["ref"], m["srcs"], m["u"], m["v"], m["conf"])
    n_good = m["good"].sum(0)
    sel = n_good >= 4
    assert sel.mean() > 0.5
    gt = m["depth_gt"]
    assert (inl[sel] >= n_good[sel]).all()
    # exact up to the float32 rounding of the matches and of the true depth map,
    # unless a uniform (outlier) match happens to fall within 2 degrees as well
    exact = sel & (inl == n_good)
    assert exact.sum() > 0.99 * sel.sum()
    np.testing.assert_allclose(depth[exact], gt[exact], rtol=3e-5)


def weighted_angle_cost(C0, d0, z, rays, w):
    e = 0.0
    for (C, d), wk in zip(rays, w):
        a = C0 + z * d0 - C
        e += wk * math.acos(np.clip(a @ d / np.linalg.norm(a) / np.linalg.norm(d), -1, 1)) ** 2
    return e


def test_selection_and_refinement_against_brute_force():
    """Python brute force with a different optimizer: all hypotheses, inliers by
    arccos angles, winner (most, lowest index), bounded Brent minimum of the
    weighted squared angles."""
    m = synth.mapping_image(np.random.default_rng(3), n_src=8, width=64, height=48, f=60.0, pixel_noise=0.7)
    depth, inl = oracle.triangulate_depth(m["ref"], m["srcs"], m["u"], m["v"], m["conf"])
    rng = np.random.default_rng(4)
    thr = math.radians(2.0)
    checked = 0
    for p in rng.choice(64 * 48, 300, replace=False):
        py, px = divmod(int(p), 64)
        C0, d0 = ray(m["ref"], px + 0.5, py + 0.5)
        used = [m["conf"][s, py, px] >= np.float32(0.05) for s in range(8)]
        rays = [ray(m["srcs"][s], float(m["u"][s, py, px]), float(m["v"][s, py, px])) for s in range(8)]

        def angle_at(z, s):
            a = C0 + z * d0 - rays[s][0]
            return math.acos(np.clip(a @ rays[s][1] / np.linalg.norm(a) / np.linalg.norm(rays[s][1]), -1, 1))

        best = (0, None, None)
        for s in range(8):
            if not used[s]:
                continue
            z = np.linalg.lstsq(np.stack([d0, -rays[s][1]], 1), rays[s][0] - C0, rcond=None)[0][0]
            if not z > 0:
                continue
            angs = [angle_at(z, k) for k in range(8)]
            if any(used[k] and abs(angs[k] - thr) < 1e-9 for k in range(8)):
                break  # a borderline inlier decision: skip the pixel
            n = sum(1 for k in range(8) if used[k] and angs[k] < thr)
            if n > best[0]:
                best = (n, s, z)
        else:
            assert inl[py, px] == best[0], (px, py)
            if best[0] > 3:
                z0 = best[2]
                S = [k for k in range(8) if used[k] and angle_at(z0, k) < thr]
                res = minimize_scalar(lambda z: weighted_angle_cost(C0, d0, z, [rays[k] for k in S],
                                                                    [float(m["conf"][k, py, px]) for k in S]),
                                      bounds=(0.4 * z0, 2.5 * z0), method="bounded",
                                      options={"xatol": 1e-12 * z0})
                # a minimum located from function values alone is good to ~sqrt(eps) of the depth
                assert abs(depth[py, px] - res.x) <= 2e-7 * z0, (px, py, depth[py, px], res.x)
                checked += 1
            else:
                assert depth[py, px] == 0.0
    assert checked > 100


def pixel_case(z_true, n_consistent, z_other=None, n_other=0, conf=None):
    """A reference pixel and sources whose matches are consistent with z_true
    (first n_consistent), with z_other (next n_other) or outliers (rest)."""
    ref = dict(fx=500.0, fy=500.0, cx=320.0, cy=240.0, R=np.eye(3), t=np.zeros(3))
    srcs, u, v = [], [], []
    C0, d0 = ray(ref, 300.5, 200.5)
    n = 8
    for s in range(n):
        ang = 2 * math.pi * s / n
        C = np.array([math.cos(ang), math.sin(ang), 0.0]) * 1.5
        R = np.eye(3)
        srcs.append(dict(fx=500.0, fy=500.0, cx=320.0, cy=240.0, R=R, t=-R @ C))
        z = z_true if s < n_consistent else (z_other if s < n_consistent + n_other else None)
        if z is None:
            X = C0 + 3.0 * d0 + np.array([0.7, -0.4, 0.9]) * (s + 1)  # a wrong point, inconsistent with the others
        else:
            X = C0 + z * d0
        Xc = R @ X - R @ C
        u.append(500.0 * Xc[0] / Xc[2] + 320.0)
        v.append(500.0 * Xc[1] / Xc[2] + 240.0)
    c = np.full(n, 0.8) if conf is None else np.asarray(conf, np.float64)
    return ref, srcs, np.array(u), np.array(v), c


def test_majority_wins_and_ties_go_to_the_lowest_source():
    ref, srcs, u, v, c = pixel_case(10.0, 5, 6.0, 3)
    n, d = oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c)
    assert n == 5 and abs(d - 10.0) < 1e-9
    ref, srcs, u, v, c = pixel_case(6.0, 4, 10.0, 4)
    n, d = oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c)
    assert n == 4 and abs(d - 6.0) < 1e-9


def test_kept_only_with_more_than_three_inliers():
    ref, srcs, u, v, c = pixel_case(10.0, 3)
    n, d = oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c)
    assert n == 3 and d == 0.0
    ref, srcs, u, v, c = pixel_case(10.0, 4)
    n, d = oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c)
    assert n == 4 and abs(d - 10.0) < 1e-9


def test_confidence_threshold_is_inclusive():
    conf = np.full(8, 0.8)
    conf[:4] = np.float32(0.05)
    ref, srcs, u, v, c = pixel_case(10.0, 4, conf=conf.astype(np.float32).astype(np.float64))
    assert oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c)[0] == 4
    conf[0] = np.nextafter(np.float32(0.05), np.float32(0))
    ref, srcs, u, v, c = pixel_case(10.0, 4, conf=conf)
    n, d = oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c)
    assert n == 3 and d == 0.0


def test_no_source_no_depth():
    ref, srcs, u, v, c = pixel_case(10.0, 8, conf=np.zeros(8))
    assert oracle.triangulate_pixel(ref, srcs, 640, 300, 200, u, v, c) == (0, 0.0)
