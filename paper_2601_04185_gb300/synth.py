"""Seeded synthetic workloads shaped like ImLoc's localization inputs.

The paper evaluates on public benchmarks (Oxford Day & Night, LaMAR,
Cambridge Landmarks, Aachen) with RoMa matches; none of that is available, so
these generators stand in for them with the same shapes: K retrieved database
views with float32 z-depth maps, thousands of dense matches per pair with a
confidence, uneven inlier ratios and pixel noise (ImLoc Sec. 3.3, Sec. 4).

This module only MAKES inputs (scene geometry, ground truth and noise).  It
holds none of the method's arithmetic: no lifting, sampling, solving, scoring
or refinement.  Both the CUDA path and the CPU oracle consume its output.

Conventions: poses are cam_from_world (X_c = R X_w + t); pixel (i, j) is
centred at (i + 0.5, j + 0.5); depth maps store z-depth, 0 where no surface
lies within [1, 50] m.
"""
from __future__ import annotations

import math

import numpy as np

CONF_MIN = np.float32(0.05)


def random_rotation(rng):
    """Haar-uniform rotation from a normalised 4-D Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def axis_angle(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * Kx + (1 - math.cos(angle)) * (Kx @ Kx)


# ---------------------------------------------------------------------------
# Direct 2D-3D correspondences (single-query and batched shapes)
# ---------------------------------------------------------------------------
def direct_query(rng, n, inlier_ratio, width, height, f, noise_px=1.0, depth_range=(2.0, 20.0),
                 weights="ones"):
    """Correspondences of one query with a known pose.

    Inliers: a uniform pixel, a uniform depth in `depth_range`, back-projected
    through the ground-truth pose; the observed pixel gets N(0, noise_px)
    noise.  Outliers: the same 3D construction but the observed pixel is
    uniform in the image.  Returns float32 arrays plus float64 ground truth.
    """
    cx, cy = width / 2.0, height / 2.0
    R = random_rotation(rng)
    t = rng.normal(size=3)
    u = rng.uniform(0, width, n)
    v = rng.uniform(0, height, n)
    d = rng.uniform(depth_range[0], depth_range[1], n)
    Xc = np.stack([(u - cx) / f * d, (v - cy) / f * d, d], axis=1)
    Xw = (Xc - t) @ R  # R^T (X_c - t), row-wise
    n_in = int(round(inlier_ratio * n))
    inl = np.zeros(n, dtype=bool)
    inl[rng.permutation(n)[:n_in]] = True
    x = np.where(inl, u + rng.normal(0, noise_px, n), rng.uniform(0, width, n))
    y = np.where(inl, v + rng.normal(0, noise_px, n), rng.uniform(0, height, n))
    if weights == "ones":
        w = np.ones(n)
    else:
        w = np.where(inl, rng.uniform(0.3, 1.0, n), rng.uniform(0.05, 1.0, n))
    return dict(x=x.astype(np.float32), y=y.astype(np.float32), X=Xw.astype(np.float32),
                w=w.astype(np.float32), K=(float(f), float(f), cx, cy), width=width, height=height,
                R_gt=R, t_gt=t, inlier=inl)


def config1(seed=0):
    """Single query, plain LO-RANSAC PnP: 2,000 correspondences, 640x480,
    f=500, principal point at the centre, R uniform, t ~ N(0, 1 m), depth
    U[2, 20] m, 30% inliers with N(0, 1 px) noise, 1,000 hypotheses, 4 px."""
    rng = np.random.default_rng(seed)
    q = direct_query(rng, 2000, 0.30, 640, 480, 500.0, noise_px=1.0)
    q.update(hypotheses=1000, tau=4.0)
    return q


def config3(seed=0, n_queries=256, n_range=(2000, 100000)):
    """Batched: queries with N log-uniform in [2k, 100k], inlier ratio
    U[5%, 70%], 4,096-16,384 hypotheses (multiples of 1,024), 1024x768, f=800."""
    rng = np.random.default_rng(seed)
    out = []
    for qi in range(n_queries):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        ratio = rng.uniform(0.05, 0.70)
        q = direct_query(rng, n, ratio, 1024, 768, 800.0, noise_px=1.0, depth_range=(2.0, 40.0), weights="conf")
        q.update(hypotheses=int(rng.integers(4, 17)) * 1024, tau=4.0, query_id=qi)
        out.append(q)
    return out


# ---------------------------------------------------------------------------
# Piecewise-planar scene, database views with depth maps, dense matches
# ---------------------------------------------------------------------------
class PlanarScene:
    """Disk-shaped planar patches plus one large backdrop, in world frame."""

    def __init__(self, rng, R_q, t_q, K, width, height, n_planes=8):
        fx, fy, cx, cy = K
        self.planes = []  # (normal_w, offset_w, centre_w, radius)
        for p in range(n_planes):
            if p == 0:
                ray = np.array([0.0, 0.0, 1.0])
                depth0 = rng.uniform(35.0, 45.0)
                tilt = rng.uniform(0, math.radians(20))
                radius = depth0 * rng.uniform(0.7, 1.2)  # leaves some 'sky' (no depth) at the corners
            else:
                u = rng.uniform(-0.1 * width, 1.1 * width)
                v = rng.uniform(-0.1 * height, 1.1 * height)
                ray = np.array([(u - cx) / fx, (v - cy) / fy, 1.0])
                depth0 = rng.uniform(3.0, 32.0)
                tilt = rng.uniform(0, math.radians(55))
                radius = rng.uniform(0.25, 0.7) * depth0
            centre_c = depth0 * ray
            n_c = -ray / np.linalg.norm(ray)
            axis = np.cross(n_c, rng.normal(size=3))
            n_c = axis_angle(axis, tilt) @ n_c
            off_c = float(n_c @ centre_c)
            n_w = R_q.T @ n_c
            off_w = off_c - float(n_c @ t_q)
            centre_w = R_q.T @ (centre_c - t_q)
            self.planes.append((n_w, off_w, centre_w, radius))

    def raycast(self, R, t, K, u, v):
        """z-depth of the first surface hit along the rays through pixels
        (u, v) of camera (R, t, K); 0 where nothing lies in [1, 50] m."""
        fx, fy, cx, cy = K
        u = np.asarray(u, dtype=np.float64)
        v = np.asarray(v, dtype=np.float64)
        shape = u.shape
        a = ((u - cx) / fx).ravel()
        b = ((v - cy) / fy).ravel()
        # world direction of the ray with unit camera-z: R^T (a, b, 1)
        C = -R.T @ t
        best = np.full(a.shape, np.inf)
        for n_w, off_w, centre_w, radius in self.planes:
            nc = R @ n_w                      # plane normal in camera axes
            den = a * nc[0] + b * nc[1] + nc[2]
            with np.errstate(divide="ignore", invalid="ignore"):
                s = (off_w - n_w @ C) / den
            # |C + s d - centre|^2 with d = R^T (a, b, 1): expand without (n, 3) temporaries
            e = R @ (C - centre_w)            # (C - centre) in camera axes
            d2 = a * a + b * b + 1.0
            ed = a * e[0] + b * e[1] + e[2]
            dist2 = (e @ e) + 2.0 * s * ed + s * s * d2
            ok = np.isfinite(s) & (s > 0) & (dist2 < radius * radius) & (s < best)
            best = np.where(ok, s, best)
        best = np.where(np.isfinite(best) & (best >= 1.0) & (best <= 50.0), best, 0.0)
        return best.reshape(shape)

    def depth_map(self, R, t, K, width, height):
        jj, ii = np.meshgrid(np.arange(height) + 0.5, np.arange(width) + 0.5, indexing="ij")
        return self.raycast(R, t, K, ii, jj).astype(np.float32)


def _project(R, t, K, Xw):
    fx, fy, cx, cy = K
    Xc = Xw @ R.T + t
    z = Xc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        return fx * Xc[:, 0] / z + cx, fy * Xc[:, 1] / z + cy, z


def _backproject(R, t, K, u, v, d):
    fx, fy, cx, cy = K
    Xc = np.stack([(u - cx) / fx * d, (v - cy) / fy * d, d], axis=1)
    return (Xc - t) @ R


def _bilinear_taps_ok(depth, u, v):
    """All four bilinear taps lie inside and carry a depth (generator-side check)."""
    h, w = depth.shape
    a = u - 0.5
    b = v - 0.5
    ok = (a >= 0) & (a < w - 1) & (b >= 0) & (b < h - 1)
    i = np.clip(np.floor(a).astype(np.int64), 0, w - 2)
    j = np.clip(np.floor(b).astype(np.int64), 0, h - 2)
    taps = np.stack([depth[j, i], depth[j, i + 1], depth[j + 1, i], depth[j + 1, i + 1]])
    return ok & np.all(taps > 0, axis=0)


def perturbed_view_pose(rng, R_q, t_q, max_rot_deg=15.0, max_shift_m=3.0):
    """A database pose near a query pose: rotation <= max_rot_deg, centre <= max_shift_m away."""
    dR = axis_angle(rng.normal(size=3), math.radians(rng.uniform(0, max_rot_deg)))
    R_d = dR @ R_q
    C_q = -R_q.T @ t_q
    dirn = rng.normal(size=3)
    C_d = C_q + dirn / np.linalg.norm(dirn) * rng.uniform(0, max_shift_m)
    return R_d, -R_d @ C_d


def pair_matches(rng, scene, R_q, t_q, K, width, height, view, n_pair, direction, ratio, pixel_noise):
    """Matches of one (query, database view) pair in one direction.

    direction 0: query pixel -> 3D by the scene -> database subpixel (visible,
    all four bilinear taps valid); direction 1: database pixel centre -> depth
    -> 3D -> query subpixel (visible from the query).  A fraction `ratio` are
    true matches with N(0, pixel_noise) on the query pixel; the rest are
    uniform.  Confidence: true U[0.3, 1], false U[0, 1]."""
    R_d, t_d, depth_true = view["R"], view["t"], view["depth_true"]
    n_in = int(round(ratio * n_pair))
    if direction == 0:
        cu = rng.uniform(0, width, 6 * n_in + 64)
        cv = rng.uniform(0, height, 6 * n_in + 64)
        zq = scene.raycast(R_q, t_q, K, cu, cv)
        Xw = _backproject(R_q, t_q, K, cu, cv, zq)
        du, dv, dz = _project(R_d, t_d, K, Xw)
        zd = scene.raycast(R_d, t_d, K, np.nan_to_num(du), np.nan_to_num(dv))
        ok = (zq > 0) & (dz > 0) & np.isfinite(du) & np.isfinite(dv)
        ok &= _bilinear_taps_ok(depth_true, np.nan_to_num(du), np.nan_to_num(dv))
        ok &= np.abs(zd - dz) < 1e-3 * np.maximum(dz, 1e-9)
        sel = np.nonzero(ok)[0][:n_in]
        in_qu, in_qv, in_du, in_dv = cu[sel], cv[sel], du[sel], dv[sel]
    else:
        valid_pix = np.flatnonzero(depth_true.ravel() > 0)
        pick = valid_pix[rng.integers(0, len(valid_pix), 6 * n_in + 64)] if len(valid_pix) else np.zeros(0, int)
        pj, pi = np.divmod(pick, width)
        du = pi + 0.5
        dv = pj + 0.5
        Xw = _backproject(R_d, t_d, K, du, dv, depth_true[pj, pi].astype(np.float64))
        qu, qv, qz = _project(R_q, t_q, K, Xw)
        ok = (qz > 0) & np.isfinite(qu) & (qu >= 0) & (qu < width) & (qv >= 0) & (qv < height)
        zq = scene.raycast(R_q, t_q, K, np.nan_to_num(qu), np.nan_to_num(qv))
        ok &= np.abs(zq - qz) < 1e-3 * np.maximum(qz, 1e-9)
        sel = np.nonzero(ok)[0][:n_in]
        in_qu, in_qv, in_du, in_dv = qu[sel], qv[sel], du[sel], dv[sel]
    n_in_eff = len(sel)
    n_out = n_pair - n_in_eff
    in_qu = in_qu + rng.normal(0, pixel_noise, n_in_eff)
    in_qv = in_qv + rng.normal(0, pixel_noise, n_in_eff)
    out_qu = rng.uniform(0, width, n_out)
    out_qv = rng.uniform(0, height, n_out)
    if direction == 0:
        out_du = rng.uniform(0, width, n_out)
        out_dv = rng.uniform(0, height, n_out)
    else:
        out_du = rng.integers(0, width, n_out) + 0.5
        out_dv = rng.integers(0, height, n_out) + 0.5
    q_u = np.concatenate([in_qu, out_qu])
    q_v = np.concatenate([in_qv, out_qv])
    d_u = np.concatenate([in_du, out_du])
    d_v = np.concatenate([in_dv, out_dv])
    conf = np.concatenate([rng.uniform(0.3, 1.0, n_in_eff), rng.uniform(0.0, 1.0, n_out)])
    truth = np.concatenate([np.ones(n_in_eff, bool), np.zeros(n_out, bool)])
    perm = rng.permutation(n_pair)
    return q_u[perm], q_v[perm], d_u[perm], d_v[perm], conf[perm], truth[perm]


def query_matches(rng, scene, R_q, t_q, K, width, height, views, view_ids, matches_per_pair, pixel_noise,
                  inlier_range):
    """Matches of a query against the listed views (segments: per view, one
    query->database and one database->query segment)."""
    cols = {k: [] for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    truth_all = []
    seg_off, seg_view, seg_dir = [0], [], []
    for slot, vid in enumerate(view_ids):
        ratio = rng.uniform(*inlier_range)
        for direction in (0, 1):
            n_pair = matches_per_pair // 2 if direction == 0 else matches_per_pair - matches_per_pair // 2
            q_u, q_v, d_u, d_v, conf, truth = pair_matches(rng, scene, R_q, t_q, K, width, height, views[vid], n_pair,
                                                           direction, ratio, pixel_noise)
            for k, a in zip(cols, (q_u, q_v, d_u, d_v, conf)):
                cols[k].append(a)
            truth_all.append(truth)
            seg_off.append(seg_off[-1] + n_pair)
            seg_view.append(slot)
            seg_dir.append(direction)
    m = {k: np.concatenate(v).astype(np.float32) for k, v in cols.items()}
    m.update(seg_off=np.array(seg_off, np.int64), seg_view=np.array(seg_view, np.int32),
             seg_dir=np.array(seg_dir, np.int32))
    return m, np.concatenate(truth_all)


def make_view(scene, R_d, t_d, K, width, height, depth_noise=0.0, rng=None):
    depth_true = scene.depth_map(R_d, t_d, K, width, height)
    depth = depth_true
    if depth_noise > 0:
        depth = (depth_true * (1.0 + rng.normal(0, depth_noise, depth_true.shape))).astype(np.float32)
    return dict(depth=depth, depth_true=depth_true, fx=K[0], fy=K[1], cx=K[2], cy=K[3], R=R_d, t=t_d)


def localization_query(rng, n_views=10, matches_per_pair=5000, width=1024, height=768, f=800.0,
                       pixel_noise=0.5, depth_noise=0.0, inlier_range=(0.10, 0.60), scene=None,
                       max_rot_deg=15.0, max_shift_m=3.0):
    """One query of the lift + RANSAC workload.

    A query camera with a random pose looks at a piecewise-planar scene; each
    of `n_views` database views is the query pose perturbed by <= 15 deg and
    <= 3 m and stores a float32 z-depth map (optionally multiplied by
    1 + N(0, depth_noise)).  Per pair, half of the matches run query->database
    (subpixel database position) and half database->query (database pixel
    centre); a fraction U[inlier_range] are true matches with N(0, pixel_noise)
    noise on the query pixel, the rest are uniform.  Confidence: inliers
    U[0.3, 1], outliers U[0, 1].
    """
    K = (f, f, width / 2.0, height / 2.0)
    R_q = random_rotation(rng)
    t_q = rng.normal(size=3)
    if scene is None:
        scene = PlanarScene(rng, R_q, t_q, K, width, height)
    views = []
    for k in range(n_views):
        R_d, t_d = perturbed_view_pose(rng, R_q, t_q, max_rot_deg, max_shift_m)
        views.append(make_view(scene, R_d, t_d, K, width, height, depth_noise, rng))
    matches, truth = query_matches(rng, scene, R_q, t_q, K, width, height, views, list(range(n_views)),
                                   matches_per_pair, pixel_noise, inlier_range)
    for v in views:
        v.pop("depth_true")
    return dict(views=views, matches=matches, K=K, width=width, height=height, R_gt=R_q, t_gt=t_q,
                truth_inlier=truth, scene=scene)


class MapStore:
    """A resident map store: one planar scene seen by `n_views` database views
    around a centre pose (<= 15 deg, <= 3 m).  Serving queries are new poses
    near the centre whose retrieved views are a subset of the store."""

    def __init__(self, seed, n_views, width=1024, height=768, f=800.0):
        rng = np.random.default_rng(seed)
        self.K = (f, f, width / 2.0, height / 2.0)
        self.width, self.height = width, height
        self.R_c = random_rotation(rng)
        self.t_c = rng.normal(size=3)
        self.scene = PlanarScene(rng, self.R_c, self.t_c, self.K, width, height)
        self.poses = [perturbed_view_pose(rng, self.R_c, self.t_c) for _ in range(n_views)]
        self.views = [None] * n_views

    def build_view(self, k):
        R_d, t_d = self.poses[k]
        v = make_view(self.scene, R_d, t_d, self.K, self.width, self.height)
        self.views[k] = v
        return v

    def query(self, rng, n_views, matches_per_pair=5000, pixel_noise=0.5, inlier_range=(0.10, 0.60)):
        """A query near the centre pose matched against `n_views` random store views."""
        R_q, t_q = perturbed_view_pose(rng, self.R_c, self.t_c, 8.0, 1.5)
        ids = sorted(rng.choice(len(self.views), size=n_views, replace=False).tolist())
        m, truth = query_matches(rng, self.scene, R_q, t_q, self.K, self.width, self.height, self.views, ids,
                                 matches_per_pair, pixel_noise, inlier_range)
        return dict(view_ids=ids, matches=m, K=self.K, R_gt=R_q, t_gt=t_q, truth_inlier=truth)


def config2(seed=0, **kw):
    """Lift + RANSAC per query: 1024x768 query, 10 views with float32 depth
    of an 8-plane scene (depth 1-50 m), 5,000 matches per pair (50k),
    inlier ratio U[10%, 60%], pixel noise N(0, 0.5 px), 10,000 hypotheses."""
    rng = np.random.default_rng(seed)
    q = localization_query(rng, **kw)
    q.update(hypotheses=10000, tau=4.0)
    return q


def config4(seed=0, n_queries=64, **kw):
    """Precision study: queries of 50k matches through the planar pipeline
    with 1% depth noise and pixel noise in {0.5, 1, 1.5, 2} px (16 each)."""
    rng = np.random.default_rng(seed)
    sigmas = [0.5, 1.0, 1.5, 2.0]
    out = []
    for qi in range(n_queries):
        q = localization_query(rng, pixel_noise=sigmas[qi * len(sigmas) // n_queries], depth_noise=0.01, **kw)
        q.update(hypotheses=10000, tau=4.0, query_id=qi)
        out.append(q)
    return out


def mapping_image(rng, n_src=8, width=560, height=560, f=480.0, inlier_prob=0.8, pixel_noise=0.5,
                  max_rot_deg=15.0, max_shift_m=3.0):
    """Input of the mapping-time dense triangulation (ImLoc Sec. 3.3 "Depth
    Estimation by Dense Matching"): a reference (mapping) camera looking at a
    piecewise-planar scene, `n_src` covisible source cameras (its pose
    perturbed by <= 15 deg / <= 3 m), and for every reference pixel one match
    per source.  A match of a pixel whose surface point is visible in the
    source (in front, inside, not occluded) is, with probability
    `inlier_prob`, the point's projection + N(0, pixel_noise) with confidence
    U[0.3, 1]; every other match is a uniform source pixel with confidence
    U[0, 1].  Returns cameras as dicts (fx, fy, cx, cy, R, t), the match
    planes u, v, conf (float32, n_src x H x W), the true reference z-depth
    and the visibility mask."""
    K = (f, f, width / 2.0, height / 2.0)
    R0 = random_rotation(rng)
    t0 = rng.normal(size=3)
    scene = PlanarScene(rng, R0, t0, K, width, height)
    depth_gt = scene.depth_map(R0, t0, K, width, height).astype(np.float64)
    jj, ii = np.meshgrid(np.arange(height) + 0.5, np.arange(width) + 0.5, indexing="ij")
    has = depth_gt > 0
    Xw = _backproject(R0, t0, K, ii.ravel(), jj.ravel(), depth_gt.ravel())
    cam = lambda R, t: dict(fx=K[0], fy=K[1], cx=K[2], cy=K[3], R=R, t=t)
    srcs = []
    u = np.zeros((n_src, height, width), np.float32)
    v = np.zeros_like(u)
    conf = np.zeros_like(u)
    vis = np.zeros((n_src, height, width), bool)
    for s in range(n_src):
        R_s, t_s = perturbed_view_pose(rng, R0, t0, max_rot_deg, max_shift_m)
        srcs.append(cam(R_s, t_s))
        us, vs, zs = _project(R_s, t_s, K, Xw)
        inside = has.ravel() & (zs > 0) & (us >= 0) & (us < width) & (vs >= 0) & (vs < height)
        hit = np.zeros_like(zs)
        hit[inside] = scene.raycast(R_s, t_s, K, us[inside], vs[inside])
        visible = inside & (np.abs(hit - zs) <= 1e-3 * np.abs(zs))
        good = visible & (rng.random(zs.shape) < inlier_prob)
        uo = rng.uniform(0, width, zs.shape)
        vo = rng.uniform(0, height, zs.shape)
        uu = np.where(good, us + rng.normal(0, pixel_noise, zs.shape), uo)
        vv = np.where(good, vs + rng.normal(0, pixel_noise, zs.shape), vo)
        cc = np.where(good, rng.uniform(0.3, 1.0, zs.shape), rng.uniform(0.0, 1.0, zs.shape))
        u[s] = uu.reshape(height, width)
        v[s] = vv.reshape(height, width)
        conf[s] = cc.reshape(height, width)
        vis[s] = good.reshape(height, width)
    return dict(ref=cam(R0, t0), srcs=srcs, u=u, v=v, conf=conf, depth_gt=depth_gt, good=vis,
                width=width, height=height)


def to_bf16_bits(x):
    """float32 array -> bfloat16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def retrieval_set(rng, n_db, n_query, dim, n_places=None, spread=0.35, noise=0.5):
    """Global retrieval descriptors (stand-ins for MegaLoc / NetVLAD features of
    the map images and the queries): database images are grouped in places
    (a random unit direction each, images of a place scattered around it),
    each query is a noisy view of one place; all L2-normalised, stored as
    bfloat16.  Returns db (n_db, dim) and queries (n_query, dim) uint16 bit
    patterns and the place of every query."""
    n_places = n_places or max(1, n_db // 20)
    centres = rng.normal(size=(n_places, dim)).astype(np.float32)
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    place = rng.integers(0, n_places, n_db)
    db = centres[place] + spread * rng.normal(size=(n_db, dim)).astype(np.float32) / np.sqrt(dim)
    db /= np.linalg.norm(db, axis=1, keepdims=True)
    qp = rng.integers(0, n_places, n_query)
    q = centres[qp] + noise * rng.normal(size=(n_query, dim)).astype(np.float32) / np.sqrt(dim)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return to_bf16_bits(db), to_bf16_bits(q), qp


def retrieval_set_torch(seed, n_db, n_query, dim, device, n_places=None, spread=0.35, noise=0.5):
    """retrieval_set generated on the GPU with torch (the same construction, a
    torch random stream): for benchmark sizes (10^5 x 8448) that numpy would
    take long to draw.  Returns bfloat16 tensors db (n_db, dim), queries
    (n_query, dim)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    n_places = n_places or max(1, n_db // 20)
    centres = torch.randn(n_places, dim, generator=g, device=device)
    centres /= centres.norm(dim=1, keepdim=True)
    place = torch.randint(0, n_places, (n_db,), generator=g, device=device)
    db = torch.empty(n_db, dim, dtype=torch.bfloat16, device=device)
    for b in range(0, n_db, 8192):
        e = min(n_db, b + 8192)
        x = centres[place[b:e]] + spread * torch.randn(e - b, dim, generator=g, device=device) / dim ** 0.5
        db[b:e] = (x / x.norm(dim=1, keepdim=True)).to(torch.bfloat16)
    qp = torch.randint(0, n_places, (n_query,), generator=g, device=device)
    q = centres[qp] + noise * torch.randn(n_query, dim, generator=g, device=device) / dim ** 0.5
    q = (q / q.norm(dim=1, keepdim=True)).to(torch.bfloat16)
    return db, q


# ---------------------------------------------------------------------------
# Multi-camera rig queries (generalized absolute pose)
# ---------------------------------------------------------------------------
def rig_layout(rng, n_cams=4, yaw_deg=(-60.0, -20.0, 20.0, 60.0), baseline=0.1):
    """A head-mounted rig in the manner of the HoloLens tracking cameras:
    camera k looks out at yaw yaw_deg[k] about the rig's y axis (with a small
    random tilt), centred within `baseline` metres of the rig origin.  Returns
    cam_from_rig rotations and translations (X_c = R_k X_r + t_k)."""
    Rs, ts = [], []
    for k in range(n_cams):
        yaw = math.radians(yaw_deg[k % len(yaw_deg)])
        R = axis_angle([0.0, 1.0, 0.0], yaw) @ axis_angle(rng.normal(size=3), rng.uniform(0, math.radians(5)))
        c = rng.uniform(-baseline, baseline, 3)
        Rs.append(R)
        ts.append(-R @ c)
    return Rs, ts


def rig_query(rng, n_per_cam=500, inlier_ratio=0.4, n_cams=4, width=640, height=480, f=450.0, noise_px=1.0,
              depth_range=(1.0, 15.0), weights="conf", baseline=0.1):
    """Correspondences of one rig query with a known rig pose (rig_from_world,
    X_r = R X_w + t).  Per camera, as direct_query: a uniform pixel and depth
    back-projected into the world; inliers observed with N(0, noise_px) noise,
    outliers at a uniform pixel.  Correspondences are grouped by camera; `cam`
    gives each one's camera."""
    R_cam, t_cam = rig_layout(rng, n_cams, baseline=baseline)
    R = random_rotation(rng)
    t = rng.normal(size=3)
    cx, cy = width / 2.0, height / 2.0
    xs, ys, Xs, ws, cams, inls = [], [], [], [], [], []
    for k in range(n_cams):
        n = n_per_cam
        u = rng.uniform(0, width, n)
        v = rng.uniform(0, height, n)
        d = rng.uniform(depth_range[0], depth_range[1], n)
        Xc = np.stack([(u - cx) / f * d, (v - cy) / f * d, d], axis=1)
        Xr = (Xc - t_cam[k]) @ R_cam[k]
        Xw = (Xr - t) @ R
        n_in = int(round(inlier_ratio * n))
        inl = np.zeros(n, dtype=bool)
        inl[rng.permutation(n)[:n_in]] = True
        xs.append(np.where(inl, u + rng.normal(0, noise_px, n), rng.uniform(0, width, n)))
        ys.append(np.where(inl, v + rng.normal(0, noise_px, n), rng.uniform(0, height, n)))
        Xs.append(Xw)
        ws.append(np.ones(n) if weights == "ones" else np.where(inl, rng.uniform(0.3, 1.0, n),
                                                                 rng.uniform(0.05, 1.0, n)))
        cams.append(np.full(n, k, np.int32))
        inls.append(inl)
    return dict(x=np.concatenate(xs).astype(np.float32), y=np.concatenate(ys).astype(np.float32),
                X=np.concatenate(Xs).astype(np.float32), w=np.concatenate(ws).astype(np.float32),
                cam=np.concatenate(cams), K=[(float(f), float(f), cx, cy)] * n_cams, R_cam=R_cam, t_cam=t_cam,
                width=width, height=height, R_gt=R, t_gt=t, inlier=np.concatenate(inls))
