"""Pins of the FP64 CPU oracle against facts it does not compute itself.

Every check here ties an oracle function to something outside it: published
known-answer values, closed forms, a library routine (SciPy bilinear
sampling, least squares, a generic minimiser), brute force on tiny inputs, or
an invariant of the mathematics.  The cases are chosen so that a dropped term,
a flipped sign, a swapped index or a transposed operand in the oracle fails
at least one of them.  CPU only.
"""
import math
import os

import numpy as np
import pytest
import scipy.ndimage
import scipy.optimize
from scipy.spatial.transform import Rotation

import oracle
from paper_2601_04185_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rot_deg(Ra, Rb):
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def centre(R, t):
    return -R.T @ t


# ---------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# ---------------------------------------------------------------------------
def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            words = [int(w, 16) for w in line.split()]
            rows.append((words[0:4], words[4:6], words[6:10]))
    return rows


def test_philox_known_answers():
    rows = load_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(oracle.philox4x32_10(ctr, key)) == want


# ---------------------------------------------------------------------------
# Minimal samples
# ---------------------------------------------------------------------------
def test_sample_worked_example_from_kat():
    # seed 0 -> key (0, 0); sample 0 of query 0, attempt 0 -> counter (0,0,0,0),
    # whose Philox output is the first known-answer vector.  index = floor(r m / 2^32).
    _, _, want = load_kat()[0]
    m = 1000
    expect = [(r * m) >> 32 for r in want[:3]]
    assert len(set(expect)) == 3
    got, att = oracle.sample(0, 0, 0, m)
    assert att == 0
    assert list(got) == expect


def test_sample_counter_layout():
    # the counter words are (sample, query, attempt, 0) and the key is (seed lo, seed hi)
    seed = 0x0123456789ABCDEF
    m = 5000
    for sid, qid in [(7, 3), (123456, 0), (1, 99)]:
        r = oracle.philox4x32_10([sid, qid, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        expect = [(int(v) * m) >> 32 for v in r[:3]]
        got, att = oracle.sample(seed, qid, sid, m)
        if len(set(expect)) == 3:
            assert att == 0 and list(got) == expect


def test_sample_distinct_and_uniform():
    m = 37
    counts = np.zeros(m)
    for s in range(6000):
        got, att = oracle.sample(42, 1, s, m)
        assert got is not None and len(set(got.tolist())) == 3
        assert 0 <= got.min() and got.max() < m
        counts[got] += 1
    expected = counts.sum() / m
    chi2 = ((counts - expected) ** 2 / expected).sum()
    # 36 degrees of freedom: 99.9th percentile is about 67
    assert chi2 < 67.0


def test_sample_retry_and_degenerate():
    # m = 3: only permutations of {0,1,2} are distinct, found by retrying
    seen_retry = False
    for s in range(200):
        got, att = oracle.sample(9, 0, s, 3)
        if got is not None:
            assert sorted(got.tolist()) == [0, 1, 2]
            seen_retry |= att > 0
    assert seen_retry
    # m = 2 can never give three distinct indices
    got, att = oracle.sample(9, 0, 5, 2)
    assert got is None and att == -1


# ---------------------------------------------------------------------------
# Subsampling (deterministic uniform stride)
# ---------------------------------------------------------------------------
def test_subsample_closed_forms():
    assert list(oracle.subsample(10, 10)) == list(range(10))
    assert list(oracle.subsample(20, 10)) == list(range(0, 20, 2))
    idx = oracle.subsample(47_331, 10_000)
    assert idx[0] == 0 and idx[-1] <= 47_330
    gaps = np.diff(idx)
    assert set(gaps.tolist()) <= {4, 5}  # floor/ceil of 4.7331
    assert len(np.unique(idx)) == 10_000
    big = oracle.subsample(3_000_000_000, 7)
    assert list(big) == [k * 3_000_000_000 // 7 for k in range(7)]


# ---------------------------------------------------------------------------
# Lift
# ---------------------------------------------------------------------------
def _one_view(depth, fx=400.0, fy=380.0, cx=30.5, cy=20.25, R=None, t=None):
    return dict(depth=np.asarray(depth, np.float32), fx=fx, fy=fy, cx=cx, cy=cy,
                R=np.eye(3) if R is None else R, t=np.zeros(3) if t is None else t)


def _matches(q_u, q_v, db_u, db_v, conf, dirs):
    n = len(q_u)
    return dict(q_u=np.float32(q_u), q_v=np.float32(q_v), db_u=np.float32(db_u), db_v=np.float32(db_v),
                conf=np.float32(conf), seg_off=np.array([0, n], np.int64), seg_view=np.array([0], np.int32),
                seg_dir=np.array([dirs], np.int32))


def test_lift_bilinear_matches_scipy_sampling():
    rng = np.random.default_rng(3)
    depth = rng.uniform(2, 30, (24, 40)).astype(np.float32)
    R = synth.random_rotation(rng)
    t = rng.normal(size=3)
    view = _one_view(depth, R=R, t=t)
    n = 400
    du = rng.uniform(0.5, 39.5 - 1e-3, n)
    dv = rng.uniform(0.5, 23.5 - 1e-3, n)
    m = _matches(rng.uniform(0, 640, n), rng.uniform(0, 480, n), du, dv, np.full(n, 0.5), 0)
    L = oracle.lift([view], m)
    assert len(L["x"]) == n and list(L["src"]) == list(range(n))
    u = m["db_u"].astype(np.float64)
    v = m["db_v"].astype(np.float64)
    # pixel centres at +0.5: sample index (row, col) = (v - 0.5, u - 0.5)
    d = scipy.ndimage.map_coordinates(depth.astype(np.float64), [v - 0.5, u - 0.5], order=1)
    Xc = L["X"] @ R.T + t
    np.testing.assert_allclose(Xc[:, 2], d, rtol=1e-12)
    # the lifted point projects back onto the database pixel
    np.testing.assert_allclose(view["fx"] * Xc[:, 0] / Xc[:, 2] + view["cx"], u, atol=1e-9)
    np.testing.assert_allclose(view["fy"] * Xc[:, 1] / Xc[:, 2] + view["cy"], v, atol=1e-9)
    np.testing.assert_array_equal(L["x"], m["q_u"].astype(np.float64))
    np.testing.assert_array_equal(L["w"], m["conf"].astype(np.float64))


def test_lift_lookup_direction_and_filters():
    depth = np.arange(1, 13, dtype=np.float32).reshape(3, 4)  # 4 wide, 3 high
    depth[1, 2] = 0.0
    depth[2, 3] = np.nan
    view = _one_view(depth)
    c05 = np.float32(0.05)
    cases = [  # (db_u, db_v, conf, expect_valid, expect_depth)
        (0.5, 0.5, 0.9, True, 1.0),
        (3.99, 0.2, 0.9, True, 4.0),            # floor -> pixel (3, 0)
        (1.7, 2.9, 0.9, True, 10.0),            # pixel (1, 2)
        (2.5, 1.5, 0.9, False, None),           # zero depth
        (3.5, 2.5, 0.9, False, None),           # NaN depth
        (4.0, 0.5, 0.9, False, None),           # right of the image
        (-0.01, 0.5, 0.9, False, None),         # left of the image
        (0.5, 0.5, float(c05), False, None),    # confidence must exceed 0.05 strictly
        (0.5, 0.5, float(np.nextafter(c05, np.float32(1))), True, 1.0),
        (float("nan"), 0.5, 0.9, False, None),
    ]
    m = _matches([1.0] * len(cases), [2.0] * len(cases), [c[0] for c in cases], [c[1] for c in cases],
                 [c[2] for c in cases], 1)
    L = oracle.lift([view], m)
    want = [i for i, c in enumerate(cases) if c[3]]
    assert list(L["src"]) == want
    np.testing.assert_allclose(L["X"][:, 2], [cases[i][4] for i in want])


def test_lift_bilinear_border_and_invalid_taps():
    depth = np.full((5, 6), 7.0, np.float32)
    depth[4, 5] = -1.0
    view = _one_view(depth)
    cases = [  # (db_u, db_v, expect_valid)
        (0.5, 0.5, True),       # first centre
        (0.4999, 1.0, False),   # left of the first centre
        (5.4999, 1.0, True),    # just inside: taps 4 and 5
        (5.5, 1.0, False),      # needs a tap at column 6
        (1.0, 4.4999, True),
        (1.0, 4.5, False),
        (5.2, 4.2, False),      # a tap with negative depth
    ]
    m = _matches([0.0] * len(cases), [0.0] * len(cases), [c[0] for c in cases], [c[1] for c in cases],
                 [0.9] * len(cases), 0)
    L = oracle.lift([view], m)
    assert list(L["src"]) == [i for i, c in enumerate(cases) if c[2]]
    np.testing.assert_allclose(L["X"][:, 2], 7.0)


def test_lift_planar_scene_invariants():
    """Noise-free planar query: lifted inliers lie on a scene plane and
    reproject into the query at the ground-truth pose."""
    rng = np.random.default_rng(11)
    q = synth.localization_query(rng, n_views=3, matches_per_pair=2000, pixel_noise=0.0)
    L = oracle.lift(q["views"], q["matches"])
    src = L["src"]
    truth = q["truth_inlier"][src]
    dirs = np.repeat(q["matches"]["seg_dir"], np.diff(q["matches"]["seg_off"]))[src]
    X = L["X"]
    planes = q["scene"].planes
    dist = np.min(np.stack([np.abs(X @ n - off) for n, off, _, _ in planes]), axis=0)
    # database pixel centres: bilinear reduces to a lookup, the point is on a plane
    # up to the float32 storage of depth (relative 6e-8 of <= 50 m)
    exact = truth & (dirs == 1)
    assert exact.sum() > 100
    assert dist[exact].max() < 2e-5
    # reprojection into the query at the ground-truth pose
    fx, fy, cx, cy = q["K"]
    Xc = X @ q["R_gt"].T + q["t_gt"]
    err = np.hypot(fx * Xc[:, 0] / Xc[:, 2] + cx - L["x"], fy * Xc[:, 1] / Xc[:, 2] + cy - L["y"])
    assert np.max(err[exact]) < 1e-3
    # subpixel database positions: z-depth of a plane is not bilinear in the
    # pixel grid, so points land within the interpolation error
    sub = truth & (dirs == 0)
    assert sub.sum() > 100
    assert np.median(err[sub]) < 0.05


# ---------------------------------------------------------------------------
# P3P
# ---------------------------------------------------------------------------
def _random_triple(rng, spread=5.0):
    R = synth.random_rotation(rng)
    t = rng.normal(size=3) * 2
    Xc = np.column_stack([rng.uniform(-spread, spread, 3), rng.uniform(-spread, spread, 3),
                          rng.uniform(2, 25, 3)])
    Xw = (Xc - t) @ R
    y = Xc / np.linalg.norm(Xc, axis=1, keepdims=True)
    return R, t, y, Xw


def test_p3p_recovers_ground_truth():
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(500):
        R, t, y, Xw = _random_triple(rng)
        sols = oracle.p3p(y, Xw)
        assert 1 <= len(sols) <= 4
        e = min(max(np.abs(Rs - R).max(), np.abs(ts - t).max() / max(1.0, np.linalg.norm(t))) for Rs, ts, _ in sols)
        worst = max(worst, e)
    assert worst <= 1e-9


def test_p3p_every_solution_is_exact_and_ordered():
    rng = np.random.default_rng(6)
    for _ in range(300):
        _, _, y, Xw = _random_triple(rng)
        sols = oracle.p3p(y, Xw)
        lam1 = [s[2][0] for s in sols]
        assert lam1 == sorted(lam1)
        for Rs, ts, lam in sols:
            np.testing.assert_allclose(Rs @ Rs.T, np.eye(3), atol=1e-12)
            assert np.linalg.det(Rs) > 0
            Xc = Xw @ Rs.T + ts
            assert np.all(Xc[:, 2] > 0)
            np.testing.assert_allclose(Xc / np.linalg.norm(Xc, axis=1, keepdims=True), y, atol=1e-9)
            np.testing.assert_allclose(np.linalg.norm(Xc, axis=1), lam, rtol=1e-9)


def test_p3p_finds_all_solutions_against_generic_root_finding():
    """Independent completeness check: solve the three distance equations with
    SciPy's generic root finder from many starts and require every positive
    solution found there to be in the oracle's list."""
    rng = np.random.default_rng(8)
    multi = 0
    for _ in range(25):
        _, _, y, Xw = _random_triple(rng, spread=12.0)
        a = [np.sum((Xw[0] - Xw[1]) ** 2), np.sum((Xw[0] - Xw[2]) ** 2), np.sum((Xw[1] - Xw[2]) ** 2)]
        b = [y[0] @ y[1], y[0] @ y[2], y[1] @ y[2]]

        def F(L):
            return [L[0] ** 2 + L[1] ** 2 - 2 * b[0] * L[0] * L[1] - a[0],
                    L[0] ** 2 + L[2] ** 2 - 2 * b[1] * L[0] * L[2] - a[1],
                    L[1] ** 2 + L[2] ** 2 - 2 * b[2] * L[1] * L[2] - a[2]]

        found = []
        scale = math.sqrt(max(a))
        for s in range(150):
            L0 = rng.uniform(0.05, 4.0, 3) * scale * 3
            sol, info, ier, _ = scipy.optimize.fsolve(F, L0, full_output=True, xtol=1e-13)
            if ier == 1 and np.all(sol > 0) and np.max(np.abs(F(sol))) < 1e-8 * max(a):
                if not any(np.allclose(sol, f, rtol=1e-6) for f in found):
                    found.append(sol)
        sols = oracle.p3p(y, Xw)
        lams = [s[2] for s in sols]
        multi += len(found) > 1
        for f in found:
            assert any(np.allclose(f, l, rtol=1e-6) for l in lams), (f, lams)
    assert multi > 0  # the sweep did meet triples with several solutions


# ---------------------------------------------------------------------------
# Scoring (confidence-weighted truncated squared reprojection error)
# ---------------------------------------------------------------------------
def test_score_single_point_offsets():
    K = (500.0, 450.0, 321.0, 239.0)  # fx != fy, cx != cy catches swapped intrinsics
    R = synth.random_rotation(np.random.default_rng(2))
    t = np.array([0.3, -0.2, 0.5])
    Xc = np.array([[1.0, -0.5, 6.0]])
    Xw = (Xc - t) @ R
    u = K[0] * 1.0 / 6.0 + K[2]
    v = K[1] * -0.5 / 6.0 + K[3]
    for dx, dy, w, want, inl in [(3.0, 0.0, 1.0, 9.0, 1), (0.0, -3.5, 2.0, 2 * 12.25, 1), (5.0, 0.0, 1.5, 1.5 * 16, 0),
                                 (2.0, 2.0, 1.0, 8.0, 1), (3.0, 3.0, 0.5, 0.5 * 16, 0)]:
        c = oracle.Corr([u + dx], [v + dy], Xw, [w])
        s, n = oracle.score(c, K, R, t, 4.0)
        assert s == pytest.approx(want, rel=1e-9) and n == inl


def test_score_at_ground_truth_equals_outlier_mass():
    rng = np.random.default_rng(4)
    n = 3000
    K = (600.0, 600.0, 400.0, 300.0)
    R = synth.random_rotation(rng)
    t = rng.normal(size=3)
    u = rng.uniform(0, 800, n); v = rng.uniform(0, 600, n); d = rng.uniform(2, 30, n)
    Xw = (np.column_stack([(u - 400) / 600 * d, (v - 300) / 600 * d, d]) - t) @ R
    out = rng.random(n) < 0.6
    ang = rng.uniform(0, 2 * np.pi, n)
    off = rng.uniform(12.0, 80.0, n)  # outliers at least 3 tau from their projection
    x = np.where(out, u + off * np.cos(ang), u)
    y = np.where(out, v + off * np.sin(ang), v)
    behind = rng.random(n) < 0.05  # a few points behind the camera: outliers
    Xw[behind] = (np.column_stack([u[behind] - 400, v[behind] - 300, -d[behind]]) - t) @ R
    w = rng.uniform(0.1, 1.0, n)
    c = oracle.Corr(x, y, Xw, w)
    s, cnt = oracle.score(c, K, R, t, 4.0)
    bad = out | behind
    assert cnt == int((~bad).sum())
    assert s == pytest.approx(16.0 * w[bad].sum(), rel=1e-9, abs=1e-6)
    # homogeneous in the weights, invariant to the order of correspondences
    s2, _ = oracle.score(oracle.Corr(x, y, Xw, 2 * w), K, R, t, 4.0)
    assert s2 == pytest.approx(2 * s, rel=1e-12)
    p = rng.permutation(n)
    s3, cnt3 = oracle.score(oracle.Corr(x[p], y[p], Xw[p], w[p]), K, R, t, 4.0)
    assert s3 == pytest.approx(s, rel=1e-12) and cnt3 == cnt
    # a subset given by indices equals the score of the gathered subset
    idx = oracle.subsample(n, 700)
    s4, c4 = oracle.score(c, K, R, t, 4.0, idx=idx)
    s5, c5 = oracle.score(oracle.Corr(x[idx], y[idx], Xw[idx], w[idx]), K, R, t, 4.0)
    assert s4 == pytest.approx(s5, rel=1e-12) and c4 == c5


# ---------------------------------------------------------------------------
# LO (Gauss-Newton on the truncated loss) and the final Cauchy refinement
# ---------------------------------------------------------------------------
def _noisy_query(seed, n=1500, ratio=0.5, noise=1.0):
    rng = np.random.default_rng(seed)
    q = synth.direct_query(rng, n, ratio, 800, 600, 700.0, noise_px=noise, weights="conf")
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    return q, c, rng


def _perturb(R, t, rng, rot_deg_=0.5, trans=0.05):
    dR = synth.axis_angle(rng.normal(size=3), math.radians(rot_deg_))
    return dR @ R, t + rng.normal(size=3) * trans


def _residuals(c, K, R, t, sel):
    fx, fy, cx, cy = K
    Xc = c.X[sel] @ R.T + t
    return np.concatenate([fx * Xc[:, 0] / Xc[:, 2] + cx - c.x[sel], fy * Xc[:, 1] / Xc[:, 2] + cy - c.y[sel]])


def test_lo_is_stationary_and_matches_scipy_least_squares():
    q, c, rng = _noisy_query(21)
    K = q["K"]
    R0, t0 = _perturb(q["R_gt"], q["t_gt"], rng, 0.3, 0.03)
    s0, _ = oracle.score(c, K, R0, t0, 4.0)
    R1, t1, s1 = oracle.lo(c, K, R0, t0, 4.0, iters=50)
    assert s1 < s0
    s1b, _ = oracle.score(c, K, R1, t1, 4.0)
    assert s1 == pytest.approx(s1b, rel=1e-12)
    # inlier set of the LO output; on it the weighted least-squares problem is
    # solved independently by SciPy (rotation-vector parametrisation)
    fx, fy, cx, cy = K
    Xc = c.X @ R1.T + t1
    r2 = (fx * Xc[:, 0] / Xc[:, 2] + cx - c.x) ** 2 + (fy * Xc[:, 1] / Xc[:, 2] + cy - c.y) ** 2
    sel = np.nonzero((Xc[:, 2] > 0) & (r2 < 16.0))[0]
    sw = np.sqrt(np.concatenate([c.w[sel], c.w[sel]]))

    def fun(p):
        Rp = Rotation.from_rotvec(p[:3]).as_matrix() @ R1
        return sw * _residuals(c, K, Rp, p[3:] + t1, sel)

    sol = scipy.optimize.least_squares(fun, np.zeros(6), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    R_ls = Rotation.from_rotvec(sol.x[:3]).as_matrix() @ R1
    t_ls = sol.x[3:] + t1
    # agreement to the flatness of a converged least-squares cost (1e-6 rad, 10 um)
    assert Rotation.from_matrix(R_ls @ R1.T).magnitude() < 1e-6
    assert np.linalg.norm(centre(R_ls, t_ls) - centre(R1, t1)) < 1e-5
    # stationarity on that set: the decrease a further Gauss-Newton step would
    # predict, f^T J (J^T J)^-1 J^T f with J from central differences of the
    # residuals, is within the stopping rule (1e-6 of the cost)
    h = 1e-7
    f0 = fun(np.zeros(6))
    J = np.stack([(fun(np.eye(6)[k] * h) - fun(-np.eye(6)[k] * h)) / (2 * h) for k in range(6)], 1)
    Jf = J.T @ f0
    predicted = float(Jf @ np.linalg.solve(J.T @ J, Jf))
    assert predicted <= 1e-6 * float(f0 @ f0)
    # first order, directly: the gradient of the weighted squared residuals on
    # that set, by central differences of the cost, is within the bound that
    # the stopping rule implies.  A Gauss-Newton step predicts the decrease
    # g^T (J^T J)^-1 g >= |g|^2 / lambda_max(J^T J) (g = J^T f), and the loop
    # stops once an accepted step lowers the truncated cost C by < 1e-6 of C,
    # so at the output |J^T f| <= sqrt(lambda_max * 1e-6 * C), i.e. the cost's
    # gradient 2 J^T f is at most twice that
    assert _grad_norm(fun) <= _stationarity_bound(J, s1)


def _grad_norm(fun, h=1e-7):
    cost = lambda p: float(fun(p) @ fun(p))  # noqa: E731
    return float(np.linalg.norm([(cost(np.eye(6)[k] * h) - cost(-np.eye(6)[k] * h)) / (2 * h) for k in range(6)]))


def _stationarity_bound(J, truncated_cost):
    return 2.0 * math.sqrt(float(np.linalg.eigvalsh(J.T @ J).max()) * 1e-6 * truncated_cost)


def test_stationarity_bound_rejects_an_unconverged_lo():
    # the same check on an LO cut off after one Gauss-Newton step fails: the
    # bound separates a converged output from one that stopped early
    q, c, rng = _noisy_query(21)
    K = q["K"]
    R0, t0 = _perturb(q["R_gt"], q["t_gt"], rng, 0.3, 0.03)
    R1, t1, s1 = oracle.lo(c, K, R0, t0, 4.0, iters=1)
    fx, fy, cx, cy = K
    Xc = c.X @ R1.T + t1
    r2 = (fx * Xc[:, 0] / Xc[:, 2] + cx - c.x) ** 2 + (fy * Xc[:, 1] / Xc[:, 2] + cy - c.y) ** 2
    sel = np.nonzero((Xc[:, 2] > 0) & (r2 < 16.0))[0]
    sw = np.sqrt(np.concatenate([c.w[sel], c.w[sel]]))

    def fun(p):
        Rp = Rotation.from_rotvec(p[:3]).as_matrix() @ R1
        return sw * _residuals(c, K, Rp, p[3:] + t1, sel)

    h = 1e-7
    J = np.stack([(fun(np.eye(6)[k] * h) - fun(-np.eye(6)[k] * h)) / (2 * h) for k in range(6)], 1)
    assert _grad_norm(fun) > 10 * _stationarity_bound(J, s1)


def test_lo_never_increases_cost_and_handles_no_inliers():
    q, c, rng = _noisy_query(22, ratio=0.2)
    K = q["K"]
    for _ in range(5):
        R0, t0 = _perturb(q["R_gt"], q["t_gt"], rng, 2.0, 0.2)
        s0, _ = oracle.score(c, K, R0, t0, 4.0)
        _, _, s1 = oracle.lo(c, K, R0, t0, 4.0)
        assert s1 <= s0
    # a pose that sees nothing: LO returns it unchanged
    Rf = q["R_gt"]
    tf = q["t_gt"] + np.array([0, 0, -1e4])
    R1, t1, s1 = oracle.lo(c, K, Rf, tf, 4.0)
    np.testing.assert_array_equal(R1, Rf)
    assert s1 == pytest.approx(16.0 * c.w.sum())


def test_refine_noise_free_recovers_ground_truth():
    q, c, rng = _noisy_query(23, ratio=0.6, noise=0.0)
    K = q["K"]
    R0, t0 = _perturb(q["R_gt"], q["t_gt"], rng, 0.2, 0.02)
    sel = np.nonzero(q["inlier"])[0]
    R1, t1, steps = oracle.refine(c, K, R0, t0, sel, 4.0, 4.0, iters=25)
    assert steps > 0
    assert rot_deg(R1, q["R_gt"]) < 1e-7
    np.testing.assert_allclose(t1, q["t_gt"], atol=1e-9)


def test_refine_matches_generic_minimiser_of_cauchy_cost():
    q, c, rng = _noisy_query(24, ratio=0.6, noise=1.5)
    K = q["K"]
    sel = np.nonzero(q["inlier"])[0]
    R0, t0 = _perturb(q["R_gt"], q["t_gt"], rng, 0.1, 0.01)
    cs = 4.0
    R1, t1, _ = oracle.refine(c, K, R0, t0, sel, cs, 4.0, iters=50)

    def cost(p):
        Rp = Rotation.from_rotvec(p[:3]).as_matrix() @ R1
        r = _residuals(c, K, Rp, p[3:] + t1, sel)
        n = len(sel)
        r2 = r[:n] ** 2 + r[n:] ** 2
        return float(np.sum(c.w[sel] * cs * cs * np.log1p(r2 / (cs * cs))))

    sol = scipy.optimize.minimize(cost, np.zeros(6), method="BFGS", options=dict(gtol=1e-10))
    assert np.linalg.norm(sol.x[:3]) < 1e-6  # radians
    assert np.linalg.norm(sol.x[3:]) < 1e-5  # metres
    # the refinement stops once a step lowers the cost by < 1e-6 of it
    assert cost(np.zeros(6)) <= sol.fun * (1 + 1e-6)


# ---------------------------------------------------------------------------
# Adaptive termination
# ---------------------------------------------------------------------------
def test_needed_iterations_closed_forms():
    assert oracle.needed_iters(0.5, 1e-4) == pytest.approx(math.log(1e-4) / math.log(0.875))
    assert oracle.needed_iters(0.5, 1e-4) == pytest.approx(68.97, abs=0.01)
    assert oracle.needed_iters(0.1, 1e-4) == pytest.approx(9205.73, abs=0.01)  # ln(1e-4)/ln(0.999)
    assert oracle.needed_iters(0.9, 1e-4) == pytest.approx(7.05, abs=0.01)  # ln(1e-4)/ln(0.271)
    assert oracle.needed_iters(1.0, 1e-4) == 0.0
    assert oracle.needed_iters(0.0, 1e-4) == math.inf


def test_adaptive_stop_at_first_round_past_needed():
    q = synth.config1(3)
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    B = 128
    r = oracle.ransac_pnp(c, q["K"], batch=B, max_iters=100000, p_miss=1e-4)
    need = oracle.needed_iters(r["subset_inliers"] / c.n, 1e-4)
    assert r["iterations"] == B * math.ceil(need / B) or r["iterations"] == B * max(1, math.ceil(need / B))
    # with the stop disabled every round runs
    r2 = oracle.ransac_pnp(c, q["K"], batch=B, max_iters=1000, p_miss=0.0)
    assert r2["iterations"] == 1000 and r2["rounds"] == 8


# ---------------------------------------------------------------------------
# End to end
# ---------------------------------------------------------------------------
def test_config1_pose_close_to_ground_truth():
    q = synth.config1(0)
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    r = oracle.ransac_pnp(c, q["K"], max_iters=q["hypotheses"], p_miss=0.0, tau=q["tau"])
    assert r["status"] == 0
    assert rot_deg(r["R"], q["R_gt"]) < 0.05
    assert np.linalg.norm(centre(r["R"], r["t"]) - centre(q["R_gt"], q["t_gt"])) < 0.02
    # the inlier set of the final pose recovers the true inliers
    agree = np.mean(r["inlier_mask"] == q["inlier"])
    assert agree > 0.98


def _tiny_scene(seed, n_in=9, n_out=3):
    rng = np.random.default_rng(seed)
    n = n_in + n_out
    K = (500.0, 500.0, 320.0, 240.0)
    R = synth.random_rotation(rng)
    t = rng.normal(size=3)
    u = rng.uniform(40, 600, n); v = rng.uniform(40, 440, n); d = rng.uniform(3, 15, n)
    Xw = (np.column_stack([(u - 320) / 500 * d, (v - 240) / 500 * d, d]) - t) @ R
    x = u.copy(); y = v.copy()
    ang = rng.uniform(0, 2 * np.pi, n_out)
    x[n_in:] += 60 * np.cos(ang)
    y[n_in:] += 60 * np.sin(ang)
    return K, R, t, x, y, Xw, np.ones(n)


def test_enumerate_all_brute_force_finds_ground_truth():
    K, R, t, x, y, Xw, w = _tiny_scene(31)
    c = oracle.Corr(x, y, Xw, w)
    r = oracle.ransac_pnp(c, K, enumerate_all=1, lo_enabled=0, final_enabled=0, p_miss=0.0)
    assert r["iterations"] == math.comb(12, 3)
    # noise-free: the best model is the true pose, its score the outlier mass
    assert r["score"] == pytest.approx(3 * 16.0, rel=1e-9)
    assert rot_deg(r["R_best"], R) < 1e-7
    assert list(np.nonzero(r["inlier_mask"])[0]) == list(range(9))


def test_permutation_invariance():
    K, R, t, x, y, Xw, w = _tiny_scene(32)
    p = np.random.default_rng(0).permutation(len(x))
    a = oracle.ransac_pnp(oracle.Corr(x, y, Xw, w), K, enumerate_all=1, p_miss=0.0)
    b = oracle.ransac_pnp(oracle.Corr(x[p], y[p], Xw[p], w[p]), K, enumerate_all=1, p_miss=0.0)
    assert rot_deg(a["R"], b["R"]) < 1e-9
    np.testing.assert_array_equal(a["inlier_mask"][p], b["inlier_mask"])
    # sampled run on a full-size query: the final pose agrees within 0.05 deg / 5 mm
    q = synth.config1(5)
    p = np.random.default_rng(1).permutation(2000)
    c1 = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    c2 = oracle.Corr(q["x"][p], q["y"][p], q["X"][p], q["w"][p])
    r1 = oracle.ransac_pnp(c1, q["K"], max_iters=1000, p_miss=0.0)
    r2 = oracle.ransac_pnp(c2, q["K"], max_iters=1000, p_miss=0.0)
    assert rot_deg(r1["R"], r2["R"]) < 0.05
    assert np.linalg.norm(centre(r1["R"], r1["t"]) - centre(r2["R"], r2["t"])) < 0.005


def test_config2_lift_then_ransac_close_to_ground_truth():
    q = synth.config2(0)
    L = oracle.lift(q["views"], q["matches"])
    c = oracle.Corr(L["x"], L["y"], L["X"], L["w"])
    r = oracle.ransac_pnp(c, q["K"], max_iters=2048, p_miss=0.0)
    assert r["status"] == 0
    assert rot_deg(r["R"], q["R_gt"]) < 0.05
    assert np.linalg.norm(centre(r["R"], r["t"]) - centre(q["R_gt"], q["t_gt"])) < 0.02
