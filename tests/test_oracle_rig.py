"""Pins of the rig oracle (supplementary "LaMAR HoloLens Results": generalized
absolute pose of a multi-camera rig, the Sec. 3.3 loop with a generalized P3P
and per-camera residuals) against facts that do not come from the oracle:
ground truth, exactness of every solution, the single-camera P3P (Grunert's
independent formulation) as the special case of coincident ray origins, a
generic root finder for completeness, closed forms of the rig projection,
SciPy least squares for LO, and noise-free recovery end to end."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import synth

scipy = pytest.importorskip("scipy")
import scipy.optimize  # noqa: E402
from scipy.spatial.transform import Rotation  # noqa: E402


def _rays(rng, spread_o=0.3):
    """Three rays of a generalized camera through three world points of a known
    rig pose: origins scattered by spread_o (0 = one centre)."""
    R = synth.random_rotation(rng)
    t = rng.normal(size=3)
    o = rng.normal(size=(3, 3)) * spread_o
    Pr = np.column_stack([rng.uniform(-4, 4, 3), rng.uniform(-4, 4, 3), rng.uniform(2, 20, 3)])
    Xw = (Pr - t) @ R
    d = Pr - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return R, t, o, d, Xw


def test_gp3p_recovers_ground_truth():
    rng = np.random.default_rng(31)
    worst = 0.0
    for _ in range(500):
        R, t, o, d, Xw = _rays(rng)
        sols = oracle.gp3p(o, d, Xw)
        assert 1 <= len(sols) <= 8
        e = min(max(np.abs(Rs - R).max(), np.abs(ts - t).max() / max(1.0, np.linalg.norm(t))) for Rs, ts, _ in sols)
        worst = max(worst, e)
    assert worst <= 1e-9


def test_gp3p_every_solution_is_exact_and_ordered():
    rng = np.random.default_rng(32)
    for _ in range(300):
        _, _, o, d, Xw = _rays(rng, spread_o=1.0)
        sols = oracle.gp3p(o, d, Xw)
        lam1 = [s[2][0] for s in sols]
        assert lam1 == sorted(lam1)
        for Rs, ts, lam in sols:
            np.testing.assert_allclose(Rs @ Rs.T, np.eye(3), atol=1e-12)
            assert np.linalg.det(Rs) > 0
            assert np.all(lam > 0)
            P = Xw @ Rs.T + ts
            np.testing.assert_allclose(P, o + lam[:, None] * d, atol=1e-9 * (1 + np.abs(P).max()))


def test_gp3p_with_one_centre_is_p3p():
    """Coincident ray origins make the problem the single-camera P3P; the
    oracle's P3P is Grunert's quartic, an independent derivation.  With the
    common centre c, a P3P pose (R, t) of the bearings is the rig pose
    (R, t + c)."""
    rng = np.random.default_rng(33)
    for _ in range(300):
        _, _, o, d, Xw = _rays(rng, spread_o=0.0)
        c = rng.normal(size=3)
        o = np.tile(c, (3, 1))
        g = oracle.gp3p(o, d, Xw)
        p = oracle.p3p(d, Xw)
        assert len(g) == len(p)
        for (Rg, tg, lg), (Rp, tp, lp) in zip(g, p):
            np.testing.assert_allclose(lg, lp, rtol=1e-8)
            np.testing.assert_allclose(Rg, Rp, atol=1e-8)
            np.testing.assert_allclose(tg, tp + c, atol=1e-7 * (1 + np.abs(tp).max()))


def test_gp3p_with_one_centre_matches_p3p_on_image_like_triples():
    """Bearings of pixels of a 640x480 image at f = 500 and points scattered by
    5 m: far, nearly degenerate solutions included (the octic's coefficients
    then span 20 orders of magnitude)."""
    rng = np.random.default_rng(46)
    for _ in range(3000):
        px = rng.uniform(-1, 1, (3, 2)) * [320, 240]
        b = np.column_stack([px / 500.0, np.ones(3)])
        b /= np.linalg.norm(b, axis=1, keepdims=True)
        X = rng.normal(size=(3, 3)) * 5
        g = oracle.gp3p(np.zeros((3, 3)), b, X)
        p = oracle.p3p(b, X)
        assert len(g) == len(p)
        for (_, _, lg), (_, _, lp) in zip(g, p):
            np.testing.assert_allclose(lg, lp, rtol=1e-6)


def test_gp3p_finds_all_solutions_against_generic_root_finding():
    """Solve the three distance equations along the rays with SciPy's generic
    root finder from many starts; every positive solution found there must be
    in the oracle's list."""
    rng = np.random.default_rng(34)
    multi = 0
    for _ in range(25):
        _, _, o, d, Xw = _rays(rng, spread_o=2.0)
        pairs = [(0, 1), (0, 2), (1, 2)]
        D2 = [np.sum((Xw[i] - Xw[j]) ** 2) for i, j in pairs]

        def F(L):
            return [np.sum((o[i] + L[i] * d[i] - o[j] - L[j] * d[j]) ** 2) - D2[e] for e, (i, j) in enumerate(pairs)]

        found = []
        scale = math.sqrt(max(D2))
        for _ in range(200):
            L0 = rng.uniform(0.05, 4.0, 3) * scale * 3
            sol, info, ier, _ = scipy.optimize.fsolve(F, L0, full_output=True, xtol=1e-13)
            if ier == 1 and np.all(sol > 0) and np.max(np.abs(F(sol))) < 1e-8 * max(D2):
                if not any(np.allclose(sol, f, rtol=1e-6) for f in found):
                    found.append(sol)
        lams = [s[2] for s in oracle.gp3p(o, d, Xw)]
        multi += len(found) > 1
        for f in found:
            assert any(np.allclose(f, lam, rtol=1e-6) for lam in lams), (f, lams)
    assert multi > 0


# ---------------------------------------------------------------------------
def _rig_of(q):
    return oracle.rig(q["K"], q["R_cam"], q["t_cam"])


def test_rig_score_with_one_identity_camera_is_the_single_camera_score():
    q = synth.direct_query(np.random.default_rng(35), 800, 0.4, 640, 480, 500.0, weights="conf")
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    rg = oracle.rig([q["K"]], [np.eye(3)], [np.zeros(3)])
    cam = np.zeros(c.n, np.int32)
    rng = np.random.default_rng(36)
    for _ in range(5):
        R = synth.axis_angle(rng.normal(size=3), rng.uniform(0, 0.05)) @ q["R_gt"]
        t = q["t_gt"] + rng.normal(size=3) * 0.05
        assert oracle.rig_score(c, cam, rg, R, t, 4.0) == oracle.score(c, q["K"], R, t, 4.0)


def test_rig_score_is_the_sum_of_per_camera_scores_with_composed_poses():
    """Camera k of the rig sees the world through cam_from_world =
    (R_k R, R_k t + t_k): the rig score is the sum over cameras of the
    single-camera scores with those composed poses."""
    q = synth.rig_query(np.random.default_rng(37), n_per_cam=300, weights="conf")
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    rg = _rig_of(q)
    rng = np.random.default_rng(38)
    for _ in range(5):
        R = synth.axis_angle(rng.normal(size=3), rng.uniform(0, 0.03)) @ q["R_gt"]
        t = q["t_gt"] + rng.normal(size=3) * 0.03
        s, n = oracle.rig_score(c, q["cam"], rg, R, t, 4.0)
        tot, cnt = 0.0, 0
        for k in range(4):
            sel = np.nonzero(q["cam"] == k)[0]
            sk, nk = oracle.score(c, q["K"][k], q["R_cam"][k] @ R, q["R_cam"][k] @ t + q["t_cam"][k], 4.0, idx=sel)
            tot += sk
            cnt += nk
        assert s == pytest.approx(tot, rel=1e-10) and n == cnt


def test_rig_score_single_point_offsets():
    """A point seen by camera 2 of a rig: exact pixel offsets give the
    closed-form truncated costs."""
    rng = np.random.default_rng(39)
    R_cam, t_cam = synth.rig_layout(rng, 3)
    K = [(500.0, 450.0, 321.0, 239.0)] * 3
    rg = oracle.rig(K, R_cam, t_cam)
    R = synth.random_rotation(rng)
    t = rng.normal(size=3)
    Xc = np.array([1.0, -0.5, 6.0])
    Xw = (R_cam[2].T @ (Xc - t_cam[2]) - t) @ R
    u = 500.0 * 1.0 / 6.0 + 321.0
    v = 450.0 * -0.5 / 6.0 + 239.0
    for dx, dy, w, want, inl in [(3.0, 0.0, 1.0, 9.0, 1), (0.0, -3.5, 2.0, 24.5, 1), (5.0, 0.0, 1.5, 24.0, 0)]:
        c = oracle.Corr([u + dx], [v + dy], Xw[None], [w])
        s, n = oracle.rig_score(c, np.array([2], np.int32), rg, R, t, 4.0)
        assert s == pytest.approx(want, rel=1e-9) and n == inl


def _rig_residuals(c, q, R, t, sel):
    out = []
    for i in sel:
        k = q["cam"][i]
        fx, fy, cx, cy = q["K"][k]
        Xc = q["R_cam"][k] @ (R @ c.X[i] + t) + q["t_cam"][k]
        out.append([fx * Xc[0] / Xc[2] + cx - c.x[i], fy * Xc[1] / Xc[2] + cy - c.y[i]])
    out = np.array(out)
    return np.concatenate([out[:, 0], out[:, 1]])


def test_rig_lo_matches_scipy_least_squares():
    q = synth.rig_query(np.random.default_rng(40), n_per_cam=150, weights="conf")
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    rg = _rig_of(q)
    rng = np.random.default_rng(41)
    R0 = synth.axis_angle(rng.normal(size=3), math.radians(0.3)) @ q["R_gt"]
    t0 = q["t_gt"] + rng.normal(size=3) * 0.01
    s0, _ = oracle.rig_score(c, q["cam"], rg, R0, t0, 4.0)
    R1, t1, s1 = oracle.rig_lo(c, q["cam"], rg, R0, t0, 4.0, iters=50)
    assert s1 < s0
    assert oracle.rig_score(c, q["cam"], rg, R1, t1, 4.0)[0] == pytest.approx(s1, rel=1e-12)
    r = _rig_residuals(c, q, R1, t1, range(c.n))
    n = c.n
    sel = np.nonzero(r[:n] ** 2 + r[n:] ** 2 < 16.0)[0]
    sw = np.sqrt(np.concatenate([c.w[sel], c.w[sel]]))

    def fun(p):
        Rp = Rotation.from_rotvec(p[:3]).as_matrix() @ R1
        return sw * _rig_residuals(c, q, Rp, Rotation.from_rotvec(p[:3]).as_matrix() @ t1 + p[3:], sel)

    sol = scipy.optimize.least_squares(fun, np.zeros(6), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    R_ls = Rotation.from_rotvec(sol.x[:3]).as_matrix() @ R1
    assert Rotation.from_matrix(R_ls @ R1.T).magnitude() < 1e-6
    t_ls = Rotation.from_rotvec(sol.x[:3]).as_matrix() @ t1 + sol.x[3:]
    assert np.linalg.norm(R_ls.T @ t_ls - R1.T @ t1) < 1e-5


def test_rig_refine_noise_free_recovers_ground_truth():
    q = synth.rig_query(np.random.default_rng(42), n_per_cam=100, inlier_ratio=1.0, noise_px=0.0)
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    rg = _rig_of(q)
    rng = np.random.default_rng(43)
    R0 = synth.axis_angle(rng.normal(size=3), math.radians(0.5)) @ q["R_gt"]
    t0 = q["t_gt"] + rng.normal(size=3) * 0.02
    R1, t1, steps = oracle.rig_refine(c, q["cam"], rg, R0, t0, np.arange(c.n), 4.0, 4.0, iters=50)
    assert steps > 0
    # float32 inputs: agreement to their rounding
    assert Rotation.from_matrix(R1 @ q["R_gt"].T).magnitude() < 1e-6
    assert np.linalg.norm(t1 - q["t_gt"]) < 1e-5


def test_rig_ransac_recovers_the_pose_with_outliers():
    q = synth.rig_query(np.random.default_rng(44), n_per_cam=400, inlier_ratio=0.35, weights="conf")
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    res = oracle.rig_ransac(c, q["cam"], _rig_of(q), max_iters=4000, batch=256, seed=7)
    assert res["status"] == 0
    assert Rotation.from_matrix(res["R"] @ q["R_gt"].T).magnitude() < math.radians(0.1)
    assert np.linalg.norm(res["R"].T @ res["t"] - q["R_gt"].T @ q["t_gt"]) < 0.01
    assert res["best_hyp"] >= 0 and res["best_hyp"] % 8 < 8
    inl = res["inlier_mask"]
    assert (inl & q["inlier"]).sum() >= 0.95 * q["inlier"].sum()


def test_rig_ransac_noise_free_minimal_pose_is_exact():
    """Cameras up to 1 m apart, noise-free inliers, no LO and no refinement:
    the best GP3P hypothesis itself is the ground-truth pose (this pins the
    rays that the loop builds from pixels and the rig)."""
    q = synth.rig_query(np.random.default_rng(47), n_per_cam=200, inlier_ratio=0.6, noise_px=0.0, baseline=1.0)
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    res = oracle.rig_ransac(c, q["cam"], _rig_of(q), max_iters=512, batch=512, seed=9, lo_enabled=0,
                            final_enabled=0)
    assert Rotation.from_matrix(res["R_best"] @ q["R_gt"].T).magnitude() < 1e-6
    assert np.linalg.norm(res["t_best"] - q["t_gt"]) < 1e-5


def test_rig_ransac_with_one_identity_camera_matches_the_single_camera_loop():
    """Same samples, GP3P poses equal to the P3P poses up to rounding: the
    same hypotheses, the same rounds and best sample, the final poses agree."""
    q = synth.direct_query(np.random.default_rng(45), 1500, 0.3, 640, 480, 500.0, weights="conf")
    c = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    rg = oracle.rig([q["K"]], [np.eye(3)], [np.zeros(3)])
    a = oracle.rig_ransac(c, np.zeros(c.n, np.int32), rg, max_iters=2048, batch=512, seed=3)
    b = oracle.ransac_pnp(c, q["K"], max_iters=2048, batch=512, seed=3)
    assert a["rounds"] == b["rounds"] and a["hypotheses"] == b["hypotheses"]
    assert a["best_hyp"] // 8 == b["best_hyp"] // 4
    np.testing.assert_allclose(a["R"], b["R"], atol=1e-9)
    np.testing.assert_allclose(a["t"], b["t"], atol=1e-8)
    assert a["num_inliers"] == b["num_inliers"]
