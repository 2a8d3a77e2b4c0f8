"""GPU LO-RANSAC of the generalized absolute pose of a camera rig (through the
C ABI; supplementary "LaMAR HoloLens Results") against the FP64 rig oracle.

Bars (as for the single-camera loop):
  minimal-sample indices      bit-exact (integer Philox arithmetic);
  GP3P poses                  per solution |R - R'|_F <= 1e-4 and
                              |t - t'| <= 1e-4 max(1, |t'|), matched as sets;
                              100% on well-conditioned samples (the pose moves
                              < 1e-5 under float32-level pixel perturbation);
  per-pose score              1e-5 relative (float32 sums);
  per-pose inlier count       exact except points within 1e-3 px of tau;
  final pose                  0.05 deg and 5 mm.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import pose_close, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = imloc.Context(0, 1 << 30)
    yield c
    c.close()


def upload(q):
    t = torch()
    c = imloc.corr_from_arrays(q["x"], q["y"], q["X"], q["w"])
    cam = t.from_numpy(np.ascontiguousarray(q["cam"], np.int32)).cuda()
    return c, cam


def rays(q, idx):
    """Rays of correspondences idx in the rig frame (test-side input plumbing
    for the oracle's GP3P)."""
    o, d = [], []
    for i in idx:
        k = int(q["cam"][i])
        fx, fy, cx, cy = q["K"][k]
        b = np.array([(float(q["x"][i]) - cx) / fx, (float(q["y"][i]) - cy) / fy, 1.0])
        b /= np.linalg.norm(b)
        d.append(q["R_cam"][k].T @ b)
        o.append(-q["R_cam"][k].T @ q["t_cam"][k])
    return np.array(o), np.array(d)


def run_debug(ctx, q, H, batch=512, **kw):
    t = torch()
    c, cam = upload(q)
    n = len(q["x"])
    opts = imloc.default_opts(max_iters=H, batch=batch, p_miss=0.0, **kw)
    R = (H + batch - 1) // batch
    dbg = dict(triples=t.full((3 * H,), -2, dtype=t.int32, device="cuda"),
               poses=t.zeros((8 * H, 12), dtype=t.float32, device="cuda"),
               scores=t.zeros((8 * H,), dtype=t.float32, device="cuda"),
               counts=t.zeros((8 * H,), dtype=t.int32, device="cuda"),
               round_best=t.zeros((R,), dtype=t.int64, device="cuda"))
    mask = t.zeros(max(n, 1), dtype=t.uint8, device="cuda")
    res = ctx.testing_rig(c, cam, imloc.rig(q["K"], q["R_cam"], q["t_cam"]), opts, n, dbg, mask=mask)
    host = {k: v.cpu().numpy() for k, v in dbg.items()}
    host["mask"] = mask[:n].cpu().numpy().astype(bool)
    return res, host


@pytest.fixture(scope="module")
def rig_run(ctx):
    q = synth.rig_query(np.random.default_rng(60), n_per_cam=400, inlier_ratio=0.35, weights="conf", baseline=0.3)
    res, dbg = run_debug(ctx, q, 2048)
    return q, res, dbg


def test_minimal_samples_bit_exact(rig_run):
    q, res, dbg = rig_run
    tri = dbg["triples"].reshape(-1, 3)
    m = len(q["x"])
    for s in range(len(tri)):
        ref, att = oracle.sample(0, 0, s, m)
        if ref is None:
            assert tri[s][0] == -1
        else:
            assert list(tri[s]) == list(ref), s


def _match(gpu, ref_R, ref_t):
    return any(np.linalg.norm(Rg - ref_R) <= 1e-4 and np.linalg.norm(tg - ref_t) <= 1e-4 * max(1.0, np.linalg.norm(ref_t))
               for Rg, tg in gpu)


def test_gp3p_poses_against_oracle(rig_run):
    q, res, dbg = rig_run
    rng = np.random.default_rng(1)
    tri = dbg["triples"].reshape(-1, 3)
    poses = dbg["poses"].reshape(-1, 8, 12)
    scores = dbg["scores"].reshape(-1, 8)
    total = matched = well = well_matched = extra = 0
    misses = []
    for s in range(len(tri)):
        if tri[s][0] < 0:
            continue
        idx = tri[s]
        o, d = rays(q, idx)
        X = q["X"][idx].astype(np.float64)
        sols = oracle.gp3p(o, d, X)
        gpu = [(poses[s, k, :9].reshape(3, 3).astype(np.float64), poses[s, k, 9:].astype(np.float64))
               for k in range(8) if not np.isnan(scores[s, k])]
        for Ro, to, lam in sols:
            total += 1
            ok = _match(gpu, Ro, to)
            matched += ok
            # conditioning: re-solve with the pixels moved by 1e-4 px
            qq = dict(q)
            qq["x"] = q["x"].astype(np.float64).copy()
            qq["y"] = q["y"].astype(np.float64).copy()
            qq["x"][idx] += rng.normal(size=3) * 1e-4
            qq["y"][idx] += rng.normal(size=3) * 1e-4
            o2, d2 = rays(qq, idx)
            moved = min([np.linalg.norm(R2 - Ro) + np.linalg.norm(t2 - to) / max(1.0, np.linalg.norm(to))
                         for R2, t2, _ in oracle.gp3p(o2, d2, X)] or [1.0])
            if moved < 1e-5:
                well += 1
                well_matched += ok
                if not ok:
                    misses.append((s, moved, len(sols), len(gpu)))
        for Rg, tg in gpu:
            if not any(np.linalg.norm(Rg - Ro) <= 1e-3 for Ro, _, _ in sols):
                extra += 1
    print(f"gp3p: {matched}/{total} matched, well-conditioned {well_matched}/{well}, extra {extra}")
    assert total > 1500
    assert well_matched == well, misses[:10]
    assert matched >= 0.995 * total
    assert extra <= 0.005 * total


def test_scores_and_counts_against_oracle(rig_run):
    q, res, dbg = rig_run
    corr = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    rg = oracle.rig(q["K"], q["R_cam"], q["t_cam"])
    poses, scores, counts = dbg["poses"], dbg["scores"], dbg["counts"]
    ids = np.nonzero(~np.isnan(scores))[0]
    assert len(ids) > 1000
    for pid in ids[::4]:
        R = poses[pid, :9].reshape(3, 3).astype(np.float64)
        t = poses[pid, 9:].astype(np.float64)
        s_ref, c_ref = oracle.rig_score(corr, q["cam"], rg, R, t, 4.0)
        assert scores[pid] == pytest.approx(s_ref, rel=1e-5, abs=1e-3), pid
        # points within 1e-3 px of tau may fall either side in float32
        near = 0
        for k in range(len(q["K"])):
            sel = np.nonzero(q["cam"] == k)[0]
            fx, fy, cx, cy = q["K"][k]
            Xc = (q["X"][sel].astype(np.float64) @ R.T + t) @ q["R_cam"][k].T + q["t_cam"][k]
            with np.errstate(divide="ignore", invalid="ignore"):
                r = np.hypot(fx * Xc[:, 0] / Xc[:, 2] + cx - q["x"][sel], fy * Xc[:, 1] / Xc[:, 2] + cy - q["y"][sel])
            near += int(np.sum((Xc[:, 2] > 0) & (np.abs(r - 4.0) <= 1e-3)))
        assert abs(int(counts[pid]) - c_ref) <= near, (pid, counts[pid], c_ref, near)


def test_round_best_is_the_argmin(rig_run):
    q, res, dbg = rig_run
    scores = dbg["scores"]
    for r in range(len(dbg["round_best"])):
        ids = np.nonzero(~np.isnan(scores[8 * 512 * r:8 * 512 * (r + 1)]))[0] + 8 * 512 * r
        key = int(dbg["round_best"][r]) & 0xFFFFFFFFFFFFFFFF
        order = np.lexsort((ids, scores[ids]))
        assert (key & 0xFFFFFFFF) == ids[order[0]]


def test_end_to_end_against_oracle(rig_run):
    q, res, dbg = rig_run
    ref = oracle.rig_ransac(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["cam"],
                            oracle.rig(q["K"], q["R_cam"], q["t_cam"]), max_iters=2048, batch=512, p_miss=0.0)
    assert res["status"] == 0 and ref["status"] == 0
    np.testing.assert_allclose(res["R"] @ res["R"].T, np.eye(3), atol=1e-9)
    assert pose_close(res["R"], res["t"], ref["R"], ref["t"])
    assert pose_close(res["R"], res["t"], q["R_gt"], q["t_gt"], deg=0.2, mm=20.0)
    assert abs(res["num_inliers"] - ref["num_inliers"]) <= max(3, 0.01 * ref["num_inliers"])
    assert res["hypotheses"] == int(np.sum(~np.isnan(dbg["scores"])))


def test_lo_and_refine_from_injected_pose(ctx):
    rng = np.random.default_rng(61)
    q = synth.rig_query(rng, n_per_cam=600, inlier_ratio=0.5, weights="conf", baseline=0.3)
    dR = synth.axis_angle(rng.normal(size=3), math.radians(0.3))
    R0, t0 = dR @ q["R_gt"], q["t_gt"] + rng.normal(size=3) * 0.02
    inj = torch().from_numpy(np.concatenate([R0.ravel(), t0]).astype(np.float32)[None]).cuda()
    R0f = inj[0, :9].cpu().numpy().astype(np.float64).reshape(3, 3)
    t0f = inj[0, 9:].cpu().numpy().astype(np.float64)
    c, cam = upload(q)
    rg = imloc.rig(q["K"], q["R_cam"], q["t_cam"])
    corr = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    org = oracle.rig(q["K"], q["R_cam"], q["t_cam"])
    n = len(q["x"])
    opts = imloc.default_opts(max_iters=1, batch=1, p_miss=0.0, final_iters=0, lo_iters=10)
    res = ctx.testing_rig(c, cam, rg, opts, n, dict(inject_poses=inj))
    R1, t1, s1 = oracle.rig_lo(corr, q["cam"], org, R0f, t0f, 4.0, iters=10)
    assert res["lo_count"] == 1
    assert pose_close(res["R_best"], res["t_best"], R1, t1, deg=0.005, mm=0.5)
    assert res["score"] == pytest.approx(s1, rel=1e-4)
    opts = imloc.default_opts(max_iters=1, batch=1, p_miss=0.0, final_iters=25, lo_iters=0)
    res = ctx.testing_rig(c, cam, rg, opts, n, dict(inject_poses=inj))
    _, inl = oracle.rig_score(corr, q["cam"], org, R0f, t0f, 4.0)
    sel = []
    for i in range(n):
        s_i, c_i = oracle.rig_score(corr, q["cam"], org, R0f, t0f, 4.0, idx=[i])
        if c_i:
            sel.append(i)
    assert len(sel) == inl
    R2, t2, _ = oracle.rig_refine(corr, q["cam"], org, R0f, t0f, sel, 4.0, 4.0, iters=25)
    assert pose_close(res["R"], res["t"], R2, t2, deg=0.005, mm=0.5)


def _batch(ctx, qs, opts_list):
    t = torch()
    xs = np.concatenate([q["x"] for q in qs]); ys = np.concatenate([q["y"] for q in qs])
    Xs = np.concatenate([q["X"] for q in qs]); ws = np.concatenate([q["w"] for q in qs])
    cams = np.concatenate([q["cam"] for q in qs]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum([len(q["x"]) for q in qs])]).astype(np.int64)
    c = imloc.corr_from_arrays(xs, ys, Xs, ws)
    cam = t.from_numpy(cams).cuda()
    d_off = t.from_numpy(off).cuda()
    rigs = [imloc.rig(q["K"], q["R_cam"], q["t_cam"]) for q in qs]
    out = t.zeros(len(qs) * imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
    masks = t.zeros(int(off[-1]), dtype=t.uint8, device="cuda")
    ctx.ransac_rig_batch(c, cam, d_off, rigs, opts_list, out, masks=masks)
    return imloc.results_from_bytes(out.cpu().numpy(), len(qs)), masks.cpu().numpy(), off


def test_batch_with_adaptive_stop_against_oracle(ctx):
    """Several rigs (2 to 5 cameras, different sizes) in one call with the
    adaptive stop: each query as the oracle runs it alone."""
    rng = np.random.default_rng(62)
    qs = [synth.rig_query(rng, n_per_cam=int(rng.integers(200, 900)), inlier_ratio=float(rng.uniform(0.25, 0.6)),
                          n_cams=int(rng.integers(2, 6)), weights="conf", baseline=0.2) for _ in range(6)]
    opts = [imloc.default_opts(max_iters=20000, batch=256, seed=5, query_id=i) for i in range(len(qs))]
    res, masks, off = _batch(ctx, qs, opts)
    for i, q in enumerate(qs):
        ref = oracle.rig_ransac(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["cam"],
                                oracle.rig(q["K"], q["R_cam"], q["t_cam"]), max_iters=20000, batch=256, seed=5,
                                query_id=i)
        assert res[i]["status"] == 0
        assert res[i]["rounds"] == ref["rounds"], (i, res[i]["rounds"], ref["rounds"])
        assert pose_close(res[i]["R"], res[i]["t"], ref["R"], ref["t"]), i
        m = masks[off[i]:off[i + 1]].astype(bool)
        assert int(m.sum()) == res[i]["num_inliers"]
        assert abs(res[i]["num_inliers"] - ref["num_inliers"]) <= max(3, 0.01 * ref["num_inliers"])


def test_one_identity_camera_matches_the_single_camera_path(ctx):
    q = synth.direct_query(np.random.default_rng(63), 2000, 0.3, 640, 480, 500.0, weights="conf")
    q.update(cam=np.zeros(2000, np.int32), K=[q["K"]], R_cam=[np.eye(3)], t_cam=[np.zeros(3)])
    res, _, _ = _batch(ctx, [q], [imloc.default_opts(max_iters=4096, batch=1024, seed=2)])
    c = imloc.corr_from_arrays(q["x"], q["y"], q["X"], q["w"])
    ref = ctx.ransac_pnp(c, q["K"][0], opts=imloc.default_opts(max_iters=4096, batch=1024, seed=2))
    assert res[0]["status"] == 0 and ref["status"] == 0
    assert pose_close(res[0]["R"], res[0]["t"], ref["R"], ref["t"])
    assert res[0]["best_hyp"] // 8 == ref["best_hyp"] // 4


def test_bad_camera_index_and_degenerate_queries(ctx):
    rng = np.random.default_rng(64)
    good = synth.rig_query(rng, n_per_cam=100, n_cams=2)
    bad = synth.rig_query(rng, n_per_cam=100, n_cams=2)
    bad["cam"] = bad["cam"].copy()
    bad["cam"][7] = 2  # the rig has cameras 0 and 1
    tiny = synth.rig_query(rng, n_per_cam=1, n_cams=2)  # 2 correspondences
    res, masks, off = _batch(ctx, [good, bad, tiny], [imloc.default_opts(max_iters=2048, batch=512)] * 3)
    assert res[0]["status"] == 0
    assert res[1]["status"] == -1  # invalid argument
    assert res[2]["status"] == -7


def test_invalid_rigs_and_options_are_rejected(ctx):
    q = synth.rig_query(np.random.default_rng(65), n_per_cam=50, n_cams=2)
    for mutate in ("no_cams", "nine_cams", "zero_focal", "enumerate"):
        rg = imloc.rig(q["K"], q["R_cam"], q["t_cam"])
        opts = imloc.default_opts(max_iters=512, batch=256)
        if mutate == "no_cams":
            rg.n_cams = 0
        elif mutate == "nine_cams":
            rg.n_cams = 9
        elif mutate == "zero_focal":
            rg.cams[1].fx = 0.0
        else:
            opts.enumerate_all = 1
        t = torch()
        c, cam = upload(q)
        off = t.tensor([0, len(q["x"])], dtype=t.int64, device="cuda")
        out = t.zeros(imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
        with pytest.raises(imloc.ImlocError):
            ctx.ransac_rig_batch(c, cam, off, [rg], [opts], out)
