"""Both scoring kernels, each forced for every call of a context
(imloc_set_scoring): the FP32 one and the tensor-core one (which large
unfused batches take by default) with each of its variants, against the FP64
oracle: per-pose truncated scores
(Sec. 3.3 MSAC cost) and inlier counts on subsets whose size is not a
multiple of the tensor-core kernel's record block, pose tiles with a ragged
last tile, the round minima, and end-to-end poses of a batched call.

Bars as for the FP32 scoring kernel: per-pose score 1e-5 relative, counts
exact except points within 1e-3 px of tau, final pose 0.05 deg / 5 mm.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import pose_close, residuals, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(params=[-1, 0, 1, 2, 3, 4],
                ids=["fp32", "tc-rec-m-80p-halves", "tc-rec-m-80p-quarters", "tc-rec-m-64p-whole", "tc-pose-m-bf16",
                     "tc-pose-m-tf32"])
def tc_ctx(request):
    c = imloc.Context(0, 1 << 30)
    if request.param < 0:
        c.set_scoring(0)
    else:
        c.set_scoring(1, request.param)
    yield c
    c.close()


def test_set_scoring_rejects_bad_values():
    c = imloc.Context(0, 1 << 20)
    for kernel, variant in ((2, -1), (-2, -1), (1, 5), (1, -2)):
        with pytest.raises(imloc.ImlocError):
            c.set_scoring(kernel, variant)
    c.set_scoring(-1, -1)
    c.close()


def injected_scores(ctx, q, n, poses, cap=10000):
    t = torch()
    inj = t.from_numpy(np.asarray(poses, np.float32)).cuda()
    P = len(poses)
    c = imloc.corr_from_arrays(q["x"][:n], q["y"][:n], q["X"][:n], q["w"][:n])
    dbg = dict(inject_poses=inj, scores=t.full((4 * P,), float("nan"), device="cuda"),
               counts=t.full((4 * P,), -1, dtype=t.int32, device="cuda"))
    opts = imloc.default_opts(max_iters=P, batch=1024, p_miss=0.0, final_iters=0, lo_iters=0, max_score_corr=cap)
    ctx.testing_ransac(c, q["K"], opts, n, dbg)
    return dbg["scores"].cpu().numpy(), dbg["counts"].cpu().numpy()


def check_against_oracle(q, n, poses, sc, ct, cap, ks):
    idx = oracle.subsample(n, min(n, cap))
    corr = oracle.Corr(q["x"][:n], q["y"][:n], q["X"][:n], q["w"][:n])
    pf = np.asarray(poses, np.float64)
    for k in ks:
        R, tt = pf[k, :9].reshape(3, 3), pf[k, 9:]
        s_ref, c_ref = oracle.score(corr, q["K"], R, tt, 4.0, idx=idx)
        assert sc[4 * k] == pytest.approx(s_ref, rel=1e-5), k
        r, z = residuals(corr.x[idx], corr.y[idx], corr.X[idx], q["K"], R, tt)
        near = int(np.sum((z > 0) & (np.abs(r - 4.0) <= 1e-3)))
        assert abs(int(ct[4 * k]) - c_ref) <= near, k


def perturbed_poses(rng, q, P, deg=3.0, t_sd=0.2):
    out = []
    for _ in range(P):
        dR = synth.axis_angle(rng.normal(size=3), math.radians(rng.uniform(0, deg)))
        out.append(np.concatenate([(dR @ q["R_gt"]).ravel(), q["t_gt"] + rng.normal(size=3) * t_sd]))
    return out


@pytest.mark.parametrize("n", [50000, 2999, 7])
def test_injected_scores_ragged_blocks_and_tiles(tc_ctx, n):
    """M = 10,000 (not a multiple of 64), 2,999 and 7 records; 1,500 poses =
    11 full tiles of 128 and a ragged one; poses include some behind the
    camera (cheirality) and the exact ground truth."""
    rng = np.random.default_rng(31 + n)
    q = synth.direct_query(rng, max(n, 64), 0.3, 1024, 768, 800.0, weights="conf")
    P = 1500
    poses = perturbed_poses(rng, q, P)
    poses[0] = np.concatenate([q["R_gt"].ravel(), q["t_gt"]])
    # a pose looking away from the scene: every point behind the camera costs tau^2
    flip = np.diag([1.0, -1.0, -1.0])
    poses[1] = np.concatenate([(flip @ q["R_gt"]).ravel(), flip @ q["t_gt"]])
    sc, ct = injected_scores(tc_ctx, q, n, poses)
    assert np.all(np.isnan(sc.reshape(-1, 4)[:, 1:]))
    check_against_oracle(q, n, poses, sc, ct, 10000, [0, 1] + list(range(2, P, 53)) + [P - 1])


def test_c1_round_minimum_is_the_argmin(tc_ctx):
    """Sampled C1 run: every valid pose's score against the oracle (a sample)
    and the round minimum equals the (score, pose id) argmin of the wave."""
    q = synth.config1(0)
    t = torch()
    H = q["hypotheses"]
    c = imloc.corr_from_arrays(q["x"], q["y"], q["X"], q["w"])
    n = len(q["x"])
    opts = imloc.default_opts(max_iters=H, batch=1024, p_miss=0.0)
    R_rounds = (H + 1023) // 1024
    dbg = dict(poses=t.zeros((4 * H, 12), dtype=t.float32, device="cuda"),
               scores=t.full((4 * H,), float("nan"), dtype=t.float32, device="cuda"),
               counts=t.full((4 * H,), -1, dtype=t.int32, device="cuda"),
               round_best=t.zeros((R_rounds,), dtype=t.int64, device="cuda"))
    tc_ctx.testing_ransac(c, q["K"], opts, n, dbg)
    poses = dbg["poses"].cpu().numpy()
    scores = dbg["scores"].cpu().numpy()
    ids = np.nonzero(~np.isnan(scores))[0]
    assert len(ids) > 1000
    corr = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    for pid in ids[::7]:
        s_ref, _ = oracle.score(corr, q["K"], poses[pid, :9].reshape(3, 3).astype(np.float64),
                                poses[pid, 9:].astype(np.float64), 4.0)
        assert scores[pid] == pytest.approx(s_ref, rel=1e-5), pid
    key = int(dbg["round_best"].cpu().numpy()[0]) & 0xFFFFFFFFFFFFFFFF
    first = ids[ids < 4 * 1024]
    order = np.lexsort((first, scores[first]))
    assert (key & 0xFFFFFFFF) == first[order[0]]


def test_batch_end_to_end(tc_ctx):
    """16 queries of 50,000 correspondences in one batched call: every pose
    against its ground truth, two against the oracle's."""
    rng = np.random.default_rng(5)
    qs = [synth.direct_query(rng, 50000, 0.3, 1024, 768, 800.0, weights="conf") for _ in range(16)]
    t = torch()
    offs = np.cumsum([0] + [len(q["x"]) for q in qs])
    cat = lambda k: np.concatenate([q[k] for q in qs])
    corr = imloc.corr_from_arrays(cat("x"), cat("y"), np.concatenate([q["X"] for q in qs]), cat("w"))
    d_offs = t.from_numpy(offs.astype(np.int64)).cuda()
    opts = [imloc.default_opts(max_iters=2048, p_miss=0.0, query_id=i, seed=5) for i in range(len(qs))]
    res_buf = t.zeros(len(qs) * imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
    tc_ctx.ransac_pnp_batch_async(corr, d_offs, [q["K"] for q in qs], opts, res_buf)
    t.cuda.synchronize()
    res = imloc.results_from_bytes(res_buf.cpu().numpy(), len(qs))
    for q, r in zip(qs, res):
        assert r["status"] == 0
        assert pose_close(r["R"], r["t"], q["R_gt"], q["t_gt"], deg=0.5, mm=100)
    for i in (0, 11):
        q = qs[i]
        ref = oracle.ransac_pnp(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["K"], max_iters=2048, p_miss=0.0,
                                query_id=i, seed=5)
        assert pose_close(res[i]["R"], res[i]["t"], ref["R"], ref["t"]), i


def test_batch_with_degenerate_and_tiny_queries(tc_ctx):
    """A batched call mixing queries of 0, 2, 3 and 5 correspondences (no or
    too few points: status -7; 3 noise-free points: exact) with full-size ones:
    the small queries get their own status, the others their poses, and no
    device error is raised."""
    rng = np.random.default_rng(11)
    sizes = [20000, 0, 2, 3, 5, 20000, 20000, 3]
    qs = [synth.direct_query(rng, max(n, 1), 0.3 if n > 10 else 1.0, 1024, 768, 800.0, noise_px=0.0 if n <= 10 else 1.0,
                             weights="conf") for n in sizes]
    t = torch()
    offs = np.cumsum([0] + sizes)
    cat = lambda k: np.concatenate([q[k][:n] for q, n in zip(qs, sizes)])
    corr = imloc.corr_from_arrays(cat("x"), cat("y"), np.concatenate([q["X"][:n] for q, n in zip(qs, sizes)]),
                                  cat("w"))
    d_offs = t.from_numpy(offs.astype(np.int64)).cuda()
    opts = [imloc.default_opts(max_iters=4096, p_miss=0.0, query_id=i, seed=9) for i in range(len(qs))]
    res_buf = t.zeros(len(qs) * imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
    tc_ctx.ransac_pnp_batch_async(corr, d_offs, [q["K"] for q in qs], opts, res_buf)
    t.cuda.synchronize()
    res = imloc.results_from_bytes(res_buf.cpu().numpy(), len(qs))
    for q, n, r in zip(qs, sizes, res):
        if n < 3:
            assert r["status"] == -7, (n, r["status"])
        elif n <= 10:
            assert r["status"] == 0 and r["num_inliers"] == n, (n, r)
        else:
            assert r["status"] == 0
            assert pose_close(r["R"], r["t"], q["R_gt"], q["t_gt"], deg=0.5, mm=100)
    assert tc_ctx.device_error() == 0


def test_batch_with_the_adaptive_stop(tc_ctx):
    """The adaptive stop (p_miss = 1e-4) on a batch: several waves of
    sampling and scoring per call, the operand rows written once.  Poses
    against the ground truth and, for two queries, the oracle's."""
    rng = np.random.default_rng(21)
    qs = [synth.direct_query(rng, 30000, r, 1024, 768, 800.0, weights="conf")
          for r in (0.5, 0.3, 0.2, 0.4, 0.6, 0.25, 0.35, 0.45)]
    t = torch()
    offs = np.cumsum([0] + [len(q["x"]) for q in qs])
    cat = lambda k: np.concatenate([q[k] for q in qs])
    corr = imloc.corr_from_arrays(cat("x"), cat("y"), np.concatenate([q["X"] for q in qs]), cat("w"))
    d_offs = t.from_numpy(offs.astype(np.int64)).cuda()
    opts = [imloc.default_opts(max_iters=10000, p_miss=1e-4, query_id=i, seed=13) for i in range(len(qs))]
    res_buf = t.zeros(len(qs) * imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
    tc_ctx.ransac_pnp_batch_async(corr, d_offs, [q["K"] for q in qs], opts, res_buf)
    t.cuda.synchronize()
    res = imloc.results_from_bytes(res_buf.cpu().numpy(), len(qs))
    for q, r in zip(qs, res):
        assert r["status"] == 0
        assert r["iterations"] < 10000  # the stop fired before the cap
        assert pose_close(r["R"], r["t"], q["R_gt"], q["t_gt"], deg=0.5, mm=100)
    for i in (1, 5):
        q = qs[i]
        ref = oracle.ransac_pnp(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["K"], max_iters=10000, p_miss=1e-4,
                                query_id=i, seed=13)
        assert pose_close(res[i]["R"], res[i]["t"], ref["R"], ref["t"]), i
    assert tc_ctx.device_error() == 0
