"""The bf16-packed scoring option (opts.score_bf16) against the FP64 oracle
and against the FP32 scoring kernel, through the C ABI.

With the option, each query's subset is stored as bf16 world coordinates
(centred and scaled per query) and every (pose, record) pair is first
classified from them; pairs that a written error bound cannot place beyond
tau are rescored in FP32 with the FP32 kernel's arithmetic.  So the inlier
counts equal the FP32 kernel's exactly, the truncated scores (Sec. 3.3 MSAC
cost) agree with them up to FP32 summation order, and both meet the oracle
bars: per-pose score 1e-5 relative, counts exact except points within
1e-3 px of tau, final poses 0.05 deg / 5 mm.
"""
import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import pose_close, torch
from test_gpu_score_kernels import check_against_oracle, perturbed_poses

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = imloc.Context(0, 1 << 30)
    c.set_scoring(0)  # the FP32 kernel for the calls without the option
    yield c
    c.close()


def scores_of(ctx, q, n, poses, bf16, cap=10000):
    t = torch()
    inj = t.from_numpy(np.asarray(poses, np.float32)).cuda()
    P = len(poses)
    c = imloc.corr_from_arrays(q["x"][:n], q["y"][:n], q["X"][:n], q["w"][:n])
    dbg = dict(inject_poses=inj, scores=t.full((4 * P,), float("nan"), device="cuda"),
               counts=t.full((4 * P,), -1, dtype=t.int32, device="cuda"),
               rescored_pairs=t.zeros(1, dtype=t.int64, device="cuda"))
    opts = imloc.default_opts(max_iters=P, batch=1024, p_miss=0.0, final_iters=0, lo_iters=0, max_score_corr=cap,
                              score_bf16=int(bf16))
    ctx.testing_ransac(c, q["K"], opts, n, dbg)
    return dbg["scores"].cpu().numpy(), dbg["counts"].cpu().numpy(), int(dbg["rescored_pairs"].item())


@pytest.mark.parametrize("n", [50000, 2999, 7])
def test_bf16_scores_equal_fp32_counts_and_meet_the_oracle_bars(ctx, n):
    """Near-ground-truth poses (many candidates), the exact ground truth and
    a pose looking away (every point behind: no candidate), on subsets of
    10,000, 2,999 (odd: a padding record) and 7 records."""
    rng = np.random.default_rng(71 + n)
    q = synth.direct_query(rng, max(n, 64), 0.3, 1024, 768, 800.0, weights="conf")
    P = 1500
    poses = perturbed_poses(rng, q, P)
    poses[0] = np.concatenate([q["R_gt"].ravel(), q["t_gt"]])
    flip = np.diag([1.0, -1.0, -1.0])
    poses[1] = np.concatenate([(flip @ q["R_gt"]).ravel(), flip @ q["t_gt"]])
    sb, cb, resc = scores_of(ctx, q, n, poses, True)
    sf, cf, _ = scores_of(ctx, q, n, poses, False)
    ok = ~np.isnan(sf)
    np.testing.assert_array_equal(np.isnan(sb), np.isnan(sf))
    np.testing.assert_array_equal(cb[ok], cf[ok])
    np.testing.assert_allclose(sb[ok], sf[ok], rtol=2e-6)
    check_against_oracle(q, n, poses, sb, cb, 10000, [0, 1] + list(range(2, P, 53)) + [P - 1])
    m = min(n, 10000)
    pairs = P * (m + (m & 1))
    assert 0 < resc < pairs


def test_bf16_sampled_round_with_few_rescored_pairs(ctx):
    """A sampled C1 round (random minimal sets: mostly wrong poses): scores
    against the oracle on a sample, the round minimum is the argmin, and the
    share of pairs that needed the FP32 rescoring is small."""
    q = synth.config1(2)
    t = torch()
    H = q["hypotheses"]
    c = imloc.corr_from_arrays(q["x"], q["y"], q["X"], q["w"])
    n = len(q["x"])
    opts = imloc.default_opts(max_iters=H, batch=1024, p_miss=0.0, score_bf16=1)
    dbg = dict(poses=t.zeros((4 * H, 12), dtype=t.float32, device="cuda"),
               scores=t.full((4 * H,), float("nan"), dtype=t.float32, device="cuda"),
               counts=t.full((4 * H,), -1, dtype=t.int32, device="cuda"),
               round_best=t.zeros((1,), dtype=t.int64, device="cuda"),
               rescored_pairs=t.zeros(1, dtype=t.int64, device="cuda"))
    ctx.testing_ransac(c, q["K"], opts, n, dbg)
    poses = dbg["poses"].cpu().numpy()
    scores = dbg["scores"].cpu().numpy()
    ids = np.nonzero(~np.isnan(scores))[0]
    assert len(ids) > 1000
    corr = oracle.Corr(q["x"], q["y"], q["X"], q["w"])
    for pid in ids[::11]:
        s_ref, _ = oracle.score(corr, q["K"], poses[pid, :9].reshape(3, 3).astype(np.float64),
                                poses[pid, 9:].astype(np.float64), 4.0)
        assert scores[pid] == pytest.approx(s_ref, rel=1e-5), pid
    key = int(dbg["round_best"].cpu().numpy()[0]) & 0xFFFFFFFFFFFFFFFF
    order = np.lexsort((ids, scores[ids]))
    assert (key & 0xFFFFFFFF) == ids[order[0]]
    frac = int(dbg["rescored_pairs"].item()) / (len(ids) * n)
    assert 0 < frac < 0.5


def test_bf16_batch_end_to_end(ctx):
    """8 queries of 20,000-50,000 correspondences in one batched call with the
    option: poses against ground truth and, for two, the oracle's."""
    rng = np.random.default_rng(15)
    qs = [synth.direct_query(rng, int(rng.integers(20000, 50000)), 0.3, 1024, 768, 800.0, weights="conf")
          for _ in range(8)]
    t = torch()
    offs = np.cumsum([0] + [len(q["x"]) for q in qs])
    cat = lambda k: np.concatenate([q[k] for q in qs])
    corr = imloc.corr_from_arrays(cat("x"), cat("y"), np.concatenate([q["X"] for q in qs]), cat("w"))
    d_offs = t.from_numpy(offs.astype(np.int64)).cuda()
    opts = [imloc.default_opts(max_iters=2048, p_miss=0.0, query_id=i, seed=5, score_bf16=1) for i in range(len(qs))]
    res_buf = t.zeros(len(qs) * imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
    ctx.ransac_pnp_batch_async(corr, d_offs, [q["K"] for q in qs], opts, res_buf)
    t.cuda.synchronize()
    res = imloc.results_from_bytes(res_buf.cpu().numpy(), len(qs))
    for q, r in zip(qs, res):
        assert r["status"] == 0
        assert pose_close(r["R"], r["t"], q["R_gt"], q["t_gt"], deg=0.5, mm=100)
    for i in (0, 5):
        q = qs[i]
        ref = oracle.ransac_pnp(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["K"], max_iters=2048, p_miss=0.0,
                                query_id=i, seed=5)
        assert pose_close(res[i]["R"], res[i]["t"], ref["R"], ref["t"]), i
    assert ctx.device_error() == 0


def test_precision_options_end_to_end_on_a_graph_stream(ctx):
    """LO / refinement in FP64 accumulation and / or with the FP64 6x6 solve,
    one after the other on the same shapes and a non-default stream (where
    the batched launch sequence is captured and replayed as a CUDA graph per
    size bucket): every final pose against the oracle's, and the variants
    within float rounding of each other (they iterate to the same fixed
    point)."""
    rng = np.random.default_rng(16)
    qs = [synth.direct_query(rng, 30000, 0.4, 1024, 768, 800.0, weights="conf") for _ in range(4)]
    t = torch()
    stream = t.cuda.Stream()
    offs = np.cumsum([0] + [len(q["x"]) for q in qs])
    cat = lambda k: np.concatenate([q[k] for q in qs])
    corr = imloc.corr_from_arrays(cat("x"), cat("y"), np.concatenate([q["X"] for q in qs]), cat("w"))
    d_offs = t.from_numpy(offs.astype(np.int64)).cuda()
    t.cuda.synchronize()
    out = {}
    variants = [(0, 0), (1, 0), (0, 1), (1, 1), (0, 0), (1, 1)]
    for k, (acc, solve) in enumerate(variants):
        opts = [imloc.default_opts(max_iters=2048, p_miss=0.0, query_id=i, seed=7, lo_fp64_accumulate=acc,
                                   lo_fp64_solve=solve) for i in range(len(qs))]
        res_buf = t.zeros(len(qs) * imloc.RESULT_BYTES, dtype=t.uint8, device="cuda")
        ctx.ransac_pnp_batch_async(corr, d_offs, [q["K"] for q in qs], opts, res_buf, stream=stream)
        stream.synchronize()
        out[k] = imloc.results_from_bytes(res_buf.cpu().numpy(), len(qs))
    for i, q in enumerate(qs):
        ref = oracle.ransac_pnp(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["K"], max_iters=2048, p_miss=0.0,
                                query_id=i, seed=7)
        for k in out:
            r = out[k][i]
            assert r["status"] == 0 and r["num_inliers"] > 0, (i, variants[k])
            assert pose_close(r["R"], r["t"], ref["R"], ref["t"]), (i, variants[k])
            assert pose_close(out[0][i]["R"], out[0][i]["t"], r["R"], r["t"], deg=0.005, mm=0.5), (i, variants[k])
