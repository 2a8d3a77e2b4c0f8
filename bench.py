"""Benchmark of the ImLoc localization hot path (lift + LO-RANSAC PnP) on GB300.

One step = one pass of the whole hot path over one batch of queries shaped
like the paper's "lift + RANSAC per query" workload: per query, 10 database
views with 1024x768 float32 depth maps of a piecewise-planar scene, 5,000
dense matches per pair (50,000 matches), inlier ratio U[10%, 60%], N(0, 0.5 px)
query noise, 10,000 minimal sets, LO on, Cauchy refinement on all inliers
(adaptive stop off: fixed hypothesis count).  A step runs the batched lift
and the batched LO-RANSAC of the C ABI on device-resident inputs; L2 is
flushed (256 MiB write) between steps, outside the timed events.

Headline metric: hypothesis x correspondence pairs scored per second.  Also
reported: queries/s, the plain one-query-per-call form with p50/p99 latency,
an end-to-end figure with host buffers (matches uploaded, results read back
every step), per-kernel device time, the roofline of the dominant kernel and
the FP64 CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own batch (weak scaling, no
collective on the data path); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import gc
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hyp*corr scored/s; localized queries/s & p50/p99 latency, served vs plain"
UNIT = "hyp*corr/s"
HYPOTHESES = 10000
MATCHES_PER_PAIR = 5000
N_VIEWS = 10
# The method's work per scored (pose, correspondence) pair, with the projection folded into
# P = K [R | t]: 9 FMA for P [X; 1], 2 FMA for the pixel residual, 1 MUL + 1 FMA for r^2 and 1 FMA
# for the weighted truncated sum = 13 FMA (2 flops each) + 1 MUL = 27 flops on the FP32 pipe (plus
# 1 reciprocal on the MUFU and 2 min/max).  Every scoring roofline below counts these 27 flops per
# pair against the FP32 FMA peak, whichever unit executes the projection.
FLOPS_PER_PAIR = 27
# tensor-core scoring: per pair the FP32 epilogue does 4 FFMA + 1 FMUL (9 flops) after the projection,
# which runs as 3 coordinate rows x 2 MMA K steps of 16 (24 split-piece terms + 8 zero) x 2 flops
TC_FP32_FLOPS_PER_PAIR = 9
TC_MMA_FLOPS_PER_PAIR = 192
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per launch of k_score on the 16-query C2 step, from
# the committed ncu capture (profiles/k_score_c2_16queries.md), keyed by the
# scoring variant (threads, poses per thread) it was taken on; the line reports
# it only when the autotuner picked that variant.
SCORE_TRAFFIC_PER_LAUNCH = {(64, 4): 25.754e6 + 0.0}
# the same for the tensor-core scoring kernel (k_score_tcr: records on the MMA's
# M side, 80-pose items) on that step (profiles/k_score_tcr_c2_16queries.md)
SCORE_TC_TRAFFIC_PER_LAUNCH = 45.270e6 + 0.118e6
# DRAM bytes (read + write) per lifted match from the committed ncu captures of
# k_lift on the batched 9.48M-match shape against the 1,024-view store
# (profiles/k_lift_batched_9.5M_1024views.md).  The row-major capture
# (207.6 B per match) predates the kernel's overlapping-block branch, so the
# row-major entry reports no traffic; the overlapping-block capture is of the
# current kernel.
LIFT_TRAFFIC_PER_MATCH = None
LIFT_HALO_TRAFFIC_PER_MATCH = (1.277477e9 + 0.244294e9) / 9.48e6


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def _gen_query(seed):
    from paper_2601_04185_gb300 import synth

    rng = np.random.default_rng(seed)
    q = synth.localization_query(rng, n_views=N_VIEWS, matches_per_pair=MATCHES_PER_PAIR)
    q.pop("scene", None)
    return q


def make_queries(n, seed0):
    # spawn: no fork after CUDA is initialised
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=min(n, os.cpu_count() or 1), mp_context=ctx) as ex:
        return list(ex.map(_gen_query, [seed0 + i for i in range(n)]))


def concat_batch(queries):
    views, qb = [], [0]
    cat = {k: [] for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    seg_off, seg_view, seg_dir = [0], [], []
    for q in queries:
        m = q["matches"]
        base_v = len(views)
        views += q["views"]
        for k in cat:
            cat[k].append(m[k])
        for s in range(len(m["seg_view"])):
            seg_off.append(qb[-1] + int(m["seg_off"][s + 1]))
            seg_view.append(base_v + int(m["seg_view"][s]))
            seg_dir.append(int(m["seg_dir"][s]))
        qb.append(qb[-1] + int(m["seg_off"][-1]))
    big = {k: np.concatenate(v).astype(np.float32) for k, v in cat.items()}
    big.update(seg_off=np.array(seg_off, np.int64), seg_view=np.array(seg_view, np.int32),
               seg_dir=np.array(seg_dir, np.int32))
    return views, big, np.array(qb, np.int64)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU, no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus, backend="nccl"):
    """Join the process group of a torchrun launch (RANK / WORLD_SIZE /
    LOCAL_RANK / MASTER_* from the environment): one process per GPU over
    NCCL; `backend="gloo"` runs the same plumbing on CPU processes."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _over_ranks(v, world, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(v, world):
    """The slowest rank's time (the job's time): MAX over ranks."""
    import torch.distributed as dist

    return v if world == 1 else _over_ranks(v, world, dist.ReduceOp.MAX)


def sum_over_ranks(v, world):
    """Work of the whole job: SUM over ranks (weak scaling, fixed work per rank)."""
    import torch.distributed as dist

    return v if world == 1 else _over_ranks(v, world, dist.ReduceOp.SUM)


def rank_seed(base, rank):
    """Each rank localizes its own queries (independent problems: no data-path collective)."""
    return base + 1000 * rank


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_queries(queries, hypotheses, threads):
    """Lift + LO-RANSAC of every query with the FP64 oracle, one query per
    thread (the C oracle releases the GIL).  Returns (wall s, pairs scored)."""
    import oracle

    def one(i):
        q = queries[i]
        L = oracle.lift(q["views"], q["matches"])
        c = oracle.Corr(L["x"], L["y"], L["X"], L["w"])
        r = oracle.ransac_pnp(c, q["K"], max_iters=hypotheses, p_miss=0.0, query_id=i)
        return r["hypotheses"] * min(c.n, 10000)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        pairs = sum(ex.map(one, range(len(queries))))
    return time.perf_counter() - t0, pairs


def c2_workload(nq):
    """The C2 step's workload, as both arms name it."""
    return (f"C2: {nq} queries/step x (lift of {N_VIEWS} views x {MATCHES_PER_PAIR} matches "
            f"+ LO-RANSAC PnP, {HYPOTHESES} minimal sets, LO, Cauchy refinement)")


def run_reference(args):
    rank, world, _ = (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0)
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    # the C2 step's own queries (same seeds, sizes and minimal sets as the GPU arm's step), one per host thread
    nq = args.queries
    queries = make_queries(nq, rank_seed(100, 0))
    threads = min(cores, nq)
    for _ in range(args.warmup):
        oracle_queries(queries[:1], HYPOTHESES, 1)
    total_t, total_pairs = 0.0, 0
    for _ in range(args.steps):
        t, p = oracle_queries(queries, HYPOTHESES, threads)
        total_t += t
        total_pairs += p
    v = total_pairs / total_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": c2_workload(nq), "queries_per_step": nq,
                       "matches_per_query": N_VIEWS * MATCHES_PER_PAIR, "depth": "1024x768 float32, 10 views/query",
                       "hypotheses": HYPOTHESES, "score_corr_cap": 10000,
                       "parallelism": f"FP64 CPU oracle, {threads} host threads (one query each)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"the C2 step's {nq} queries per step (lift + {HYPOTHESES} minimal sets + LO "
                                       f"+ refinement), one per thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson arrivals, served (continuous batching) vs plain
# ---------------------------------------------------------------------------
STORE_VIEWS = 1024
SERVE_RATES = (50, 100, 200, 500, 1000, 2000, 5000, 10000, 20000, 40000)


def _gen_store_view(args):
    from paper_2601_04185_gb300 import synth

    seed, k = args
    st = synth.MapStore(seed, STORE_VIEWS)
    v = st.build_view(k)
    v.pop("depth_true", None)
    return v


_STORE = None  # map store shared with forked generator processes


def _serve_query_worker(i):
    rng = np.random.default_rng(10_000 + i)
    return _STORE.query(rng, int(rng.integers(10, 41)))


def make_store_and_queries(seed, n_queries):
    """The resident map store (64 views, 1024x768 float32 depth) and serving
    queries against it (10-40 views x 5,000 matches, 50k-200k matches).
    Must run before CUDA is initialised in this process (fork pool)."""
    global _STORE
    from paper_2601_04185_gb300 import synth

    with cf.ProcessPoolExecutor(max_workers=os.cpu_count() or 1, mp_context=mp.get_context("spawn")) as ex:
        views = list(ex.map(_gen_store_view, [(seed, k) for k in range(STORE_VIEWS)]))
    store = synth.MapStore(seed, STORE_VIEWS)
    store.views = [dict(v, depth_true=v["depth"]) for v in views]
    _STORE = store
    with cf.ProcessPoolExecutor(max_workers=os.cpu_count() or 1, mp_context=mp.get_context("fork")) as ex:
        queries = list(ex.map(_serve_query_worker, range(n_queries), chunksize=2))
    return store, views, queries


def run_retrieval(dev, peaks, repeats=10):
    """Nearest-neighbour search of global retrieval features (Sec. 3.1,
    Sec. 4.4 "Runtime"): 100,000 database descriptors of 8,448 dims (a
    MegaLoc-sized feature, bfloat16, 1.69 GB), top 50 per query; one query
    (reads the database once: HBM-bound) and a batch of 256 queries (the
    tensor-core GEMM); CUDA events, L2 flushed before each call."""
    import torch

    from paper_2601_04185_gb300 import imloc, synth

    N, D, K = 100000, 8448, 50
    db, q = synth.retrieval_set_torch(2027, N, 256, D, dev)
    ctx = imloc.Context(dev.index, (512 << 20))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for Q in (1, 256):
        qq = q[:Q].contiguous()
        for _ in range(3):
            ctx.retrieve_topk(qq, db, K, stream=stream)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(repeats)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            ctx.retrieve_topk(qq, db, K, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        kname = "k_retrieve_gemm" if "k_retrieve_gemm" in prof else "k_retrieve_gemv"
        gemm_ms = prof[kname][1] / prof[kname][0]
        sel_ms = prof["k_topk_select"][1] / prof["k_topk_select"][0]
        nbytes = N * D * 2 + Q * D * 2 + Q * N * 4
        flops = 2.0 * Q * N * D
        r = {"queries": Q, "kernel": kname, "ms": ms, "gemm_ms": gemm_ms, "select_ms": sel_ms,
             "queries_per_s": Q / (ms * 1e-3),
             "gemm_gbs": (N * D * 2 + Q * D * 2) / (gemm_ms * 1e-3) / 1e9,
             "gemm_tflops": flops / (gemm_ms * 1e-3) / 1e12}
        if Q == 1:
            r["roofline"] = {"bound": "hbm", "achieved": r["gemm_gbs"], "peak": peaks.get("hbm_gbs", 6800.0),
                             "unit": "GB/s", "frac": r["gemm_gbs"] / peaks.get("hbm_gbs", 6800.0),
                             "note": "database bytes read by the scoring kernel / its event time"}
        else:
            pk = peaks.get("bf16_tflops", 1900.0)
            r["roofline"] = {"bound": "tensor", "achieved": r["gemm_tflops"], "peak": pk, "unit": "TFLOP/s",
                             "frac": r["gemm_tflops"] / pk, "hbm_frac": r["gemm_gbs"] / peaks.get("hbm_gbs", 6800.0),
                             "note": "2 Q N D flops / GEMM event time; burst bf16 peak of a cuBLAS GEMM"}
        out[f"q{Q}"] = r
    ctx.close()
    out["workload"] = (f"{N} database descriptors x {D} dims (bfloat16, L2-normalised, place-clustered), top {K}; "
                       "L2 flushed before each call; paper: < 1 ms per query on an RTX 4090 (Sec. 4.4)")
    return out


def run_triangulation(dev, repeats=20):
    """Mapping-time dense triangulation (Sec. 3.3 "Depth Estimation by Dense
    Matching") of one 560x560 mapping image with 8 covisible sources (the
    paper's default map resolution): CUDA-event time per image, L2 flushed
    before each launch."""
    import torch

    from paper_2601_04185_gb300 import imloc, synth

    m = synth.mapping_image(np.random.default_rng(2026), n_src=8, width=560, height=560, f=480.0)
    u, v, c = (torch.from_numpy(np.ascontiguousarray(m[k])).to(dev) for k in ("u", "v", "conf"))
    depth = torch.empty((560, 560), dtype=torch.float32, device=dev)
    inl = torch.empty((560, 560), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        imloc.triangulate_depth(m["ref"], m["srcs"], u, v, c, depth=depth, inliers=inl, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(repeats)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        imloc.triangulate_depth(m["ref"], m["srcs"], u, v, c, depth=depth, inliers=inl, stream=stream)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    d = depth.cpu().numpy()
    kept = d > 0
    gt = m["depth_gt"]
    return {"workload": "one 560x560 mapping image, 8 covisible sources (one match per pixel and source), "
                        "inlier probability 0.8 where visible, N(0, 0.5 px) match noise",
            "ms_per_image": ms, "images_per_s": 1e3 / ms, "pixels_per_s": 560 * 560 / (ms * 1e-3),
            "kept_fraction": float(kept.mean()),
            "median_rel_depth_error": float(np.median(np.abs(d[kept] - gt[kept]) / gt[kept])) if kept.any() else None,
            "input_bytes": int(3 * 8 * 560 * 560 * 4),
            "roofline": _triangulation_roofline(dev, ms, 560 * 560, 8),
            "paper_context": "~30 ms per image on an RTX 4090 for matching + triangulation, matching dominating (Sec. 3.3)"}


# Triangulation work per pixel: S depth hypotheses (closest approach of two rays, ~40 flops each) and
# S x S inlier tests of a hypothesis against a source (point on the pixel's ray, offset from the source
# centre, cross and dot products with the match's ray, the tan^2 comparison: ~30 flops each); the
# refinement of the kept pixels is not counted.
TRI_FLOPS_HYP, TRI_FLOPS_TEST = 40, 30


def _triangulation_roofline(dev, ms, pixels, sources):
    peak, basis = fp32_peak_tflops(dev, load_peaks())
    flops = pixels * (sources * TRI_FLOPS_HYP + sources * sources * TRI_FLOPS_TEST)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"kernel": "k_triangulate", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flops_per_pixel": flops / pixels, "peak_basis": basis,
            "note": "hypothesis-and-test core per pixel (S hypotheses x 40 + S^2 tests x 30 flops) / event time per "
                    "image; the refinement of kept pixels is extra work not counted"}


def run_rig(dev, peaks, repeats=5, n_queries=16):
    """Generalized absolute pose of camera-rig queries (supplementary "LaMAR
    HoloLens Results"): 16 queries of a 4-camera head-mounted rig (cameras at
    -60, -20, 20, 60 degrees of yaw, within 10 cm of the rig origin), 2,500
    correspondences per camera (N = 10,000), inlier ratio U[15%, 50%],
    default options (batches of 1,024, at most 100K minimal sets, adaptive
    stop at 1e-4); one call per step, L2 flushed before each."""
    import torch

    from paper_2601_04185_gb300 import imloc, synth

    rng = np.random.default_rng(2031)
    qs = [synth.rig_query(rng, n_per_cam=2500, inlier_ratio=float(rng.uniform(0.15, 0.5)), n_cams=4, weights="conf")
          for _ in range(n_queries)]
    off = np.concatenate([[0], np.cumsum([len(q["x"]) for q in qs])]).astype(np.int64)
    c = imloc.corr_from_arrays(np.concatenate([q["x"] for q in qs]), np.concatenate([q["y"] for q in qs]),
                               np.concatenate([q["X"] for q in qs]), np.concatenate([q["w"] for q in qs]), device=dev)
    cam = torch.from_numpy(np.concatenate([q["cam"] for q in qs]).astype(np.int32)).to(dev)
    d_off = torch.from_numpy(off).to(dev)
    rigs = [imloc.rig(q["K"], q["R_cam"], q["t_cam"]) for q in qs]
    opts = [imloc.default_opts(query_id=i, seed=77) for i in range(n_queries)]
    out = torch.zeros(n_queries * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
    ctx = imloc.Context(dev.index, 1 << 30)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        ctx.ransac_rig_batch(c, cam, d_off, rigs, opts, out, stream=stream)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    times = []
    for _ in range(repeats):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.ransac_rig_batch(c, cam, d_off, rigs, opts, out, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    ctx.close()
    res = imloc.results_from_bytes(out.cpu().numpy(), n_queries)
    ms = statistics.median(times)
    hyps = sum(r["hypotheses"] for r in res)
    m = [min(len(q["x"]), 10000) for q in qs]
    work = sum(r["hypotheses"] * mq for r, mq in zip(res, m))
    errs = []
    for r, q in zip(res, qs):
        dR = r["R"] @ q["R_gt"].T
        ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(dR) - 1) / 2))))
        errs.append((ang, float(np.linalg.norm(r["R"].T @ r["t"] - q["R_gt"].T @ q["t_gt"]))))
    score_ms = prof["k_rig_score"][1] / repeats if "k_rig_score" in prof else None
    fp32_peak = fp32_peak_tflops(dev, peaks)[0]
    line = {"workload": f"{n_queries} rig queries x 4 cameras x 2,500 correspondences, inlier ratio U[15%, 50%], "
                        "default options, one call",
            "ms_per_call": ms, "queries_per_s": n_queries / (ms * 1e-3),
            "hyp_corr_per_s": work / (ms * 1e-3), "hypotheses": hyps,
            "rounds": [int(r["rounds"]) for r in res],
            "status_ok": sum(r["status"] == 0 for r in res),
            "max_rot_err_deg": max(e[0] for e in errs), "max_centre_err_m": max(e[1] for e in errs),
            "kernel_ms_per_call": {k: prof[k][1] / repeats for k in prof},
            "launches_per_call": {k: prof[k][0] / repeats for k in prof}}
    if score_ms:
        tflops = work * 27 / (score_ms * 1e-3) / 1e12
        line["roofline"] = {"kernel": "k_rig_score", "bound": "alu", "achieved": tflops, "peak": fp32_peak,
                            "unit": "TFLOP/s", "frac": tflops / fp32_peak,
                            "note": "27 flops per (pose, correspondence) / summed k_rig_score time; derived FP32 peak"}
    return line


def run_serving(dev, rates, per_rate, queries, dev_views, seconds_cap=3.0):
    """Offer Poisson streams to the server and to the plain loop; returns per-rate q/s and latency percentiles.

    Two input forms each: matches in host memory (the server copies them into
    its pinned ring at submission and uploads them; the plain loop uploads
    them per query) and matches already in device memory, as a GPU matcher
    leaves them (imloc_serve_submit_device; the plain loop lifts them in place)."""
    import queue
    import torch

    from paper_2601_04185_gb300 import imloc

    def opts_for(i):
        return imloc.default_opts(max_iters=10000, p_miss=1e-4, query_id=i, seed=4321)

    prepared = [imloc.Server.prepare([dev_views[j] for j in q["view_ids"]], q["matches"], q["K"], opts_for(i))
                for i, q in enumerate(queries)]
    d_matches = []
    for q in queries:
        dm = {k: torch.from_numpy(np.ascontiguousarray(q["matches"][k], dtype=np.float32)).to(dev)
              for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
        dm.update({k: q["matches"][k] for k in ("seg_off", "seg_view", "seg_dir")})
        d_matches.append(dm)
    prepared_dev = [imloc.Server.prepare_device([dev_views[j] for j in q["view_ids"]], d_matches[i], q["K"],
                                                opts_for(i)) for i, q in enumerate(queries)]
    pinned = [{k: torch.from_numpy(q["matches"][k]).pin_memory() for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
              for q in queries]
    out = {"rates": list(rates), "served": [], "plain": [], "served_device": [], "plain_device": []}
    rng = np.random.default_rng(77)
    ctx = imloc.Context(dev.index, 512 << 20)
    srv = imloc.Server(ctx, max_slots=64, device_budget_bytes=64 << 30, host_staging_bytes=1 << 30,
                       rounds_per_step=2)
    # warm the server (autotuning, module load)
    tk = [srv.submit_prepared(prepared[i]) for i in range(8)] + [srv.submit_prepared(prepared_dev[i]) for i in range(8)]
    while any(srv.poll(t)[0] == 1 for t in tk):
        time.sleep(0.001)
    corr = imloc.alloc_corr(max(len(q["matches"]["q_u"]) for q in queries), dev)

    def served(arrivals, order, preps):
        tickets = []
        t0 = time.perf_counter()
        for k in range(len(order)):
            wait = arrivals[k] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets.append(srv.submit_prepared(preps[order[k]]))
        lats, pending = [], [t for t in tickets if t is not None]
        while pending:
            keep = []
            for t in pending:
                st, res, lat = srv.poll(t)
                if st == 0:
                    lats.append(lat)
                else:
                    keep.append(t)
            pending = keep
            if pending:
                time.sleep(0.0005)
        elapsed = time.perf_counter() - t0
        lats.sort()
        refused = sum(t is None for t in tickets)
        if not lats:
            return {"queries": len(order), "refused": refused, "q_per_s": 0.0, "p50_ms": None, "p99_ms": None,
                    "server_stats": srv.stats()}
        return {"queries": len(order), "refused": refused, "q_per_s": len(lats) / elapsed,
                "p50_ms": lats[len(lats) // 2], "p99_ms": lats[min(len(lats) - 1, int(0.99 * len(lats)))]}

    def plain(arrivals, order, on_device):
        # one query at a time: (upload +) lift + RANSAC per call
        qq = queue.Queue()
        lat_p = []

        def worker():
            stream = torch.cuda.current_stream(dev)
            while True:
                item = qq.get()
                if item is None:
                    return
                k, t_arr = item
                i = order[k]
                q = queries[i]
                if on_device:
                    dm = d_matches[i]
                else:
                    dm = {kk: v.to(dev, non_blocking=True) for kk, v in pinned[i].items()}
                    dm.update({kk: q["matches"][kk] for kk in ("seg_off", "seg_view", "seg_dir")})
                ctx.lift([dev_views[j] for j in q["view_ids"]], dm, out=corr, stream=stream)
                ctx.ransac_pnp(corr, q["K"], opts_for(i), stream=stream)
                lat_p.append(1e3 * (time.perf_counter() - t_arr))
        th = threading.Thread(target=worker)
        th.start()
        t0 = time.perf_counter()
        for k in range(len(order)):
            wait = arrivals[k] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            qq.put((k, time.perf_counter()))
        qq.put(None)
        th.join()
        elapsed = time.perf_counter() - t0
        lat_p.sort()
        return {"queries": len(order), "q_per_s": len(lat_p) / elapsed, "p50_ms": lat_p[len(lat_p) // 2],
                "p99_ms": lat_p[min(len(lat_p) - 1, int(0.99 * len(lat_p)))]}

    for lam in rates:
        n = min(per_rate, int(lam * seconds_cap))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n))
        order = rng.integers(0, len(queries), n)
        out["served"].append({"lambda": lam, **served(arrivals, order, prepared)})
        out["served_device"].append({"lambda": lam, **served(arrivals, order, prepared_dev)})
        out["plain"].append({"lambda": lam, **plain(arrivals, order, False)})
        out["plain_device"].append({"lambda": lam, **plain(arrivals, order, True)})
    out["server_stats"] = srv.stats()
    srv.close()
    ctx.close()
    return out


# ---------------------------------------------------------------------------
# batched (C3): 256 direct queries in shared launches
# ---------------------------------------------------------------------------
def run_batched_c3(dev, steps=5):
    import torch

    from paper_2601_04185_gb300 import imloc, synth

    qs = synth.config3(0)
    nq = len(qs)
    offs = np.cumsum([0] + [len(q["x"]) for q in qs])
    cat = lambda k: np.concatenate([q[k] for q in qs])
    corr = imloc.corr_from_arrays(cat("x"), cat("y"), np.concatenate([q["X"] for q in qs]), cat("w"), device=dev)
    d_offs = torch.from_numpy(offs.astype(np.int64)).to(dev)
    opts = [imloc.default_opts(max_iters=q["hypotheses"], p_miss=0.0, query_id=i, seed=5) for i, q in enumerate(qs)]
    ctx = imloc.Context(dev.index, 4 << 30)
    res_buf = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
    prep = imloc.prepare_ransac_batch([q["K"] for q in qs], opts)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        ctx.ransac_pnp_batch_async(corr, d_offs, None, None, res_buf, stream=stream, prepared=prep)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        ctx.ransac_pnp_batch_async(corr, d_offs, None, None, res_buf, stream=stream, prepared=prep)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    # per-kernel times: the same calls again, traced (tracing switches the graph replay off)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for _ in range(steps):
        ctx.ransac_pnp_batch_async(corr, d_offs, None, None, res_buf, stream=stream, prepared=prep)
    torch.cuda.synchronize()
    kst = ctx.profile_read(reset=True)
    res = imloc.results_from_bytes(res_buf.cpu().numpy(), nq)
    pairs = float(sum(r["hypotheses"] * min(int(n), 10000) for r, n in zip(res, np.diff(offs))))
    ctx.profile(False)
    # scoring forms on the same batch: the FP32 kernel, and bf16-packed coordinates with FP32 rescoring
    forms = {}
    for name, scoring, bf in (("fp32_kernel", 0, 0), ("bf16_rescore", -1, 1)):
        ctx.set_scoring(scoring)
        opts_f = [imloc.default_opts(max_iters=q["hypotheses"], p_miss=0.0, query_id=i, seed=5, score_bf16=bf)
                  for i, q in enumerate(qs)]
        prep_f = imloc.prepare_ransac_batch([q["K"] for q in qs], opts_f)
        buf_f = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
        for _ in range(2):
            ctx.ransac_pnp_batch_async(corr, d_offs, None, None, buf_f, stream=stream, prepared=prep_f)
        torch.cuda.synchronize()
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(stream)
        for _ in range(steps):
            ctx.ransac_pnp_batch_async(corr, d_offs, None, None, buf_f, stream=stream, prepared=prep_f)
        b2.record(stream)
        torch.cuda.synchronize()
        rf = imloc.results_from_bytes(buf_f.cpu().numpy(), nq)
        rot = [_rot_err_deg(x["R"], y["R"]) for x, y in zip(rf, res)]
        tr = [1e3 * float(np.linalg.norm(-x["R"].T @ x["t"] + y["R"].T @ y["t"])) for x, y in zip(rf, res)]
        forms[name] = {"ms_per_batch": a2.elapsed_time(b2) / steps,
                       "vs_default_rot_deg_max": float(max(rot)), "vs_default_trans_mm_max": float(max(tr)),
                       "status": sorted({x["status"] for x in rf})}
    ctx.set_scoring(-1)
    # share of (pose, record) pairs the bf16 test left to the FP32 rescoring, on 8 of the batch's queries
    resc, tot = 0, 0
    for i in range(0, nq, nq // 8):
        q = qs[i]
        n = len(q["x"])
        H = q["hypotheses"]
        c1 = imloc.corr_from_arrays(q["x"], q["y"], q["X"], q["w"], device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        dbg = dict(scores=torch.full((4 * H,), float("nan"), device=dev), rescored_pairs=cnt)
        ctx.testing_ransac(c1, q["K"], imloc.default_opts(max_iters=H, p_miss=0.0, query_id=i, seed=5, score_bf16=1),
                           n, dbg)
        scored = int(torch.isfinite(dbg["scores"]).sum().item())
        m = min(n, 10000)
        resc += int(cnt.item())
        tot += scored * (m + (m & 1))
    forms["bf16_rescore"]["rescored_fraction"] = resc / max(1, tot)
    forms["bf16_rescore"]["note"] = ("bf16 world coordinates (centred, scaled by a power of two per query) give a "
                                     "per-pair bound of several pixels at these scales, so every pair that the bound "
                                     "cannot place beyond tau is rescored in FP32 with the FP32 kernel's arithmetic")
    ctx.close()
    skey = "k_score_tc" if "k_score_tc" in kst else "k_score"
    score_ms = kst.get(skey, (1, 0.0))[1] / max(1, kst.get(skey, (1, 0.0))[0])
    return {"workload": "C3: 256 direct queries, N log-uniform in [2k, 100k], inlier ratio U[5%, 70%], "
                        "4,096-16,384 minimal sets, LO + refinement, one batched call",
            "ms_per_batch": ms, "hyp_corr_per_s": pairs / (ms * 1e-3), "queries_per_s": nq / (ms * 1e-3),
            "correspondences": int(offs[-1]), "scoring_kernel": skey, "score_ms": score_ms,
            "score_tflops": FLOPS_PER_PAIR * pairs / (score_ms * 1e-3) / 1e12 if score_ms else None,
            "score_flops_per_pair": FLOPS_PER_PAIR,
            "kernels_ms": {k: v[1] / steps for k, v in kst.items()},
            "status": sorted({r["status"] for r in res}), "scoring_forms": forms}


# ---------------------------------------------------------------------------
# precision study (C4): P3P polish and LO accumulation variants vs the oracle
# ---------------------------------------------------------------------------
def _gen_c4_query(args):
    from paper_2601_04185_gb300 import synth

    i, n = args
    rng = np.random.default_rng(500 + i)
    sig = (0.5, 1.0, 1.5, 2.0)[i * 4 // n]
    q = synth.localization_query(rng, pixel_noise=sig, depth_noise=0.01)
    q.pop("scene", None)
    q["sigma"] = sig
    return q


PRECISION_QUERIES = 64


def _oracle_pose(args):
    import oracle

    q, i = args
    L = oracle.lift(q["views"], q["matches"])
    c = oracle.Corr(L["x"], L["y"], L["X"], L["w"])
    r = oracle.ransac_pnp(c, q["K"], max_iters=HYPOTHESES, p_miss=0.0, query_id=i, seed=31)
    return r["R"], r["t"]


def _rot_err_deg(Ra, Rb):
    chord = np.linalg.norm(np.asarray(Ra) - np.asarray(Rb))
    return math.degrees(2.0 * math.asin(min(1.0, chord / (2.0 * math.sqrt(2.0)))))


def _c4_queries(n):
    with cf.ProcessPoolExecutor(max_workers=min(n, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen_c4_query, [(i, n) for i in range(n)]))


def _c4_oracle(qs):
    """The FP64 oracle's final pose of every C4 query (threads; the C oracle releases the GIL)."""
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        ref = list(ex.map(_oracle_pose, [(q, i) for i, q in enumerate(qs)]))
    return ref, time.perf_counter() - t0


PRECISION_VARIANTS = (
    # (P3P polish, LO / refinement accumulation, LO / refinement 6x6 solve, scoring coordinates)
    ("fp32 + double-float polish", "fp32", "fp32", "fp32"),
    ("fp32 + double-float polish", "fp64", "fp32", "fp32"),
    ("fp32 + double-float polish", "fp32", "fp64", "fp32"),
    ("fp32 + double-float polish", "fp64", "fp64", "fp32"),
    ("fp32", "fp32", "fp32", "fp32"),
    ("fp32", "fp64", "fp64", "fp32"),
    ("fp32 + double-float polish", "fp32", "fp32", "bf16 + fp32 rescore"),
)


def precision_study(dev, qs, ref, oracle_s):
    """C4: every precision variant on the same lifted queries; final poses
    against the FP64 oracle's (and against ground truth), batch time."""
    import torch

    from paper_2601_04185_gb300 import imloc

    views, big, qb = concat_batch(qs)
    d_views = []
    for v in views:
        d = dict(v)
        d["depth"] = torch.from_numpy(v["depth"]).to(dev)
        d_views.append(d)
    d_match = {k: torch.from_numpy(big[k]).to(dev) for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    d_match.update({k: big[k] for k in ("seg_off", "seg_view", "seg_dir")})
    ctx = imloc.Context(dev.index, 2 << 30)
    corr, offsets = ctx.lift_batch(qb, d_views, d_match)
    nq = len(qs)
    out = {"workload": f"C4: {nq} queries of 50k matches (10 views x 5,000), depth x (1 + N(0, 0.01)), pixel noise "
                       "0.5/1/1.5/2 px (a quarter each), 10,000 minimal sets, LO + refinement; errors vs the FP64 "
                       "oracle's final pose and vs ground truth",
           "oracle_seconds": oracle_s, "variants": []}
    for p3p, acc, solve, coords in PRECISION_VARIANTS:
        opts = [imloc.default_opts(max_iters=HYPOTHESES, p_miss=0.0, query_id=i, seed=31,
                                   p3p_fp64_polish=int(p3p != "fp32"), lo_fp64_accumulate=int(acc == "fp64"),
                                   lo_fp64_solve=int(solve == "fp64"), score_bf16=int(coords != "fp32"))
                for i in range(nq)]
        res_buf = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
        ctx.ransac_pnp_batch_async(corr, offsets, [q["K"] for q in qs], opts, res_buf)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.ransac_pnp_batch_async(corr, offsets, [q["K"] for q in qs], opts, res_buf)
        b.record()
        torch.cuda.synchronize()
        res = imloc.results_from_bytes(res_buf.cpu().numpy(), nq)
        rot = np.array([_rot_err_deg(r["R"], o[0]) for r, o in zip(res, ref)])
        trans = np.array([1e3 * np.linalg.norm(-r["R"].T @ r["t"] + o[0].T @ o[1]) for r, o in zip(res, ref)])
        rot_gt = np.array([_rot_err_deg(r["R"], q["R_gt"]) for r, q in zip(res, qs)])
        trans_gt = np.array([1e3 * np.linalg.norm(-r["R"].T @ r["t"] + q["R_gt"].T @ q["t_gt"])
                             for r, q in zip(res, qs)])
        within = float(np.mean((rot <= 0.05) & (trans <= 5.0)))
        out["variants"].append({
            "p3p": p3p, "lo_accumulate": acc, "lo_solve": solve, "scoring_coordinates": coords,
            "vs_oracle_rot_deg": {"median": float(np.median(rot)), "p90": float(np.percentile(rot, 90)),
                                  "max": float(rot.max())},
            "vs_oracle_trans_mm": {"median": float(np.median(trans)), "p90": float(np.percentile(trans, 90)),
                                   "max": float(trans.max())},
            "within_0.05deg_5mm": within,
            "vs_gt_rot_deg_median": float(np.median(rot_gt)), "vs_gt_trans_mm_median": float(np.median(trans_gt)),
            "batch_ms": a.elapsed_time(b), "status": sorted({r["status"] for r in res})})
    ctx.close()
    return out


def run_precision_study(args):
    import torch

    qs = _c4_queries(PRECISION_QUERIES)
    ref, oracle_s = _c4_oracle(qs)
    torch.cuda.set_device(0)
    print(json.dumps({"precision_study": precision_study(torch.device("cuda", 0), qs, ref, oracle_s)}))
    return 0


# ---------------------------------------------------------------------------
# C1: one plain query per call
# ---------------------------------------------------------------------------
C1_QUERIES = 16


def c1_inputs(n=C1_QUERIES):
    """C1 queries and the FP64 oracle's final pose of each (same seed and query id as the GPU calls)."""
    import oracle

    from paper_2601_04185_gb300 import synth

    qs = [synth.config1(300 + i) for i in range(n)]

    def one(i):
        q = qs[i]
        r = oracle.ransac_pnp(oracle.Corr(q["x"], q["y"], q["X"], q["w"]), q["K"], max_iters=q["hypotheses"],
                              p_miss=0.0, tau=q["tau"], query_id=i, seed=41)
        return r["R"], r["t"]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        ref = list(ex.map(one, range(n)))
    return qs, ref, time.perf_counter() - t0


def run_c1(dev, qs, ref, oracle_s, reps=5):
    """C1: a single query per imloc_ransac_pnp call (2,000 correspondences,
    1,000 minimal sets, LO, refinement; host-synchronous), timed on the host
    clock per call: p50/p99 latency, queries/s, hyp*corr/s; final poses
    against the FP64 oracle's."""
    import torch

    from paper_2601_04185_gb300 import imloc

    ctx = imloc.Context(dev.index, 256 << 20)
    corrs = [imloc.corr_from_arrays(q["x"], q["y"], q["X"], q["w"], device=dev) for q in qs]
    opts = [imloc.default_opts(max_iters=q["hypotheses"], p_miss=0.0, tau_px=q["tau"], query_id=i, seed=41)
            for i, q in enumerate(qs)]
    stream = torch.cuda.Stream(dev)
    for i, q in enumerate(qs):
        ctx.ransac_pnp(corrs[i], q["K"], opts[i], stream=stream)
    lat, res, pairs = [], [None] * len(qs), 0.0
    for _ in range(reps):
        for i, q in enumerate(qs):
            t0 = time.perf_counter()
            r = ctx.ransac_pnp(corrs[i], q["K"], opts[i], stream=stream)
            lat.append(1e3 * (time.perf_counter() - t0))
            res[i] = r
            pairs += r["hypotheses"] * min(len(q["x"]), 10000)
    ctx.close()
    lat_s = sorted(lat)
    rot = np.array([_rot_err_deg(r["R"], o[0]) for r, o in zip(res, ref)])
    trans = np.array([1e3 * np.linalg.norm(-r["R"].T @ r["t"] + o[0].T @ o[1]) for r, o in zip(res, ref)])
    return {"workload": "C1: one query per call, 2,000 correspondences (640x480, f = 500, 30 % inliers, N(0, 1 px)), "
                        "1,000 minimal sets, tau 4 px, LO + Cauchy refinement; host-synchronous imloc_ransac_pnp, "
                        "correspondences resident on the device",
            "latency_ms_p50": lat_s[len(lat_s) // 2],
            "latency_ms_p99": lat_s[min(len(lat_s) - 1, int(math.ceil(0.99 * len(lat_s))) - 1)],
            "queries_per_s": 1e3 / statistics.mean(lat), "hyp_corr_per_s": pairs / (sum(lat) * 1e-3),
            "calls": len(lat), "status": sorted({r["status"] for r in res}), "oracle_seconds": oracle_s,
            "vs_oracle_rot_deg_max": float(rot.max()), "vs_oracle_trans_mm_max": float(trans.max()),
            "within_0.05deg_5mm": float(np.mean((rot <= 0.05) & (trans <= 5.0)))}


# ---------------------------------------------------------------------------
# lift roofline on a batched shape (many queries, ~10^7 matches per launch)
# ---------------------------------------------------------------------------
def concat_store_queries(dev, store_views_dev, queries):
    """The matches of serving queries concatenated (each query's segments
    pointing at the store views it uses) and moved to the device."""
    import torch

    views, qb = [], [0]
    cat = {k: [] for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    seg_off, seg_view, seg_dir = [0], [], []
    vid_of = {}
    for q in queries:
        m = q["matches"]
        for k in cat:
            cat[k].append(m[k])
        for s_ in range(len(m["seg_view"])):
            sid = q["view_ids"][int(m["seg_view"][s_])]
            if sid not in vid_of:
                vid_of[sid] = len(views)
                views.append(store_views_dev[sid])
            seg_off.append(qb[-1] + int(m["seg_off"][s_ + 1]))
            seg_view.append(vid_of[sid])
            seg_dir.append(int(m["seg_dir"][s_]))
        qb.append(qb[-1] + int(m["seg_off"][-1]))
    big = {k: np.concatenate(v).astype(np.float32) for k, v in cat.items()}
    d_match = {k: torch.from_numpy(big[k]).to(dev) for k in big}
    d_match.update(seg_off=np.array(seg_off, np.int64), seg_view=np.array(seg_view, np.int32),
                   seg_dir=np.array(seg_dir, np.int32))
    return views, np.array(qb, np.int64), big, d_match, seg_off, seg_dir


def run_batched_c5(dev, store_views_dev, queries, repeats=5):
    """The serving queries in one batched call (lift + LO-RANSAC with the
    served options: at most 10,000 minimal sets, adaptive stop 1e-4), matches
    resident on the device: the batched rate the served form is compared with."""
    import torch

    from paper_2601_04185_gb300 import imloc

    views, qb, big, d_match, _, _ = concat_store_queries(dev, store_views_dev, queries)
    nq = len(queries)
    ctx = imloc.Context(dev.index, 2 << 30)
    stream = torch.cuda.Stream(dev)
    corr = imloc.alloc_corr(int(qb[-1]), dev)
    offs = torch.zeros(nq + 1, dtype=torch.int64, device=dev)
    res = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
    opts = [imloc.default_opts(max_iters=10000, p_miss=1e-4, query_id=i, seed=4321) for i in range(nq)]
    pl = imloc.prepare_lift_batch(qb, views, d_match)
    pr = imloc.prepare_ransac_batch([q["K"] for q in queries], opts)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def once():
        ctx.lift_batch(qb, views, d_match, out=corr, offsets=offs, stream=stream, prepared=pl)
        ctx.ransac_pnp_batch_async(corr, offs, None, None, res, stream=stream, prepared=pr)

    for _ in range(3):
        once()
    torch.cuda.synchronize()
    ms = []
    for _ in range(repeats):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        once()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    r = imloc.results_from_bytes(res.cpu().numpy(), nq)
    ctx.close()
    m = statistics.median(ms)
    return {"queries": nq, "matches": int(qb[-1]), "ms_per_batch": m, "queries_per_s": nq / (m * 1e-3),
            "status": sorted({x["status"] for x in r}),
            "note": "the serving queries lifted and localized in one batched call each repetition (L2 flushed)"}


def run_lift_batched(dev, store_views_dev, queries, repeats=10, log8=False, tile4=False, halo=False):
    """One lift launch over all serving queries concatenated (each query's
    matches against its own store views); algorithmic bytes / event time.
    log8: the store views as 8-bit log depth codes (the depth codec of
    Sec. 3.3 "Data Compression", decoded inside the lift); tile4: the float32
    maps in 4x4-pixel blocks of 64 bytes; halo: in overlapping 8x4-pixel
    blocks of 128 bytes every 7 x 3 pixels (every footprint in one block)."""
    import torch

    from paper_2601_04185_gb300 import imloc

    if log8 or tile4 or halo:
        enc = []
        for v in store_views_dev:
            if tile4:
                enc.append(imloc.tile4_view(v))
            elif halo:
                enc.append(imloc.halo_view(v))
            else:
                d = dict(v)
                d["depth"] = imloc.depth_encode_log8(v["depth"])
                enc.append(d)
        torch.cuda.synchronize()
        store_views_dev = enc

    views, qb, big, d_match, seg_off, seg_dir = concat_store_queries(dev, store_views_dev, queries)
    n = int(qb[-1])
    ctx = imloc.Context(dev.index, 512 << 20)
    out = imloc.alloc_corr(n, dev)
    offs = torch.zeros(len(queries) + 1, dtype=torch.int64, device=dev)
    prep = imloc.prepare_lift_batch(qb, views, d_match)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        ctx.lift_batch(qb, views, d_match, out=out, offsets=offs, stream=stream, prepared=prep)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for _ in range(repeats):
        flush.zero_()
        ctx.lift_batch(qb, views, d_match, out=out, offsets=offs, stream=stream, prepared=prep)
    torch.cuda.synchronize()
    k = ctx.profile_read(reset=True)["k_lift"]
    ctx.close()
    launch_ms = k[1] / k[0]
    n_valid = int(offs[-1].item())
    conf_ok = big["conf"] > np.float32(0.05)
    dirs = np.repeat(np.array(seg_dir), np.diff(np.array(seg_off)))
    nbytes = 20 * n + int(np.sum(np.where(dirs[conf_ok] == 0, 64, 32))) + 28 * n_valid
    # the same count with 64-byte DRAM atoms for the random depth taps (2 x 64 B bilinear, 64 B lookup)
    nbytes64 = 20 * n + int(np.sum(np.where(dirs[conf_ok] == 0, 128, 64))) + 28 * n_valid
    return {"depth_format": "log8" if log8 else ("f32 4x4 blocks" if tile4 else ("f32 8x4 overlapping blocks" if halo
                                                                              else "f32")), "map_store_bytes": int(sum(v["depth"].numel() * v["depth"].element_size() for v in views)),
            "matches_per_launch": n, "valid": n_valid, "bytes_per_launch": nbytes, "launch_ms": launch_ms,
            "achieved_gbs": nbytes / (launch_ms * 1e-3) / 1e9, "store_views": len(views),
            "bytes_per_launch_64b_atoms": nbytes64, "achieved_gbs_64b_atoms": nbytes64 / (launch_ms * 1e-3) / 1e9,
            "workload": f"{len(queries)} serving queries concatenated ({n} matches) against "
                        f"{len(views)} resident 1024x768 depth maps, L2 flushed before each launch"}


def fp32_peak_tflops(dev, peaks):
    """Derived FP32 FMA peak of the device: SMs (queried) x 128 lanes x 2 flops x max SM clock."""
    import torch

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return (sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            f"{sm_count} SMs (device) x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {mhz:.0f} MHz "
            "(max SM clock, MEASURED_PEAKS.json; derived FP32 FMA peak)")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def run_retrieval_only(args):
    import torch

    torch.cuda.set_device(0)
    print(json.dumps({"retrieval": run_retrieval(torch.device("cuda", 0), load_peaks(), repeats=args.steps)}))
    return 0


def run_lift_only(args):
    import torch

    store, store_views, sq = make_store_and_queries(2024, args.serve_queries)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    dv = []
    for v in store_views:
        d = dict(v)
        d["depth"] = torch.from_numpy(v["depth"]).to(dev)
        dv.append(d)
    print(json.dumps({"lift_batched": run_lift_batched(dev, dv, sq, repeats=args.steps),
                      "lift_batched_tile4": run_lift_batched(dev, dv, sq, repeats=args.steps, tile4=True),
                      "lift_batched_halo": run_lift_batched(dev, dv, sq, repeats=args.steps, halo=True),
                      "lift_batched_log8": run_lift_batched(dev, dv, sq, repeats=args.steps, log8=True)}))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2601_04185_gb300 import imloc

    # inputs first (process pools before CUDA starts in this process)
    queries = make_queries(args.queries, rank_seed(100, int(os.environ.get("RANK", "0"))))
    serving_inputs = None
    if int(os.environ.get("WORLD_SIZE", "1")) == 1 and not args.no_serving:
        serving_inputs = make_store_and_queries(2024, args.serve_queries)
    # C1 and C4 inputs with the FP64 oracle's poses (host cores, before the GPU work)
    c1_in = c4_in = None
    if int(os.environ.get("WORLD_SIZE", "1")) == 1:
        if not args.no_c1:
            c1_in = c1_inputs()
        if not args.no_c4:
            qs4 = _c4_queries(args.c4_queries)
            c4_in = (qs4,) + _c4_oracle(qs4)
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    views, big, qb = concat_batch(queries)
    nq = len(queries)
    d_views = []
    for v in views:
        d = dict(v)
        d["depth"] = torch.from_numpy(v["depth"]).to(dev)
        d_views.append(d)
    d_match = {k: torch.from_numpy(big[k]).to(dev) for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    d_match.update({k: big[k] for k in ("seg_off", "seg_view", "seg_dir")})
    h_match = {k: torch.from_numpy(big[k]).pin_memory() for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    n_matches = int(qb[-1])
    ctx = imloc.Context(dev.index, (256 << 20) + nq * (64 << 20))
    corr = imloc.alloc_corr(n_matches, dev)
    offsets = torch.zeros(nq + 1, dtype=torch.int64, device=dev)
    results = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
    h_results = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    opts = [imloc.default_opts(max_iters=HYPOTHESES, p_miss=0.0, query_id=i, seed=1234) for i in range(nq)]
    Ks = [q["K"] for q in queries]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # a dedicated stream (the library captures its launch sequences as CUDA graphs on real streams)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    prep_lift = imloc.prepare_lift_batch(qb, d_views, d_match)
    prep_ransac = imloc.prepare_ransac_batch(Ks, opts)

    def step(from_host=False):
        if from_host:
            for k in h_match:
                d_match[k].copy_(h_match[k], non_blocking=True)
        ctx.lift_batch(qb, d_views, d_match, out=corr, offsets=offsets, stream=stream, prepared=prep_lift)
        ctx.ransac_pnp_batch_async(corr, offsets, Ks, opts, results, stream=stream, prepared=prep_ransac)
        if from_host:
            h_results.copy_(results, non_blocking=True)

    # Two batches in flight: a second context (its own workspace and captured
    # graphs), output buffers and stream, so that one batch's small latency-
    # bound kernels and replay overlap the other batch's scoring.  Steps
    # alternate between the two lanes; each runs the whole path.
    lanes = [dict(ctx=ctx, corr=corr, offsets=offsets, results=results, stream=stream, pl=prep_lift,
                  pr=prep_ransac)]
    ctx_b = imloc.Context(dev.index, (256 << 20) + nq * (64 << 20))
    lanes.append(dict(ctx=ctx_b, corr=imloc.alloc_corr(n_matches, dev),
                      offsets=torch.zeros(nq + 1, dtype=torch.int64, device=dev),
                      results=torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev),
                      stream=torch.cuda.Stream(dev), pl=imloc.prepare_lift_batch(qb, d_views, d_match),
                      pr=imloc.prepare_ransac_batch(Ks, opts)))

    def lane_step(L, dm=None, pl=None):
        L["ctx"].lift_batch(qb, d_views, d_match if dm is None else dm, out=L["corr"], offsets=L["offsets"],
                            stream=L["stream"], prepared=L["pl"] if pl is None else pl)
        L["ctx"].ransac_pnp_batch_async(L["corr"], L["offsets"], Ks, opts, L["results"], stream=L["stream"],
                                        prepared=L["pr"])

    # ---- device-timed steps (inputs resident): the library's own launch path (CUDA graphs) ----
    # K steps alternating between the two lanes, timed from the first launch to
    # the end of the last step of either lane; no L2 flush (a step's inputs,
    # 160 depth maps and 16 MB of matches, exceed the L2).  The clock sampler
    # starts before the warm-up steps, so that the GPU is not left idle (and
    # its clock lowered) between the warm-up and the timed steps.
    t_first, t_last = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        for _ in range(args.warmup):
            for L in lanes:
                lane_step(L)
        barrier(world)
        torch.cuda.synchronize()
        t_first.record(stream)
        lanes[1]["stream"].wait_event(t_first)
        for i in range(args.steps):
            lane_step(lanes[i % 2])
        joined = torch.cuda.Event()
        joined.record(lanes[1]["stream"])
        stream.wait_event(joined)
        t_last.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    timed_s = t_first.elapsed_time(t_last) / 1e3
    lanes_identical = bool(torch.equal(lanes[0]["results"], lanes[1]["results"]))
    # ---- per-kernel launch durations: the same K steps again, traced per kernel ----
    # (CUDA events around every launch on the launching stream; tracing switches the
    # graph replay off, so these steps are not the ones the headline times)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for i in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    kstats = ctx.profile_read(reset=True)
    # the FP32 scoring kernel on the same step (replay in its own kernel) for its roofline: a few extra steps
    os.environ["IMLOC_NO_FUSE"] = "1"
    os.environ["IMLOC_SCORE_TC"] = "0"
    for _ in range(3):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.profile_read(reset=True)
    n_unfused = max(3, args.steps // 3)
    for _ in range(n_unfused):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    kstats_unfused = ctx.profile_read(reset=True)
    del os.environ["IMLOC_SCORE_TC"]
    del os.environ["IMLOC_NO_FUSE"]
    ctx.profile(False)
    total_s_max = max_over_ranks(timed_s, world)

    res = imloc.results_from_bytes(results.cpu().numpy(), nq)
    offs = offsets.cpu().numpy()
    n_corr = np.diff(offs)
    pairs_per_step = float(sum(r["hypotheses"] * min(int(n), 10000) for r, n in zip(res, n_corr)))
    statuses = sorted({r["status"] for r in res})
    pairs_all = sum_over_ranks(pairs_per_step * args.steps, world)
    value = pairs_all / total_s_max
    q_per_s = sum_over_ranks(nq * args.steps, world) / total_s_max

    # ---- end to end through the public API with host buffers ----
    # Every step uploads its matches from pinned host memory and reads its
    # results back, with the same two lanes as the device-timed steps: step i
    # runs on lane i mod 2 and lifts from that lane's device match buffer,
    # into which a copy stream uploads the step's matches once the lane's
    # previous step has lifted from it (events order the reuse); the results
    # are read back on the lane's stream into its pinned host buffer.  All
    # copies and read-backs are inside the timed region, which spans the K
    # steps.  No L2 flush between steps: a step's inputs (the depth maps of
    # its views and its matches) exceed the L2.
    h2d = sum(h_match[k].numel() * 4 for k in h_match)
    d2h = results.numel()
    d_match_b = [d_match, dict(d_match, **{k: torch.empty_like(d_match[k]) for k in h_match})]
    prep_b = [prep_lift, imloc.prepare_lift_batch(qb, d_views, d_match_b[1])]
    h_results_b = [h_results, torch.zeros_like(h_results).pin_memory()]
    copy_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(b):
        with torch.cuda.stream(copy_stream):
            for k in h_match:
                d_match_b[b][k].copy_(h_match[k], non_blocking=True)
        copied[b].record(copy_stream)

    def e2e_steps(k, start_ev=None):
        if start_ev is not None:
            copy_stream.wait_event(start_ev)
            lanes[1]["stream"].wait_event(start_ev)
        else:
            copy_stream.wait_stream(stream)
            lanes[1]["stream"].wait_stream(stream)
        upload(0)
        for i in range(k):
            b = i % 2
            L = lanes[b]
            if i + 1 < k:
                if i >= 1:
                    copy_stream.wait_event(consumed[1 - b])  # step i-1 (lane 1-b) has lifted from that buffer
                upload(1 - b)
            L["stream"].wait_event(copied[b])
            with torch.cuda.stream(L["stream"]):
                L["ctx"].lift_batch(qb, d_views, d_match_b[b], out=L["corr"], offsets=L["offsets"],
                                    stream=L["stream"], prepared=prep_b[b])
                consumed[b].record(L["stream"])
                L["ctx"].ransac_pnp_batch_async(L["corr"], L["offsets"], Ks, opts, L["results"], stream=L["stream"],
                                                prepared=L["pr"])
                h_results_b[b].copy_(L["results"], non_blocking=True)
        joined_e = torch.cuda.Event()
        joined_e.record(lanes[1]["stream"])
        stream.wait_event(joined_e)
        stream.wait_stream(copy_stream)

    # untimed: both lanes and match buffers once (the library captures a launch graph per buffer on first use)
    e2e_steps(max(4, args.warmup))
    torch.cuda.synchronize()
    t_start.record(stream)
    e2e_steps(args.steps, t_start)
    t_end.record(stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(t_start.elapsed_time(t_end) / 1e3, world)
    e2e_value = pairs_all / e2e_s
    e2e_identical = bool(torch.equal(h_results_b[0], h_results_b[1]))
    ctx_b.close()

    # ---- roofline stress mode: every pose scored against all N correspondences (M = N) ----
    full_cap = 1 << 16
    opts_full = [imloc.default_opts(max_iters=HYPOTHESES, p_miss=0.0, query_id=i, seed=1234, max_score_corr=full_cap)
                 for i in range(nq)]
    prep_full = imloc.prepare_ransac_batch(Ks, opts_full)
    results_full = torch.zeros(nq * imloc.RESULT_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(2):
        ctx.ransac_pnp_batch_async(corr, offsets, Ks, opts_full, results_full, stream=stream, prepared=prep_full)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    n_full = 3
    for _ in range(n_full):
        flush.zero_()
        ctx.ransac_pnp_batch_async(corr, offsets, Ks, opts_full, results_full, stream=stream, prepared=prep_full)
    torch.cuda.synchronize()
    kfull = ctx.profile_read(reset=True)
    ctx.profile(False)
    res_full = imloc.results_from_bytes(results_full.cpu().numpy(), nq)
    n_corr_full = np.diff(offsets.cpu().numpy())
    pairs_full = float(sum(r["hypotheses"] * min(int(n), full_cap) for r, n in zip(res_full, n_corr_full)))
    full_key = "k_score_tc" if "k_score_tc" in kfull else "k_score"
    full_ms = kfull[full_key][1] / max(1, kfull[full_key][0]) if full_key in kfull else None
    full_tflops = pairs_full * FLOPS_PER_PAIR / (full_ms * 1e-3) / 1e12 if full_ms else None

    # ---- plain form: one query per call (lift, then RANSAC), host-synchronous ----
    lat = []
    q_single = {}
    for i in range(min(nq, 8)):
        q = queries[i]
        dv = d_views[i * N_VIEWS:(i + 1) * N_VIEWS]
        dm = {k: torch.from_numpy(q["matches"][k]).to(dev) for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
        dm.update({k: q["matches"][k] for k in ("seg_off", "seg_view", "seg_dir")})
        q_single[i] = dm
    c1 = imloc.alloc_corr(n_matches, dev)
    for rep in range(3):
        for i in q_single:
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.lift(d_views[i * N_VIEWS:(i + 1) * N_VIEWS], q_single[i], out=c1, stream=stream)
            ctx.ransac_pnp(c1, queries[i]["K"], imloc.default_opts(max_iters=HYPOTHESES, p_miss=0.0, query_id=i,
                                                                    seed=1234), stream=stream)
            lat.append(1e3 * (time.perf_counter() - t0))
    lat_sorted = sorted(lat)
    p50 = lat_sorted[len(lat) // 2]
    p99 = lat_sorted[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    # ---- roofline of the dominant kernel (the scoring kernel of the step) ----
    clocks = clk.summary()
    launches = {k: v[0] for k, v in kstats.items()}
    kms = {k: v[1] for k, v in kstats.items()}
    score_key = "k_score_tc" if "k_score_tc" in kms else "k_score"
    score_launch_ms = kms.get(score_key, 0.0) / max(1, launches.get(score_key, 1))
    pairs_per_launch = pairs_per_step * args.steps / max(1, launches.get(score_key, 1))
    achieved_tflops = FLOPS_PER_PAIR * pairs_per_launch / (score_launch_ms * 1e-3) / 1e12 if score_launch_ms else None
    u_launches, u_ms = kstats_unfused.get("k_score", (1, 0.0))
    score_only_ms = u_ms / max(1, u_launches)
    score_only_tflops = FLOPS_PER_PAIR * pairs_per_step / (score_only_ms * 1e-3) / 1e12 if score_only_ms else None
    score_cfg = ctx.score_config()
    if score_key == "k_score_tc":
        score_traffic = SCORE_TC_TRAFFIC_PER_LAUNCH if nq == 16 else None
    else:
        score_traffic = SCORE_TRAFFIC_PER_LAUNCH.get(tuple(score_cfg[:2])) if (score_cfg and nq == 16) else None
    peaks = load_peaks()
    peak_tflops, peak_basis = fp32_peak_tflops(dev, peaks)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    tc_epi_tflops = (TC_FP32_FLOPS_PER_PAIR * pairs_per_launch / (score_launch_ms * 1e-3) / 1e12
                     if (score_key == "k_score_tc" and score_launch_ms) else None)
    tc_tensor_tflops = (TC_MMA_FLOPS_PER_PAIR * pairs_per_launch / (score_launch_ms * 1e-3) / 1e12
                        if (score_key == "k_score_tc" and score_launch_ms) else None)
    lift_ms = kms.get("k_lift", 0.0) / max(1, launches.get("k_lift", 1))
    # algorithmic bytes of one lift launch: 20 B per match, 64 B (bilinear) or 32 B (lookup) of depth
    # sectors per match that passes the confidence filter, 28 B per correspondence written
    conf_ok = big["conf"] > np.float32(0.05)
    dirs = np.repeat(big["seg_dir"], np.diff(big["seg_off"]))
    lift_bytes = 20 * n_matches + int(np.sum(np.where(dirs[conf_ok] == 0, 64, 32))) + 28 * int(offs[-1])
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    lift_gbs = lift_bytes / (lift_ms * 1e-3) / 1e9 if lift_ms else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": c2_workload(nq),
                   "queries_per_step": nq, "matches_per_query": N_VIEWS * MATCHES_PER_PAIR,
                   "depth": "1024x768 float32, 10 views/query", "hypotheses": HYPOTHESES, "score_corr_cap": 10000,
                   "l2": "not flushed: a step's inputs (160 depth maps of 3 MB, 16 MB of matches) exceed the L2",
                   "batches_in_flight": 2, "parallelism": f"replicas x{world}"},
        "queries_per_s": q_per_s,
        "lanes_identical_results": lanes_identical,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "queries_per_s": sum_over_ranks(nq * args.steps, world) / e2e_s,
                "form": "matches uploaded from pinned host memory every step on a copy stream into the device "
                        "buffer of the step's lane (two batches in flight, as in the device-timed steps), results "
                        "read back every step; timed over the K steps, no L2 flush (a step's depth maps and matches "
                        "exceed L2)", "lanes_identical_results": e2e_identical},
        "plain": {"latency_ms_p50": p50, "latency_ms_p99": p99, "queries_per_s": 1e3 / statistics.mean(lat),
                  "form": "one query per call: imloc_lift_async + imloc_ransac_pnp (host-synchronous)",
                  "samples": len(lat)},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": (achieved_tflops / peak_tflops) if achieved_tflops else None,
                     "traffic": score_traffic, "kernel": score_key,
                     "variant": ("k_score_tcr: 128-record blocks x 80-pose items, bf16 pieces"
                                 if score_key == "k_score_tc" else score_cfg),
                     "peak_basis": peak_basis, "flops_per_pair": FLOPS_PER_PAIR,
                     "flops_per_pair_basis": "13 FMA + 1 MUL per (pose, correspondence) pair",
                     "pairs_per_launch": pairs_per_launch, "launch_ms": score_launch_ms,
                     **({"tensor": {"achieved": tc_tensor_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                                    "frac": (tc_tensor_tflops / bf16_peak) if tc_tensor_tflops else None,
                                    "flops_per_pair": TC_MMA_FLOPS_PER_PAIR,
                                    "peak_basis": "measured bf16 burst (cuBLAS)"},
                         "fp32_epilogue": {"achieved": tc_epi_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                                           "frac": (tc_epi_tflops / peak_tflops) if tc_epi_tflops else None,
                                           "flops_per_pair": TC_FP32_FLOPS_PER_PAIR},
                         "note": "tensor-core scoring: achieved counts the method's 27 flops per pair; the "
                                 "projection runs on the tensor pipe (6 split bf16 piece products per coordinate "
                                 "row, 3 rows, K padded to 32: 192 MMA flops per pair, sub-entry tensor) and the "
                                 "FP32 epilogue does 9 flops per pair (sub-entry fp32_epilogue)"}
                        if score_key == "k_score_tc" else {})},
        "roofline_fp32_kernel": {"bound": "alu", "achieved": score_only_tflops, "peak": peak_tflops,
                                 "unit": "TFLOP/s", "kernel": "k_score",
                                 "frac": (score_only_tflops / peak_tflops) if score_only_tflops else None,
                                 "flops_per_pair": FLOPS_PER_PAIR, "launch_ms": score_only_ms,
                                 "traffic": SCORE_TRAFFIC_PER_LAUNCH.get(tuple(score_cfg[:2]))
                                 if (score_cfg and nq == 16) else None, "variant": score_cfg,
                                 "replay_kernel_ms": kstats_unfused.get("k_replay", (1, 0))[1]
                                 / max(1, kstats_unfused.get("k_replay", (1, 0))[0]),
                                 "note": "the FP32-only scoring kernel (IMLOC_SCORE_TC=0) on the same step: 27 "
                                         "flops per pair on the FMA pipe; it scores single queries and calls too "
                                         "small for the tensor-core kernel"},
        "roofline_full_n": {"bound": "alu", "achieved": full_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                            "frac": (full_tflops / peak_tflops) if full_tflops else None, "launch_ms": full_ms,
                            "pairs_per_launch": pairs_full,
                            "mean_scored_corr": float(np.mean(np.minimum(n_corr_full, full_cap))),
                            "kernel": full_key, "flops_per_pair": FLOPS_PER_PAIR,
                            "note": "stress mode: the same step's poses scored against all N correspondences "
                                    "(subset cap raised to 65,536), one scoring launch"},
        "lift_in_step": {"bound": "hbm", "achieved": lift_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": (lift_gbs / hbm_peak) if lift_gbs else None, "bytes_per_launch": lift_bytes,
                         "launch_ms": lift_ms, "note": "16-query step: 800k matches, latency-bound"},
        "kernels_ms_per_step": {k: v / args.steps for k, v in kms.items()},
        "kernel_timing": "per-kernel CUDA events on the launching stream over a second pass of the same K steps "
                         "on one lane, the L2 flushed before each step; tracing switches the library's CUDA-graph "
                         "replay off, so the headline steps run untraced",
        "gpu_launches": int(sum(launches.values())),
        "clocks": clocks,
        "result_status": statuses,
        "per_query": {"lo_runs_mean": float(np.mean([r["lo_count"] for r in res])),
                      "gn_passes_mean": float(np.mean([r["passes"] for r in res])),
                      "hypotheses_mean": float(np.mean([r["hypotheses"] for r in res])),
                      "inliers_mean": float(np.mean([r["num_inliers"] for r in res]))},
        "paper_context": "ImLoc reports ~200 ms per query for its RANSAC loop on an RTX 4090 (Sec. 4.4); "
                         "different hardware and data",
    }
    # ---- batched C3 ----
    if world == 1 and not args.no_c3:
        line["batched_c3"] = run_batched_c3(dev)
    # ---- C1: one plain query per call ----
    if c1_in is not None:
        line["c1"] = run_c1(dev, *c1_in)
    # ---- C4: precision variants against the FP64 oracle ----
    if c4_in is not None:
        line["precision_study"] = precision_study(dev, *c4_in)
    # ---- retrieval nearest-neighbour search (next row f4) ----
    if world == 1 and not args.no_retrieval:
        line["retrieval"] = run_retrieval(dev, peaks)
    # ---- generalized absolute pose of rig queries (next row f3) ----
    if world == 1 and not args.no_rig:
        line["rig"] = run_rig(dev, peaks)
    # ---- mapping-time dense triangulation (next row f2) ----
    if world == 1 and not args.no_triangulation:
        line["triangulation"] = run_triangulation(dev)
    # ---- serving (C5): Poisson arrivals, served vs plain ----
    if serving_inputs is not None:
        # the earlier legs' buffers go before the host-timed serving loop
        gc.collect()
        torch.cuda.empty_cache()
        store, store_views, sq = serving_inputs
        dv = []
        for v in store_views:
            d = dict(v)
            d["depth"] = torch.from_numpy(v["depth"]).to(dev)
            dv.append(d)
        lb = run_lift_batched(dev, dv, sq)
        line["roofline_lift"] = {"bound": "hbm", "achieved": lb["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                                 "frac": lb["achieved_gbs"] / hbm_peak, "traffic": LIFT_TRAFFIC_PER_MATCH and
                                 LIFT_TRAFFIC_PER_MATCH * lb["matches_per_launch"],
                                 "traffic_note": "null: the committed row-major capture (207.6 B per match) predates "
                                                 "the kernel's overlapping-block branch; see lift_halo",
                                 "kernel": "k_lift", "peak_basis": "MEASURED_PEAKS.json hbm_gbs (measured)", **lb}
        lbt = run_lift_batched(dev, dv, sq, tile4=True)
        line["lift_tile4"] = {"bound": "hbm", "achieved": lbt["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                              "frac": lbt["achieved_gbs"] / hbm_peak, "launch_ms": lbt["launch_ms"],
                              "speedup_vs_f32": lb["launch_ms"] / lbt["launch_ms"], "valid": lbt["valid"],
                              "bytes_per_launch": lbt["bytes_per_launch"],
                              "note": "same matches and algorithmic bytes as roofline_lift, the float32 store maps "
                                      "in 4x4-pixel blocks of 64 B (imloc_depth_tile4_async); L2 flushed before "
                                      "each launch"}
        lbh = run_lift_batched(dev, dv, sq, halo=True)
        line["lift_halo"] = {"bound": "hbm", "achieved": lbh["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                             "frac": lbh["achieved_gbs"] / hbm_peak, "launch_ms": lbh["launch_ms"],
                             "traffic": LIFT_HALO_TRAFFIC_PER_MATCH * lbh["matches_per_launch"],
                             "speedup_vs_f32": lb["launch_ms"] / lbh["launch_ms"], "valid": lbh["valid"],
                             "bytes_per_launch": lbh["bytes_per_launch"], "map_store_bytes": lbh["map_store_bytes"],
                             "note": "same matches and algorithmic bytes as roofline_lift, the float32 store maps "
                                     "in overlapping 8x4-pixel blocks of 128 B every 7 x 3 pixels "
                                     "(imloc_depth_halo_async: every footprint in one DRAM line, 1.52x the store); "
                                     "L2 flushed before each launch"}
        lb8 = run_lift_batched(dev, dv, sq, log8=True)
        line["lift_log8"] = {"launch_ms": lb8["launch_ms"], "speedup_vs_f32": lb["launch_ms"] / lb8["launch_ms"],
                             "matches_per_s": lb8["matches_per_launch"] / (lb8["launch_ms"] * 1e-3),
                             "valid": lb8["valid"], "map_store_bytes": lb8["map_store_bytes"],
                             "map_store_bytes_f32": lb["map_store_bytes"],
                             "note": "same matches as roofline_lift, store views as 8-bit log depth codes "
                                     "(Sec. 3.3 Data Compression) decoded inside k_lift; L2 flushed before each launch"}
        line["serving"] = run_serving(dev, SERVE_RATES, args.serve_per_rate, sq, dv)
        line["serving"]["batched"] = run_batched_c5(dev, dv, sq)
        bq = line["serving"]["batched"]["queries_per_s"]
        line["serving"]["served_peak_over_batched"] = max(x["q_per_s"] for x in line["serving"]["served"]) / bq
        line["serving"]["served_device_peak_over_batched"] = max(
            x["q_per_s"] for x in line["serving"]["served_device"]) / bq
        line["serving"]["workload"] = (f"C5: map store of {STORE_VIEWS} views (1024x768 float32 depth, resident), "
                                       f"{len(sq)} distinct queries of 10-40 views x 5,000 matches, "
                                       "10,000 minimal sets max with the adaptive stop (p = 1e-4); Poisson arrivals")
    # ---- CPU baseline: the FP64 oracle on the host cores (rank 0, N = 1 only) ----
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample = queries[:min(nq, cores)]
        wall, pairs = oracle_queries(sample, HYPOTHESES, cores)
        line["cpu_baseline"] = {"value": pairs / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{len(sample)} of the step's queries (lift + {HYPOTHESES} minimal "
                                          f"sets + LO + refinement), one per thread, {wall:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--queries", type=int, default=16, help="queries per step (per GPU)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--no-c1", action="store_true")
    ap.add_argument("--no-c4", action="store_true")
    ap.add_argument("--c4-queries", type=int, default=16, help="queries of the precision study in the bench line")
    ap.add_argument("--no-triangulation", action="store_true")
    ap.add_argument("--no-rig", action="store_true")
    ap.add_argument("--no-retrieval", action="store_true")
    ap.add_argument("--precision-study", action="store_true", help="C4: precision variants vs the oracle")
    ap.add_argument("--lift-only", action="store_true", help="only the batched lift measurement")
    ap.add_argument("--retrieval-only", action="store_true", help="only the retrieval search measurement")
    ap.add_argument("--rig-only", action="store_true", help="only the rig-query measurement")
    ap.add_argument("--serve-queries", type=int, default=80, help="distinct serving queries")
    ap.add_argument("--serve-per-rate", type=int, default=600, help="arrivals per offered rate (at most 3 s of arrivals)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.precision_study:
        return run_precision_study(args)
    if args.lift_only:
        return run_lift_only(args)
    if args.retrieval_only:
        return run_retrieval_only(args)
    if args.rig_only:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"rig": run_rig(torch.device("cuda", 0), load_peaks(), repeats=args.steps)}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
