"""Thin Python binding of ``libimloc.so`` (C ABI in ``include/imloc.h``).

Argument marshalling only: every step of the localization path runs in the
CUDA kernels of the library.  PyTorch provides device memory and streams.
There is no fallback: if the library is missing or no CUDA device is present
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libimloc.so")

IMLOC_OK = 0
IMLOC_PENDING = 1
STATUS = {0: "ok", 1: "pending", -1: "invalid argument", -2: "out of workspace memory", -3: "rejected",
          -4: "timeout", -5: "cuda error", -6: "not found", -7: "degenerate", -8: "capacity"}


class Camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class Pose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


DEPTH_F32, DEPTH_LOG8, DEPTH_F32_TILE4, DEPTH_F32_HALO = 0, 1, 2, 3


class View(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32), ("pitch", C.c_int64),
                ("cam", Camera), ("pose", Pose), ("depth_format", C.c_int32), ("reserved", C.c_int32)]


class TriangulateOpts(C.Structure):
    _fields_ = [("angle_deg", C.c_float), ("conf_min", C.c_float), ("keep_more_than", C.c_int32),
                ("refine_iters", C.c_int32)]


class Segment(C.Structure):
    _fields_ = [("begin", C.c_int64), ("view", C.c_int32), ("direction", C.c_int32)]


class Matches(C.Structure):
    _fields_ = [("q_u", C.c_void_p), ("q_v", C.c_void_p), ("db_u", C.c_void_p), ("db_v", C.c_void_p),
                ("conf", C.c_void_p), ("n", C.c_int64), ("segments", C.POINTER(Segment)), ("n_segments", C.c_int32)]


class Corr(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("X", C.c_void_p), ("Y", C.c_void_p), ("Z", C.c_void_p),
                ("w", C.c_void_p), ("src", C.c_void_p), ("count", C.c_void_p), ("capacity", C.c_int64)]


class RansacOpts(C.Structure):
    _fields_ = [("tau_px", C.c_double), ("max_score_corr", C.c_int32), ("batch", C.c_int32),
                ("max_iters", C.c_int32), ("lo_iters", C.c_int32), ("p_miss", C.c_double),
                ("final_iters", C.c_int32), ("p3p_fp64_polish", C.c_int32), ("cauchy_scale", C.c_double),
                ("seed", C.c_uint64), ("query_id", C.c_uint32), ("enumerate_all", C.c_int32),
                ("lo_fp64_accumulate", C.c_int32), ("lo_fp64_solve", C.c_int32), ("score_bf16", C.c_int32),
                ("reserved", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("R_best", C.c_double * 9), ("t_best", C.c_double * 3),
                ("score", C.c_double), ("num_inliers", C.c_int64), ("subset_inliers", C.c_int64),
                ("iterations", C.c_int64), ("rounds", C.c_int64), ("lo_count", C.c_int64), ("hypotheses", C.c_int64),
                ("best_hyp", C.c_int64), ("status", C.c_int32), ("passes", C.c_int32)]


RIG_MAX_CAMERAS = 8


class Rig(C.Structure):
    _fields_ = [("n_cams", C.c_int32), ("reserved", C.c_int32), ("cams", Camera * RIG_MAX_CAMERAS),
                ("cam_from_rig", Pose * RIG_MAX_CAMERAS)]


def rig(Ks, R_cam, t_cam) -> Rig:
    """Ks: per camera (fx, fy, cx, cy); R_cam, t_cam: cam_from_rig per camera."""
    r = Rig()
    r.n_cams = len(Ks)
    for k, K in enumerate(Ks):
        r.cams[k] = camera(K)
        r.cam_from_rig[k].R[:] = [float(a) for a in np.asarray(R_cam[k], dtype=np.float64).ravel()]
        r.cam_from_rig[k].t[:] = [float(a) for a in np.asarray(t_cam[k], dtype=np.float64).ravel()]
    return r


class ServeConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_queue", C.c_int32), ("device_budget_bytes", C.c_size_t),
                ("host_staging_bytes", C.c_size_t), ("rounds_per_step", C.c_int32), ("reserved", C.c_int32)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("rejected", C.c_int64), ("admitted", C.c_int64),
                ("completed", C.c_int64), ("steps", C.c_int64), ("pending", C.c_int64), ("resident", C.c_int64),
                ("device_bytes_in_use", C.c_size_t)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


class Debug(C.Structure):
    _fields_ = [("triples", C.c_void_p), ("poses", C.c_void_p), ("scores", C.c_void_p), ("counts", C.c_void_p),
                ("round_best", C.c_void_p), ("inject_poses", C.c_void_p), ("n_inject", C.c_int64),
                ("rescored_pairs", C.c_void_p)]


# every symbol declared in include/imloc.h and include/imloc_testing.h
EXPORTS = ["imloc_create", "imloc_destroy", "imloc_status_str", "imloc_last_cuda_error", "imloc_device_error",
           "imloc_lift_async", "imloc_lift_batch_async", "imloc_ransac_default_opts", "imloc_ransac_pnp",
           "imloc_ransac_pnp_batch_async", "imloc_testing_ransac", "imloc_profile_enable", "imloc_profile_read",
           "imloc_lift_noalloc_async", "imloc_serve_default_config", "imloc_serve_create", "imloc_serve_submit",
           "imloc_serve_poll", "imloc_serve_read_stats", "imloc_serve_destroy", "imloc_score_config",
           "imloc_set_scoring",
           "imloc_depth_encode_log8_async", "imloc_depth_decode_log8_async", "imloc_triangulate_default_opts",
           "imloc_triangulate_depth_async", "imloc_retrieve_topk_async", "imloc_ransac_rig_batch",
           "imloc_testing_rig", "imloc_testing_lift_stalled", "imloc_serve_submit_device",
           "imloc_depth_tile4_async", "imloc_depth_halo_async"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libimloc.so and declare the signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    L = C.CDLL(path)
    P, V = C.POINTER, C.c_void_p
    L.imloc_create.argtypes = [P(V), C.c_int, C.c_size_t]
    L.imloc_destroy.argtypes = [V]
    L.imloc_destroy.restype = None
    L.imloc_status_str.argtypes = [C.c_int]
    L.imloc_status_str.restype = C.c_char_p
    L.imloc_last_cuda_error.argtypes = []
    L.imloc_last_cuda_error.restype = C.c_char_p
    L.imloc_device_error.argtypes = [V]
    L.imloc_lift_async.argtypes = [V, P(View), C.c_int32, P(Matches), P(Corr), V]
    L.imloc_lift_batch_async.argtypes = [V, C.c_int32, P(C.c_int64), P(View), C.c_int32, P(Matches), P(Corr), V, V]
    L.imloc_ransac_default_opts.argtypes = [P(RansacOpts)]
    L.imloc_ransac_default_opts.restype = None
    L.imloc_ransac_pnp.argtypes = [V, P(Corr), P(Camera), P(RansacOpts), P(Result), V, V]
    L.imloc_ransac_pnp_batch_async.argtypes = [V, C.c_int32, P(Corr), V, P(Camera), P(RansacOpts), V, V, V]
    L.imloc_testing_ransac.argtypes = [V, P(Corr), P(Camera), P(RansacOpts), P(Debug), P(Result), V, V]
    L.imloc_lift_noalloc_async.argtypes = [P(View), C.c_int32, P(Matches), P(Corr), V]
    L.imloc_testing_lift_stalled.argtypes = [V, P(View), C.c_int32, P(Matches), P(Corr), C.c_int32, C.c_uint32, V]
    L.imloc_serve_default_config.argtypes = [P(ServeConfig)]
    L.imloc_serve_default_config.restype = None
    L.imloc_serve_create.argtypes = [V, P(ServeConfig), P(V)]
    L.imloc_serve_submit.argtypes = [V, P(View), C.c_int32, P(Matches), P(Camera), P(RansacOpts), P(C.c_uint64)]
    L.imloc_serve_submit_device.argtypes = [V, P(View), C.c_int32, P(Matches), P(Camera), P(RansacOpts),
                                            P(C.c_uint64)]
    L.imloc_serve_poll.argtypes = [V, C.c_uint64, P(Result), P(C.c_double)]
    L.imloc_serve_read_stats.argtypes = [V, P(ServeStats)]
    L.imloc_serve_destroy.argtypes = [V]
    L.imloc_profile_enable.argtypes = [V, C.c_int]
    L.imloc_profile_read.argtypes = [V, P(KernelStat), C.c_int32, P(C.c_int32), C.c_int]
    L.imloc_score_config.argtypes = [V, P(C.c_int32), P(C.c_int32), P(C.c_int32)]
    L.imloc_set_scoring.argtypes = [V, C.c_int32, C.c_int32]
    L.imloc_retrieve_topk_async.argtypes = [V, V, C.c_int32, V, C.c_int64, C.c_int32, C.c_int32, V, V, V]
    L.imloc_triangulate_default_opts.argtypes = [P(TriangulateOpts)]
    L.imloc_triangulate_default_opts.restype = None
    L.imloc_triangulate_depth_async.argtypes = [P(Camera), P(Pose), C.c_int32, C.c_int32, P(Camera), P(Pose),
                                                C.c_int32, V, V, V, C.c_int64, P(TriangulateOpts), V, V, V]
    L.imloc_ransac_rig_batch.argtypes = [V, C.c_int32, P(Corr), V, V, P(Rig), P(RansacOpts), V, V, V]
    L.imloc_testing_rig.argtypes = [V, P(Corr), V, P(Rig), P(RansacOpts), P(Debug), P(Result), V, V]
    L.imloc_depth_encode_log8_async.argtypes = [V, C.c_int32, C.c_int32, C.c_int64, V, C.c_int64, V]
    L.imloc_depth_decode_log8_async.argtypes = [V, C.c_int32, C.c_int32, C.c_int64, V, C.c_int64, V]
    L.imloc_depth_tile4_async.argtypes = [V, C.c_int32, C.c_int32, C.c_int64, V, C.c_int64, V]
    L.imloc_depth_halo_async.argtypes = [V, C.c_int32, C.c_int32, C.c_int64, V, C.c_int64, V]
    _lib = L
    return L


class ImlocError(RuntimeError):
    pass


def _check(rc, what):
    if rc != IMLOC_OK:
        msg = load().imloc_status_str(rc).decode()
        if rc == -5:
            msg += ": " + load().imloc_last_cuda_error().decode()
        raise ImlocError(f"{what}: {msg} ({rc})")


def _torch():
    import torch

    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def default_opts(**kw) -> RansacOpts:
    o = RansacOpts()
    load().imloc_ransac_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def camera(K, width=0, height=0) -> Camera:
    fx, fy, cx, cy = [float(a) for a in K]
    return Camera(fx, fy, cx, cy, int(width), int(height))


def result_dict(r: Result) -> dict:
    return dict(R=np.array(r.R).reshape(3, 3), t=np.array(r.t), R_best=np.array(r.R_best).reshape(3, 3),
                t_best=np.array(r.t_best), score=r.score, num_inliers=r.num_inliers,
                subset_inliers=r.subset_inliers, iterations=r.iterations, rounds=r.rounds, lo_count=r.lo_count,
                hypotheses=r.hypotheses, best_hyp=r.best_hyp, status=r.status, passes=r.passes)


def alloc_corr(capacity: int, device="cuda"):
    """Device buffers of a correspondence set (structure of arrays)."""
    torch = _torch()
    cap = max(int(capacity), 1)
    out = {k: torch.empty(cap, dtype=torch.float32, device=device) for k in ("x", "y", "X", "Y", "Z", "w")}
    out["src"] = torch.empty(cap, dtype=torch.int32, device=device)
    out["count"] = torch.zeros(1, dtype=torch.int32, device=device)
    out["capacity"] = int(capacity)
    return out


def corr_from_arrays(x, y, X, w, device="cuda"):
    """Upload a host correspondence set (float32) into device buffers."""
    torch = _torch()
    X = np.asarray(X, dtype=np.float32).reshape(-1, 3)
    n = len(X)
    c = alloc_corr(n, device)
    for k, a in (("x", x), ("y", y), ("X", X[:, 0]), ("Y", X[:, 1]), ("Z", X[:, 2]), ("w", w)):
        if n:
            c[k][:n].copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    c["count"].fill_(n)
    return c


def _corr_struct(c, capacity=None) -> Corr:
    return Corr(*[_ptr(c[k]) for k in ("x", "y", "X", "Y", "Z", "w", "src")], _ptr(c.get("count")),
                int(c["capacity"] if capacity is None else capacity))


def _views_struct(views):
    arr = (View * len(views))()
    for i, v in enumerate(views):
        d = v["depth"]
        arr[i].depth = d.data_ptr()
        arr[i].pitch = int(d.stride(0))
        if v.get("layout") in ("tile4", "halo"):
            # blocked float32 map (depth_tile4 / depth_halo): rows of blocks, the image size given with the view
            H, W = int(v["height"]), int(v["width"])
            arr[i].depth_format = DEPTH_F32_TILE4 if v["layout"] == "tile4" else DEPTH_F32_HALO
        else:
            H, W = int(d.shape[0]), int(d.shape[1])
            # uint8 maps hold 8-bit log codes (depth_encode_log8), float32 maps metres
            arr[i].depth_format = DEPTH_LOG8 if d.element_size() == 1 else DEPTH_F32
        arr[i].height, arr[i].width = H, W
        arr[i].cam = Camera(float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"]), W, H)
        arr[i].pose.R[:] = [float(a) for a in np.asarray(v["R"], dtype=np.float64).ravel()]
        arr[i].pose.t[:] = [float(a) for a in np.asarray(v["t"], dtype=np.float64).ravel()]
    return arr


def _matches_struct(m):
    seg_off = np.asarray(m["seg_off"], dtype=np.int64)
    n_seg = len(seg_off) - 1
    segs = (Segment * max(n_seg, 1))()
    for s in range(n_seg):
        segs[s].begin = int(seg_off[s])
        segs[s].view = int(m["seg_view"][s])
        segs[s].direction = int(m["seg_dir"][s])
    n = int(seg_off[-1]) if n_seg > 0 else 0
    st = Matches(*[_ptr(m[k]) for k in ("q_u", "q_v", "db_u", "db_v", "conf")], n, segs, n_seg)
    return st, segs


class Prepared:
    """Marshalled arguments kept alive for repeated calls (no per-call Python work)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def prepare_lift_batch(query_begin, views, matches):
    vs = _views_struct(views)
    ms, keep = _matches_struct(matches)
    qb = np.ascontiguousarray(query_begin, dtype=np.int64)
    return Prepared(vs=vs, n_views=len(views), ms=ms, keep=keep, qb=qb, nq=len(qb) - 1,
                    qb_ptr=qb.ctypes.data_as(C.POINTER(C.c_int64)), tensors=(views, matches))


def prepare_ransac_batch(Ks, opts):
    nq = len(Ks)
    return Prepared(nq=nq, cams=(Camera * nq)(*[camera(K) for K in Ks]), opts=(RansacOpts * nq)(*opts))


class Context:
    """One libimloc context (device workspace) bound to a CUDA device."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        self.lib = load()
        h = C.c_void_p()
        _check(self.lib.imloc_create(C.byref(h), int(device), int(workspace_bytes)), "imloc_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.imloc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_error(self):
        return self.lib.imloc_device_error(self.h)

    def profile(self, on: bool):
        _check(self.lib.imloc_profile_enable(self.h, 1 if on else 0), "imloc_profile_enable")

    def set_scoring(self, kernel: int = -1, tc_variant: int = -1):
        """Scoring kernel of later RANSAC calls: -1 by call size, 0 the FP32
        kernel, 1 the tensor-core kernel; tc_variant -1 default, else 0-4."""
        _check(self.lib.imloc_set_scoring(self.h, int(kernel), int(tc_variant)), "imloc_set_scoring")

    def score_config(self):
        """(threads, poses per thread, poses per tile) of the scoring variant the
        autotuner chose, or None before the first tuning."""
        t, h, tile = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        rc = self.lib.imloc_score_config(self.h, C.byref(t), C.byref(h), C.byref(tile))
        if rc == -6:
            return None
        _check(rc, "imloc_score_config")
        return (t.value, h.value, tile.value)

    # ---- retrieval nearest-neighbour search ----
    def retrieve_topk(self, queries, db, k, out_score=None, out_index=None, stream=None):
        """queries (Q, D), db (N, D): CUDA tensors of bfloat16 values or their
        16-bit patterns (int16 / uint16), row-major.  Returns (scores float32
        (Q, k), database indices int32 (Q, k)), best first."""
        import torch

        assert queries.is_cuda and db.is_cuda and queries.is_contiguous() and db.is_contiguous()
        assert queries.element_size() == 2 and db.element_size() == 2 and queries.shape[1] == db.shape[1]
        Q, D = queries.shape
        N = db.shape[0]
        if out_score is None:
            out_score = torch.empty((Q, k), dtype=torch.float32, device=queries.device)
        if out_index is None:
            out_index = torch.empty((Q, k), dtype=torch.int32, device=queries.device)
        _check(self.lib.imloc_retrieve_topk_async(self.h, C.c_void_p(queries.data_ptr()), Q, C.c_void_p(db.data_ptr()),
                                                  N, D, k, C.c_void_p(out_score.data_ptr()),
                                                  C.c_void_p(out_index.data_ptr()), _stream_handle(stream)),
               "imloc_retrieve_topk_async")
        return out_score, out_index

    def profile_read(self, reset=True):
        """{kernel name: (launches, total device ms)} of the traced launches."""
        arr = (KernelStat * 64)()
        n = C.c_int32(0)
        _check(self.lib.imloc_profile_read(self.h, arr, 64, C.byref(n), 1 if reset else 0), "imloc_profile_read")
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(n.value, 64))}

    # ---- lifting ----
    def lift(self, views, matches, out=None, stream=None):
        """views: list of dicts (depth: cuda float32 HxW tensor, fx, fy, cx, cy, R, t);
        matches: dict of cuda float32 tensors q_u, q_v, db_u, db_v, conf plus host seg_off, seg_view, seg_dir."""
        vs = _views_struct(views)
        ms, keep = _matches_struct(matches)
        if out is None:
            out = alloc_corr(ms.n, matches["q_u"].device)
        cs = _corr_struct(out)
        _check(self.lib.imloc_lift_async(self.h, vs, len(views), C.byref(ms), C.byref(cs), _stream(stream)),
               "imloc_lift_async")
        return out

    def testing_lift_stalled(self, views, matches, out, skip_tiles=1, spin_limit=64, stream=None):
        """Test hook: the lift with its first tiles never taken, so that the look-back waits end by their
        iteration limit (imloc_testing_lift_stalled); returns the call's status."""
        vs = _views_struct(views)
        ms, keep = _matches_struct(matches)
        cs = _corr_struct(out)
        return self.lib.imloc_testing_lift_stalled(self.h, vs, len(views), C.byref(ms), C.byref(cs), int(skip_tiles),
                                                   int(spin_limit), _stream(stream))

    def lift_batch(self, query_begin, views, matches, out=None, offsets=None, stream=None, prepared=None):
        torch = _torch()
        p = prepared if prepared is not None else prepare_lift_batch(query_begin, views, matches)
        dev = matches["q_u"].device
        if out is None:
            out = alloc_corr(p.ms.n, dev)
        if offsets is None:
            offsets = torch.zeros(p.nq + 1, dtype=torch.int64, device=dev)
        cs = _corr_struct(out)
        _check(self.lib.imloc_lift_batch_async(self.h, p.nq, p.qb_ptr, p.vs, p.n_views, C.byref(p.ms), C.byref(cs),
                                               _ptr(offsets), _stream(stream)), "imloc_lift_batch_async")
        return out, offsets

    # ---- RANSAC ----
    def ransac_pnp(self, corr, K, opts=None, n=None, mask=None, stream=None):
        """corr: device buffers (alloc_corr / corr_from_arrays / lift output); N from corr['count']
        unless `n` is given.  Returns a result dict (host)."""
        o = opts if opts is not None else default_opts()
        cs = _corr_struct(corr)
        if n is not None:
            cs.count = None
            cs.capacity = int(n)
        res = Result()
        rc = self.lib.imloc_ransac_pnp(self.h, C.byref(cs), C.byref(camera(K)), C.byref(o), C.byref(res),
                                       _ptr(mask), _stream(stream))
        if rc not in (IMLOC_OK, -7):
            _check(rc, "imloc_ransac_pnp")
        return result_dict(res)

    def ransac_pnp_batch_async(self, corr, offsets, Ks, opts, results, masks=None, stream=None, prepared=None):
        """results: cuda uint8 tensor of n_queries * sizeof(Result) bytes (see RESULT_BYTES)."""
        p = prepared if prepared is not None else prepare_ransac_batch(Ks, opts)
        cs = _corr_struct(corr)
        _check(self.lib.imloc_ransac_pnp_batch_async(self.h, p.nq, C.byref(cs), _ptr(offsets), p.cams, p.opts,
                                                     _ptr(results), _ptr(masks), _stream(stream)),
               "imloc_ransac_pnp_batch_async")

    def ransac_rig_batch(self, corr, cam, offsets, rigs, opts, results, masks=None, stream=None):
        """Rig queries (generalized absolute pose).  cam: device int32 camera index per correspondence;
        offsets: device int64 (n_queries + 1); rigs: list of Rig; opts: list of RansacOpts;
        results: cuda uint8 tensor of n_queries * RESULT_BYTES.  Returns when the results are written."""
        nq = len(rigs)
        cs = _corr_struct(corr)
        _check(self.lib.imloc_ransac_rig_batch(self.h, nq, C.byref(cs), _ptr(cam), _ptr(offsets),
                                               (Rig * nq)(*rigs), (RansacOpts * nq)(*opts), _ptr(results),
                                               _ptr(masks), _stream(stream)), "imloc_ransac_rig_batch")

    def testing_rig(self, corr, cam, rg, opts, n, debug: dict, mask=None, stream=None):
        cs = _corr_struct(corr, capacity=n)
        cs.count = None
        dbg = Debug(_ptr(debug.get("triples")), _ptr(debug.get("poses")), _ptr(debug.get("scores")),
                    _ptr(debug.get("counts")), _ptr(debug.get("round_best")), _ptr(debug.get("inject_poses")),
                    int(debug["inject_poses"].shape[0]) if debug.get("inject_poses") is not None else 0,
                    _ptr(debug.get("rescored_pairs")))
        res = Result()
        _check(self.lib.imloc_testing_rig(self.h, C.byref(cs), _ptr(cam), C.byref(rg), C.byref(opts), C.byref(dbg),
                                          C.byref(res), _ptr(mask), _stream(stream)), "imloc_testing_rig")
        return result_dict(res)

    def testing_ransac(self, corr, K, opts, n, debug: dict, mask=None, stream=None):
        cs = _corr_struct(corr, capacity=n)
        cs.count = None
        dbg = Debug(_ptr(debug.get("triples")), _ptr(debug.get("poses")), _ptr(debug.get("scores")),
                    _ptr(debug.get("counts")), _ptr(debug.get("round_best")), _ptr(debug.get("inject_poses")),
                    int(debug["inject_poses"].shape[0]) if debug.get("inject_poses") is not None else 0,
                    _ptr(debug.get("rescored_pairs")))
        res = Result()
        _check(self.lib.imloc_testing_ransac(self.h, C.byref(cs), C.byref(camera(K)), C.byref(opts), C.byref(dbg),
                                             C.byref(res), _ptr(mask), _stream(stream)), "imloc_testing_ransac")
        return result_dict(res)


class Server:
    """Continuous-batching server (imloc_serve_*): submit host matches, poll results."""

    def __init__(self, ctx: Context, **cfg):
        self.lib = load()
        c = ServeConfig()
        self.lib.imloc_serve_default_config(C.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        h = C.c_void_p()
        _check(self.lib.imloc_serve_create(ctx.h, C.byref(c), C.byref(h)), "imloc_serve_create")
        self.h = h
        self.cfg = c

    @staticmethod
    def prepare(views, matches, K, opts):
        """Marshal one query: views with device depth maps, matches as host float32 arrays."""
        vs = _views_struct(views)
        arrs = [np.ascontiguousarray(matches[k], dtype=np.float32) for k in ("q_u", "q_v", "db_u", "db_v", "conf")]
        seg_off = np.asarray(matches["seg_off"], dtype=np.int64)
        n_seg = len(seg_off) - 1
        segs = (Segment * max(n_seg, 1))()
        for s_ in range(n_seg):
            segs[s_].begin = int(seg_off[s_])
            segs[s_].view = int(matches["seg_view"][s_])
            segs[s_].direction = int(matches["seg_dir"][s_])
        n = int(seg_off[-1]) if n_seg > 0 else 0
        ms = Matches(*[a.ctypes.data for a in arrs], n, segs, n_seg)
        return Prepared(vs=vs, n_views=len(views), ms=ms, keep=(arrs, segs, views), cam=camera(K), opts=opts)

    def submit(self, views, matches, K, opts):
        return self.submit_prepared(self.prepare(views, matches, K, opts))

    @staticmethod
    def prepare_device(views, matches, K, opts):
        """Marshal one query whose matches are cuda float32 tensors (kept alive by the returned object,
        which must outlive the query's result)."""
        vs = _views_struct(views)
        ms, segs = _matches_struct(matches)
        return Prepared(vs=vs, n_views=len(views), ms=ms, keep=(matches, segs, views), cam=camera(K), opts=opts,
                        device=True)

    def submit_prepared(self, p):
        """Returns the ticket, or None when the server refuses the query."""
        t = C.c_uint64(0)
        fn = self.lib.imloc_serve_submit_device if getattr(p, "device", False) else self.lib.imloc_serve_submit
        rc = fn(self.h, p.vs, p.n_views, C.byref(p.ms), C.byref(p.cam), C.byref(p.opts), C.byref(t))
        if rc == -3:
            return None
        _check(rc, "imloc_serve_submit")
        return t.value

    def poll(self, ticket):
        """(status, result dict or None, latency ms or None); status 1 = pending, -6 = unknown ticket."""
        r = Result()
        lat = C.c_double(0.0)
        rc = self.lib.imloc_serve_poll(self.h, C.c_uint64(ticket), C.byref(r), C.byref(lat))
        if rc == 0:
            return 0, result_dict(r), lat.value
        return rc, None, None

    def stats(self):
        st = ServeStats()
        rc = self.lib.imloc_serve_read_stats(self.h, C.byref(st))
        d = {k: getattr(st, k) for k, _ in ServeStats._fields_}
        d["worker_status"] = rc
        return d

    def close(self):
        if getattr(self, "h", None):
            self.lib.imloc_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


RESULT_BYTES = C.sizeof(Result)


def results_from_bytes(buf: np.ndarray, nq: int):
    """Decode `nq` device results copied to host as bytes."""
    arr = (Result * nq).from_buffer_copy(np.ascontiguousarray(buf).tobytes())
    return [result_dict(arr[i]) for i in range(nq)]


# ---- depth codec (8-bit log codes; no context needed) ----
def _stream_handle(stream):
    import torch

    st = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(st.cuda_stream)


def depth_encode_log8(depth, out=None, stream=None):
    """float32 CUDA tensor HxW (metres) -> uint8 CUDA tensor HxW of codes
    (0 = no depth, 1..255 log levels over [0.25, 128] m), asynchronous."""
    import torch

    assert depth.dtype == torch.float32 and depth.dim() == 2 and depth.is_cuda and depth.stride(1) == 1
    H, W = depth.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.uint8, device=depth.device)
    _check(load().imloc_depth_encode_log8_async(C.c_void_p(depth.data_ptr()), W, H, depth.stride(0),
                                                C.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)),
           "imloc_depth_encode_log8_async")
    return out


def depth_tile4(depth, stream=None):
    """float32 CUDA tensor HxW -> the 4x4-blocked layout (imloc_depth_tile4_async): a float32 CUDA tensor of
    ceil(H/4) block rows x 16 ceil(W/4) elements.  Use it as a view's depth with layout="tile4" and the
    view's width and height."""
    import torch

    assert depth.dtype == torch.float32 and depth.dim() == 2 and depth.is_cuda and depth.stride(1) == 1
    H, W = depth.shape
    out = torch.empty(((H + 3) // 4, 16 * ((W + 3) // 4)), dtype=torch.float32, device=depth.device)
    _check(load().imloc_depth_tile4_async(C.c_void_p(depth.data_ptr()), W, H, depth.stride(0),
                                          C.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)),
           "imloc_depth_tile4_async")
    return out


def tile4_view(v):
    """A view dict with its float32 depth map re-laid out in 4x4 blocks."""
    d = dict(v)
    H, W = v["depth"].shape
    d.update(depth=depth_tile4(v["depth"]), layout="tile4", width=W, height=H)
    return d


def depth_halo(depth, stream=None):
    """float32 CUDA tensor HxW -> the overlapping-block layout (imloc_depth_halo_async): a float32 CUDA tensor
    of (H-1)//3+1 block rows x 32 ((W-1)//7+1) elements.  Use it as a view's depth with layout="halo" and the
    view's width and height."""
    import torch

    assert depth.dtype == torch.float32 and depth.dim() == 2 and depth.is_cuda and depth.stride(1) == 1
    H, W = depth.shape
    out = torch.empty(((H - 1) // 3 + 1, 32 * ((W - 1) // 7 + 1)), dtype=torch.float32, device=depth.device)
    _check(load().imloc_depth_halo_async(C.c_void_p(depth.data_ptr()), W, H, depth.stride(0),
                                         C.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)),
           "imloc_depth_halo_async")
    return out


def halo_view(v):
    """A view dict with its float32 depth map re-laid out in overlapping 8x4 blocks."""
    d = dict(v)
    H, W = v["depth"].shape
    d.update(depth=depth_halo(v["depth"]), layout="halo", width=W, height=H)
    return d


def depth_decode_log8(codes, out=None, stream=None):
    """uint8 CUDA tensor of codes -> float32 CUDA tensor (metres, 0 for code 0)."""
    import torch

    assert codes.dtype == torch.uint8 and codes.dim() == 2 and codes.is_cuda and codes.stride(1) == 1
    H, W = codes.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=codes.device)
    _check(load().imloc_depth_decode_log8_async(C.c_void_p(codes.data_ptr()), W, H, codes.stride(0),
                                                C.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)),
           "imloc_depth_decode_log8_async")
    return out


# ---- dense triangulation of a mapping depth map ----
def triangulate_opts(**kw):
    o = TriangulateOpts()
    load().imloc_triangulate_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _cam_pose(c, width=0, height=0):
    cam = Camera(float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"]), int(width), int(height))
    pose = Pose()
    pose.R[:] = [float(a) for a in np.asarray(c["R"], dtype=np.float64).ravel()]
    pose.t[:] = [float(a) for a in np.asarray(c["t"], dtype=np.float64).ravel()]
    return cam, pose


def triangulate_depth(ref, srcs, u, v, conf, opts=None, depth=None, inliers=None, stream=None):
    """ref, srcs: camera dicts (fx, fy, cx, cy, R, t); u, v, conf: float32 CUDA
    tensors (n_src, H, W).  Returns (depth float32 HxW, inliers uint8 HxW)."""
    import torch

    S, H, W = u.shape
    for t in (u, v, conf):
        assert t.dtype == torch.float32 and t.is_cuda and t.is_contiguous() and tuple(t.shape) == (S, H, W)
    if depth is None:
        depth = torch.empty((H, W), dtype=torch.float32, device=u.device)
    if inliers is None:
        inliers = torch.empty((H, W), dtype=torch.uint8, device=u.device)
    rc, rp = _cam_pose(ref, W, H)
    cams = (Camera * S)()
    poses = (Pose * S)()
    for i, c in enumerate(srcs):
        cams[i], poses[i] = _cam_pose(c)
    o = opts if opts is not None else triangulate_opts()
    _check(load().imloc_triangulate_depth_async(C.byref(rc), C.byref(rp), W, H, cams, poses, S,
                                                C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()),
                                                C.c_void_p(conf.data_ptr()), H * W, C.byref(o),
                                                C.c_void_p(depth.data_ptr()), C.c_void_p(inliers.data_ptr()),
                                                _stream_handle(stream)),
           "imloc_triangulate_depth_async")
    return depth, inliers
