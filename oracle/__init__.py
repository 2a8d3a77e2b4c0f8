"""ctypes front end of the FP64 CPU oracle (``oracle/imloc_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It does not import
the CUDA library and the CUDA library does not import it; both consume the
same seeded inputs from ``paper_2601_04185_gb300.synth``.

Every function converts numpy arrays to the plain C layout of the oracle and
back; no arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None


class OrcView(C.Structure):
    _fields_ = [("depth", C.POINTER(C.c_float)), ("width", C.c_int64), ("height", C.c_int64),
                ("pitch", C.c_int64), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("R", C.c_double * 9), ("t", C.c_double * 3)]


class OrcCorr(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("X", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double))]


class OrcCam(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double)]


class OrcOpts(C.Structure):
    _fields_ = [("tau", C.c_double), ("max_score_corr", C.c_int64), ("batch", C.c_int64),
                ("max_iters", C.c_int64), ("p_miss", C.c_double), ("lo_iters", C.c_int64),
                ("final_iters", C.c_int64), ("cauchy_scale", C.c_double), ("seed", C.c_uint64),
                ("query_id", C.c_uint32), ("enumerate_all", C.c_int32), ("lo_enabled", C.c_int32),
                ("final_enabled", C.c_int32)]


class OrcResult(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("R_best", C.c_double * 9),
                ("t_best", C.c_double * 3), ("score", C.c_double), ("num_inliers", C.c_int64),
                ("subset_inliers", C.c_int64), ("iterations", C.c_int64), ("rounds", C.c_int64),
                ("lo_count", C.c_int64), ("hypotheses", C.c_int64), ("best_hyp", C.c_int64),
                ("status", C.c_int32)]


class OrcRig(C.Structure):
    _fields_ = [("n_cams", C.c_int64), ("cam", OrcCam * 8), ("R", (C.c_double * 9) * 8), ("t", (C.c_double * 3) * 8)]


class OrcTriCam(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("R", C.c_double * 9), ("t", C.c_double * 3)]


class OrcTriOpts(C.Structure):
    _fields_ = [("angle_deg", C.c_double), ("conf_min", C.c_double), ("keep_more_than", C.c_int64),
                ("refine_iters", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        # a test may point at another build of the same source (mutation checks)
        path = os.environ.get("IMLOC_ORACLE_LIB") or _build()
        L = C.CDLL(path)
        P = C.POINTER
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_lift.restype = C.c_int64
        L.orc_lift.argtypes = [P(OrcView), C.c_int64] + [P(C.c_float)] * 5 + [
            P(C.c_int64), P(C.c_int32), P(C.c_int32), C.c_int64, C.c_float] + [P(C.c_double)] * 4 + [P(C.c_int64)]
        L.orc_subsample.argtypes = [C.c_int64, C.c_int64, P(C.c_int64)]
        L.orc_sample.restype = C.c_int
        L.orc_sample.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, P(C.c_int64)]
        L.orc_p3p.restype = C.c_int
        L.orc_p3p.argtypes = [P(C.c_double)] * 5
        L.orc_score.restype = C.c_double
        L.orc_score.argtypes = [P(OrcCorr), P(C.c_int64), C.c_int64, P(OrcCam), P(C.c_double),
                                P(C.c_double), C.c_double, P(C.c_int64)]
        L.orc_lo.restype = C.c_double
        L.orc_lo.argtypes = [P(OrcCorr), P(C.c_int64), C.c_int64, P(OrcCam), C.c_double, C.c_int64,
                             P(C.c_double), P(C.c_double)]
        L.orc_refine.restype = C.c_int
        L.orc_refine.argtypes = [P(OrcCorr), P(C.c_int64), C.c_int64, P(OrcCam), C.c_double, C.c_double,
                                 C.c_int64, P(C.c_double), P(C.c_double)]
        L.orc_needed_iters.restype = C.c_double
        L.orc_needed_iters.argtypes = [C.c_double, C.c_double]
        L.orc_depth_decode_log8.restype = C.c_double
        L.orc_depth_decode_log8.argtypes = [C.c_uint8]
        L.orc_depth_encode_log8.restype = C.c_uint8
        L.orc_depth_encode_log8.argtypes = [C.c_float]
        L.orc_depth_encode_log8_n.argtypes = [P(C.c_float), C.c_int64, P(C.c_uint8)]
        L.orc_depth_decode_log8_n.argtypes = [P(C.c_uint8), C.c_int64, P(C.c_double)]
        L.orc_angle.restype = C.c_double
        L.orc_angle.argtypes = [P(C.c_double), P(C.c_double)]
        L.orc_closest_depth.restype = C.c_double
        L.orc_closest_depth.argtypes = [P(C.c_double)] * 4
        L.orc_triangulate_pixel.restype = C.c_int64
        L.orc_triangulate_pixel.argtypes = [P(OrcTriCam), C.c_int64, C.c_int64, C.c_int64, P(OrcTriCam), C.c_int64,
                                            P(C.c_double), P(C.c_double), P(C.c_double), P(OrcTriOpts),
                                            P(C.c_double)]
        L.orc_triangulate_depth.argtypes = [P(OrcTriCam), C.c_int64, C.c_int64, P(OrcTriCam), C.c_int64,
                                            P(C.c_float), P(C.c_float), P(C.c_float), C.c_int64, P(OrcTriOpts),
                                            P(C.c_double), P(C.c_int64)]
        L.orc_bf16_to_double.restype = C.c_double
        L.orc_bf16_to_double.argtypes = [C.c_uint16]
        L.orc_retrieve_topk.argtypes = [P(C.c_uint16), C.c_int64, P(C.c_uint16), C.c_int64, C.c_int64, C.c_int64,
                                        P(C.c_double), P(C.c_int64)]
        L.orc_gp3p.restype = C.c_int
        L.orc_gp3p.argtypes = [P(C.c_double)] * 6
        L.orc_rig_score.restype = C.c_double
        L.orc_rig_score.argtypes = [P(OrcCorr), P(C.c_int32), P(C.c_int64), C.c_int64, P(OrcRig), P(C.c_double),
                                    P(C.c_double), C.c_double, P(C.c_int64)]
        L.orc_rig_lo.restype = C.c_double
        L.orc_rig_lo.argtypes = [P(OrcCorr), P(C.c_int32), P(C.c_int64), C.c_int64, P(OrcRig), C.c_double,
                                 C.c_int64, P(C.c_double), P(C.c_double)]
        L.orc_rig_refine.restype = C.c_int
        L.orc_rig_refine.argtypes = [P(OrcCorr), P(C.c_int32), P(C.c_int64), C.c_int64, P(OrcRig), C.c_double,
                                     C.c_double, C.c_int64, P(C.c_double), P(C.c_double)]
        L.orc_rig_ransac.restype = C.c_int
        L.orc_rig_ransac.argtypes = [P(OrcCorr), P(C.c_int32), P(OrcRig), P(OrcOpts), P(OrcResult), P(C.c_uint8),
                                     P(C.c_int64), P(C.c_double), C.c_int64]
        L.orc_ransac_pnp.restype = C.c_int
        L.orc_ransac_pnp.argtypes = [P(OrcCorr), P(OrcCam), P(OrcOpts), P(OrcResult), P(C.c_uint8),
                                     P(C.c_int64), P(C.c_double), C.c_int64]
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def lift(views, matches, conf_min=np.float32(0.05)):
    """views: list of dicts (depth f32 HxW, fx, fy, cx, cy, R 3x3, t 3);
    matches: dict q_u, q_v, db_u, db_v, conf (f32), seg_off (n_seg+1), seg_view, seg_dir.
    Returns dict x, y, X (n,3), w, src (float64 / int64)."""
    keep = []
    arr = (OrcView * len(views))()
    for i, v in enumerate(views):
        d = np.ascontiguousarray(v["depth"], dtype=np.float32)
        keep.append(d)
        arr[i].depth = _ptr(d, C.c_float)
        arr[i].height, arr[i].width = d.shape
        arr[i].pitch = d.shape[1]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"]))
        arr[i].R[:] = [float(a) for a in np.asarray(v["R"], dtype=np.float64).ravel()]
        arr[i].t[:] = [float(a) for a in np.asarray(v["t"], dtype=np.float64).ravel()]
    f = {k: np.ascontiguousarray(matches[k], dtype=np.float32) for k in ("q_u", "q_v", "db_u", "db_v", "conf")}
    seg_off = np.ascontiguousarray(matches["seg_off"], dtype=np.int64)
    seg_view = np.ascontiguousarray(matches["seg_view"], dtype=np.int32)
    seg_dir = np.ascontiguousarray(matches["seg_dir"], dtype=np.int32)
    n = len(f["q_u"])
    x = np.zeros(n); y = np.zeros(n); X = np.zeros((n, 3)); w = np.zeros(n); src = np.zeros(n, dtype=np.int64)
    nv = lib().orc_lift(arr, len(views), *[_ptr(f[k], C.c_float) for k in ("q_u", "q_v", "db_u", "db_v", "conf")],
                        _ptr(seg_off, C.c_int64), _ptr(seg_view, C.c_int32), _ptr(seg_dir, C.c_int32),
                        len(seg_view), C.c_float(float(conf_min)), _ptr(x, C.c_double), _ptr(y, C.c_double),
                        _ptr(X, C.c_double), _ptr(w, C.c_double), _ptr(src, C.c_int64))
    return dict(x=x[:nv], y=y[:nv], X=X[:nv], w=w[:nv], src=src[:nv])


def subsample(n, m):
    idx = np.zeros(m, dtype=np.int64)
    lib().orc_subsample(n, m, _ptr(idx, C.c_int64))
    return idx


def sample(seed, query_id, sample_id, m):
    out = np.zeros(3, dtype=np.int64)
    att = lib().orc_sample(C.c_uint64(seed), C.c_uint32(query_id), C.c_uint32(sample_id), m, _ptr(out, C.c_int64))
    return (out if att >= 0 else None), att


def p3p(bearings, points):
    """bearings (3,3) unit rows, points (3,3) -> list of (R, t, lambdas)."""
    y = np.ascontiguousarray(bearings, dtype=np.float64).ravel().copy()
    X = np.ascontiguousarray(points, dtype=np.float64).ravel().copy()
    R = np.zeros(36); t = np.zeros(12); lam = np.zeros(12)
    ns = lib().orc_p3p(_ptr(y, C.c_double), _ptr(X, C.c_double), _ptr(R, C.c_double), _ptr(t, C.c_double),
                       _ptr(lam, C.c_double))
    return [(R[9 * k:9 * k + 9].reshape(3, 3).copy(), t[3 * k:3 * k + 3].copy(), lam[3 * k:3 * k + 3].copy())
            for k in range(ns)]


class Corr:
    """Holds float64 copies of a correspondence set and its C view."""

    def __init__(self, x, y, X, w):
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        self.X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 3))
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.c = OrcCorr(len(self.x), _ptr(self.x, C.c_double), _ptr(self.y, C.c_double),
                         _ptr(self.X, C.c_double), _ptr(self.w, C.c_double))

    @property
    def n(self):
        return len(self.x)


def _cam(K):
    fx, fy, cx, cy = [float(a) for a in K]
    return OrcCam(fx, fy, cx, cy)


def score(corr: Corr, K, R, t, tau, idx=None):
    cam = _cam(K)
    Rd = np.ascontiguousarray(R, dtype=np.float64).ravel().copy()
    td = np.ascontiguousarray(t, dtype=np.float64).ravel().copy()
    cnt = C.c_int64(0)
    if idx is None:
        s = lib().orc_score(C.byref(corr.c), None, corr.n, C.byref(cam), _ptr(Rd, C.c_double), _ptr(td, C.c_double),
                            tau, C.byref(cnt))
    else:
        ii = np.ascontiguousarray(idx, dtype=np.int64)
        s = lib().orc_score(C.byref(corr.c), _ptr(ii, C.c_int64), len(ii), C.byref(cam), _ptr(Rd, C.c_double),
                            _ptr(td, C.c_double), tau, C.byref(cnt))
    return s, cnt.value


def lo(corr: Corr, K, R, t, tau, iters=10, idx=None):
    cam = _cam(K)
    Rd = np.ascontiguousarray(R, dtype=np.float64).ravel().copy()
    td = np.ascontiguousarray(t, dtype=np.float64).ravel().copy()
    if idx is None:
        s = lib().orc_lo(C.byref(corr.c), None, corr.n, C.byref(cam), tau, iters, _ptr(Rd, C.c_double),
                         _ptr(td, C.c_double))
    else:
        ii = np.ascontiguousarray(idx, dtype=np.int64)
        s = lib().orc_lo(C.byref(corr.c), _ptr(ii, C.c_int64), len(ii), C.byref(cam), tau, iters,
                         _ptr(Rd, C.c_double), _ptr(td, C.c_double))
    return Rd.reshape(3, 3), td, s


def refine(corr: Corr, K, R, t, sel, cauchy_c, tau, iters=25):
    cam = _cam(K)
    Rd = np.ascontiguousarray(R, dtype=np.float64).ravel().copy()
    td = np.ascontiguousarray(t, dtype=np.float64).ravel().copy()
    ss = np.ascontiguousarray(sel, dtype=np.int64)
    steps = lib().orc_refine(C.byref(corr.c), _ptr(ss, C.c_int64), len(ss), C.byref(cam), cauchy_c, tau, iters,
                             _ptr(Rd, C.c_double), _ptr(td, C.c_double))
    return Rd.reshape(3, 3), td, steps


def needed_iters(eps, p_miss):
    return lib().orc_needed_iters(float(eps), float(p_miss))


def default_opts(**kw):
    o = dict(tau=4.0, max_score_corr=10000, batch=1024, max_iters=100000, p_miss=1e-4, lo_iters=10,
             final_iters=25, cauchy_scale=None, seed=0, query_id=0, enumerate_all=0, lo_enabled=1,
             final_enabled=1)
    o.update(kw)
    if o["cauchy_scale"] is None:
        o["cauchy_scale"] = o["tau"]
    return o


def ransac_pnp(corr: Corr, K, max_rounds=256, **kw):
    o = default_opts(**kw)
    opts = OrcOpts(**o)
    cam = _cam(K)
    res = OrcResult()
    mask = np.zeros(max(corr.n, 1), dtype=np.uint8)
    rb_id = np.full(max_rounds, -1, dtype=np.int64)
    rb_sc = np.full(max_rounds, np.inf)
    lib().orc_ransac_pnp(C.byref(corr.c), C.byref(cam), C.byref(opts), C.byref(res), _ptr(mask, C.c_uint8),
                         _ptr(rb_id, C.c_int64), _ptr(rb_sc, C.c_double), max_rounds)
    nr = min(res.rounds, max_rounds)
    return dict(status=res.status, R=np.array(res.R).reshape(3, 3), t=np.array(res.t),
                R_best=np.array(res.R_best).reshape(3, 3), t_best=np.array(res.t_best), score=res.score,
                num_inliers=res.num_inliers, subset_inliers=res.subset_inliers, iterations=res.iterations,
                rounds=res.rounds, lo_count=res.lo_count, hypotheses=res.hypotheses, best_hyp=res.best_hyp,
                inlier_mask=mask[:corr.n].astype(bool), round_best_id=rb_id[:nr], round_best_score=rb_sc[:nr])


# ---- depth codec (Sec. 3.3 "Data Compression", Sec. 4.3 "Depth Quantization") ----
def depth_encode_log8(depth):
    """float32 depth array -> uint8 codes (0 = no depth, 1..255 log levels over [0.25, 128] m)."""
    d = np.ascontiguousarray(depth, dtype=np.float32)
    out = np.zeros(d.shape, dtype=np.uint8)
    L = lib()
    L.orc_depth_encode_log8_n(_ptr(d, C.c_float), d.size, _ptr(out, C.c_uint8))
    return out


def depth_decode_log8(codes):
    """uint8 codes -> float64 depth (0 for code 0)."""
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.zeros(c.shape, dtype=np.float64)
    lib().orc_depth_decode_log8_n(_ptr(c, C.c_uint8), c.size, _ptr(out, C.c_double))
    return out


# ---- dense triangulation (Sec. 3.3 "Depth Estimation by Dense Matching") ----
def tri_cam(cam):
    """cam: dict fx, fy, cx, cy, R (3x3), t (3)"""
    c = OrcTriCam()
    c.fx, c.fy, c.cx, c.cy = (float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"]))
    c.R[:] = [float(a) for a in np.asarray(cam["R"], np.float64).ravel()]
    c.t[:] = [float(a) for a in np.asarray(cam["t"], np.float64).ravel()]
    return c


def tri_opts(angle_deg=2.0, conf_min=0.05, keep_more_than=3, refine_iters=500):
    return OrcTriOpts(float(angle_deg), float(conf_min), int(keep_more_than), int(refine_iters))


def angle(a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    return lib().orc_angle(_ptr(a, C.c_double), _ptr(b, C.c_double))


def closest_depth(C0, d0, C1, d1):
    arrs = [np.ascontiguousarray(x, np.float64) for x in (C0, d0, C1, d1)]
    return lib().orc_closest_depth(*[_ptr(a, C.c_double) for a in arrs])


def triangulate_pixel(ref, srcs, width, px, py, u, v, conf, **kw):
    """one pixel: (inliers, depth); u, v, conf: one value per source"""
    r = tri_cam(ref)
    arr = (OrcTriCam * len(srcs))(*[tri_cam(c) for c in srcs])
    uu, vv, cc = (np.ascontiguousarray(x, np.float64) for x in (u, v, conf))
    o = tri_opts(**kw)
    d = C.c_double(0.0)
    n = lib().orc_triangulate_pixel(C.byref(r), width, px, py, arr, len(srcs), _ptr(uu, C.c_double),
                                    _ptr(vv, C.c_double), _ptr(cc, C.c_double), C.byref(o), C.byref(d))
    return int(n), d.value


def triangulate_depth(ref, srcs, u, v, conf, **kw):
    """u, v, conf: float32 arrays (n_src, H, W). Returns depth (H, W) float64, inliers (H, W) int64."""
    u, v, conf = (np.ascontiguousarray(x, np.float32) for x in (u, v, conf))
    S, H, W = u.shape
    r = tri_cam(ref)
    arr = (OrcTriCam * S)(*[tri_cam(c) for c in srcs])
    o = tri_opts(**kw)
    depth = np.zeros((H, W), np.float64)
    inl = np.zeros((H, W), np.int64)
    lib().orc_triangulate_depth(C.byref(r), W, H, arr, S, _ptr(u, C.c_float), _ptr(v, C.c_float),
                                _ptr(conf, C.c_float), H * W, C.byref(o), _ptr(depth, C.c_double),
                                _ptr(inl, C.c_int64))
    return depth, inl


# ---- retrieval nearest-neighbour search (Sec. 3.1, Sec. 4.4 "Runtime") ----
def bf16_to_double(bits):
    return lib().orc_bf16_to_double(int(bits))


def retrieve_topk(queries_bf16, db_bf16, k):
    """queries_bf16: uint16 (Q, D), db_bf16: uint16 (N, D) bfloat16 bit patterns.
    Returns scores (Q, k) float64 and indices (Q, k) int64."""
    q = np.ascontiguousarray(queries_bf16, np.uint16)
    d = np.ascontiguousarray(db_bf16, np.uint16)
    Q, D = q.shape
    N = d.shape[0]
    sc = np.zeros((Q, k), np.float64)
    ix = np.zeros((Q, k), np.int64)
    lib().orc_retrieve_topk(_ptr(q, C.c_uint16), Q, _ptr(d, C.c_uint16), N, D, k, _ptr(sc, C.c_double),
                            _ptr(ix, C.c_int64))
    return sc, ix


# ---- generalized absolute pose of a camera rig (supplementary "LaMAR HoloLens Results") ----
def rig(cams, R_cam, t_cam):
    """cams: list of (fx, fy, cx, cy); R_cam, t_cam: cam_from_rig per camera."""
    r = OrcRig()
    r.n_cams = len(cams)
    for k, K in enumerate(cams):
        r.cam[k] = _cam(K)
        r.R[k][:] = [float(a) for a in np.asarray(R_cam[k], np.float64).ravel()]
        r.t[k][:] = [float(a) for a in np.asarray(t_cam[k], np.float64).ravel()]
    return r


def gp3p(origins, dirs, points):
    """origins, dirs (unit), points: (3, 3) -> list of (R, t, lambdas), ascending lambda_1."""
    o = np.ascontiguousarray(origins, np.float64).ravel().copy()
    d = np.ascontiguousarray(dirs, np.float64).ravel().copy()
    X = np.ascontiguousarray(points, np.float64).ravel().copy()
    R = np.zeros(72); t = np.zeros(24); lam = np.zeros(24)
    ns = lib().orc_gp3p(*[_ptr(a, C.c_double) for a in (o, d, X, R, t, lam)])
    return [(R[9 * k:9 * k + 9].reshape(3, 3).copy(), t[3 * k:3 * k + 3].copy(), lam[3 * k:3 * k + 3].copy())
            for k in range(ns)]


def _pose(R, t):
    return (np.ascontiguousarray(R, np.float64).ravel().copy(), np.ascontiguousarray(t, np.float64).ravel().copy())


def rig_score(corr: Corr, cam_of, rg, R, t, tau, idx=None):
    co = np.ascontiguousarray(cam_of, np.int32)
    Rd, td = _pose(R, t)
    cnt = C.c_int64(0)
    ii = None if idx is None else np.ascontiguousarray(idx, np.int64)
    s = lib().orc_rig_score(C.byref(corr.c), _ptr(co, C.c_int32), None if ii is None else _ptr(ii, C.c_int64),
                            corr.n if ii is None else len(ii), C.byref(rg), _ptr(Rd, C.c_double),
                            _ptr(td, C.c_double), tau, C.byref(cnt))
    return s, cnt.value


def rig_lo(corr: Corr, cam_of, rg, R, t, tau, iters=10, idx=None):
    co = np.ascontiguousarray(cam_of, np.int32)
    Rd, td = _pose(R, t)
    ii = None if idx is None else np.ascontiguousarray(idx, np.int64)
    s = lib().orc_rig_lo(C.byref(corr.c), _ptr(co, C.c_int32), None if ii is None else _ptr(ii, C.c_int64),
                         corr.n if ii is None else len(ii), C.byref(rg), tau, iters, _ptr(Rd, C.c_double),
                         _ptr(td, C.c_double))
    return Rd.reshape(3, 3), td, s


def rig_refine(corr: Corr, cam_of, rg, R, t, sel, cauchy_c, tau, iters=25):
    co = np.ascontiguousarray(cam_of, np.int32)
    Rd, td = _pose(R, t)
    ss = np.ascontiguousarray(sel, np.int64)
    steps = lib().orc_rig_refine(C.byref(corr.c), _ptr(co, C.c_int32), _ptr(ss, C.c_int64), len(ss), C.byref(rg),
                                 cauchy_c, tau, iters, _ptr(Rd, C.c_double), _ptr(td, C.c_double))
    return Rd.reshape(3, 3), td, steps


def rig_ransac(corr: Corr, cam_of, rg, max_rounds=256, **kw):
    o = default_opts(**kw)
    opts = OrcOpts(**o)
    co = np.ascontiguousarray(cam_of, np.int32)
    res = OrcResult()
    mask = np.zeros(max(corr.n, 1), dtype=np.uint8)
    rb_id = np.full(max_rounds, -1, dtype=np.int64)
    rb_sc = np.full(max_rounds, np.inf)
    lib().orc_rig_ransac(C.byref(corr.c), _ptr(co, C.c_int32), C.byref(rg), C.byref(opts), C.byref(res),
                         _ptr(mask, C.c_uint8), _ptr(rb_id, C.c_int64), _ptr(rb_sc, C.c_double), max_rounds)
    nr = min(res.rounds, max_rounds)
    return dict(status=res.status, R=np.array(res.R).reshape(3, 3), t=np.array(res.t),
                R_best=np.array(res.R_best).reshape(3, 3), t_best=np.array(res.t_best), score=res.score,
                num_inliers=res.num_inliers, subset_inliers=res.subset_inliers, iterations=res.iterations,
                rounds=res.rounds, lo_count=res.lo_count, hypotheses=res.hypotheses, best_hyp=res.best_hyp,
                inlier_mask=mask[:corr.n].astype(bool), round_best_id=rb_id[:nr], round_best_score=rb_sc[:nr])
