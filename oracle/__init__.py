"""ctypes wrapper of the CPU oracle (plain C, FP64 solver) of one Adaptive
Position-Based Fluids step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the benchmark's CPU-baseline / reference leg. The product path never
imports it.

Parity status of each function (what pins it) is listed in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import build as _build

ORC_LOD_FIXED = 0
ORC_LOD_DTC = 1
ORC_LOD_DTVS = 2
DEPTH_EMPTY_BITS = 0x7F7F7F7F
ORC_LAMBDA_STALE = 0
ORC_LAMBDA_ZERO = 1
ORC_LAMBDA_RECOMPUTE = 2


class OrcView(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32),
        ("tan_half_fov", C.c_float),
        ("dir", C.c_float * 3),
        ("up", C.c_float * 3),
        ("radius", C.c_float),
        ("brute_force", C.c_int32),
        ("outside_level", C.c_int32),
    ]


def make_view(width: int, height: int, tan_half_fov: float, direction, up=(0.0, 0.0, 1.0), radius: float = 0.025,
              brute_force: bool = False, outside_level: int = 0) -> OrcView:
    """The DTVS camera image; outside_level is N_i of a particle outside the
    view (0: n_min, reading 20)."""
    v = OrcView()
    v.width, v.height = int(width), int(height)
    v.tan_half_fov = float(tan_half_fov)
    v.dir[:] = [float(a) for a in direction]
    v.up[:] = [float(a) for a in up]
    v.radius = float(radius)
    v.brute_force = int(bool(brute_force))
    v.outside_level = int(outside_level)
    return v


ORC_MAX_OBSTACLES = 8
ORC_OBSTACLE_SPHERE, ORC_OBSTACLE_BOX, ORC_OBSTACLE_CONE = 1, 2, 3


class OrcObstacle(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_float * 3), ("b", C.c_float * 3)]


class OrcParams(C.Structure):
    _fields_ = [
        ("h", C.c_float), ("dt", C.c_float), ("mass", C.c_float), ("rho0", C.c_float),
        ("eps", C.c_float), ("scorr_k", C.c_float), ("scorr_dq", C.c_float), ("xsph_c", C.c_float),
        ("scorr_n", C.c_int32),
        ("gravity", C.c_float * 3),
        ("grid_lo", C.c_float * 3), ("grid_hi", C.c_float * 3),
        ("box_lo", C.c_float * 3), ("box_hi", C.c_float * 3),
        ("n_min", C.c_int32), ("n_max", C.c_int32), ("lod_mode", C.c_int32),
        ("eye", C.c_float * 3),
        ("d_near", C.c_float), ("d_far", C.c_float),
        ("lambda_mode", C.c_int32), ("lod_rounding", C.c_int32),
        ("view", OrcView),
        ("stabil_iters", C.c_int32), ("stabil_s", C.c_int32),
        ("n_obstacles", C.c_int32),
        ("obstacles", OrcObstacle * ORC_MAX_OBSTACLES),
    ]


class OrcRecord(C.Structure):
    _fields_ = [
        ("xpred", C.POINTER(C.c_float)),
        ("level_presort", C.POINTER(C.c_int32)),
        ("keys", C.POINTER(C.c_uint32)),
        ("order", C.POINTER(C.c_int32)),
        ("cell_start", C.POINTER(C.c_uint32)),
        ("cell_cap", C.c_int64),
        ("nbr_off", C.POINTER(C.c_int32)),
        ("nbr_idx", C.POINTER(C.c_int32)),
        ("nbr_cap", C.c_int64),
        ("active_count", C.POINTER(C.c_int32)),
        ("rec_iters", C.c_int32),
        ("lam", C.POINTER(C.c_double)),
        ("rho", C.POINTER(C.c_double)),
        ("xs", C.POINTER(C.c_double)),
        ("x_final", C.POINTER(C.c_double)),
        ("v_final", C.POINTER(C.c_double)),
        ("d_range", C.c_float * 2),
        ("dims", C.c_int32 * 3),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.orc_poly6.restype = C.c_double
        L.orc_poly6.argtypes = [C.c_double, C.c_double]
        L.orc_spiky.restype = C.c_double
        L.orc_spiky.argtypes = [C.c_double, C.c_double]
        L.orc_spiky_grad.restype = None
        L.orc_spiky_grad.argtypes = [P(C.c_double), C.c_double, P(C.c_double)]
        L.orc_rest_density.restype = C.c_double
        L.orc_rest_density.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_grid_dims.argtypes = [P(OrcParams), P(C.c_int32)]
        L.orc_lod_levels.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_int32), P(C.c_float)]
        L.orc_predict.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_float), P(C.c_float)]
        L.orc_cell_keys.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_uint32)]
        L.orc_counting_sort.argtypes = [C.c_int32, P(C.c_uint32), C.c_int64, P(C.c_int32), P(C.c_uint32)]
        L.orc_neighbors.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_int32), P(C.c_int32),
                                    C.c_int64]
        L.orc_constraint.argtypes = [P(OrcParams), C.c_int32, P(C.c_double), P(C.c_int32), P(C.c_int32),
                                     C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double),
                                     P(C.c_double)]
        L.orc_delta_p.argtypes = [P(OrcParams), C.c_int32, P(C.c_double), P(C.c_double), P(C.c_int32),
                                  P(C.c_int32), P(C.c_double)]
        L.orc_xsph.argtypes = [P(OrcParams), C.c_int32, P(C.c_double), P(C.c_double), P(C.c_int32),
                               P(C.c_int32), P(C.c_double)]
        L.orc_step.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_float), P(C.c_int32),
                               P(OrcRecord)]
        L.orc_density_stats.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_double),
                                        P(C.c_double)]
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_set_threads.restype = C.c_int32
        L.orc_obstacle_project.argtypes = [P(OrcObstacle), P(C.c_double), P(C.c_double)]
        L.orc_obstacle_project.restype = C.c_int
        L.orc_view_basis.argtypes = [P(OrcView), P(C.c_float), P(C.c_float), P(C.c_float)]
        L.orc_pixel_ray.argtypes = [P(OrcView), C.c_int32, C.c_int32, P(C.c_float)]
        L.orc_depth_image.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_float)]
        L.orc_dtvs_distance.argtypes = [P(OrcParams), C.c_int32, P(C.c_float), P(C.c_float), P(C.c_float)]
        for f in ("orc_grid_dims", "orc_lod_levels", "orc_predict", "orc_cell_keys", "orc_counting_sort",
                  "orc_neighbors", "orc_constraint", "orc_delta_p", "orc_xsph", "orc_step",
                  "orc_density_stats", "orc_view_basis", "orc_pixel_ray", "orc_depth_image", "orc_dtvs_distance"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} returned {rc}")


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(ctype))


def make_params(cfg=None, *, rho0: float, box_lo=None, box_hi=None, eye=(0.0, 0.0, 0.0),
                d_near: float = 0.0, d_far: float = 0.0, lambda_mode: int = ORC_LAMBDA_STALE,
                lod_rounding: int = 0, view: Optional[OrcView] = None, obstacles=(), **over) -> OrcParams:
    """Parameters from a scenes.SceneConfig (or keyword overrides)."""
    vals = {}
    if cfg is not None:
        vals.update(h=cfg.h, dt=cfg.dt, mass=cfg.mass, eps=cfg.eps, scorr_k=cfg.scorr_k,
                    scorr_dq=cfg.scorr_dq, xsph_c=cfg.xsph_c, scorr_n=cfg.scorr_n, gravity=cfg.gravity,
                    grid_lo=cfg.box_lo, grid_hi=cfg.box_hi, n_min=cfg.n_min, n_max=cfg.n_max,
                    lod_mode=cfg.lod_mode)
    vals.update(over)
    p = OrcParams()
    for k in ("h", "dt", "mass", "eps", "scorr_k", "scorr_dq", "xsph_c"):
        setattr(p, k, float(vals[k]))
    p.rho0 = float(rho0)
    p.scorr_n = int(vals["scorr_n"])
    p.gravity[:] = [float(g) for g in vals["gravity"]]
    p.grid_lo[:] = [float(g) for g in vals["grid_lo"]]
    p.grid_hi[:] = [float(g) for g in vals["grid_hi"]]
    blo = vals["grid_lo"] if box_lo is None else box_lo
    bhi = vals["grid_hi"] if box_hi is None else box_hi
    p.box_lo[:] = [float(g) for g in blo]
    p.box_hi[:] = [float(g) for g in bhi]
    p.n_min = int(vals["n_min"])
    p.n_max = int(vals["n_max"])
    p.lod_mode = int(vals["lod_mode"])
    p.eye[:] = [float(e) for e in eye]
    p.d_near = float(d_near)
    p.d_far = float(d_far)
    p.lambda_mode = int(lambda_mode)
    p.lod_rounding = int(lod_rounding)
    if view is not None:
        p.view = view
    if cfg is not None:
        vals.setdefault("stabil_iters", getattr(cfg, "stabil_iters", 0))
        vals.setdefault("stabil_s", getattr(cfg, "stabil_s", 1))
        if not obstacles:
            obstacles = getattr(cfg, "obstacles", ())
    p.stabil_iters = int(vals.get("stabil_iters", 0))
    p.stabil_s = int(vals.get("stabil_s", 1))
    p.n_obstacles = len(obstacles)
    for k, (kind, a, b) in enumerate(obstacles):
        p.obstacles[k].kind = int(kind)
        p.obstacles[k].a[:] = [float(t) for t in a]
        p.obstacles[k].b[:] = [float(t) for t in b]
    return p


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's per-particle loops (n <= 0: keep the current
    count); returns the count in use. Results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def poly6(r2: float, h: float) -> float:
    return lib().orc_poly6(r2, h)


def spiky(r: float, h: float) -> float:
    return lib().orc_spiky(r, h)


def spiky_grad(r, h: float) -> np.ndarray:
    rr = np.ascontiguousarray(r, np.float64)
    g = np.zeros(3)
    lib().orc_spiky_grad(_ptr(rr, C.c_double), h, _ptr(g, C.c_double))
    return g


def rest_density(h: float, mass: float, spacing: float) -> float:
    return lib().orc_rest_density(h, mass, spacing)


def grid_dims(p: OrcParams):
    d = np.zeros(3, np.int32)
    _check(lib().orc_grid_dims(C.byref(p), _ptr(d, C.c_int32)), "orc_grid_dims")
    return d


def lod_levels(p: OrcParams, x: np.ndarray):
    x = np.ascontiguousarray(x, np.float32)
    n = x.shape[0]
    lv = np.zeros(n, np.int32)
    rng = np.zeros(2, np.float32)
    _check(lib().orc_lod_levels(C.byref(p), n, _ptr(x, C.c_float), _ptr(lv, C.c_int32),
                                _ptr(rng, C.c_float)), "orc_lod_levels")
    return lv, rng


def obstacle_project(kind, a, b, x):
    """(inside, nearest surface point) of a point for one obstacle, FP64."""
    o = OrcObstacle()
    o.kind = int(kind)
    o.a[:] = [float(t) for t in a]
    o.b[:] = [float(t) for t in b]
    xx = np.ascontiguousarray(x, np.float64)
    q = np.zeros(3)
    inside = lib().orc_obstacle_project(C.byref(o), _ptr(xx, C.c_double), _ptr(q, C.c_double))
    return bool(inside), q


def view_basis(v: OrcView):
    f, r, u = (np.zeros(3, np.float32) for _ in range(3))
    _check(lib().orc_view_basis(C.byref(v), _ptr(f, C.c_float), _ptr(r, C.c_float), _ptr(u, C.c_float)),
           "orc_view_basis")
    return f, r, u


def pixel_ray(v: OrcView, px: int, py: int) -> np.ndarray:
    ray = np.zeros(3, np.float32)
    _check(lib().orc_pixel_ray(C.byref(v), px, py, _ptr(ray, C.c_float)), "orc_pixel_ray")
    return ray


def depth_image(p: OrcParams, x: np.ndarray) -> np.ndarray:
    """(height, width) float32 depth image; empty pixels hold the float with bits 0x7f7f7f7f."""
    x = np.ascontiguousarray(x, np.float32)
    d = np.zeros((p.view.height, p.view.width), np.float32)
    _check(lib().orc_depth_image(C.byref(p), x.shape[0], _ptr(x, C.c_float), _ptr(d, C.c_float)),
           "orc_depth_image")
    return d


def dtvs_distance(p: OrcParams, x: np.ndarray, depth: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    depth = np.ascontiguousarray(depth, np.float32)
    out = np.zeros(x.shape[0], np.float32)
    _check(lib().orc_dtvs_distance(C.byref(p), x.shape[0], _ptr(x, C.c_float), _ptr(depth, C.c_float),
                                   _ptr(out, C.c_float)), "orc_dtvs_distance")
    return out


def predict(p: OrcParams, x: np.ndarray, v: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    out = np.zeros_like(x)
    _check(lib().orc_predict(C.byref(p), x.shape[0], _ptr(x, C.c_float), _ptr(v, C.c_float),
                             _ptr(out, C.c_float)), "orc_predict")
    return out


def cell_keys(p: OrcParams, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    k = np.zeros(x.shape[0], np.uint32)
    _check(lib().orc_cell_keys(C.byref(p), x.shape[0], _ptr(x, C.c_float), _ptr(k, C.c_uint32)),
           "orc_cell_keys")
    return k


def counting_sort(keys: np.ndarray, ncell: int):
    keys = np.ascontiguousarray(keys, np.uint32)
    n = keys.shape[0]
    order = np.zeros(n, np.int32)
    start = np.zeros(ncell + 1, np.uint32)
    _check(lib().orc_counting_sort(n, _ptr(keys, C.c_uint32), ncell, _ptr(order, C.c_int32),
                                   _ptr(start, C.c_uint32)), "orc_counting_sort")
    return order, start


def neighbors(p: OrcParams, x: np.ndarray):
    """CSR (off, idx) of neighbour sets in input indices, lists ascending."""
    x = np.ascontiguousarray(x, np.float32)
    n = x.shape[0]
    off = np.zeros(n + 1, np.int32)
    cap = max(64 * n, 1)
    while True:
        idx = np.zeros(cap, np.int32)
        rc = lib().orc_neighbors(C.byref(p), n, _ptr(x, C.c_float), _ptr(off, C.c_int32),
                                 _ptr(idx, C.c_int32), cap)
        if rc == -2:
            cap = int(off[n]) + 1
            continue
        _check(rc, "orc_neighbors")
        return off, idx[: off[n]].copy()


def constraint(p: OrcParams, xs: np.ndarray, off: np.ndarray, idx: np.ndarray, i: int):
    """(rho, C, grad (deg+1, 3), lambda) for particle i (Eq. 4-6)."""
    xs = np.ascontiguousarray(xs, np.float64)
    deg = int(off[i + 1] - off[i])
    grad = np.zeros((deg + 1, 3))
    rho, Cv, lam = C.c_double(), C.c_double(), C.c_double()
    off = np.ascontiguousarray(off, np.int32)
    idx = np.ascontiguousarray(idx if len(idx) else np.zeros(1, np.int32), np.int32)
    _check(lib().orc_constraint(C.byref(p), xs.shape[0], _ptr(xs, C.c_double), _ptr(off, C.c_int32),
                                _ptr(idx, C.c_int32), i, C.byref(rho), C.byref(Cv),
                                _ptr(grad, C.c_double), C.byref(lam)), "orc_constraint")
    return rho.value, Cv.value, grad, lam.value


def delta_p(p: OrcParams, xs, lam, off, idx) -> np.ndarray:
    xs = np.ascontiguousarray(xs, np.float64)
    lam = np.ascontiguousarray(lam, np.float64)
    off = np.ascontiguousarray(off, np.int32)
    idx = np.ascontiguousarray(idx if len(idx) else np.zeros(1, np.int32), np.int32)
    dp = np.zeros_like(xs)
    _check(lib().orc_delta_p(C.byref(p), xs.shape[0], _ptr(xs, C.c_double), _ptr(lam, C.c_double),
                             _ptr(off, C.c_int32), _ptr(idx, C.c_int32), _ptr(dp, C.c_double)),
           "orc_delta_p")
    return dp


def xsph(p: OrcParams, xs, v, off, idx) -> np.ndarray:
    xs = np.ascontiguousarray(xs, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    off = np.ascontiguousarray(off, np.int32)
    idx = np.ascontiguousarray(idx if len(idx) else np.zeros(1, np.int32), np.int32)
    out = np.zeros_like(v)
    _check(lib().orc_xsph(C.byref(p), xs.shape[0], _ptr(xs, C.c_double), _ptr(v, C.c_double),
                          _ptr(off, C.c_int32), _ptr(idx, C.c_int32), _ptr(out, C.c_double)),
           "orc_xsph")
    return out


def density_stats(p: OrcParams, x: np.ndarray, want_rho: bool = False):
    x = np.ascontiguousarray(x, np.float32)
    n = x.shape[0]
    stats = np.zeros(4)
    rho = np.zeros(max(n, 1)) if want_rho else None
    _check(lib().orc_density_stats(C.byref(p), n, _ptr(x, C.c_float), _ptr(rho, C.c_double),
                                   _ptr(stats, C.c_double)), "orc_density_stats")
    return (stats, rho[:n]) if want_rho else stats


class Step:
    """Result of one oracle step with optional records (numpy arrays)."""


def step(p: OrcParams, x: np.ndarray, v: np.ndarray, ids: Optional[np.ndarray] = None, *,
         record: bool = False, rec_iters: int = 0, want_final64: bool = False) -> Step:
    """Run one step of Fig. 7. Inputs are not modified; returns a Step with
    x, v, ids (new state in sorted order) and, if record, the stage records."""
    x = np.array(x, np.float32, order="C", copy=True)
    v = np.array(v, np.float32, order="C", copy=True)
    n = x.shape[0]
    ids = np.arange(n, dtype=np.int32) if ids is None else np.array(ids, np.int32, copy=True)
    r = OrcRecord()
    out = Step()
    keep = []
    dims = grid_dims(p)
    ncell = int(dims[0]) * int(dims[1]) * int(dims[2])

    def alloc(name, shape, dtype, ctype):
        a = np.zeros(shape, dtype)
        keep.append(a)
        setattr(r, name, _ptr(a, ctype))
        setattr(out, name, a)
        return a

    if record:
        alloc("xpred", (max(n, 1), 3), np.float32, C.c_float)
        alloc("level_presort", max(n, 1), np.int32, C.c_int32)
        alloc("keys", max(n, 1), np.uint32, C.c_uint32)
        alloc("order", max(n, 1), np.int32, C.c_int32)
        alloc("cell_start", ncell + 1, np.uint32, C.c_uint32)
        r.cell_cap = ncell + 1
        alloc("nbr_off", n + 1, np.int32, C.c_int32)
        alloc("active_count", int(p.n_max) + 2, np.int32, C.c_int32)
    if rec_iters > 0:
        r.rec_iters = rec_iters
        alloc("lam", (rec_iters, max(n, 1)), np.float64, C.c_double)
        alloc("rho", (rec_iters, max(n, 1)), np.float64, C.c_double)
        alloc("xs", (rec_iters, max(n, 1), 3), np.float64, C.c_double)
    if want_final64:
        alloc("x_final", (max(n, 1), 3), np.float64, C.c_double)
        alloc("v_final", (max(n, 1), 3), np.float64, C.c_double)
    cap = 64 * n if record else 0
    while True:
        if record:
            alloc("nbr_idx", max(cap, 1), np.int32, C.c_int32)
            r.nbr_cap = cap
        xx, vv, ii = x.copy(), v.copy(), ids.copy()
        rc = lib().orc_step(C.byref(p), n, _ptr(xx, C.c_float), _ptr(vv, C.c_float), _ptr(ii, C.c_int32),
                            C.byref(r))
        if rc == -2 and record:
            cap *= 2
            continue
        _check(rc, "orc_step")
        break
    out.x, out.v, out.ids = xx[:n], vv[:n], ii[:n]
    out.dims = np.array(r.dims[:], np.int32)
    out.d_range = np.array(r.d_range[:], np.float32)
    if record:
        out.xpred = out.xpred[:n]
        out.level_presort = out.level_presort[:n]
        out.keys = out.keys[:n]
        out.order = out.order[:n]
        out.nbr_idx = out.nbr_idx[: out.nbr_off[n]]
    if rec_iters > 0:
        out.lam = out.lam[:, :n]
        out.rho = out.rho[:, :n]
        out.xs = out.xs[:, :n]
    if want_final64:
        out.x_final = out.x_final[:n]
        out.v_final = out.v_final[:n]
    return out


def run(p_fn, x, v, steps: int):
    """Run ``steps`` oracle steps; p_fn(step) -> OrcParams for that step.
    Returns (x, v, ids) in the final state order."""
    ids = np.arange(x.shape[0], dtype=np.int32)
    for s in range(steps):
        st = step(p_fn(s), x, v, ids)
        x, v, ids = st.x, st.v, st.ids
    return x, v, ids


