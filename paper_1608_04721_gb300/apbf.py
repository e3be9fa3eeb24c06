"""Thin ctypes binding of the C ABI in include/apbf.h (same names).

Argument marshalling only: every step of the simulation runs in the CUDA
library libapbf.so. PyTorch, when present, lends device memory (the scene
arena) and the current CUDA stream. If the library has not been built the
import still works, but the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# APBF_LIBRARY=debug selects the build with device-side invariant checks
# (libapbf_debug.so); any other value is taken as a path to the library.
_CHOICE = os.environ.get("APBF_LIBRARY", "")
LIB_PATH = (os.path.join(_HERE, "libapbf_debug.so") if _CHOICE == "debug"
            else _CHOICE or os.path.join(_HERE, "libapbf.so"))

# status codes
APBF_OK = 0
APBF_ERR_INVALID_ARG = 1
APBF_ERR_OUT_OF_MEMORY = 2
APBF_ERR_CUDA = 3
APBF_ERR_TIMEOUT = 4
APBF_ERR_BAD_STATE = 5
APBF_ERR_NEIGHBOR_OVERFLOW = 6
APBF_ERR_NOT_SUPPORTED = 7
APBF_ERR_CHECK_FAILED = 8

APBF_LOD_FIXED = 0
APBF_LOD_DTC = 1
APBF_LOD_DTVS = 2
APBF_FLAG_NO_GRAPH = 1

STAGES = ["depth_image", "predict", "scan", "scatter", "reorder", "neighbors", "levels", "lambda", "deltap",
          "finalize"]
(APBF_STAGE_LOD_RANGE, APBF_STAGE_PREDICT, APBF_STAGE_SCAN, APBF_STAGE_SCATTER, APBF_STAGE_REORDER,
 APBF_STAGE_NEIGHBORS, APBF_STAGE_LEVELS, APBF_STAGE_LAMBDA, APBF_STAGE_DELTAP, APBF_STAGE_FINALIZE) = range(10)
APBF_STAGE_COUNT = 11
APBF_STAGE_PRESTAB = 10
APBF_MAX_OBSTACLES = 8
APBF_OBSTACLE_SPHERE, APBF_OBSTACLE_BOX, APBF_OBSTACLE_CONE = 1, 2, 3

(APBF_DBG_KEYS, APBF_DBG_STATE_IDS, APBF_DBG_LEVEL_PRESORT, APBF_DBG_SORTED_IDS, APBF_DBG_CELL_START,
 APBF_DBG_XPRED, APBF_DBG_LEVEL, APBF_DBG_NBR_COUNT, APBF_DBG_NBR, APBF_DBG_ACTIVE, APBF_DBG_LEVEL_COUNT,
 APBF_DBG_LAMBDA, APBF_DBG_RHO, APBF_DBG_XSTAR, APBF_DBG_DRANGE, APBF_DBG_DEPTH,
 APBF_DBG_LOD_DISTANCE) = range(17)


class apbf_scene_desc(C.Structure):
    _fields_ = [
        ("n", C.c_uint32),
        ("pos", C.POINTER(C.c_float)),
        ("vel", C.POINTER(C.c_float)),
        ("grid_lo", C.c_float * 3), ("grid_hi", C.c_float * 3),
        ("box_lo", C.c_float * 3), ("box_hi", C.c_float * 3),
        ("h", C.c_float), ("dt", C.c_float), ("mass", C.c_float), ("rho0", C.c_float), ("eps", C.c_float),
        ("scorr_k", C.c_float), ("scorr_dq", C.c_float),
        ("scorr_n", C.c_uint32),
        ("xsph_c", C.c_float),
        ("gravity", C.c_float * 3),
        ("n_min", C.c_uint32), ("n_max", C.c_uint32), ("lod_mode", C.c_uint32),
        ("stabil_iters", C.c_uint32), ("stabil_s", C.c_uint32),
        ("max_neighbors", C.c_uint32),
        ("flags", C.c_uint32),
    ]


class apbf_step_info(C.Structure):
    _fields_ = [
        ("particle_iterations", C.c_uint64),
        ("neighbor_pairs", C.c_uint64),
        ("lambda_pairs", C.c_uint64),
        ("active_count", C.c_uint32 * 256),
        ("d_range", C.c_float * 2),
        ("total_particle_iterations", C.c_uint64),
    ]


class apbf_obstacle(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("a", C.c_float * 3), ("b", C.c_float * 3)]


class apbf_tune_result(C.Structure):
    _fields_ = [
        ("block", C.c_uint32),
        ("mask_threshold", C.c_float),
        ("ms_per_step", C.c_double),
        ("tried", C.c_uint32),
        ("blocks", C.c_uint32 * 16),
        ("thresholds", C.c_float * 16),
        ("ms", C.c_double * 16),
    ]


class apbf_server_desc(C.Structure):
    _fields_ = [
        ("physics", C.POINTER(apbf_scene_desc)),
        ("max_particles", C.c_uint32),
        ("max_cells", C.c_uint32),
        ("max_scenes", C.c_uint32),
        ("budget_bytes", C.c_size_t),
        ("target_step_ms", C.c_double),
    ]


class apbf_request(C.Structure):
    _fields_ = [
        ("scene", C.POINTER(apbf_scene_desc)),
        ("eye", C.c_float * 3),
        ("steps", C.c_uint32),
        ("pos_out", C.POINTER(C.c_float)),
        ("vel_out", C.POINTER(C.c_float)),
        ("obstacles", C.c_void_p),
        ("n_obstacles", C.c_uint32),
    ]


class apbf_tick_info(C.Structure):
    _fields_ = [
        ("tick", C.c_uint64),
        ("resident_scenes", C.c_uint32),
        ("resident_particles", C.c_uint32),
        ("admitted", C.c_uint32),
        ("completed", C.c_uint32),
        ("queued", C.c_uint32),
        ("failed", C.c_uint32),
        ("prev_step_ms", C.c_double),
        ("total_particle_iterations", C.c_uint64),
        ("particle_limit", C.c_uint32),
        ("pad", C.c_uint32),
    ]


class apbf_request_info(C.Structure):
    _fields_ = [
        ("state", C.c_uint32),
        ("steps_done", C.c_uint32),
        ("n", C.c_uint32),
        ("steps", C.c_uint32),
        ("submit_tick", C.c_uint64),
        ("admit_tick", C.c_uint64),
        ("done_tick", C.c_uint64),
        ("status", C.c_int32),
        ("pad", C.c_uint32),
    ]


APBF_REQ_QUEUED, APBF_REQ_RESIDENT, APBF_REQ_DONE, APBF_REQ_FAILED = 0, 1, 2, 3

EXPORTS = [
    "apbf_status_string", "apbf_rest_density", "apbf_scene_bytes", "apbf_create_scene", "apbf_set_camera",
    "apbf_set_box", "apbf_step", "apbf_read_state", "apbf_density_stats", "apbf_get_step_info", "apbf_sync",
    "apbf_last_error", "apbf_destroy_scene", "apbf_set_timing", "apbf_timing_report", "apbf_debug_step_to",
    "apbf_debug_read", "apbf_debug_dims", "apbf_density_stats_static", "apbf_batch_bytes", "apbf_create_batch",
    "apbf_set_camera_at", "apbf_set_box_at", "apbf_set_tuning", "apbf_autotune", "apbf_server_bytes",
    "apbf_server_create", "apbf_server_submit", "apbf_server_tick", "apbf_server_query", "apbf_server_last_error",
    "apbf_server_destroy", "apbf_set_view", "apbf_set_view_outside_level", "apbf_set_obstacles", "apbf_read_positions_async",
    "apbf_debug_checks_enabled", "apbf_debug_plant",
]
APBF_STATIC_MAX_PARTICLES = 65536
APBF_STATIC_MAX_CELLS = 262144

_lib = None


class ApbfError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {_status_name(status)} ({status}): {message}")
        self.status = status


def _status_name(st: int) -> str:
    try:
        return lib().apbf_status_string(st).decode()
    except Exception:
        return str(st)


def lib():
    """The loaded libapbf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                               f"g.build()\"` (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        P, V = C.POINTER, C.c_void_p
        L.apbf_status_string.restype = C.c_char_p
        L.apbf_status_string.argtypes = [C.c_int]
        L.apbf_rest_density.argtypes = [C.c_float, C.c_float, C.c_float, P(C.c_double)]
        L.apbf_scene_bytes.argtypes = [P(apbf_scene_desc), P(C.c_size_t)]
        L.apbf_create_scene.argtypes = [P(apbf_scene_desc), V, V, C.c_size_t, P(V)]
        L.apbf_set_camera.argtypes = [V, P(C.c_float), P(C.c_float), C.c_float, C.c_float]
        L.apbf_set_box.argtypes = [V, P(C.c_float), P(C.c_float)]
        L.apbf_step.argtypes = [V, C.c_uint32]
        L.apbf_read_state.argtypes = [V, P(C.c_float), P(C.c_float), P(C.c_uint8), P(C.c_float)]
        L.apbf_density_stats.argtypes = [V, P(C.c_double)]
        L.apbf_get_step_info.argtypes = [V, P(apbf_step_info)]
        L.apbf_sync.argtypes = [V]
        L.apbf_read_positions_async.argtypes = [V, V]
        L.apbf_last_error.restype = C.c_char_p
        L.apbf_last_error.argtypes = [V]
        L.apbf_destroy_scene.restype = None
        L.apbf_destroy_scene.argtypes = [V]
        L.apbf_set_timing.argtypes = [V, C.c_int]
        L.apbf_timing_report.argtypes = [V, P(C.c_double), P(C.c_uint64)]
        L.apbf_debug_step_to.argtypes = [V, C.c_uint32, C.c_uint32]
        L.apbf_debug_read.argtypes = [V, C.c_uint32, V, C.c_size_t]
        L.apbf_debug_dims.argtypes = [V, P(C.c_int32), P(C.c_uint32), P(C.c_uint32)]
        L.apbf_debug_checks_enabled.restype = C.c_int
        L.apbf_debug_checks_enabled.argtypes = []
        L.apbf_debug_plant.argtypes = [V, C.c_uint32]
        L.apbf_batch_bytes.argtypes = [P(apbf_scene_desc), C.c_uint32, P(C.c_size_t)]
        L.apbf_create_batch.argtypes = [P(apbf_scene_desc), C.c_uint32, V, V, C.c_size_t, P(V)]
        L.apbf_set_camera_at.argtypes = [V, C.c_uint32, P(C.c_float), P(C.c_float), C.c_float, C.c_float]
        L.apbf_set_box_at.argtypes = [V, C.c_uint32, P(C.c_float), P(C.c_float)]
        L.apbf_set_tuning.argtypes = [V, C.c_uint32, C.c_float]
        L.apbf_autotune.argtypes = [V, C.c_uint32, P(apbf_tune_result)]
        L.apbf_density_stats_static.argtypes = [V, C.c_uint32, C.c_float, C.c_float, C.c_float, P(C.c_float),
                                                P(C.c_float), V, V]
        L.apbf_set_obstacles.argtypes = [V, C.c_uint32, P(apbf_obstacle), C.c_uint32]
        L.apbf_set_view.argtypes = [V, C.c_uint32, C.c_uint32, C.c_float, P(C.c_float), C.c_float]
        L.apbf_set_view_outside_level.argtypes = [V, C.c_uint32]
        L.apbf_server_bytes.argtypes = [P(apbf_server_desc), P(C.c_size_t), P(C.c_uint32), P(C.c_uint32)]
        L.apbf_server_create.argtypes = [P(apbf_server_desc), V, P(V)]
        L.apbf_server_submit.argtypes = [V, P(apbf_request), P(C.c_uint64)]
        L.apbf_server_tick.argtypes = [V, P(apbf_tick_info)]
        L.apbf_server_query.argtypes = [V, C.c_uint64, P(apbf_request_info)]
        L.apbf_server_last_error.restype = C.c_char_p
        L.apbf_server_last_error.argtypes = [V]
        L.apbf_server_destroy.restype = None
        L.apbf_server_destroy.argtypes = [V]
        for f in EXPORTS:
            if f not in ("apbf_status_string", "apbf_last_error", "apbf_destroy_scene", "apbf_server_last_error",
                         "apbf_server_destroy"):
                getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(st: int, where: str, scene=None):
    if st != APBF_OK:
        h = scene.handle if scene is not None else None
        raise ApbfError(st, where, lib().apbf_last_error(h).decode())


def _fptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


class Scene:
    """Handle of a created scene or batch; keeps the arena and inputs alive."""

    def __init__(self, handle, n, desc, keep, counts=None):
        self.handle = handle
        self.n = n
        self.desc = desc
        self._keep = keep
        self.counts = [n] if counts is None else list(counts)  # particles per scene

    @property
    def scenes(self) -> int:
        return len(self.counts)

    def __del__(self):
        try:
            if self.handle:
                lib().apbf_destroy_scene(self.handle)
                self.handle = None
        except Exception:
            pass


def make_desc(*, pos: np.ndarray, vel: Optional[np.ndarray] = None, grid_lo, grid_hi, box_lo=None, box_hi=None,
              h: float, dt: float, mass: float, rho0: float, eps: float, scorr_k: float, scorr_dq: float,
              scorr_n: int, xsph_c: float, gravity, n_min: int, n_max: int, lod_mode: int, stabil_iters: int = 0,
              stabil_s: int = 1, max_neighbors: int = 0, flags: int = 0):
    """Fill an apbf_scene_desc; returns (desc, arrays to keep alive)."""
    pos = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float32).reshape(-1, 3)
    d = apbf_scene_desc()
    d.n = pos.shape[0]
    d.pos = _fptr(pos) if pos.size else None
    d.vel = _fptr(vel) if vel is not None and vel.size else None
    d.grid_lo[:] = [float(v) for v in grid_lo]
    d.grid_hi[:] = [float(v) for v in grid_hi]
    d.box_lo[:] = [float(v) for v in (grid_lo if box_lo is None else box_lo)]
    d.box_hi[:] = [float(v) for v in (grid_hi if box_hi is None else box_hi)]
    d.h, d.dt, d.mass, d.rho0, d.eps = h, dt, mass, rho0, eps
    d.scorr_k, d.scorr_dq, d.scorr_n, d.xsph_c = scorr_k, scorr_dq, scorr_n, xsph_c
    d.gravity[:] = [float(v) for v in gravity]
    d.n_min, d.n_max, d.lod_mode = n_min, n_max, lod_mode
    d.stabil_iters, d.stabil_s, d.max_neighbors, d.flags = stabil_iters, stabil_s, max_neighbors, flags
    return d, (pos, vel)


def desc_from_config(cfg, pos, vel, rho0: float, **over):
    """apbf_scene_desc from a scenes.SceneConfig (plain field mapping)."""
    kw = dict(pos=pos, vel=vel, grid_lo=cfg.box_lo, grid_hi=cfg.box_hi, h=cfg.h, dt=cfg.dt, mass=cfg.mass,
              rho0=rho0, eps=cfg.eps, scorr_k=cfg.scorr_k, scorr_dq=cfg.scorr_dq, scorr_n=cfg.scorr_n,
              xsph_c=cfg.xsph_c, gravity=cfg.gravity, n_min=cfg.n_min, n_max=cfg.n_max, lod_mode=cfg.lod_mode,
              stabil_iters=getattr(cfg, "stabil_iters", 0), stabil_s=getattr(cfg, "stabil_s", 1))
    kw.update(over)
    return make_desc(**kw)


# ------------------------------------------------------------ entry points

def apbf_status_string(status: int) -> str:
    return lib().apbf_status_string(status).decode()


def apbf_rest_density(h: float, mass: float, spacing: float) -> float:
    out = C.c_double()
    _check(lib().apbf_rest_density(h, mass, spacing, C.byref(out)), "apbf_rest_density")
    return out.value


def apbf_scene_bytes(desc) -> int:
    d = desc[0] if isinstance(desc, tuple) else desc
    out = C.c_size_t()
    _check(lib().apbf_scene_bytes(C.byref(d), C.byref(out)), "apbf_scene_bytes")
    return out.value


def _stream_and_arena(nbytes_fn, stream, device_arena):
    torch = None
    try:
        import torch as _torch
        torch = _torch if _torch.cuda.is_available() else None
    except Exception:
        torch = None
    if stream is None:
        stream_ptr = torch.cuda.current_stream().cuda_stream if torch is not None else 0
    elif hasattr(stream, "cuda_stream"):
        stream_ptr = stream.cuda_stream
    else:
        stream_ptr = int(stream)
    arena_ptr, arena_bytes, arena_keep = None, 0, None
    if isinstance(device_arena, str) and device_arena == "torch":
        if torch is not None:
            nbytes = nbytes_fn()
            arena_keep = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            arena_ptr = (arena_keep.data_ptr() + 255) // 256 * 256
            arena_bytes = nbytes
    elif device_arena is None:
        pass
    elif hasattr(device_arena, "data_ptr"):
        arena_keep = device_arena
        arena_ptr = device_arena.data_ptr()
        arena_bytes = device_arena.numel() * device_arena.element_size()
    else:
        arena_ptr, arena_bytes = int(device_arena[0]), int(device_arena[1])
    return stream_ptr, arena_ptr, arena_bytes, arena_keep


def apbf_batch_bytes(descs) -> int:
    arr, _ = _desc_array(descs)
    out = C.c_size_t()
    _check(lib().apbf_batch_bytes(arr, len(arr), C.byref(out)), "apbf_batch_bytes")
    return out.value


def _desc_array(descs):
    items = [d[0] if isinstance(d, tuple) else d for d in descs]
    keep = [d[1] for d in descs if isinstance(d, tuple)]
    arr = (apbf_scene_desc * len(items))(*items)
    return arr, keep


def apbf_create_batch(descs, stream=None, device_arena="torch") -> Scene:
    """descs: a list of apbf_scene_desc (or make_desc pairs); other arguments
    as in apbf_create_scene."""
    arr, keep = _desc_array(descs)
    stream_ptr, arena_ptr, arena_bytes, arena_keep = _stream_and_arena(lambda: apbf_batch_bytes(descs), stream,
                                                                       device_arena)
    h = C.c_void_p()
    _check(lib().apbf_create_batch(arr, len(arr), C.c_void_p(stream_ptr), C.c_void_p(arena_ptr), arena_bytes,
                                   C.byref(h)), "apbf_create_batch")
    counts = [int(d.n) for d in arr]
    return Scene(h, sum(counts), arr[0], (keep, arena_keep, arr), counts)


def apbf_set_camera_at(scene: Scene, index: int, eye, direction=(1.0, 0.0, 0.0), d_near: float = 0.0,
                       d_far: float = 0.0):
    e = (C.c_float * 3)(*[float(v) for v in eye])
    d = (C.c_float * 3)(*[float(v) for v in direction])
    _check(lib().apbf_set_camera_at(scene.handle, index, e, d, d_near, d_far), "apbf_set_camera_at", scene)


def apbf_set_box_at(scene: Scene, index: int, lo, hi):
    a = (C.c_float * 3)(*[float(v) for v in lo])
    b = (C.c_float * 3)(*[float(v) for v in hi])
    _check(lib().apbf_set_box_at(scene.handle, index, a, b), "apbf_set_box_at", scene)


def apbf_create_scene(desc, stream=None, device_arena="torch") -> Scene:
    """desc: apbf_scene_desc or the (desc, keep) pair of make_desc.
    stream: a CUDA stream handle (int) or a torch.cuda.Stream; None = torch's
    current stream (or the default stream without torch).
    device_arena: "torch" (a torch.uint8 CUDA tensor lent to the library),
    None (the library allocates), or a torch tensor / (pointer, bytes) pair."""
    keep = ()
    if isinstance(desc, tuple):
        desc, keep = desc
    torch = None
    try:
        import torch as _torch
        torch = _torch if _torch.cuda.is_available() else None
    except Exception:
        torch = None
    if stream is None:
        stream_ptr = torch.cuda.current_stream().cuda_stream if torch is not None else 0
    elif hasattr(stream, "cuda_stream"):
        stream_ptr = stream.cuda_stream
    else:
        stream_ptr = int(stream)
    arena_ptr, arena_bytes, arena_keep = None, 0, None
    if isinstance(device_arena, str) and device_arena == "torch":
        if torch is not None:
            nbytes = apbf_scene_bytes(desc)
            arena_keep = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = arena_keep.data_ptr()
            arena_ptr = (base + 255) // 256 * 256
            arena_bytes = nbytes
    elif device_arena is None:
        pass
    elif hasattr(device_arena, "data_ptr"):
        arena_keep = device_arena
        arena_ptr = device_arena.data_ptr()
        arena_bytes = device_arena.numel() * device_arena.element_size()
    else:
        arena_ptr, arena_bytes = int(device_arena[0]), int(device_arena[1])
    h = C.c_void_p()
    st = lib().apbf_create_scene(C.byref(desc), C.c_void_p(stream_ptr), C.c_void_p(arena_ptr), arena_bytes,
                                 C.byref(h))
    _check(st, "apbf_create_scene")
    return Scene(h, desc.n, desc, (keep, arena_keep))


def apbf_set_camera(scene: Scene, eye, direction=(1.0, 0.0, 0.0), d_near: float = 0.0, d_far: float = 0.0):
    e = (C.c_float * 3)(*[float(v) for v in eye])
    d = (C.c_float * 3)(*[float(v) for v in direction])
    _check(lib().apbf_set_camera(scene.handle, e, d, d_near, d_far), "apbf_set_camera", scene)


def apbf_set_box(scene: Scene, lo, hi):
    a = (C.c_float * 3)(*[float(v) for v in lo])
    b = (C.c_float * 3)(*[float(v) for v in hi])
    _check(lib().apbf_set_box(scene.handle, a, b), "apbf_set_box", scene)


def apbf_step(scene: Scene, nsteps: int = 1):
    _check(lib().apbf_step(scene.handle, nsteps), "apbf_step", scene)


def apbf_read_state(scene: Scene, pos=True, vel=True, n_iter=False, rho=False):
    """Each argument: False (skip), True (allocate) or a preallocated numpy
    array (e.g. in pinned memory). Returns a dict of the requested arrays in
    particle-id order."""
    n = scene.n
    out = {}

    def take(name, want, shape, dtype):
        if want is False or want is None:
            return None
        a = np.empty(shape, dtype) if want is True else want
        assert a.dtype == dtype and a.flags["C_CONTIGUOUS"] and a.size == int(np.prod(shape))
        out[name] = a
        return a

    p = take("pos", pos, (n, 3), np.float32)
    v = take("vel", vel, (n, 3), np.float32)
    it = take("n_iter", n_iter, (n,), np.uint8)
    r = take("rho", rho, (n,), np.float32)
    st = lib().apbf_read_state(scene.handle, _fptr(p), _fptr(v),
                               None if it is None else it.ctypes.data_as(C.POINTER(C.c_uint8)), _fptr(r))
    _check(st, "apbf_read_state", scene)
    return out


def apbf_read_positions_async(scene: Scene, pos_ptr: int):
    """Queue a copy of the positions (n x 3 float32, particle-id order) to the
    host memory at pos_ptr (a pinned buffer's address, e.g. a pinned torch
    tensor's data_ptr()); it is complete after apbf_sync. The buffer must
    stay alive until then."""
    _check(lib().apbf_read_positions_async(scene.handle, C.c_void_p(int(pos_ptr))), "apbf_read_positions_async",
           scene)


def apbf_density_stats(scene: Scene) -> np.ndarray:
    out = np.zeros(4)
    _check(lib().apbf_density_stats(scene.handle, out.ctypes.data_as(C.POINTER(C.c_double))),
           "apbf_density_stats", scene)
    return out


def apbf_get_step_info(scene: Scene) -> dict:
    info = apbf_step_info()
    _check(lib().apbf_get_step_info(scene.handle, C.byref(info)), "apbf_get_step_info", scene)
    return dict(particle_iterations=int(info.particle_iterations), neighbor_pairs=int(info.neighbor_pairs),
                lambda_pairs=int(info.lambda_pairs), active_count=np.array(info.active_count[:], np.int64),
                d_range=np.array(info.d_range[:], np.float32),
                total_particle_iterations=int(info.total_particle_iterations))


def apbf_sync(scene: Scene):
    _check(lib().apbf_sync(scene.handle), "apbf_sync", scene)


def apbf_last_error(scene: Optional[Scene] = None) -> str:
    return lib().apbf_last_error(scene.handle if scene is not None else None).decode()


def apbf_destroy_scene(scene: Scene):
    if scene.handle:
        lib().apbf_destroy_scene(scene.handle)
        scene.handle = None


def apbf_set_timing(scene: Scene, enable: bool):
    _check(lib().apbf_set_timing(scene.handle, 1 if enable else 0), "apbf_set_timing", scene)


def apbf_timing_report(scene: Scene):
    ms = np.zeros(APBF_STAGE_COUNT)
    ln = np.zeros(APBF_STAGE_COUNT, np.uint64)
    _check(lib().apbf_timing_report(scene.handle, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                    ln.ctypes.data_as(C.POINTER(C.c_uint64))), "apbf_timing_report", scene)
    return ms, ln


def apbf_debug_step_to(scene: Scene, stage: int, iteration: int = 0):
    _check(lib().apbf_debug_step_to(scene.handle, stage, iteration), "apbf_debug_step_to", scene)


def apbf_debug_checks_enabled() -> bool:
    return bool(lib().apbf_debug_checks_enabled())


def apbf_debug_plant(scene: Scene, what: int):
    _check(lib().apbf_debug_plant(scene.handle, what), "apbf_debug_plant", scene)


def apbf_debug_dims(scene: Scene):
    dims = (C.c_int32 * 3)()
    ncell, mx = C.c_uint32(), C.c_uint32()
    _check(lib().apbf_debug_dims(scene.handle, dims, C.byref(ncell), C.byref(mx)), "apbf_debug_dims", scene)
    return np.array(dims[:], np.int32), ncell.value, mx.value


def apbf_debug_read(scene: Scene, field: int) -> np.ndarray:
    n = scene.n
    dims, ncell, mx = apbf_debug_dims(scene)
    n_max = int(scene.desc.n_max)
    shapes = {
        APBF_DBG_KEYS: ((n,), np.uint32), APBF_DBG_STATE_IDS: ((n,), np.uint32),
        APBF_DBG_LEVEL_PRESORT: ((n,), np.uint8), APBF_DBG_SORTED_IDS: ((n,), np.uint32),
        APBF_DBG_CELL_START: ((ncell + 1,), np.uint32), APBF_DBG_XPRED: ((n, 4), np.float32),
        APBF_DBG_LEVEL: ((n,), np.uint8), APBF_DBG_NBR_COUNT: ((n,), np.uint8),
        APBF_DBG_NBR: ((mx, n), np.uint32), APBF_DBG_ACTIVE: ((n,), np.uint32),
        APBF_DBG_LEVEL_COUNT: ((n_max + 2,), np.uint32), APBF_DBG_LAMBDA: ((n,), np.float32),
        APBF_DBG_RHO: ((n,), np.float32), APBF_DBG_XSTAR: ((n, 4), np.float32),
        APBF_DBG_DRANGE: ((2 * scene.scenes,), np.float32),
        APBF_DBG_DEPTH: ((getattr(scene, "view", (0, 0))[1], getattr(scene, "view", (0, 0))[0]), np.float32),
        APBF_DBG_LOD_DISTANCE: ((n,), np.float32),
    }
    shape, dt = shapes[field]
    a = np.empty(shape, dt)
    _check(lib().apbf_debug_read(scene.handle, field, C.c_void_p(a.ctypes.data if a.size else 0), a.nbytes),
           "apbf_debug_read", scene)
    return a


def apbf_density_stats_static(pos_dev, n: int, h: float, mass: float, rho0: float, grid_lo, grid_hi, stats_dev,
                              stream=None):
    """Allocation-free density statistics of device positions (see the C
    header). pos_dev and stats_dev are device pointers (ints) or CUDA tensors
    (float32 of 3n values, float64 of 4 values); stream as in apbf_create_scene."""
    def ptr(x):
        return x.data_ptr() if hasattr(x, "data_ptr") else int(x)
    if stream is None:
        try:
            import torch
            stream_ptr = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        except Exception:
            stream_ptr = 0
    else:
        stream_ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    lo = (C.c_float * 3)(*[float(v) for v in grid_lo])
    hi = (C.c_float * 3)(*[float(v) for v in grid_hi])
    _check(lib().apbf_density_stats_static(C.c_void_p(ptr(pos_dev)), n, h, mass, rho0, lo, hi,
                                           C.c_void_p(ptr(stats_dev)), C.c_void_p(stream_ptr)),
           "apbf_density_stats_static")


def apbf_set_tuning(scene: Scene, block: int, mask_threshold: float):
    _check(lib().apbf_set_tuning(scene.handle, block, mask_threshold), "apbf_set_tuning", scene)


def apbf_autotune(scene: Scene, trial_steps: int = 5) -> dict:
    r = apbf_tune_result()
    _check(lib().apbf_autotune(scene.handle, trial_steps, C.byref(r)), "apbf_autotune", scene)
    trials = [(int(r.blocks[k]), float(r.thresholds[k]), float(r.ms[k])) for k in range(r.tried)]
    return dict(block=int(r.block), mask_threshold=float(r.mask_threshold), ms_per_step=float(r.ms_per_step),
                trials=trials)


# ---------------------------------------------------------------- serving


class Server:
    """Handle of an apbf_server; keeps submitted requests' output buffers alive
    until they are retired."""

    def __init__(self, handle, physics_keep, max_particles, max_cells):
        self.handle = handle
        self._physics_keep = physics_keep
        self._outputs = {}
        self.max_particles = max_particles
        self.max_cells = max_cells

    def __del__(self):
        try:
            if self.handle:
                lib().apbf_server_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _server_check(st: int, where: str, server=None):
    if st != APBF_OK:
        h = server.handle if server is not None else None
        raise ApbfError(st, where, lib().apbf_server_last_error(h).decode())


def _server_desc(physics, max_particles=0, max_cells=0, max_scenes=0, budget_bytes=0, target_step_ms=0.0):
    phys = physics[0] if isinstance(physics, tuple) else physics
    d = apbf_server_desc()
    d.physics = C.pointer(phys)
    d.max_particles, d.max_cells, d.max_scenes, d.budget_bytes = max_particles, max_cells, max_scenes, budget_bytes
    d.target_step_ms = float(target_step_ms)
    return d, phys


def apbf_server_bytes(physics, max_particles=0, max_cells=0, max_scenes=0, budget_bytes=0, target_step_ms=0.0):
    """(pool bytes, particle capacity, cell capacity) of a server description."""
    d, _ = _server_desc(physics, max_particles, max_cells, max_scenes, budget_bytes, target_step_ms)
    nb, npart, ncell = C.c_size_t(), C.c_uint32(), C.c_uint32()
    _server_check(lib().apbf_server_bytes(C.byref(d), C.byref(nb), C.byref(npart), C.byref(ncell)),
                  "apbf_server_bytes")
    return nb.value, npart.value, ncell.value


def apbf_server_create(physics, max_particles=0, max_cells=0, max_scenes=0, budget_bytes=0, stream=None,
                       target_step_ms=0.0) -> Server:
    d, phys = _server_desc(physics, max_particles, max_cells, max_scenes, budget_bytes, target_step_ms)
    _, npart, ncell = apbf_server_bytes(physics, max_particles, max_cells, max_scenes, budget_bytes, target_step_ms)
    stream_ptr, _, _, _ = _stream_and_arena(lambda: 0, stream, None)
    h = C.c_void_p()
    _server_check(lib().apbf_server_create(C.byref(d), C.c_void_p(stream_ptr), C.byref(h)), "apbf_server_create")
    return Server(h, phys, npart, ncell)


def apbf_server_submit(server: Server, desc, eye, steps: int, want_pos=True, want_vel=False, obstacles=()) -> int:
    """Queue a scene (a make_desc / desc_from_config pair or an apbf_scene_desc)
    with optional obstacles ((kind, a, b), ...); returns its ticket. Results:
    apbf_server_result(server, ticket) once done."""
    d = desc[0] if isinstance(desc, tuple) else desc
    n = int(d.n)
    pos = np.empty((n, 3), np.float32) if want_pos else None
    vel = np.empty((n, 3), np.float32) if want_vel else None
    r = apbf_request()
    r.scene = C.pointer(d)
    r.eye[:] = [float(e) for e in eye]
    r.steps = steps
    r.pos_out = _fptr(pos)
    r.vel_out = _fptr(vel)
    obs = (apbf_obstacle * max(1, len(obstacles)))()
    for k, (kind, a, b) in enumerate(obstacles):
        obs[k].kind = int(kind)
        obs[k].a[:] = [float(t) for t in a]
        obs[k].b[:] = [float(t) for t in (list(b) + [0.0, 0.0, 0.0])[:3]]
    r.obstacles = C.cast(obs, C.c_void_p) if obstacles else None
    r.n_obstacles = len(obstacles)
    t = C.c_uint64()
    _server_check(lib().apbf_server_submit(server.handle, C.byref(r), C.byref(t)), "apbf_server_submit", server)
    server._outputs[t.value] = (pos, vel)
    return t.value


def apbf_server_tick(server: Server) -> dict:
    info = apbf_tick_info()
    _server_check(lib().apbf_server_tick(server.handle, C.byref(info)), "apbf_server_tick", server)
    return {f: getattr(info, f) for f, _ in apbf_tick_info._fields_ if f != "pad"}


def apbf_server_query(server: Server, ticket: int) -> dict:
    info = apbf_request_info()
    _server_check(lib().apbf_server_query(server.handle, ticket, C.byref(info)), "apbf_server_query", server)
    return {f: getattr(info, f) for f, _ in apbf_request_info._fields_ if f != "pad"}


def apbf_server_result(server: Server, ticket: int):
    """(pos, vel) arrays of a finished request (None where not requested); the
    server stops holding them."""
    q = apbf_server_query(server, ticket)
    if q["state"] != APBF_REQ_DONE:
        raise ApbfError(APBF_ERR_BAD_STATE, "apbf_server_result", f"request {ticket} is not done (state {q['state']})")
    return server._outputs.pop(ticket)


def apbf_server_destroy(server: Server):
    if server.handle:
        lib().apbf_server_destroy(server.handle)
        server.handle = None


def apbf_set_view(scene: Scene, width: int, height: int, tan_half_fov: float, up=(0.0, 0.0, 1.0),
                  radius: float = 0.025):
    """Camera image of the DTVS model (see include/apbf.h)."""
    u = (C.c_float * 3)(*[float(a) for a in up])
    _check(lib().apbf_set_view(scene.handle, width, height, tan_half_fov, u, radius), "apbf_set_view", scene)
    scene.view = (int(width), int(height))


def apbf_set_view_outside_level(scene: Scene, level: int):
    """N_i of the DTVS particles outside the view (0: n_min; see include/apbf.h)."""
    _check(lib().apbf_set_view_outside_level(scene.handle, int(level)), "apbf_set_view_outside_level", scene)


def apbf_set_obstacles(scene: Scene, obstacles, index: int = 0):
    """obstacles: sequence of (kind, a, b) with kind APBF_OBSTACLE_*; see include/apbf.h."""
    arr = (apbf_obstacle * max(1, len(obstacles)))()
    for k, (kind, a, b) in enumerate(obstacles):
        arr[k].kind = int(kind)
        arr[k].a[:] = [float(t) for t in a]
        arr[k].b[:] = [float(t) for t in (list(b) + [0.0, 0.0, 0.0])[:3]]
    _check(lib().apbf_set_obstacles(scene.handle, index, arr, len(obstacles)), "apbf_set_obstacles", scene)
