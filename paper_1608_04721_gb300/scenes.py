"""Seeded synthetic scenes for the adaptive PBF solver.

This module only *generates inputs*: particle lattices with jitter, the scene
parameters, and per-step scene drivers (camera path, moving wall). It holds
none of the solver's arithmetic (no kernels, no densities, no constraints), so
both the CUDA path and the CPU oracle can take their inputs from it.

The paper publishes no scene geometry (Sec. 7 gives only particle counts and
iteration ranges, Table 1). The scenes below are synthetic stand-ins of the
same kind and size class: dam-break blocks on a lattice of spacing h/2 with
uniform jitter, in an axis-aligned box.

Random numbers come from a counter-based generator: draw k of stream s is
``splitmix64(seed + (k + 1) * GOLDEN + s * STREAM)`` where splitmix64 is the
finaliser published by Steele, Lea and Flood ("Fast splittable pseudorandom
number generators", OOPSLA 2014); the uniform value is the top 24 bits scaled
by 2**-24.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

LOD_FIXED = 0
LOD_DTC = 1
LOD_DTVS = 2


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied element-wise to uint64 counters."""
    z = np.asarray(counter, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` uniforms in [0, 1) (float64 holding 24-bit values)."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = np.uint64(seed) + k * GOLDEN + np.uint64(stream) * _STREAM
    r = splitmix64(ctr)
    return (r >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


@dataclasses.dataclass
class SceneConfig:
    """One synthetic workload. Lengths in metres, time in seconds."""
    name: str
    lattice: Tuple[int, int, int]          # particles along x, y, z
    spacing: float                          # lattice spacing (h/2)
    block_lo: Tuple[float, float, float]    # corner of the fluid block
    box_lo: Tuple[float, float, float]      # static container / grid extent
    box_hi: Tuple[float, float, float]
    h: float = 0.1
    dt: float = 1.0 / 60.0
    mass: float = 1.0
    eps: float = 100.0
    # The tensile term s_corr = -k (W/W(dq))^n is added to lambda (Eq. 7),
    # and lambda has units of length^2 (Eq. 4: C is dimensionless, grad C is
    # 1/length). The workload's k = 0.1 is read in units of h^2, i.e.
    # k = 0.1 h^2 = 1e-3 m^2 at h = 0.1 m; eps = 100 m^-2 is 1/h^2 in the
    # same units. Taken as 0.1 m^2 the term outweighs lambda ~5x at the
    # lattice spacing and the dam break explodes in its first step.
    scorr_k: float = 0.001
    scorr_n: int = 4
    scorr_dq: float = 0.02                  # 0.2 h, as a distance
    xsph_c: float = 0.01
    gravity: Tuple[float, float, float] = (0.0, 0.0, -9.81)
    jitter: float = 0.001                   # U(+-0.01 h)
    n_min: int = 4
    n_max: int = 4
    lod_mode: int = LOD_FIXED
    steps: int = 20
    seed: int = 1608_04721
    camera: str = "none"                    # "none" | "fixed" | "spline"
    eye: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    wall: str = "none"                      # "none" | "oscillate_xlo"
    wall_amplitude: float = 0.5
    wall_period: float = 2.0
    rho0: Optional[float] = None            # None: the caller supplies the lattice rest density
    stabil_iters: int = 0                   # pre-stabilisation iterations (Sec. 4.3)
    stabil_s: int = 1                       # S: particles of level < S are pre-stabilised (S <= 1: none)
    obstacles: tuple = ()                   # ((kind, a, b), ...) analytic solids, see apbf_set_obstacles
    blocks: tuple = ()                      # more block corners: the lattice repeated at each (ids in order)
    target: Optional[Tuple[float, float, float]] = None  # "fixed" camera looks at this point (else +x)

    @property
    def n(self) -> int:
        return int(self.lattice[0] * self.lattice[1] * self.lattice[2]) * max(1, len(self.blocks))

    def replace(self, **kw) -> "SceneConfig":
        return dataclasses.replace(self, **kw)


def config_dam_break_4k() -> SceneConfig:
    """16x16x16 = 4096 particles, plain PBF with N = 4, 1.6 m cube, 20 steps."""
    return SceneConfig(name="pbf_dam_break_4096", lattice=(16, 16, 16), spacing=0.05,
                       block_lo=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0), box_hi=(1.6, 1.6, 1.6),
                       n_min=4, n_max=4, lod_mode=LOD_FIXED, steps=20)


def config_dam_break_131k(lod_mode: int = LOD_DTC, n_min: int = 5, n_max: int = 10) -> SceneConfig:
    """64x64x32 = 131072 particles in a 6.4x3.2x3.2 m box, camera 4 m outside
    the x = 0 end wall, N_i in 5..10 (or plain PBF with a fixed N)."""
    # Time step 0.0016 s, the paper's (Sec. 7). At 1/60 s the 1.6 m column is
    # crushed at 5..10 iterations: mean |rho/rho0 - 1| reaches 8.4 % by step 12
    # and rises, and the 128-entry neighbour lists overflow within 300 steps.
    return SceneConfig(name="apbf_dam_break_131072", lattice=(64, 64, 32), spacing=0.05,
                       block_lo=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0), box_hi=(6.4, 3.2, 3.2),
                       n_min=n_min, n_max=n_max, lod_mode=lod_mode, steps=300, dt=0.0016,
                       camera="fixed", eye=(-4.0, 1.6, 1.6))


def config_ocean_1m(lod_mode: int = LOD_DTC, n_min: int = 3, n_max: int = 15) -> SceneConfig:
    """128x128x64 = 1,048,576 particles (6.4x6.4x3.2 m) in a 9.6x6.4x4.8 m
    basin whose x_lo wall oscillates (amplitude 0.5 m, period 2 s); camera on
    a seeded closed cubic spline at z in [4.0, 4.8) m; N_i in 3..15."""
    # Time step 0.0016 s, the paper's (Sec. 7). At 1/60 s this 3.2 m deep
    # column crushed by the moving wall overflows 128 neighbours per particle
    # within 100 steps even with plain PBF and 15 iterations, and the adaptive
    # run (3 iterations at the bottom) at 1/120 s as well.
    return SceneConfig(name="apbf_ocean_1048576", lattice=(128, 128, 64), spacing=0.05,
                       block_lo=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0), box_hi=(9.6, 6.4, 4.8),
                       n_min=n_min, n_max=n_max, lod_mode=lod_mode, steps=600, dt=0.0016,
                       camera="spline", wall="oscillate_xlo")


def config_multi_dam_break_225k(lod_mode: int = LOD_DTC, n_min: int = 4, n_max: int = 8) -> SceneConfig:
    """Analogue of the paper's multi dam break (Sec. 7.3): four blocks of
    38x38x39 particles (225,264 in all) in the corners of a 6.4x6.4x3.2 m box
    around a central cone (base radius 1.2 m, height 1.6 m), N_i in 4..8 from
    a fixed camera above one corner looking at the centre, pre-stabilisation
    of the levels below 6 (two iterations), time step 0.0016 s (Sec. 7)."""
    w = 38 * 0.05
    corners = ((0.0, 0.0, 0.0), (6.4 - w, 0.0, 0.0), (0.0, 6.4 - w, 0.0), (6.4 - w, 6.4 - w, 0.0))
    cone = (3, (3.2, 3.2, 0.0), (1.2, 1.6, 0.0))  # APBF_OBSTACLE_CONE
    return SceneConfig(name="apbf_multi_dam_break_225264", lattice=(38, 38, 39), spacing=0.05,
                       block_lo=corners[0], blocks=corners, box_lo=(0.0, 0.0, 0.0), box_hi=(6.4, 6.4, 3.2),
                       n_min=n_min, n_max=n_max, lod_mode=lod_mode, steps=300, dt=0.0016, camera="fixed",
                       eye=(-2.0, -2.0, 3.5), target=(3.2, 3.2, 0.8), stabil_s=6, stabil_iters=2,
                       obstacles=(cone,))


def config_batch_256(count: int = 256, seed: int = 1608_04721, n_lo: int = 2048, n_hi: int = 65536,
                     n_min: int = 4, n_max: int = 8, steps: int = 100, dt: float = 0.0016):
    """Independent dam-break scenes for batched stepping: particle counts
    log-uniform in [n_lo, n_hi], block aspect ratio (x : y) uniform in 1..4
    with depth z = y, the block in the low-x half of a box twice its length
    and 1.5 times its height, a camera 3 m outside the box's x = 0 wall at a
    random height; N_i in n_min..n_max from the distance to the camera.
    The time step is the paper's 0.0016 s (Sec. 7): at 1/60 s the tallest
    columns (about 1.75 m) collapse within 50 steps at 4..8 iterations."""
    u = uniform01(seed, 2, 4 * count).reshape(count, 4)
    out = []
    for k in range(count):
        n_target = math.exp(math.log(n_lo) + u[k, 0] * (math.log(n_hi) - math.log(n_lo)))
        aspect = 1.0 + 3.0 * u[k, 1]
        ny = max(2, int(round((n_target / aspect) ** (1.0 / 3.0))))
        nx = max(2, int(round(aspect * ny)))
        nz = ny
        s = 0.05
        bx, by, bz = nx * s, ny * s, nz * s
        box_hi = (round(2.0 * bx + 0.1, 2), round(by + 0.1, 2), round(1.5 * bz + 0.1, 2))
        eye = (-3.0, 0.5 * box_hi[1], float(0.2 + u[k, 2] * box_hi[2]))
        out.append(SceneConfig(name=f"batch_{k:03d}", lattice=(nx, ny, nz), spacing=s, block_lo=(0.0, 0.0, 0.0),
                               box_lo=(0.0, 0.0, 0.0), box_hi=box_hi, n_min=n_min, n_max=n_max, lod_mode=LOD_DTC,
                               steps=steps, seed=seed + 7919 * (k + 1), camera="fixed", eye=eye, dt=dt))
    return out


def serve_arrivals(rate: float = 200.0, seconds: float = 60.0, templates: int = 64, seed: int = 1608_04721,
                   steps_lo: int = 30, steps_hi: int = 300):
    """Arrival schedule of a served workload: a Poisson process of the given
    rate (exponential gaps from seeded uniforms) over `seconds`; each arrival
    names a scene template (uniform over `templates`) and a step count
    (uniform integer in steps_lo..steps_hi). Returns a list of
    (arrival time in s, template index, steps)."""
    expected = int(rate * seconds * 1.5) + 64
    u = uniform01(seed, 3, 3 * expected).reshape(expected, 3)
    out = []
    t = 0.0
    for k in range(expected):
        t += -math.log(1.0 - u[k, 0]) / rate
        if t >= seconds:
            break
        out.append((t, int(u[k, 1] * templates), steps_lo + int(u[k, 2] * (steps_hi - steps_lo + 1))))
    return out


def config_serve_templates(count: int = 64, seed: int = 1608_04721 + 5):
    """Scene templates of the served workload: the batch generator's dam
    breaks with 4096..262144 particles (log-uniform) and N_i in 5..10."""
    return config_batch_256(count=count, seed=seed, n_lo=4096, n_hi=262144, n_min=5, n_max=10)


CONFIGS = {
    "dam_break_4k": config_dam_break_4k,
    "dam_break_131k": config_dam_break_131k,
    "ocean_1m": config_ocean_1m,
    "multi_dam_break_225k": config_multi_dam_break_225k,
}


def lattice_positions(cfg: SceneConfig) -> np.ndarray:
    """Block lattice p = block_lo + (i + 0.5) s + U(+-jitter) per axis (the
    same lattice at each corner of cfg.blocks, block after block, if given).

    Particle order (= particle id) is lattice order: x fastest, then y, then z.
    Three draws per particle in that order (x, y, z). Computed in float64 and
    rounded once to float32. Returns an (n, 3) float32 array.
    """
    nx, ny, nz = cfg.lattice
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    corners = cfg.blocks if cfg.blocks else (cfg.block_lo,)
    base = np.concatenate([np.asarray(c, np.float64)[None, :] + (idx + 0.5) * cfg.spacing for c in corners])
    if cfg.jitter > 0.0:
        u = uniform01(cfg.seed, 0, 3 * cfg.n).reshape(cfg.n, 3)
        base = base + (2.0 * u - 1.0) * cfg.jitter
    return base.astype(np.float32)


def make_scene(cfg: SceneConfig):
    """Initial state: positions (n,3) float32 in id order and zero velocities."""
    pos = lattice_positions(cfg)
    vel = np.zeros_like(pos)
    return pos, vel


def _spline_points(cfg: SceneConfig) -> np.ndarray:
    u = uniform01(cfg.seed, 1, 24).reshape(8, 3)
    lo = np.asarray(cfg.box_lo, np.float64)
    hi = np.asarray(cfg.box_hi, np.float64)
    pts = np.empty((8, 3))
    pts[:, 0] = lo[0] + u[:, 0] * (hi[0] - lo[0])
    pts[:, 1] = lo[1] + u[:, 1] * (hi[1] - lo[1])
    pts[:, 2] = 4.0 + u[:, 2] * 0.8
    return pts


def camera_at(cfg: SceneConfig, step: int):
    """Camera (eye, dir) for step ``step`` (0-based), float32 arrays.

    "fixed": cfg.eye looking +x. "spline": a closed uniform Catmull-Rom
    spline through 8 seeded points, traversed once every cfg.steps steps,
    looking at the initial block centre. Only the eye matters for the
    distance-to-camera LOD.
    """
    if cfg.camera == "spline":
        pts = _spline_points(cfg)
        u = (step % cfg.steps) / cfg.steps * 8.0
        k = int(math.floor(u))
        t = u - k
        p0, p1, p2, p3 = (pts[(k + d) % 8] for d in (-1, 0, 1, 2))
        t2, t3 = t * t, t * t * t
        eye = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)
        nx, ny, nz = cfg.lattice
        centre = np.asarray(cfg.block_lo) + 0.5 * cfg.spacing * np.asarray([nx, ny, nz])
        d = centre - eye
        d = d / max(np.linalg.norm(d), 1e-12)
        return eye.astype(np.float32), d.astype(np.float32)
    eye = np.asarray(cfg.eye, np.float32)
    if cfg.target is not None:
        d = np.asarray(cfg.target, np.float64) - np.asarray(cfg.eye, np.float64)
        return eye, (d / np.linalg.norm(d)).astype(np.float32)
    return eye, np.asarray([1.0, 0.0, 0.0], np.float32)


def box_at(cfg: SceneConfig, step: int):
    """Collision box (lo, hi) for step ``step``: the static box, or with the
    x_lo wall at A (1 - cos(2 pi t / T)), t = step * dt, which starts at rest."""
    lo = np.asarray(cfg.box_lo, np.float64).copy()
    hi = np.asarray(cfg.box_hi, np.float64)
    if cfg.wall == "oscillate_xlo":
        t = step * cfg.dt
        lo[0] = lo[0] + cfg.wall_amplitude * (1.0 - math.cos(2.0 * math.pi * t / cfg.wall_period))
    return lo.astype(np.float32), hi.astype(np.float32)
