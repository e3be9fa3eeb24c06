"""Pins of the oracle's obstacle contacts (Sec. 6, the collision response of Fig. 7) and
pre-stabilisation (Sec. 4.3, the pre-stabilisation loop of Fig. 7), checked against geometry
and closed forms computed here:

  orc_obstacle_project  the projection of an interior point is the nearest point of a dense
                        sampling of the solid's surface (sphere, block, cone), within the
                        sampling resolution; points outside are left alone
  orc_step contacts     after a PBF step no particle is strictly inside an obstacle
  pre-stabilisation     a particle at rest inside an obstacle leaves it with zero velocity when
                        pre-stabilised and with the closed-form ejection speed depth/dt when not
                        (Fig. 6); a particle moving outward keeps its own velocity; only levels
                        below S are pre-stabilised; S = 1 changes nothing
"""
import math

import numpy as np
import pytest

import oracle as O

SPHERE = (O.ORC_OBSTACLE_SPHERE, (0.2, -0.1, 0.3), (0.5, 0.0, 0.0))
BLOCK = (O.ORC_OBSTACLE_BOX, (-0.3, 0.0, 0.1), (0.5, 0.4, 0.9))
CONE = (O.ORC_OBSTACLE_CONE, (0.1, 0.2, 0.0), (0.6, 0.9, 0.0))


def _surface(kind, a, b, res):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if kind == O.ORC_OBSTACLE_SPHERE:
        m = int(4 * math.pi * b[0] ** 2 / res ** 2)
        k = np.arange(m) + 0.5
        phi = np.arccos(1 - 2 * k / m)
        th = math.pi * (1 + 5 ** 0.5) * k
        return a + b[0] * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    if kind == O.ORC_OBSTACLE_BOX:
        pts = []
        for ax in range(3):
            o1, o2 = [t for t in range(3) if t != ax]
            u = np.arange(a[o1], b[o1] + res / 2, res)
            w = np.arange(a[o2], b[o2] + res / 2, res)
            U, Wg = np.meshgrid(u, w, indexing="ij")
            for face in (a[ax], b[ax]):
                P = np.zeros((U.size, 3))
                P[:, ax], P[:, o1], P[:, o2] = face, U.ravel(), Wg.ravel()
                pts.append(P)
        return np.concatenate(pts)
    R, H = b[0], b[1]
    pts = []
    for rr in np.arange(0, R + res / 2, res):                     # base disc
        m = max(1, int(2 * math.pi * rr / res))
        th = 2 * math.pi * np.arange(m) / m
        pts.append(np.stack([a[0] + rr * np.cos(th), a[1] + rr * np.sin(th), np.full(m, a[2])], 1))
    L = math.hypot(R, H)
    for t in np.arange(0, L + res / 2, res):                      # slant surface, from the rim up
        rr, zz = R * (1 - t / L), H * t / L
        m = max(1, int(2 * math.pi * rr / res))
        th = 2 * math.pi * np.arange(m) / m
        pts.append(np.stack([a[0] + rr * np.cos(th), a[1] + rr * np.sin(th), np.full(m, a[2] + zz)], 1))
    return np.concatenate(pts)


def _interior(kind, a, b, rng, count):
    a, b = np.asarray(a, float), np.asarray(b, float)
    out = []
    while len(out) < count:
        if kind == O.ORC_OBSTACLE_SPHERE:
            x = a + rng.uniform(-b[0], b[0], 3)
            ok = np.linalg.norm(x - a) < 0.98 * b[0]
        elif kind == O.ORC_OBSTACLE_BOX:
            x = rng.uniform(a, b)
            ok = True
        else:
            x = a + np.array([rng.uniform(-b[0], b[0]), rng.uniform(-b[0], b[0]), rng.uniform(0, b[1])])
            rho = math.hypot(x[0] - a[0], x[1] - a[1])
            ok = x[2] > a[2] + 0.01 and rho / b[0] + (x[2] - a[2]) / b[1] < 0.98
        if ok:
            out.append(x)
    return np.array(out)


@pytest.mark.parametrize("obst", [SPHERE, BLOCK, CONE], ids=["sphere", "block", "cone"])
def test_projection_is_the_nearest_surface_point(obst):
    kind, a, b = obst
    res = 0.006
    surf = _surface(kind, a, b, res)
    rng = np.random.default_rng(kind)
    for x in _interior(kind, a, b, rng, 60):
        inside, q = O.obstacle_project(kind, a, b, x)
        assert inside
        d_s = np.linalg.norm(surf - x, axis=1)
        # q is on the surface (a sample lies within the resolution) ...
        assert np.linalg.norm(surf - q, axis=1).min() < res
        # ... and no surface sample is nearer to x than q (beyond the resolution)
        assert np.linalg.norm(q - x) <= d_s.min() + 1e-9
        assert np.linalg.norm(q - x) >= d_s.min() - res


@pytest.mark.parametrize("obst", [SPHERE, BLOCK, CONE], ids=["sphere", "block", "cone"])
def test_points_outside_are_left_alone(obst):
    kind, a, b = obst
    rng = np.random.default_rng(7)
    surf = _surface(kind, a, b, 0.02)
    for s in surf[rng.choice(len(surf), 40, replace=False)]:
        x = s + rng.normal(size=3) * 0.0
        c = np.asarray(a, float) + (np.array([0, 0, b[1] / 3]) if kind == O.ORC_OBSTACLE_CONE else
                                    (np.asarray(b, float) - np.asarray(a, float)) / 2 * (kind == O.ORC_OBSTACLE_BOX))
        out = x + 0.05 * (x - c) / np.linalg.norm(x - c)      # pushed away from an interior point
        inside, q = O.obstacle_project(kind, a, b, out)
        if not inside:
            assert np.array_equal(q, out)
    for x in [np.array([5.0, 5.0, 5.0]), np.array([-3.0, 0.0, 0.2])]:
        inside, q = O.obstacle_project(kind, a, b, x)
        assert not inside and np.array_equal(q, x)


def _params(*, n_min, n_max, lod_mode, stabil_s, stabil_iters, obstacles, eye=(0.0, 0.0, 0.0), gravity=0.0):
    return O.make_params(None, rho0=1000.0, h=0.1, dt=0.01, mass=1.0, eps=100.0, scorr_k=0.0, scorr_dq=0.0,
                         xsph_c=0.0, scorr_n=4, gravity=(0.0, 0.0, gravity), grid_lo=(-2.0, -2.0, -2.0),
                         grid_hi=(2.0, 2.0, 2.0), n_min=n_min, n_max=n_max, lod_mode=lod_mode, eye=eye,
                         stabil_s=stabil_s, stabil_iters=stabil_iters, obstacles=obstacles)


def test_prestabilised_particle_leaves_without_ejection_velocity():
    """Fig. 6: a particle resting inside an obstacle. Without pre-stabilisation
    the contact response moves only x*, so v = depth/dt; with it, x and x*
    move together and the particle leaves at rest."""
    c, R = np.array([0.0, 0.0, 0.0]), 0.5
    x = np.array([[0.1, 0.05, 0.2]], np.float32)          # isolated: no neighbours, no Delta p
    depth = R - np.linalg.norm(x[0].astype(np.float64) - c)
    obst = [(O.ORC_OBSTACLE_SPHERE, c, (R, 0, 0))]
    for S, expect_speed in ((1, depth / 0.01), (4, 0.0)):
        p = _params(n_min=3, n_max=3, lod_mode=O.ORC_LOD_FIXED, stabil_s=S, stabil_iters=1, obstacles=obst)
        st = O.step(p, x.copy(), np.zeros_like(x))
        assert abs(np.linalg.norm(st.x[0].astype(np.float64) - c) - R) < 1e-6       # on the surface
        assert abs(np.linalg.norm(st.v[0]) - expect_speed) < 1e-3 * max(1.0, expect_speed)


def test_prestabilisation_keeps_the_particles_own_velocity():
    """A particle inside a sphere moving outward along the normal, slowly
    enough that x* is still inside: pre-stabilisation shifts x and x*
    together, so x* leaves the sphere and the particle keeps its velocity;
    without it the contact response puts x* on the surface and the particle
    is ejected at (R - |x - c|)/dt."""
    c, R, dt = np.array([0.0, 0.0, 0.0]), 0.5, 0.01
    x = np.array([[0.3, 0.0, 0.0]], np.float32)
    v0 = np.array([[5.0, 0.0, 0.0]], np.float32)          # x* = 0.35: still inside
    obst = [(O.ORC_OBSTACLE_SPHERE, c, (R, 0, 0))]
    for S, expect in ((4, 5.0), (1, (R - 0.3) / dt)):
        p = _params(n_min=3, n_max=3, lod_mode=O.ORC_LOD_FIXED, stabil_s=S, stabil_iters=1, obstacles=obst)
        st = O.step(p, x.copy(), v0.copy())
        assert abs(st.v[0, 0] - expect) < 1e-3 * expect and abs(st.v[0, 1]) + abs(st.v[0, 2]) < 1e-6
        assert np.linalg.norm(st.x[0].astype(np.float64) - c) >= R - 1e-6


def test_only_levels_below_S_are_prestabilised():
    c, R = np.array([0.0, 0.0, 0.0]), 0.6
    # two isolated particles inside the sphere; the camera near the first gives it the top level
    x = np.array([[0.0, 0.0, 0.45], [0.0, 0.0, -0.45]], np.float32)
    obst = [(O.ORC_OBSTACLE_SPHERE, c, (R, 0, 0))]
    p = _params(n_min=2, n_max=6, lod_mode=O.ORC_LOD_DTC, stabil_s=4, stabil_iters=2, obstacles=obst,
                eye=(0.0, 0.0, 1.5))
    lv, _ = O.lod_levels(p, x)
    assert lv[0] == 6 and lv[1] == 2
    st = O.step(p, x.copy(), np.zeros_like(x))
    v = st.v[np.argsort(st.ids)]
    assert np.linalg.norm(v[1]) < 1e-6                     # level 2 < S: pre-stabilised
    assert abs(np.linalg.norm(v[0]) - (R - 0.45) / 0.01) < 1e-2   # level 6 >= S: ejected


def test_S1_changes_nothing():
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.4, 0.4, size=(150, 3)).astype(np.float32)
    v = rng.normal(size=(150, 3)).astype(np.float32) * 0.1
    obst = [SPHERE, CONE]
    a = O.step(_params(n_min=2, n_max=5, lod_mode=O.ORC_LOD_DTC, stabil_s=1, stabil_iters=4, obstacles=obst,
                       eye=(1.0, 0.0, 0.0), gravity=-9.81), x.copy(), v.copy())
    b = O.step(_params(n_min=2, n_max=5, lod_mode=O.ORC_LOD_DTC, stabil_s=1, stabil_iters=0, obstacles=obst,
                       eye=(1.0, 0.0, 0.0), gravity=-9.81), x.copy(), v.copy())
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)


def test_no_particle_ends_inside_an_obstacle_after_a_pbf_step():
    """Disjoint obstacles (projections onto overlapping solids, applied one
    after the other, can push a particle from one into the next)."""
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.2, 1.2, size=(600, 3)).astype(np.float32)
    obst = [(O.ORC_OBSTACLE_SPHERE, (-0.7, 0.0, 0.0), (0.4, 0, 0)),
            (O.ORC_OBSTACLE_BOX, (0.2, -0.3, -0.3), (0.6, 0.3, 0.3)),
            (O.ORC_OBSTACLE_CONE, (0.0, 0.8, -0.5), (0.35, 0.9, 0))]
    p = _params(n_min=3, n_max=3, lod_mode=O.ORC_LOD_FIXED, stabil_s=1, stabil_iters=0, obstacles=obst,
                gravity=-9.81)
    st = O.step(p, x, np.zeros_like(x))
    for pos in st.x.astype(np.float64):
        for kind, a, b in obst:
            inside, q = O.obstacle_project(kind, a, b, pos)
            assert not inside or np.linalg.norm(q - pos) < 1e-6
