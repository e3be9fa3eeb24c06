"""Pins of the oracle's DTVS adaption model (Sec. 4.1, Sec. 6) against the
geometry of a pinhole camera and of spheres, computed here independently in
float64 (nothing re-types the oracle's FP32 sequence):

  orc_view_basis     orthonormal, right-handed, forward = dir, image up toward world up
  orc_pixel_ray      float64 pinhole rays through pixel centres; the centre pixel of an
                     odd-sized image looks along dir; image x to the right, row 0 at the top
  orc_depth_image    per pixel: closed-form ray-sphere distance of the nearest sphere,
                     empty where no sphere is hit; independent of the particle order;
                     the bounding-box cull equals testing every pixel
  orc_dtvs_distance  visible particles at 0; a particle hidden behind another on the same
                     ray at the gap between them; -1 behind the camera / outside the image
  orc_lod_levels     (DTVS) visible wall at n_max, farthest hidden particle at n_min,
                     particles outside the view at n_min and outside the automatic range
"""
import math

import numpy as np
import pytest

import oracle as O

EMPTY = np.frombuffer(np.uint32(O.DEPTH_EMPTY_BITS).tobytes(), np.float32)[0]


def _params(eye, view, n_min=2, n_max=6, d_near=0.0, d_far=0.0):
    return O.make_params(None, rho0=1000.0, h=0.1, dt=0.01, mass=1.0, eps=100.0, scorr_k=0.0, scorr_dq=0.0,
                         xsph_c=0.0, scorr_n=4, gravity=(0.0, 0.0, -9.81), grid_lo=(-50.0, -50.0, -50.0),
                         grid_hi=(50.0, 50.0, 50.0), n_min=n_min, n_max=n_max, lod_mode=O.ORC_LOD_DTVS, eye=eye,
                         d_near=d_near, d_far=d_far, view=view)


def _basis64(direction, up):
    f = np.asarray(direction, np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r = r / np.linalg.norm(r)
    return f, r, np.cross(r, f)


def _ray64(view, px, py):
    f, r, u = _basis64(list(view.dir), list(view.up))
    t = float(view.tan_half_fov)
    sx = ((2 * px + 1) / view.width - 1.0) * t * view.width / view.height
    sy = (1.0 - (2 * py + 1) / view.height) * t
    d = f + sx * r + sy * u
    return d / np.linalg.norm(d)


EPS32 = 2.0 ** -24


def _hit64(ray, rel, radius):
    """Closed-form ray-sphere entry distance and the squared half chord."""
    b = float(ray @ rel)
    disc = b * b - (float(rel @ rel) - radius * radius)
    return (b - math.sqrt(disc) if disc >= 0 and b > 0 else None), disc


def _fp32_depth_bound(rel, radius, disc):
    """Error bound of an FP32 evaluation of the entry distance: a few units
    in the last place of |rel| from the dot product and the ray, plus the
    propagation of the half chord's absolute error ~ r |rel| eps through the
    square root (derivative 1 / (2 sqrt(disc)))."""
    L = float(np.linalg.norm(rel))
    return EPS32 * (8.0 * L + 12.0 * radius * L / math.sqrt(disc))


def test_basis_is_orthonormal_right_handed_and_upright():
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.normal(size=3)
        v = O.make_view(64, 48, 0.5, d, up=(0.0, 0.0, 1.0))
        f, r, u = (x.astype(np.float64) for x in O.view_basis(v))
        F = d / np.linalg.norm(d)
        assert np.allclose(f, F, atol=1e-6)
        assert abs(f @ r) < 1e-6 and abs(f @ u) < 1e-6 and abs(r @ u) < 1e-6
        assert np.allclose([f @ f, r @ r, u @ u], 1.0, atol=1e-6)
        assert np.allclose(np.cross(r, u), -f, atol=1e-6) or np.allclose(np.cross(u, r), f, atol=1e-6)
        assert abs(r[2]) < 1e-6 and u[2] > 0.0   # horizontal right axis, image up toward +z


def test_pixel_rays_are_pinhole_rays():
    v = O.make_view(33, 21, math.tan(math.radians(30)), (1.0, 0.5, -0.3))
    for px, py in [(0, 0), (32, 0), (0, 20), (32, 20), (16, 10), (7, 13)]:
        assert np.allclose(O.pixel_ray(v, px, py), _ray64(v, px, py), atol=2e-7)
    f, _, _ = O.view_basis(v)
    assert np.array_equal(O.pixel_ray(v, 16, 10), f)   # centre of an odd image: exactly forward
    # image x grows to the right, rows grow downward
    _, r, u = _basis64(list(v.dir), list(v.up))
    assert O.pixel_ray(v, 32, 10) @ r > 0 > O.pixel_ray(v, 0, 10) @ r
    assert O.pixel_ray(v, 16, 0) @ u > 0 > O.pixel_ray(v, 16, 20) @ u


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_depth_of_one_sphere_is_the_closed_form(seed):
    rng = np.random.default_rng(seed)
    eye = rng.uniform(-1, 1, size=3)
    d = rng.normal(size=3)
    v = O.make_view(80, 60, 0.4, d, radius=0.15)
    f, r, u = _basis64(d, (0, 0, 1))
    c = eye + 3.0 * f + 0.3 * rng.uniform(-1, 1) * r + 0.2 * rng.uniform(-1, 1) * u
    x = c.astype(np.float32)[None, :]
    p = _params(eye, v)
    img = O.depth_image(p, x)
    rel = x[0].astype(np.float64) - np.asarray(p.eye, np.float64)
    hits = 0
    for py in range(v.height):
        for px in range(v.width):
            t, disc = _hit64(_ray64(v, px, py), rel, float(np.float32(0.15)))
            if disc > 1e-4:
                hits += 1
                assert abs(img[py, px] - t) <= _fp32_depth_bound(rel, 0.15, disc), (px, py)
            elif disc < -1e-4:
                assert img[py, px] == EMPTY, (px, py)
    assert hits > 20


def test_depth_keeps_the_nearest_sphere_in_any_order():
    v = O.make_view(31, 31, 0.3, (0.0, 1.0, 0.0), radius=0.2)
    eye = np.zeros(3)
    x = np.array([[0.0, 5.0, 0.0], [0.0, 3.0, 0.0], [0.05, 4.0, 0.02]], np.float32)
    p = _params(eye, v)
    img = O.depth_image(p, x)
    assert abs(img[15, 15] - (3.0 - 0.2)) < 1e-6          # the front sphere's surface
    for perm in ([2, 1, 0], [1, 0, 2], [0, 2, 1]):
        assert np.array_equal(O.depth_image(p, x[perm]), img)


def test_distance_to_the_visible_surface_along_a_ray():
    v = O.make_view(31, 31, 0.3, (0.0, 1.0, 0.0), radius=0.2)
    eye = np.zeros(3)
    x = np.array([[0.0, 3.0, 0.0],      # visible
                  [0.0, 4.5, 0.0],      # hidden 1.5 m behind it on the same ray
                  [0.0, -2.0, 0.0],     # behind the camera
                  [9.0, 3.0, 0.0],      # far outside the field of view
                  [0.5, 3.0, 0.0]],     # beside the front one, in view, nothing in front
                 np.float32)
    p = _params(eye, v)
    d = O.dtvs_distance(p, x, O.depth_image(p, x))
    assert d[0] == 0.0 and d[4] == 0.0
    assert abs(d[1] - 1.5) < 1e-5
    assert d[2] == -1.0 and d[3] == -1.0


def test_dtvs_levels_of_a_wall_with_particles_behind_it():
    v = O.make_view(64, 64, 0.6, (1.0, 0.0, 0.0), radius=0.05)
    eye = np.zeros(3)
    ys, zs = np.meshgrid(np.arange(-10, 11) * 0.1, np.arange(-10, 11) * 0.1, indexing="ij")
    wall = np.stack([np.full(ys.size, 2.0), ys.ravel(), zs.ravel()], 1)   # touching spheres at x = 2
    behind = np.array([[2.5, 0.0, 0.0], [3.0, 0.3, 0.2], [4.0, -0.2, 0.1]])
    outside = np.array([[-1.0, 0.0, 0.0]])
    x = np.concatenate([wall, behind, outside]).astype(np.float32)
    p = _params(eye, v, n_min=2, n_max=6)
    lv, rng = O.lod_levels(p, x)
    nw = len(wall)
    assert np.all(lv[:nw] == 6)                 # the visible surface gets the highest level
    assert lv[nw + 2] == 2                      # farthest behind the surface: the lowest
    assert lv[nw] >= lv[nw + 1] >= lv[nw + 2]   # deeper behind the surface, lower level
    assert lv[-1] == 2                          # outside the view: n_min
    # the range ends at the deepest particle's distance behind the wall along its own pixel's ray
    # (float64: the nearest wall sphere that ray enters); the outside particle did not enter it
    c = x[nw + 2].astype(np.float64)
    f, r, u = _basis64(list(v.dir), list(v.up))
    t = float(v.tan_half_fov)
    px = int(math.floor(((c @ r) / (c @ f) / t + 1.0) * 0.5 * v.width))
    py = int(math.floor((1.0 - (c @ u) / (c @ f) / t) * 0.5 * v.height))
    ray = _ray64(v, px, py)
    hits = [h for h in (_hit64(ray, w.astype(np.float64), 0.05)[0] for w in x[:nw].astype(np.float32)) if h]
    expect = (np.linalg.norm(c) - 0.05) - min(hits)
    assert rng[0] == 0.0 and abs(rng[1] - expect) < 1e-5


def test_nothing_in_view_gives_n_min_everywhere():
    v = O.make_view(16, 16, 0.5, (-1.0, 0.0, 0.0), radius=0.05)
    x = np.random.default_rng(0).uniform(1, 2, size=(50, 3)).astype(np.float32)
    lv, rng = O.lod_levels(_params(np.zeros(3), v, n_min=3, n_max=7), x)
    assert np.all(lv == 3) and rng[0] == 0.0 and rng[1] == 0.0


def test_outside_level_option_changes_only_the_particles_outside_the_view():
    """view.outside_level gives the particles outside the view that level and
    leaves every other level and the automatic range as they are; a level
    outside n_min..n_max is refused."""
    v0 = O.make_view(64, 64, 0.6, (1.0, 0.0, 0.0), radius=0.05)
    v1 = O.make_view(64, 64, 0.6, (1.0, 0.0, 0.0), radius=0.05, outside_level=6)
    rng = np.random.default_rng(3)
    inside = np.stack([rng.uniform(2.0, 4.0, 40), rng.uniform(-0.5, 0.5, 40), rng.uniform(-0.5, 0.5, 40)], 1)
    outside = np.stack([rng.uniform(-4.0, -1.0, 10), rng.uniform(-1, 1, 10), rng.uniform(-1, 1, 10)], 1)
    x = np.concatenate([inside, outside]).astype(np.float32)
    lv0, r0 = O.lod_levels(_params(np.zeros(3), v0, n_min=2, n_max=6), x)
    lv1, r1 = O.lod_levels(_params(np.zeros(3), v1, n_min=2, n_max=6), x)
    assert np.all(lv0[40:] == 2) and np.all(lv1[40:] == 6)
    assert np.array_equal(lv0[:40], lv1[:40]) and np.array_equal(r0, r1)
    with pytest.raises(Exception):
        O.lod_levels(_params(np.zeros(3), O.make_view(64, 64, 0.6, (1.0, 0.0, 0.0), radius=0.05,
                                                      outside_level=7), n_min=2, n_max=6), x)


@pytest.mark.parametrize("seed", [0, 1])
def test_bounding_box_cull_equals_every_pixel(seed):
    rng = np.random.default_rng(seed)
    eye = np.array([-2.0, 0.3, 0.5])
    x = rng.uniform(-0.5, 0.5, size=(300, 3)).astype(np.float32)
    x[:40] += np.float32(2.0)                  # some beside the camera, partly off-image
    x[40:50, 0] -= np.float32(2.6)             # some behind the camera or straddling it
    for radius in (0.02, 0.3):
        v_box = O.make_view(48, 40, 0.7, (1.0, 0.1, -0.05), radius=radius)
        v_all = O.make_view(48, 40, 0.7, (1.0, 0.1, -0.05), radius=radius, brute_force=True)
        a = O.depth_image(_params(eye, v_box), x)
        b = O.depth_image(_params(eye, v_all), x)
        assert np.array_equal(a, b)
        assert np.any(a != EMPTY)
