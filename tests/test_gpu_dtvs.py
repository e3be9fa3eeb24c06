"""Parity of the CUDA DTVS adaption model (Sec. 4.1, Sec. 6) with the oracle.

The depth image, each particle's distance behind the visible surface and its
level are integer decisions taken in FP32 on both sides with the same
rounded operations, so they must match bit-exactly; the step that follows
must match the oracle within the one-step tolerances of test_gpu_parity."""
import math

import numpy as np
import pytest

import oracle
from paper_1608_04721_gb300 import apbf, build, scenes
from tests.multistep import compare_runs
from tests.test_gpu_parity import check_final, check_stages, rest_density

pytestmark = pytest.mark.gpu

TAN30 = math.tan(math.radians(30.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    apbf.lib()


def make(cfg, eye, direction, view, *, d_near=0.0, d_far=0.0, flags=0, step=0):
    """view = (width, height, tan_half_fov, up, radius)"""
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    scene = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0, flags=flags))
    apbf.apbf_set_camera(scene, eye, direction, d_near, d_far)
    W, H, t, up, rad = view
    apbf.apbf_set_view(scene, W, H, t, up, rad)
    lo, hi = scenes.box_at(cfg, step)
    apbf.apbf_set_box(scene, lo, hi)
    p = oracle.make_params(cfg, rho0=r0, eye=eye, d_near=d_near, d_far=d_far, box_lo=lo, box_hi=hi,
                           view=oracle.make_view(W, H, t, direction, up=up, radius=rad))
    return scene, p, x, v


def check_lod(scene, p, x):
    """Depth image, distances and levels of the first step, bit for bit."""
    apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_REORDER)
    depth_ref = oracle.depth_image(p, x)
    depth = apbf.apbf_debug_read(scene, apbf.APBF_DBG_DEPTH)
    assert np.array_equal(depth.view(np.uint32), depth_ref.view(np.uint32))
    dist_ref = oracle.dtvs_distance(p, x, depth_ref)
    dist = apbf.apbf_debug_read(scene, apbf.APBF_DBG_LOD_DISTANCE)
    assert np.array_equal(dist.view(np.uint32), dist_ref.view(np.uint32))
    lv_ref, _ = oracle.lod_levels(p, x)
    lv = apbf.apbf_debug_read(scene, apbf.APBF_DBG_LEVEL_PRESORT).astype(np.int32)
    assert np.array_equal(lv, lv_ref)
    return depth_ref, dist_ref, lv_ref


def _dam(lattice=(20, 20, 13), n_min=2, n_max=7):
    return scenes.config_dam_break_4k().replace(lattice=lattice, lod_mode=scenes.LOD_DTVS, n_min=n_min,
                                                 n_max=n_max, camera="fixed")


CASES = {
    # oblique camera over the block: a visible top and front, hidden interior
    "oblique_5200": lambda: (_dam(), (-0.8, -0.6, 1.4), (0.8, 0.7, -0.8), (160, 120, TAN30, (0, 0, 1), 0.025)),
    # camera at the block's side, odd image, large spheres
    "side_1000_big_spheres": lambda: (_dam((10, 10, 10), 1, 5), (-1.0, 0.25, 0.25), (1.0, 0.0, 0.0),
                                      (63, 47, 0.5, (0, 0, 1), 0.06)),
    # camera inside the fluid block: spheres around the eye are not rendered,
    # particles behind the camera are outside the view
    "eye_inside_1000": lambda: (_dam((10, 10, 10), 2, 6), (0.25, 0.25, 0.25), (1.0, 0.3, 0.2),
                                (64, 64, 0.8, (0, 0, 1), 0.03)),
    # narrow view: most particles outside the image
    "narrow_view_5200": lambda: (_dam(), (-1.5, 0.5, 0.3), (1.0, 0.0, 0.0), (32, 24, 0.05, (0, 0, 1), 0.025)),
    # large spheres close to the camera: their tiles exhaust the tile-list capacity
    # (16 per particle + 65536), so many spheres take the one-block-per-sphere path
    "huge_spheres_1000": lambda: (_dam((10, 10, 10), 2, 6), (-0.35, 0.25, 0.3), (1.0, 0.05, -0.1),
                                  (512, 512, 0.9, (0, 0, 1), 0.2)),
    # a single pixel
    "one_pixel_1000": lambda: (_dam((10, 10, 10), 1, 4), (-1.0, 0.25, 0.25), (1.0, 0.0, 0.0),
                               (1, 1, 0.4, (0, 0, 1), 0.025)),
    # a very wide view (~172 degrees vertically): the corner angle is past the
    # range in which the frustum cull is used, so every sphere is binned
    "wide_view_1000": lambda: (_dam((10, 10, 10), 1, 5), (-0.06, 0.25, 0.25), (1.0, 0.1, 0.05),
                               (96, 64, 15.0, (0, 0, 1), 0.03)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dtvs_stagewise_parity(name):
    cfg, eye, direction, view = CASES[name]()
    scene, p, x, v = make(cfg, eye, direction, view)
    depth, dist, lv = check_lod(scene, p, x)
    if name != "one_pixel_1000":
        assert len(np.unique(lv)) > 1
    st = check_stages(cfg, scene, p, x, v)
    check_final(cfg, scene, p, st)


def test_dtvs_two_phase_render_after_steps_is_bitwise():
    """After a few steps the renderer draws the spheres of particles with few
    neighbours first and leaves out, tile by tile, the others that cannot come
    out in front; the image, distances and levels must still equal the
    oracle's for the same positions."""
    cfg, eye, direction, view = CASES["oblique_5200"]()
    scene, p, x, v = make(cfg, eye, direction, view)
    apbf.apbf_step(scene, 3)
    st = apbf.apbf_read_state(scene, pos=True, vel=True)
    cnt = apbf.apbf_debug_read(scene, apbf.APBF_DBG_NBR_COUNT)
    assert np.any(cnt < 28) and np.any(cnt >= 28)          # both phases have spheres
    apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_REORDER)
    ids = apbf.apbf_debug_read(scene, apbf.APBF_DBG_STATE_IDS).astype(np.int64)
    xs = st["pos"][ids]                                     # positions in the scene's state order
    depth_ref = oracle.depth_image(p, xs)
    depth = apbf.apbf_debug_read(scene, apbf.APBF_DBG_DEPTH)
    assert np.array_equal(depth.view(np.uint32), depth_ref.view(np.uint32))
    dist = apbf.apbf_debug_read(scene, apbf.APBF_DBG_LOD_DISTANCE)
    assert np.array_equal(dist.view(np.uint32), oracle.dtvs_distance(p, xs, depth_ref).view(np.uint32))
    lv = apbf.apbf_debug_read(scene, apbf.APBF_DBG_LEVEL_PRESORT).astype(np.int32)
    assert np.array_equal(lv, oracle.lod_levels(p, xs)[0])


def test_dtvs_user_distance_range():
    cfg, eye, direction, view = CASES["oblique_5200"]()
    scene, p, x, v = make(cfg, eye, direction, view, d_near=0.05, d_far=0.4)
    _, dist, lv = check_lod(scene, p, x)
    inview = dist >= 0
    assert np.all(lv[dist >= 0.4] == cfg.n_min) and np.all(lv[inview & (dist <= 0.05)] == cfg.n_max)


def test_dtvs_looking_away_gives_n_min_and_steps():
    cfg = _dam((10, 10, 10), 2, 6)
    scene, p, x, v = make(cfg, (-1.0, 0.25, 0.25), (-1.0, 0.0, 0.0), (64, 48, TAN30, (0, 0, 1), 0.025))
    _, dist, lv = check_lod(scene, p, x)
    assert np.all(dist == -1.0) and np.all(lv == 2)
    st = oracle.step(p, x, v, record=True, rec_iters=1)
    check_final(cfg, scene, p, st)


def test_dtvs_outside_level_option():
    """apbf_set_view_outside_level: particles outside a narrow view take the
    set level (bit for bit with the oracle's view.outside_level) and the step
    matches the oracle; 0 restores n_min; levels outside n_min..n_max and
    non-DTVS scenes are refused."""
    cfg, eye, direction, view = CASES["narrow_view_5200"]()
    scene, p, x, v = make(cfg, eye, direction, view)
    apbf.apbf_set_view_outside_level(scene, cfg.n_max)
    W, H, t, up, rad = view
    p.view = oracle.make_view(W, H, t, direction, up=up, radius=rad, outside_level=cfg.n_max)
    _, dist, lv = check_lod(scene, p, x)
    assert np.any(dist < 0) and np.all(lv[dist < 0] == cfg.n_max)
    st = check_stages(cfg, scene, p, x, v, iters=False)
    check_final(cfg, scene, p, st)
    for bad in (cfg.n_min - 1, cfg.n_max + 1):
        with pytest.raises(apbf.ApbfError) as e:
            apbf.apbf_set_view_outside_level(scene, bad)
        assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    apbf.apbf_destroy_scene(scene)
    scene, p, x, v = make(cfg, eye, direction, view)
    apbf.apbf_set_view_outside_level(scene, cfg.n_max)
    apbf.apbf_set_view_outside_level(scene, 0)  # back to n_min
    _, dist, lv = check_lod(scene, p, x)
    assert np.all(lv[dist < 0] == cfg.n_min)
    apbf.apbf_destroy_scene(scene)
    plain = apbf.apbf_create_scene(apbf.desc_from_config(scenes.config_dam_break_4k().replace(lattice=(4, 4, 4)),
                                                         *scenes.make_scene(scenes.config_dam_break_4k().replace(
                                                             lattice=(4, 4, 4))), rest_density(cfg)))
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_set_view_outside_level(plain, 2)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    apbf.apbf_destroy_scene(plain)


def test_dtvs_131k_one_step_parity():
    cfg = scenes.config_dam_break_131k(lod_mode=scenes.LOD_DTVS)
    eye, direction = (-4.0, 1.6, 2.6), (1.0, 0.0, -0.35)
    scene, p, x, v = make(cfg, eye, direction, (1280, 720, TAN30, (0, 0, 1), 0.025))
    check_lod(scene, p, x)
    rng = np.random.default_rng(3)
    st = check_stages(cfg, scene, p, x, v, sample=rng.choice(cfg.n, 4096, replace=False))
    check_final(cfg, scene, p, st)


def test_dtvs_one_step_parity_1m_bench_configuration():
    """The benchmark's DTVS line: the 1,048,576-particle ocean scene under its
    spline camera at 1280 x 720 with spheres of half the particle spacing:
    depth image, distances and levels bit for bit, sampled neighbour sets, the
    first iteration's lambda and rho for every particle, and the final state."""
    cfg = scenes.config_ocean_1m().replace(lod_mode=scenes.LOD_DTVS)
    eye, direction = scenes.camera_at(cfg, 0)
    view = (1280, 720, TAN30, (0, 0, 1), 0.5 * cfg.spacing)
    scene, p, x, v = make(cfg, tuple(float(a) for a in eye), tuple(float(a) for a in direction), view)
    depth, dist, lv = check_lod(scene, p, x)
    assert len(np.unique(lv)) > 3
    rng = np.random.default_rng(5)
    st = check_stages(cfg, scene, p, x, v, iters=False, sample=rng.choice(cfg.n, 2048, replace=False))
    check_final(cfg, scene, p, st)


def test_dtvs_graph_equals_eager_and_follows_camera_and_view_changes():
    cfg, eye, direction, view = CASES["oblique_5200"]()
    g, p, x, v = make(cfg, eye, direction, view)
    e, _, _, _ = make(cfg, eye, direction, view, flags=apbf.APBF_FLAG_NO_GRAPH)
    for s in (g, e):
        for k in range(4):
            apbf.apbf_set_camera(s, (eye[0] + 0.1 * k, eye[1], eye[2]), direction)
            if k == 2:
                apbf.apbf_set_view(s, 200, 100, 0.4, (0, 0, 1), 0.03)
            apbf.apbf_step(s, 1)
    a = apbf.apbf_read_state(g, pos=True, vel=True, n_iter=True)
    b = apbf.apbf_read_state(e, pos=True, vel=True, n_iter=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_dtvs_multi_step_density_statistics_match_oracle():
    """15 steps of a 5200-particle dam break under DTVS, compared by density
    statistics per step (chaotic flow, tests/multistep.py): mean within 0.2
    points, 99th percentile within 0.2 points plus the oracle's own spread."""
    cfg, eye, direction, view = CASES["oblique_5200"]()
    scene, p, x, v = make(cfg, eye, direction, view)
    compare_runs(scene, p, x, v, 15)

def test_dtvs_invalid_uses():
    cfg, eye, direction, view = CASES["side_1000_big_spheres"]()
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_step(s, 1)                         # no view yet
    assert e.value.status == apbf.APBF_ERR_BAD_STATE
    apbf.apbf_set_camera(s, eye, (0.0, 0.0, 1.0))
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_set_view(s, 64, 48, 0.5, (0, 0, 1), 0.03)   # up parallel to the direction
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    apbf.apbf_set_camera(s, eye, direction)
    for bad in [(0, 48, 0.5, (0, 0, 1), 0.03), (64, 48, 0.0, (0, 0, 1), 0.03), (64, 48, 0.5, (0, 0, 1), -1.0),
                (20000, 48, 0.5, (0, 0, 1), 0.03)]:
        with pytest.raises(apbf.ApbfError) as e:
            apbf.apbf_set_view(s, *bad)
        assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    apbf.apbf_set_view(s, 64, 48, 0.5, (0, 0, 1), 0.03)
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_set_camera(s, eye, (0.0, 0.0, -2.0))         # now parallel to the view's up
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    apbf.apbf_step(s, 2)
    # DTC scenes have no view; DTVS batches and servers are not built
    dtc = apbf.apbf_create_scene(apbf.desc_from_config(cfg.replace(lod_mode=scenes.LOD_DTC), x, v, r0))
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_set_view(dtc, 64, 48, 0.5, (0, 0, 1), 0.03)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    d = apbf.desc_from_config(cfg, x, v, r0)
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_batch([d, d])
    assert e.value.status == apbf.APBF_ERR_NOT_SUPPORTED
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_server_create(d, max_particles=10000)
    assert e.value.status == apbf.APBF_ERR_NOT_SUPPORTED
