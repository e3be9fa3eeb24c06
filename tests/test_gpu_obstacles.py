"""Parity of the CUDA obstacle contacts (the collision response of Fig. 7, Sec. 6) and
pre-stabilisation (Sec. 4.3, the pre-stabilisation loop of Fig. 7) with the oracle, with the
one-step tolerances of test_gpu_parity (positions 1e-5 h, velocities
1e-5 h / dt). The obstacles overlap the initial fluid block, so contacts
act from the first iteration and pre-stabilisation has work to do."""
import numpy as np
import pytest

import oracle
from paper_1608_04721_gb300 import apbf, build, scenes
from tests.multistep import compare_runs
from tests.test_gpu_parity import check_final, check_stages, rest_density

pytestmark = pytest.mark.gpu

S, B, C = apbf.APBF_OBSTACLE_SPHERE, apbf.APBF_OBSTACLE_BOX, apbf.APBF_OBSTACLE_CONE


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    apbf.lib()


def make(cfg, obstacles, eye=(-1.0, 0.5, 0.4)):
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    scene = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    apbf.apbf_set_camera(scene, eye)
    apbf.apbf_set_obstacles(scene, obstacles)
    p = oracle.make_params(cfg, rho0=r0, eye=eye, obstacles=obstacles)
    return scene, p, x, v


def _dam(**kw):
    base = dict(lattice=(16, 16, 12), lod_mode=scenes.LOD_FIXED, n_min=4, n_max=4, camera="fixed")
    base.update(kw)
    return scenes.config_dam_break_4k().replace(**base)


# Shallow overlaps with the block (particles at (i + 1/2) 0.05 m): a sphere dented into the x = 0 face
# near the camera, one into the far face, a cone resting on the top layer and a block cutting a thin
# slab off the y = 0 face; no particle is deeper than a lattice spacing, as when fluid reaches a
# surface (deep overlaps project whole columns of particles onto one surface point, where pairs
# nearly coincide and the spiky gradient's 1/r makes the solve ill-conditioned).
OBST = [(S, (-0.11, 0.5, 0.3), (0.15, 0, 0)), (S, (1.11, 0.3, 0.3), (0.15, 0, 0)),
        (C, (0.5, 0.5, 0.61), (0.2, 0.3, 0)), (B, (0.3, -0.1, -0.1), (0.7, 0.045, 0.2))]


def _inside_any(x, obstacles, tol=0.0):
    """Particles deeper than tol inside some obstacle (a position projected onto a surface and
    rounded to FP32 may sit a few 1e-8 m inside)."""
    def deep(p):
        for k, a, b in obstacles:
            inside, q = oracle.obstacle_project(k, a, b, p)
            if inside and np.linalg.norm(q - p) > tol:
                return True
        return False
    return sum(deep(p) for p in x.astype(np.float64))


def test_pbf_contacts_stagewise_parity():
    cfg = _dam()
    scene, p, x, v = make(cfg, OBST)
    assert _inside_any(x, OBST) > 20               # particles start inside every obstacle
    st = check_stages(cfg, scene, p, x, v)
    check_final(cfg, scene, p, st)
    pos = apbf.apbf_read_state(scene, pos=True, vel=False)["pos"]
    assert _inside_any(pos, OBST, tol=1e-6) == 0   # all were active in the last iteration


@pytest.mark.parametrize("stabil_s,iters", [(5, 1), (5, 3), (7, 2)])
def test_apbf_prestabilisation_stagewise_parity(stabil_s, iters):
    cfg = _dam(lattice=(20, 20, 13), lod_mode=scenes.LOD_DTC, n_min=2, n_max=7, stabil_s=stabil_s,
               stabil_iters=iters)
    scene, p, x, v = make(cfg, OBST)
    lv, _ = oracle.lod_levels(p, x)
    low = lv < stabil_s
    inside = np.array([any(oracle.obstacle_project(k, a, b, q)[0] for k, a, b in OBST) for q in x.astype(float)])
    assert np.any(low & inside) and np.any(~low & inside)   # both kinds of penetrating particle
    st = check_stages(cfg, scene, p, x, v)
    check_final(cfg, scene, p, st)


def test_obstacles_in_a_batch_match_each_scene_alone_bitwise():
    cfgs = [_dam(lattice=(20, 20, 13), lod_mode=scenes.LOD_DTC, n_min=2, n_max=6, stabil_s=4, stabil_iters=2),
            _dam(lattice=(12, 18, 10), lod_mode=scenes.LOD_DTC, n_min=2, n_max=6, stabil_s=4, stabil_iters=2)]
    obst = [OBST, [(S, (0.3, 0.4, -0.1), (0.14, 0, 0))]]
    r0 = rest_density(cfgs[0])
    descs, alone = [], []
    for k, c in enumerate(cfgs):
        x, v = scenes.make_scene(c)
        descs.append(apbf.desc_from_config(c, x, v, r0))
        s = apbf.apbf_create_scene(apbf.desc_from_config(c, x, v, r0))
        apbf.apbf_set_camera(s, (-1.0, 0.5, 0.4))
        apbf.apbf_set_obstacles(s, obst[k])
        apbf.apbf_step(s, 4)
        alone.append(apbf.apbf_read_state(s, pos=True, vel=True))
    batch = apbf.apbf_create_batch(descs)
    for k in range(2):
        apbf.apbf_set_camera_at(batch, k, (-1.0, 0.5, 0.4))
        apbf.apbf_set_obstacles(batch, obst[k], index=k)
    apbf.apbf_step(batch, 4)
    got = apbf.apbf_read_state(batch, pos=True, vel=True)
    o = 0
    for k, c in enumerate(cfgs):
        for f in ("pos", "vel"):
            assert np.array_equal(got[f][o:o + c.n], alone[k][f]), (k, f)
        o += c.n


def test_prestabilisation_multi_step_statistics_match_oracle():
    """12 steps with obstacles and pre-stabilisation below level 5, compared by
    density statistics per step (tests/multistep.py)."""
    cfg = _dam(lattice=(20, 20, 13), lod_mode=scenes.LOD_DTC, n_min=2, n_max=7, stabil_s=5, stabil_iters=2)
    scene, p, x, v = make(cfg, OBST)
    compare_runs(scene, p, x, v, 12)

def test_obstacle_arguments_are_validated():
    cfg = _dam()
    scene, _, _, _ = make(cfg, [])
    for bad in ([(S, (0, 0, 0), (0.0, 0, 0))], [(B, (0, 0, 0), (1, -1, 1))], [(C, (0, 0, 0), (0.2, 0.0, 0))],
                [(9, (0, 0, 0), (1, 1, 1))], [(S, (0, 0, float("nan")), (0.1, 0, 0))], [OBST[0]] * 9):
        with pytest.raises(apbf.ApbfError) as e:
            apbf.apbf_set_obstacles(scene, bad)
        assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_set_obstacles(scene, OBST, index=1)
    apbf.apbf_set_obstacles(scene, OBST)
    apbf.apbf_set_obstacles(scene, [])
    apbf.apbf_step(scene, 1)


def test_one_step_parity_multi_dam_break_225k():
    """The multi-dam-break workload (four blocks around the cone, N_i 4..8,
    pre-stabilisation below level 6) in the launch configuration the
    benchmark times: all integer stages, sampled neighbour sets, every
    iteration's lambda, rho and x*, and the final state."""
    cfg = scenes.config_multi_dam_break_225k()
    x, v = scenes.make_scene(cfg)
    # each block moved rigidly 0.54 m along both axes toward the cone, so that its inner bottom
    # corner dents the cone by at most 2.8 cm, and moving toward it at 1 m/s: contacts in the first step
    per = cfg.n // 4
    for k, (sx, sy) in enumerate([(1, 1), (-1, 1), (1, -1), (-1, -1)]):
        x[k * per:(k + 1) * per] += np.array([0.54 * sx, 0.54 * sy, 0.0], np.float32)
        v[k * per:(k + 1) * per] = np.array([0.7071 * sx, 0.7071 * sy, 0.0], np.float32)
    r0 = rest_density(cfg)
    eye, direction = scenes.camera_at(cfg, 0)
    scene = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    apbf.apbf_set_camera(scene, eye, direction)
    apbf.apbf_set_obstacles(scene, cfg.obstacles)
    p = oracle.make_params(cfg, rho0=r0, eye=eye)
    assert _inside_any(x, cfg.obstacles) > 12
    rng = np.random.default_rng(4)
    st = check_stages(cfg, scene, p, x, v, sample=rng.choice(cfg.n, 3000, replace=False))
    check_final(cfg, scene, p, st, x0=x)
