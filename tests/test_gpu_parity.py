"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer stages (LOD levels, cell keys, sorted order, cell starts, neighbour
sets, active sets) must match bit-exactly; FP32 results must match the FP64
oracle within the stated tolerances:
  rho_i           relative 1e-5
  lambda_i        1e-5 * max_i |lambda_ref| (C_i ~ 0 in the interior makes a
                  per-particle relative error meaningless)
  positions       1e-5 * h after each iteration and after the step
  velocities      1e-5 * h / dt (the position tolerance over one step)
"""
import numpy as np
import pytest

import oracle
from paper_1608_04721_gb300 import apbf, build, scenes
from tests.multistep import compare_runs

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    apbf.lib()


def rest_density(cfg) -> float:
    return float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))


def make(cfg, *, eye=None, d_near=0.0, d_far=0.0, box=None, step=0, **over):
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    scene = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0, **over))
    if eye is None:
        eye = scenes.camera_at(cfg, step)[0]
    lo, hi = (scenes.box_at(cfg, step) if box is None else box)
    apbf.apbf_set_camera(scene, eye, (1.0, 0.0, 0.0), d_near, d_far)
    apbf.apbf_set_box(scene, lo, hi)
    p = oracle.make_params(cfg, rho0=r0, eye=eye, d_near=d_near, d_far=d_far, box_lo=lo, box_hi=hi,
                           **{k: v for k, v in over.items() if k in ("n_min", "n_max", "lod_mode")})
    return scene, p, x, v


def cell_coords(keys, dims):
    keys = keys.astype(np.int64)
    return np.stack([keys % dims[0], (keys // dims[0]) % dims[1], keys // (dims[0] * dims[1])], 1)


def check_stages(cfg, scene, p, x, v, *, iters=True, sample=None):
    n = cfg.n
    n_max = int(p.n_max)
    st = oracle.step(p, x, v, record=True, rec_iters=n_max if iters else 1)
    # a1-a3: levels and keys, pre-sort (= id) order
    apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_PREDICT)
    assert np.array_equal(apbf.apbf_debug_read(scene, apbf.APBF_DBG_KEYS), st.keys)
    # a4-a6 and the neighbour lists; the levels come from the reorder pass
    apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_NEIGHBORS)
    assert np.array_equal(apbf.apbf_debug_read(scene, apbf.APBF_DBG_LEVEL_PRESORT).astype(np.int32),
                          st.level_presort)
    assert np.array_equal(apbf.apbf_debug_read(scene, apbf.APBF_DBG_SORTED_IDS).astype(np.int32), st.order)
    assert np.array_equal(apbf.apbf_debug_read(scene, apbf.APBF_DBG_CELL_START), st.cell_start)
    xpred = apbf.apbf_debug_read(scene, apbf.APBF_DBG_XPRED)[:, :3]
    assert np.array_equal(xpred, st.xpred[st.order])
    cnt = apbf.apbf_debug_read(scene, apbf.APBF_DBG_NBR_COUNT).astype(np.int64)
    nbr = apbf.apbf_debug_read(scene, apbf.APBF_DBG_NBR)
    assert np.array_equal(cnt, np.diff(st.nbr_off))
    dims, _, _ = apbf.apbf_debug_dims(scene)
    cells = cell_coords(st.keys[st.order], dims)
    rows = range(n) if sample is None else sample
    for q in rows:
        e = nbr[: cnt[q], q]
        got = e.astype(np.int64)
        ref = st.nbr_idx[st.nbr_off[q]:st.nbr_off[q + 1]]
        assert np.array_equal(np.sort(got), np.sort(ref)), q
        assert np.all(np.abs(cells[got] - cells[q]) <= 1), q   # one of the 27 cells around q's
        # padding to a multiple of 4 entries: slot n (the far record)
        pad = nbr[cnt[q]: min(-(-cnt[q] // 4) * 4, nbr.shape[0]), q]
        assert np.all(pad == n), q
    lvl = st.level_presort[st.order]
    if cfg.lod_mode in (scenes.LOD_DTC, scenes.LOD_DTVS) and p.n_max > p.n_min:
        apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_LEVELS)
        lc = apbf.apbf_debug_read(scene, apbf.APBF_DBG_LEVEL_COUNT).astype(np.int64)
        assert np.array_equal(lc, st.active_count)
        # the neighbour search places each particle in the active list
        apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_NEIGHBORS)
        act = apbf.apbf_debug_read(scene, apbf.APBF_DBG_ACTIVE).astype(np.int64)
        assert np.array_equal(act, np.lexsort((np.arange(n), -lvl)))
    # a8-a9 per iteration
    h = float(p.h)
    for l in range(1, (n_max if iters else 1) + 1):
        apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_LAMBDA, l)
        lam = apbf.apbf_debug_read(scene, apbf.APBF_DBG_LAMBDA).astype(np.float64)
        rho = apbf.apbf_debug_read(scene, apbf.APBF_DBG_RHO).astype(np.float64)
        lam_ref = st.lam[l - 1]
        scale = np.abs(lam_ref).max()
        err = np.abs(lam - lam_ref).max()
        assert err <= 1e-5 * scale, f"iteration {l}: lambda error {err:.3g} vs scale {scale:.3g}"
        act = lvl >= l
        rerr = np.abs(rho[act] / st.rho[l - 1][act] - 1).max()
        assert rerr <= 1e-5, f"iteration {l}: rho relative error {rerr:.3g}"
        if not iters:
            break
        apbf.apbf_debug_step_to(scene, apbf.APBF_STAGE_DELTAP, l)
        xs = apbf.apbf_debug_read(scene, apbf.APBF_DBG_XSTAR)[:, :3].astype(np.float64)
        xerr = np.abs(xs - st.xs[l - 1]).max()
        assert xerr <= 1e-5 * h, f"iteration {l}: x* error {xerr:.3g} m"
    return st


def check_final(cfg, scene, p, st, x0=None):
    apbf.apbf_step(scene, 1)
    got = apbf.apbf_read_state(scene, pos=True, vel=True, n_iter=True)
    inv = np.argsort(st.ids)
    h = float(p.h)
    xerr = np.abs(got["pos"].astype(np.float64) - st.x[inv]).max()
    verr = np.abs(got["vel"].astype(np.float64) - st.v[inv]).max()
    assert xerr <= 1e-5 * h, f"positions after the step differ by {xerr:.3g} m"
    assert verr <= 1e-5 * h / float(p.dt), f"velocities after the step differ by {verr:.3g} m/s"
    lv, _ = oracle.lod_levels(p, scenes.make_scene(cfg)[0] if x0 is None else x0)
    assert np.array_equal(got["n_iter"].astype(np.int32), lv)
    lo, hi = np.asarray(p.box_lo[:], np.float32), np.asarray(p.box_hi[:], np.float32)
    assert np.all(got["pos"] >= lo) and np.all(got["pos"] <= hi)


SMALL = {
    "pbf_4096": lambda: (scenes.config_dam_break_4k(), {}),
    "apbf_5200": lambda: (scenes.config_dam_break_4k().replace(lattice=(20, 20, 13), lod_mode=scenes.LOD_DTC,
                                                               n_min=2, n_max=7, camera="fixed",
                                                               eye=(-1.0, 0.5, 0.3)), {}),
    "apbf_ragged_1000_user_range": lambda: (
        scenes.config_dam_break_4k().replace(lattice=(10, 10, 10), lod_mode=scenes.LOD_DTC, n_min=1, n_max=5,
                                             camera="fixed", eye=(-0.5, 0.2, 0.9)),
        dict(d_near=0.7, d_far=1.3)),
    "apbf_33": lambda: (scenes.config_dam_break_4k().replace(lattice=(11, 3, 1), lod_mode=scenes.LOD_DTC,
                                                             n_min=1, n_max=3, camera="fixed", eye=(2.0, 0.1, 0.1)),
                        {}),
    # a 30 m grid spans 1.0e9 units of 2^-25 m, so the solver takes the coarser unit 2^-24 m; the
    # block sits 25 m from the grid origin and near x = 0, where FP32 positions resolve 1e-5 h
    # (at 20 m the FP32 spacing alone is 1.9e-6 m)
    "apbf_long_grid_4096": lambda: (
        scenes.config_dam_break_4k().replace(box_lo=(-25.0, 0.0, 0.0), box_hi=(5.0, 1.6, 1.6),
                                             block_lo=(0.0, 0.0, 0.0), lod_mode=scenes.LOD_DTC, n_min=2,
                                             n_max=5, camera="fixed", eye=(-1.0, 0.8, 0.8)), {}),
}


@pytest.mark.parametrize("name", ["pbf_4096", "apbf_5200", "apbf_ragged_1000_user_range", "apbf_33"])
def test_step_counters_match_the_oracle(name):
    """apbf_get_step_info's counts, which the benchmark's roofline divides by,
    are exact: neighbour pairs = sum_i |N_i|, lambda pairs = sum_i N_i |N_i|
    (particle i visits its list in N_i lambda passes), particle-iterations =
    sum_i N_i, and |P_l| per iteration (Eq. 9-10)."""
    cfg, kw = SMALL[name]()
    scene, p, x, v = make(cfg, **kw)
    st = oracle.step(p, x, v, record=True, rec_iters=1)
    apbf.apbf_step(scene, 1)
    info = apbf.apbf_get_step_info(scene)
    deg = np.diff(st.nbr_off).astype(np.int64)          # sorted order
    lvl = st.level_presort[st.order].astype(np.int64)   # sorted order
    assert info["neighbor_pairs"] == int(deg.sum())
    assert info["lambda_pairs"] == int((deg * lvl).sum())
    assert info["particle_iterations"] == int(lvl.sum())
    n_max = int(p.n_max)
    assert np.array_equal(info["active_count"][1:n_max + 1], [int((lvl >= l).sum()) for l in range(1, n_max + 1)])
    assert not info["active_count"][n_max + 1:].any()
    apbf.apbf_destroy_scene(scene)


@pytest.mark.parametrize("name", list(SMALL))
def test_stagewise_parity_small(name):
    cfg, kw = SMALL[name]()
    scene, p, x, v = make(cfg, **kw)
    st = check_stages(cfg, scene, p, x, v)
    check_final(cfg, scene, p, st)


def test_list_capacity_not_a_multiple_of_four():
    """max_neighbors set to the step's longest list (or one more), whichever is
    not a multiple of 4: the longest lists end in a padded block inside the
    allocation, and every stage and the step still match the oracle."""
    cfg, kw = SMALL["apbf_5200"]()
    scene, p, x, v = make(cfg, **kw)
    st = oracle.step(p, x, v, record=True, rec_iters=1)
    longest = int(np.diff(st.nbr_off).max())
    cap = longest if longest % 4 else longest + 1
    scene, p, x, v = make(cfg, max_neighbors=cap, **kw)
    st = check_stages(cfg, scene, p, x, v)
    check_final(cfg, scene, p, st)


def test_one_step_parity_131k():
    cfg = scenes.config_dam_break_131k()
    scene, p, x, v = make(cfg)
    rng = np.random.default_rng(0)
    st = check_stages(cfg, scene, p, x, v, sample=rng.choice(cfg.n, 4096, replace=False))
    check_final(cfg, scene, p, st)


def test_one_step_parity_1m_bench_configuration():
    """The benchmark's workload (1,048,576 particles, N_i in 3..15, moving
    wall and spline camera) in the launch configuration the benchmark times
    (captured graph): all integer stages, sampled neighbour sets, and for
    every particle lambda and rho of each of the 15 iterations and x* after
    each, then the final state."""
    cfg = scenes.config_ocean_1m()
    scene, p, x, v = make(cfg, step=0)
    rng = np.random.default_rng(1)
    st = check_stages(cfg, scene, p, x, v, iters=True, sample=rng.choice(cfg.n, 2048, replace=False))
    check_final(cfg, scene, p, st)


def test_multi_step_density_statistics_1m_bench_configuration():
    """Five steps of the benchmark's 1,048,576-particle ocean (moving wall,
    spline camera, N_i in 3..15) against the oracle: mean, 99th and 99.9th
    percentile of |rho/rho0 - 1| within 0.2 points at every step."""
    cfg = scenes.config_ocean_1m()
    scene, p0, x, v = make(cfg, step=0)

    def params(k):
        eye, d = scenes.camera_at(cfg, k)
        lo, hi = scenes.box_at(cfg, k)
        apbf.apbf_set_camera(scene, eye, d)
        apbf.apbf_set_box(scene, lo, hi)
        return oracle.make_params(cfg, rho0=rest_density(cfg), eye=eye, box_lo=lo, box_hi=hi)

    compare_runs(scene, params, x, v, 5, strict=True)


def test_apbf_with_every_level_at_nmax_is_bitwise_pbf():
    """Eq. 9-11: with every N_i = N_max, P_l = P_1 and APBF is PBF. The camera
    range puts every particle at the nearest level, so the adaptive scene
    still runs the level partition and the compacted-list kernels."""
    base = scenes.config_dam_break_4k().replace(lattice=(16, 16, 12))
    x, v = scenes.make_scene(base)
    r0 = rest_density(base)
    a = apbf.apbf_create_scene(apbf.desc_from_config(base, x, v, r0, n_min=6, n_max=6,
                                                     lod_mode=apbf.APBF_LOD_FIXED))
    b = apbf.apbf_create_scene(apbf.desc_from_config(base, x, v, r0, n_min=2, n_max=6, lod_mode=apbf.APBF_LOD_DTC))
    apbf.apbf_set_camera(b, (-1.0, 0.3, 0.3), (1.0, 0.0, 0.0), 50.0, 60.0)
    for s in (a, b):
        apbf.apbf_step(s, 3)
    ra = apbf.apbf_read_state(a, pos=True, vel=True)
    rb = apbf.apbf_read_state(b, pos=True, vel=True)
    assert np.array_equal(ra["pos"], rb["pos"]) and np.array_equal(ra["vel"], rb["vel"])


def test_graph_replay_equals_eager_launches_bitwise():
    cfg = scenes.config_dam_break_4k().replace(lattice=(16, 16, 12), lod_mode=scenes.LOD_DTC, n_min=2, n_max=6,
                                               camera="fixed", eye=(-1.0, 0.4, 0.4))
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    g = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    e = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0, flags=apbf.APBF_FLAG_NO_GRAPH))
    for s in (g, e):
        apbf.apbf_set_camera(s, cfg.eye)
        for k in range(4):
            apbf.apbf_set_box(s, (0.02 * k, 0.0, 0.0), (1.6, 1.6, 1.6))
            apbf.apbf_step(s, 1)
    a = apbf.apbf_read_state(g, pos=True, vel=True, n_iter=True, rho=True)
    b = apbf.apbf_read_state(e, pos=True, vel=True, n_iter=True, rho=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_checkpoint_resume_is_bitwise():
    cfg = scenes.config_dam_break_4k().replace(lod_mode=scenes.LOD_DTC, n_min=2, n_max=5, camera="fixed",
                                               eye=(-1.0, 0.5, 0.5))
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    full = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    apbf.apbf_set_camera(full, cfg.eye)
    apbf.apbf_step(full, 3)
    mid = apbf.apbf_read_state(full, pos=True, vel=True)
    apbf.apbf_step(full, 4)
    end = apbf.apbf_read_state(full, pos=True, vel=True)
    res = apbf.apbf_create_scene(apbf.desc_from_config(cfg, mid["pos"], mid["vel"], r0))
    apbf.apbf_set_camera(res, cfg.eye)
    apbf.apbf_step(res, 4)
    got = apbf.apbf_read_state(res, pos=True, vel=True)
    assert np.array_equal(got["pos"], end["pos"]) and np.array_equal(got["vel"], end["vel"])


def test_multi_step_density_statistics_match_oracle():
    """20 steps of the 4096-particle dam break (chaotic, so compared by
    statistics, tests/multistep.py): mean |rho/rho0 - 1| within 0.2 points
    at every step and its 99th percentile (the robust maximum) within 0.2
    points plus the chaotic spread of the oracle itself."""
    cfg = scenes.config_dam_break_4k()
    scene, p, x, v = make(cfg)
    g, o = compare_runs(scene, p, x, v, cfg.steps)
    assert abs(g[:, 0].max() - o[:, 0].max()) <= 0.002


def test_multi_step_density_statistics_131k():
    """12 steps of the 131,072-particle APBF dam break (N_i 5..10, camera 4 m
    outside the end wall) at dt = 1/60 s against the oracle: mean, 99th and
    99.9th percentile of |rho/rho0 - 1| within 0.2 points at every step."""
    cfg = scenes.config_dam_break_131k().replace(dt=1 / 60)  # the larger step moves the flow more
    scene, p, x, v = make(cfg)
    compare_runs(scene, p, x, v, 12, strict=True)


def test_empty_scene():
    cfg = scenes.config_dam_break_4k()
    d = apbf.make_desc(pos=np.zeros((0, 3), np.float32), grid_lo=cfg.box_lo, grid_hi=cfg.box_hi, h=cfg.h, dt=cfg.dt,
                       mass=1.0, rho0=8078.2, eps=cfg.eps, scorr_k=cfg.scorr_k, scorr_dq=cfg.scorr_dq,
                       scorr_n=cfg.scorr_n, xsph_c=cfg.xsph_c, gravity=cfg.gravity, n_min=1, n_max=3,
                       lod_mode=apbf.APBF_LOD_DTC)
    s = apbf.apbf_create_scene(d)
    apbf.apbf_set_camera(s, (0, 0, 0))
    apbf.apbf_step(s, 2)
    out = apbf.apbf_read_state(s, pos=True, vel=True, n_iter=True, rho=True)
    assert out["pos"].shape == (0, 3)
    assert np.array_equal(apbf.apbf_density_stats(s), np.zeros(4))


def test_single_particle_free_fall_matches_oracle():
    cfg = scenes.config_dam_break_4k()
    x = np.array([[0.8, 0.8, 1.2]], np.float32)
    v = np.array([[0.3, 0.0, -0.5]], np.float32)
    r0 = rest_density(cfg)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    p = oracle.make_params(cfg, rho0=r0)
    for _ in range(5):
        apbf.apbf_step(s, 1)
        st = oracle.step(p, x, v)
        x, v = st.x, st.v
    got = apbf.apbf_read_state(s, pos=True, vel=True)
    assert np.abs(got["pos"] - x).max() <= 1e-6 and np.abs(got["vel"] - v).max() <= 1e-5


def test_one_cell_cluster_and_box_faces():
    """All of a cluster's particles in one cell (every pair a neighbour),
    coincident particles on the box's upper corner (last cell index, r = 0
    pairs) and particles resting on the floor."""
    cfg = scenes.config_dam_break_4k()
    rng = np.random.default_rng(3)
    x = (0.405 + 0.09 * rng.random((24, 3))).astype(np.float32)
    x[:4] = np.float32(1.6)
    x[4:8, 2] = np.float32(0.0)
    v = np.zeros_like(x)
    r0 = rest_density(cfg)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    p = oracle.make_params(cfg, rho0=r0)
    st = oracle.step(p, x, v, record=True)
    apbf.apbf_debug_step_to(s, apbf.APBF_STAGE_NEIGHBORS)
    assert np.array_equal(apbf.apbf_debug_read(s, apbf.APBF_DBG_SORTED_IDS).astype(np.int32), st.order)
    cnt = apbf.apbf_debug_read(s, apbf.APBF_DBG_NBR_COUNT).astype(np.int64)
    assert np.array_equal(cnt, np.diff(st.nbr_off))
    apbf.apbf_step(s, 1)
    got = apbf.apbf_read_state(s, pos=True, vel=True)
    inv = np.argsort(st.ids)
    err = np.abs(got["pos"] - st.x[inv]).max()
    assert err <= 1e-5 * cfg.h, err


def test_async_position_readback_equals_sync_readback():
    """Positions queued to pinned host memory while the next step runs arrive
    intact: two alternating buffers hold the same bits as a synchronous read
    of an identical scene after the same step, and a synchronous read after
    an asynchronous one is unaffected."""
    import torch

    cfg = scenes.config_dam_break_4k()
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    a = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    b = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    bufs = [torch.empty((cfg.n, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    refs = []
    for k in range(6):
        apbf.apbf_step(a, 1)
        apbf.apbf_read_positions_async(a, bufs[k % 2].data_ptr())
        apbf.apbf_step(b, 1)
        refs.append(apbf.apbf_read_state(b, pos=True, vel=False)["pos"])
        if k % 2 == 1:
            apbf.apbf_sync(a)
            assert np.array_equal(bufs[0].numpy(), refs[k - 1]), k
            assert np.array_equal(bufs[1].numpy(), refs[k]), k
    apbf.apbf_step(a, 1)
    apbf.apbf_read_positions_async(a, bufs[0].data_ptr())
    got = apbf.apbf_read_state(a, pos=True, vel=False)["pos"]
    apbf.apbf_step(b, 1)
    ref = apbf.apbf_read_state(b, pos=True, vel=False)["pos"]
    apbf.apbf_sync(a)
    assert np.array_equal(got, ref) and np.array_equal(bufs[0].numpy(), ref)
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_read_positions_async(a, 0)
    apbf.apbf_destroy_scene(a)
    apbf.apbf_destroy_scene(b)


def test_neighbor_overflow_is_reported_and_sticky():
    cfg = scenes.config_dam_break_4k()
    rng = np.random.default_rng(4)
    x = (0.8 + 0.02 * rng.random((100, 3))).astype(np.float32)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, None, rest_density(cfg), max_neighbors=16))
    apbf.apbf_step(s, 1)
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_read_state(s)
    assert e.value.status == apbf.APBF_ERR_NEIGHBOR_OVERFLOW
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_step(s, 1)
    assert e.value.status == apbf.APBF_ERR_NEIGHBOR_OVERFLOW
    # other scenes are unaffected
    y, w = scenes.make_scene(cfg.replace(lattice=(4, 4, 4)))
    ok = apbf.apbf_create_scene(apbf.desc_from_config(cfg, y, w, rest_density(cfg)))
    apbf.apbf_step(ok, 1)
    apbf.apbf_read_state(ok)


def test_moving_wall_one_step_parity_along_a_trajectory():
    """An oscillating x_lo wall (0.1 m, 0.2 s, up to 3 m/s) sweeping into the
    block at the ocean workload's time step: at several states of the
    oracle's trajectory, one GPU step from that state (scene re-created from
    it) matches the oracle's step within the one-step tolerance. (Multi-step
    runs are chaotic and are compared by statistics.)"""
    cfg = scenes.config_dam_break_4k().replace(lattice=(12, 12, 8), wall="oscillate_xlo", wall_amplitude=0.1,
                                               wall_period=0.2, dt=0.0016, lod_mode=scenes.LOD_DTC, n_min=2,
                                               n_max=5, camera="fixed", eye=(2.5, 0.4, 0.3))
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    ids = np.arange(cfg.n, dtype=np.int32)
    checked = 0
    for k in range(26):
        lo, hi = scenes.box_at(cfg, k)
        p = oracle.make_params(cfg, rho0=r0, eye=cfg.eye, box_lo=lo, box_hi=hi)
        if k in (14, 18, 22, 25):
            inv = np.argsort(ids)
            s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x[inv], v[inv], r0))
            apbf.apbf_set_box(s, lo, hi)
            apbf.apbf_set_camera(s, cfg.eye)
            apbf.apbf_step(s, 1)
            got = apbf.apbf_read_state(s, pos=True, vel=True)
            apbf.apbf_destroy_scene(s)
        st = oracle.step(p, x, v, ids)
        x, v, ids = st.x, st.v, st.ids
        if k in (14, 18, 22, 25):
            inv = np.argsort(ids)
            err = np.abs(got["pos"] - x[inv]).max()
            assert err <= 1e-5 * cfg.h, (k, err)
            assert np.all(got["pos"][:, 0] >= lo[0])
            checked += 1
    assert checked == 4 and scenes.box_at(cfg, 25)[0][0] > 0.05   # the wall has entered the block


def test_invalid_calls_on_a_live_scene():
    cfg = scenes.config_dam_break_4k().replace(lattice=(4, 4, 4))
    x, v = scenes.make_scene(cfg)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, rest_density(cfg)))
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_set_box(s, (0, 0, 0), (2.0, 1.6, 1.6))
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_set_camera(s, (np.nan, 0, 0))
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_debug_step_to(s, apbf.APBF_STAGE_LAMBDA, 99)
    apbf.apbf_step(s, 1)  # still usable
    apbf.apbf_sync(s)


def test_caller_arena_refusals_and_use():
    """A scene in caller-provided device memory: a misaligned arena is refused
    (INVALID_ARG) and a short one too (OUT_OF_MEMORY), before any device work;
    an arena of exactly apbf_scene_bytes steps bit-identically to a scene whose
    memory the library allocates."""
    import torch

    cfg = scenes.config_dam_break_4k().replace(lattice=(8, 8, 8))
    x, v = scenes.make_scene(cfg)
    desc = apbf.desc_from_config(cfg, x, v, rest_density(cfg))
    need = apbf.apbf_scene_bytes(desc)
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_scene(desc, device_arena=(base + 16, need))
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_scene(desc, device_arena=(base, need - 256))
    assert e.value.status == apbf.APBF_ERR_OUT_OF_MEMORY
    mine = apbf.apbf_create_scene(desc, device_arena=(base, need))
    lib_owned = apbf.apbf_create_scene(desc, device_arena=None)
    for s in (mine, lib_owned):
        apbf.apbf_step(s, 3)
    a = apbf.apbf_read_state(mine, pos=True, vel=True)
    b = apbf.apbf_read_state(lib_owned, pos=True, vel=True)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["vel"], b["vel"])
    apbf.apbf_destroy_scene(mine)
    apbf.apbf_destroy_scene(lib_owned)
    del buf
