"""Serving loop: scenes arrive over time, queue for room in the resident pool,
are stepped together one step per tick and leave when done. Each scene's
result must be bit-identical to the same scene stepped alone, whatever else
shared the pool with it, wherever it sat in the pool, and whether it ran
alone (the single-scene kernels) or in a batch."""
import numpy as np
import pytest

import oracle
from paper_1608_04721_gb300 import apbf, build, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    apbf.lib()


def _configs(count, seed):
    cfgs = scenes.config_batch_256(count=count, seed=seed, n_lo=400, n_hi=4000, n_min=3, n_max=7)
    out = []
    for k, c in enumerate(cfgs):
        if k % 3 == 2:  # a grid away from the origin
            c = c.replace(block_lo=(0.5, -1.0, 0.3), box_lo=(0.5, -1.0, 0.3),
                          box_hi=(c.box_hi[0] + 0.5, c.box_hi[1] - 1.0, c.box_hi[2] + 0.3),
                          eye=(c.eye[0] + 0.5, c.eye[1] - 1.0, c.eye[2]))
        out.append(c)
    return out


def _alone(desc, eye, steps):
    s = apbf.apbf_create_scene(desc)
    apbf.apbf_set_camera(s, eye)
    apbf.apbf_step(s, steps)
    st = apbf.apbf_read_state(s, pos=True, vel=True)
    apbf.apbf_destroy_scene(s)
    return st["pos"], st["vel"]


def test_each_scene_matches_itself_alone_bitwise():
    cfgs = _configs(9, 31)
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0) for c in cfgs]
    steps = [6, 3, 9, 4, 7, 2, 5, 8, 3]
    arrive = [0, 3, 3, 4, 6, 6, 7, 12, 12]   # scene 0 runs alone for three ticks
    largest = max(c.n for c in cfgs)
    srv = apbf.apbf_server_create(descs[0], max_particles=int(2.2 * largest), max_cells=4 * 10**6, max_scenes=8)
    tickets = {}
    log = []
    tick = 0
    while True:
        for k in range(len(cfgs)):
            if arrive[k] == tick:
                tickets[k] = apbf.apbf_server_submit(srv, descs[k], cfgs[k].eye, steps[k], want_pos=True,
                                                     want_vel=True)
        info = apbf.apbf_server_tick(srv)
        log.append(info)
        tick += 1
        if len(tickets) == len(cfgs) and info["resident_scenes"] == 0 and info["queued"] == 0:
            break
        assert tick < 200
    assert any(i["queued"] > 0 for i in log), "the capacity never made a request wait"
    assert any(i["resident_scenes"] == 1 for i in log) and max(i["resident_scenes"] for i in log) >= 3
    assert sum(i["admitted"] for i in log) == len(cfgs) == sum(i["completed"] for i in log)
    for k in range(len(cfgs)):
        q = apbf.apbf_server_query(srv, tickets[k])
        assert q["state"] == apbf.APBF_REQ_DONE and q["steps_done"] == steps[k]
        assert q["done_tick"] - q["admit_tick"] == steps[k]
        pos, vel = apbf.apbf_server_result(srv, tickets[k])
        ref_pos, ref_vel = _alone(descs[k], cfgs[k].eye, steps[k])
        assert np.array_equal(pos, ref_pos), k
        assert np.array_equal(vel, ref_vel), k
    # FIFO: no request was admitted before one that arrived earlier
    adm = [apbf.apbf_server_query(srv, tickets[k])["admit_tick"] for k in range(len(cfgs))]
    order = sorted(range(len(cfgs)), key=lambda k: (arrive[k], k))
    assert all(adm[a] <= adm[b] for a, b in zip(order, order[1:]))
    apbf.apbf_server_destroy(srv)


def test_serving_templates_match_alone_and_the_oracle():
    """Scenes of the served workload's own templates (4,096-262,144 particles,
    N_i 5..10, at rest, as the benchmark submits them): the smallest, the
    largest and three others served together through a pool that forces one
    to queue, each bit-identical to itself alone; the largest also against
    the oracle's step."""
    temps = scenes.config_serve_templates()
    sizes = np.array([c.n for c in temps])
    picks = [int(sizes.argmin()), int(sizes.argmax()), 5, 20, 40]
    cfgs = [temps[k] for k in picks]
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    xs = [scenes.make_scene(c)[0] for c in cfgs]
    descs = [apbf.desc_from_config(c, x, None, r0) for c, x in zip(cfgs, xs)]
    cap = sum(c.n for c in cfgs) - min(c.n for c in cfgs[1:]) // 2
    srv = apbf.apbf_server_create(descs[0], max_particles=cap, max_cells=16 * 10**6, max_scenes=8)
    steps = [3, 2, 4, 3, 2]
    t = [apbf.apbf_server_submit(srv, descs[k], cfgs[k].eye, steps[k], want_vel=True) for k in range(len(cfgs))]
    log = []
    for _ in range(40):
        info = apbf.apbf_server_tick(srv)
        log.append(info)
        if info["resident_scenes"] == 0 and info["queued"] == 0:
            break
    assert any(i["queued"] > 0 for i in log), "the capacity never made a request wait"
    for k in range(len(cfgs)):
        pos, vel = apbf.apbf_server_result(srv, t[k])
        ref_pos, ref_vel = _alone(descs[k], cfgs[k].eye, steps[k])
        assert np.array_equal(pos, ref_pos) and np.array_equal(vel, ref_vel), k
    # the largest template after its first step, against the oracle
    big = 1
    s1 = apbf.apbf_create_scene(descs[big])
    apbf.apbf_set_camera(s1, cfgs[big].eye)
    apbf.apbf_step(s1, 1)
    got = apbf.apbf_read_state(s1, pos=True, vel=True)
    p = oracle.make_params(cfgs[big], rho0=r0, eye=cfgs[big].eye)
    st = oracle.step(p, xs[big], np.zeros_like(xs[big]))
    inv = np.argsort(st.ids)
    assert np.abs(got["pos"] - st.x[inv]).max() <= 1e-5 * cfgs[big].h
    assert np.abs(got["vel"] - st.v[inv]).max() <= 1e-5 * cfgs[big].h / cfgs[big].dt
    apbf.apbf_destroy_scene(s1)
    apbf.apbf_server_destroy(srv)


def test_one_scene_after_another_reuses_the_pool():
    cfgs = _configs(3, 5)
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0) for c in cfgs]
    srv = apbf.apbf_server_create(descs[0], max_particles=max(c.n for c in cfgs), max_cells=4 * 10**6,
                                  max_scenes=1)
    t = [apbf.apbf_server_submit(srv, descs[k], cfgs[k].eye, 4 + k) for k in range(3)]
    for _ in range(40):
        info = apbf.apbf_server_tick(srv)
        assert info["resident_scenes"] <= 1
        if info["resident_scenes"] == 0 and info["queued"] == 0:
            break
    for k in range(3):
        pos, _ = apbf.apbf_server_result(srv, t[k])
        assert np.array_equal(pos, _alone(descs[k], cfgs[k].eye, 4 + k)[0]), k
    apbf.apbf_server_destroy(srv)


def test_server_rejects_what_can_never_run():
    cfgs = _configs(2, 9)
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    d0 = apbf.desc_from_config(cfgs[0], *scenes.make_scene(cfgs[0]), r0)
    srv = apbf.apbf_server_create(d0, max_particles=cfgs[0].n, max_cells=4 * 10**6, max_scenes=4)
    # more particles than the pool holds
    big = cfgs[0].replace(lattice=(cfgs[0].lattice[0] + 2,) + tuple(cfgs[0].lattice[1:]))
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_server_submit(srv, apbf.desc_from_config(big, *scenes.make_scene(big), r0), big.eye, 3)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    # other physics
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_server_submit(srv, apbf.desc_from_config(cfgs[0], *scenes.make_scene(cfgs[0]), r0, dt=0.001),
                                cfgs[0].eye, 3)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_server_submit(srv, d0, cfgs[0].eye, 0)
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_server_query(srv, 12345)
    # the server still works after rejected calls
    t = apbf.apbf_server_submit(srv, d0, cfgs[0].eye, 2)
    assert apbf.apbf_server_query(srv, t)["state"] == apbf.APBF_REQ_QUEUED
    for _ in range(4):
        apbf.apbf_server_tick(srv)
    assert apbf.apbf_server_query(srv, t)["state"] == apbf.APBF_REQ_DONE
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_server_result(srv, 777)
    apbf.apbf_server_destroy(srv)


def test_served_scenes_with_obstacles_and_prestabilisation_match_alone():
    cfgs = scenes.config_batch_256(count=4, seed=77, n_lo=500, n_hi=3000, n_min=2, n_max=6)
    cfgs = [c.replace(stabil_s=4, stabil_iters=2) for c in cfgs]
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0) for c in cfgs]
    # a sphere dented into each block's far face and a cone on its top, per scene
    obst = []
    for c in cfgs:
        nx, ny, nz = c.lattice
        w, d, hgt = nx * c.spacing, ny * c.spacing, nz * c.spacing
        obst.append([(apbf.APBF_OBSTACLE_SPHERE, (w + 0.11, 0.5 * d, 0.5 * hgt), (0.15, 0, 0)),
                     (apbf.APBF_OBSTACLE_CONE, (0.5 * w, 0.5 * d, hgt - 0.015), (0.2, 0.3, 0))])
    srv = apbf.apbf_server_create(descs[0], max_particles=sum(c.n for c in cfgs), max_cells=4 * 10**6, max_scenes=4)
    steps = [5, 3, 6, 4]
    t = [apbf.apbf_server_submit(srv, descs[k], cfgs[k].eye, steps[k], want_vel=True, obstacles=obst[k])
         for k in range(4)]
    for _ in range(20):
        info = apbf.apbf_server_tick(srv)
        if info["resident_scenes"] == 0 and info["queued"] == 0:
            break
    for k in range(4):
        pos, vel = apbf.apbf_server_result(srv, t[k])
        s = apbf.apbf_create_scene(descs[k])
        apbf.apbf_set_camera(s, cfgs[k].eye)
        apbf.apbf_set_obstacles(s, obst[k])
        apbf.apbf_step(s, steps[k])
        ref = apbf.apbf_read_state(s, pos=True, vel=True)
        assert np.array_equal(pos, ref["pos"]) and np.array_equal(vel, ref["vel"]), k
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_server_submit(srv, descs[0], cfgs[0].eye, 2, obstacles=[(9, (0, 0, 0), (1, 1, 1))])
    apbf.apbf_server_destroy(srv)


def _run_server(srv, descs, eyes, steps, arrive, crowded=()):
    """Tick until every request has left; returns (tickets, tick infos)."""
    tickets, log, tick = {}, [], 0
    while True:
        for k in range(len(descs)):
            if arrive[k] == tick:
                tickets[k] = apbf.apbf_server_submit(srv, descs[k], eyes[k], steps[k], want_pos=True, want_vel=True)
        info = apbf.apbf_server_tick(srv)
        log.append(info)
        tick += 1
        if len(tickets) == len(descs) and info["resident_scenes"] == 0 and info["queued"] == 0:
            return tickets, log
        assert tick < 400


def _alone_total_iterations(desc, eye, steps):
    s = apbf.apbf_create_scene(desc)
    apbf.apbf_set_camera(s, eye)
    apbf.apbf_step(s, steps)
    t = apbf.apbf_get_step_info(s)["total_particle_iterations"]
    apbf.apbf_destroy_scene(s)
    return t


def test_neighbour_overflow_fails_only_its_request():
    """A request whose 300 particles sit in a 2 cm cube (299 neighbours each,
    over the list capacity) fails with APBF_ERR_NEIGHBOR_OVERFLOW at its first
    step; the scenes sharing the pool with it finish bit-identical to
    themselves alone, and the server keeps serving."""
    cfgs = _configs(4, 77)
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0) for c in cfgs]
    c = cfgs[1]
    rng = np.random.default_rng(5)
    lo = np.asarray(c.box_lo, np.float64) + 0.3
    xc = (lo + 0.02 * rng.random((300, 3))).astype(np.float32)
    bad = apbf.desc_from_config(c, xc, None, r0)
    descs.insert(2, bad)
    eyes = [cc.eye for cc in cfgs]
    eyes.insert(2, c.eye)
    steps = [5, 6, 4, 7, 3]
    arrive = [0, 0, 1, 1, 2]
    srv = apbf.apbf_server_create(descs[0], max_particles=60000, max_cells=4 * 10**6, max_scenes=8)
    tickets, log = _run_server(srv, descs, eyes, steps, arrive)
    assert sum(i["failed"] for i in log) == 1
    q = apbf.apbf_server_query(srv, tickets[2])
    assert q["state"] == apbf.APBF_REQ_FAILED and q["status"] == apbf.APBF_ERR_NEIGHBOR_OVERFLOW
    assert q["done_tick"] == q["admit_tick"] + 1
    for k in (0, 1, 3, 4):
        q = apbf.apbf_server_query(srv, tickets[k])
        assert q["state"] == apbf.APBF_REQ_DONE and q["status"] == apbf.APBF_OK, k
        pos, vel = apbf.apbf_server_result(srv, tickets[k])
        ref_pos, ref_vel = _alone(descs[k], eyes[k], steps[k])
        assert np.array_equal(pos, ref_pos) and np.array_equal(vel, ref_vel), k
    # still serving after the failure
    t = apbf.apbf_server_submit(srv, descs[0], eyes[0], 2)
    for _ in range(4):
        apbf.apbf_server_tick(srv)
    assert apbf.apbf_server_query(srv, t)["state"] == apbf.APBF_REQ_DONE
    apbf.apbf_server_destroy(srv)


def test_latency_target_limits_residency_and_keeps_results():
    """With a step-latency target far below any step, admission keeps one
    scene resident at a time (a request is always admitted into an empty
    pool); the results are still each scene's own, and the pool's running
    total of particle-iterations is exactly the sum of the scenes' totals
    alone."""
    cfgs = _configs(5, 91)
    r0 = float(np.float32(oracle.rest_density(cfgs[0].h, cfgs[0].mass, cfgs[0].spacing)))
    descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0) for c in cfgs]
    eyes = [c.eye for c in cfgs]
    steps = [4, 3, 5, 2, 3]
    arrive = [0, 0, 0, 1, 1]
    srv = apbf.apbf_server_create(descs[0], max_particles=60000, max_cells=4 * 10**6, max_scenes=8,
                                  target_step_ms=1e-6)
    tickets, log = _run_server(srv, descs, eyes, steps, arrive)
    assert max(i["resident_scenes"] for i in log) == 1
    assert all(i["particle_limit"] < 60000 for i in log)
    for k in range(len(cfgs)):
        pos, vel = apbf.apbf_server_result(srv, tickets[k])
        ref_pos, ref_vel = _alone(descs[k], eyes[k], steps[k])
        assert np.array_equal(pos, ref_pos) and np.array_equal(vel, ref_vel), k
    total = sum(_alone_total_iterations(descs[k], eyes[k], steps[k]) for k in range(len(cfgs)))
    assert log[-1]["total_particle_iterations"] == total
    apbf.apbf_server_destroy(srv)
    # without a target the same arrivals share the pool
    srv = apbf.apbf_server_create(descs[0], max_particles=60000, max_cells=4 * 10**6, max_scenes=8)
    tickets, log = _run_server(srv, descs, eyes, steps, arrive)
    assert max(i["resident_scenes"] for i in log) >= 3
    assert log[-1]["total_particle_iterations"] == total
    apbf.apbf_server_destroy(srv)


def test_running_particle_iterations_equal_the_per_step_counts():
    """apbf_step_info.total_particle_iterations is the sum of every step's
    particle_iterations (sum_l |P_l|, Eq. 10); the autotuner's trial steps do
    not count."""
    c = _configs(1, 5)[0]
    r0 = float(np.float32(oracle.rest_density(c.h, c.mass, c.spacing)))
    s = apbf.apbf_create_scene(apbf.desc_from_config(c, *scenes.make_scene(c), r0))
    apbf.apbf_set_camera(s, c.eye)
    total = 0
    for k in range(6):
        apbf.apbf_step(s, 1)
        info = apbf.apbf_get_step_info(s)
        total += info["particle_iterations"]
        assert info["total_particle_iterations"] == total
        if k == 2:
            apbf.apbf_autotune(s, 2)
            assert apbf.apbf_get_step_info(s)["total_particle_iterations"] == total
    assert total > c.n * c.n_min
    apbf.apbf_destroy_scene(s)
