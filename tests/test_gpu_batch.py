"""Batched stepping: independent scenes of uneven sizes stepped together,
one launch per stage over all of them.

A scene inside a batch must evolve bit-identically to the same scene stepped
alone (the per-scene arithmetic and order do not change), and each scene of a
batch must match the oracle's step within the one-step tolerances."""
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


def rest_density(cfg) -> float:
    return float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))


def _batch_configs(count, seed):
    cfgs = scenes.config_batch_256(count=count, seed=seed, n_lo=300, n_hi=6000)
    # shift some grids away from the origin so that scene geometry differs beyond the size
    out = []
    for k, c in enumerate(cfgs):
        if k % 3 == 1:
            c = c.replace(block_lo=(1.0, -0.5, 0.25), box_lo=(1.0, -0.5, 0.25),
                          box_hi=(c.box_hi[0] + 1.0, c.box_hi[1] - 0.5, c.box_hi[2] + 0.25),
                          eye=(c.eye[0] + 1.0, c.eye[1] - 0.5, c.eye[2]))
        out.append(c)
    return out


def _drive(s, k, cfg, step, index=None):
    eye = np.asarray(cfg.eye, np.float32)
    lo, hi = np.asarray(cfg.box_lo, np.float32), np.asarray(cfg.box_hi, np.float32)
    lo = lo.copy()
    lo[0] = lo[0] + np.float32(0.01 * step * (k % 2))   # a wall moving in odd scenes
    if index is None:
        apbf.apbf_set_camera(s, eye)
        apbf.apbf_set_box(s, lo, hi)
    else:
        apbf.apbf_set_camera_at(s, index, eye)
        apbf.apbf_set_box_at(s, index, lo, hi)
    return eye, lo, hi


def test_scenes_in_a_batch_match_the_same_scenes_alone_bitwise():
    cfgs = _batch_configs(7, 11)
    r0 = rest_density(cfgs[0])
    descs, states = [], []
    for c in cfgs:
        x, v = scenes.make_scene(c)
        descs.append(apbf.desc_from_config(c, x, v, r0))
    batch = apbf.apbf_create_batch(descs)
    alone = [apbf.apbf_create_scene(d) for d in descs]
    for step in range(6):
        for k, c in enumerate(cfgs):
            _drive(batch, k, c, step, index=k)
            _drive(alone[k], k, c, step)
        apbf.apbf_step(batch, 1)
        for a in alone:
            apbf.apbf_step(a, 1)
    got = apbf.apbf_read_state(batch, pos=True, vel=True, n_iter=True, rho=True)
    off = 0
    for k, a in enumerate(alone):
        ref = apbf.apbf_read_state(a, pos=True, vel=True, n_iter=True, rho=True)
        n = cfgs[k].n
        for f in ref:
            assert np.array_equal(got[f][off:off + n], ref[f]), (k, f)
        off += n
    assert off == batch.n
    info = apbf.apbf_get_step_info(batch)
    for key in ("particle_iterations", "neighbor_pairs", "lambda_pairs"):
        assert info[key] == sum(apbf.apbf_get_step_info(a)[key] for a in alone), key



def test_deep_and_regular_solver_kernels_agree_bitwise():
    """A scene with fewer particles than the solver kernels hold resident
    threads is stepped by their deep-batch variants (two entry blocks of
    gathers in flight per thread); a batch of ~400k particles by the regular
    ones. The variants visit the same pairs in the same order, so each scene
    in the batch keeps the bits it has alone."""
    cfgs = scenes.config_batch_256(count=48, seed=5, n_lo=6000, n_hi=12000)
    assert sum(c.n for c in cfgs) > 2 * 152 * 5 * 256 and max(c.n for c in cfgs) < 152 * 3 * 256
    r0 = rest_density(cfgs[0])
    descs = []
    for c in cfgs:
        x, v = scenes.make_scene(c)
        descs.append(apbf.desc_from_config(c, x, v, r0))
    batch = apbf.apbf_create_batch(descs)
    alone = [apbf.apbf_create_scene(d) for d in descs]
    for step in range(3):
        for k, c in enumerate(cfgs):
            _drive(batch, k, c, step, index=k)
            _drive(alone[k], k, c, step)
        apbf.apbf_step(batch, 1)
        for a in alone:
            apbf.apbf_step(a, 1)
    got = apbf.apbf_read_state(batch, pos=True, vel=True, rho=True)
    off = 0
    for k, a in enumerate(alone):
        ref = apbf.apbf_read_state(a, pos=True, vel=True, rho=True)
        n = cfgs[k].n
        for f in ref:
            assert np.array_equal(got[f][off:off + n], ref[f]), (k, f)
        off += n
        apbf.apbf_destroy_scene(a)
    apbf.apbf_destroy_scene(batch)


def test_each_scene_of_a_batch_matches_the_oracle_after_one_step():
    cfgs = _batch_configs(4, 23)
    r0 = rest_density(cfgs[0])
    descs, inputs = [], []
    for c in cfgs:
        x, v = scenes.make_scene(c)
        descs.append(apbf.desc_from_config(c, x, v, r0))
        inputs.append((x, v))
    batch = apbf.apbf_create_batch(descs)
    params = []
    for k, c in enumerate(cfgs):
        eye, lo, hi = _drive(batch, k, c, 3, index=k)
        params.append(oracle.make_params(c, rho0=r0, eye=eye, box_lo=lo, box_hi=hi))
    apbf.apbf_step(batch, 1)
    got = apbf.apbf_read_state(batch, pos=True, vel=True, n_iter=True)
    off = 0
    for k, c in enumerate(cfgs):
        x, v = inputs[k]
        st = oracle.step(params[k], x, v)
        inv = np.argsort(st.ids)
        n = c.n
        assert np.abs(got["pos"][off:off + n] - st.x[inv]).max() <= 1e-5 * c.h, k
        assert np.abs(got["vel"][off:off + n] - st.v[inv]).max() <= 1e-5 * c.h / c.dt, k
        lv, _ = oracle.lod_levels(params[k], x)
        assert np.array_equal(got["n_iter"][off:off + n].astype(np.int32), lv), k
        off += n


def test_full_size_batch_256_sampled_scenes_match_the_oracle():
    """The benchmark's batch (256 dam breaks of 2,048-65,536 particles, 4.8 M
    in all, seeded as the benchmark's rank 0) stepped once as one graph: the
    smallest, the largest and two other scenes match the oracle's step."""
    cfgs = scenes.config_batch_256(seed=1608_04721)
    r0 = rest_density(cfgs[0])
    inputs = [scenes.make_scene(c) for c in cfgs]
    batch = apbf.apbf_create_batch([apbf.desc_from_config(c, x, v, r0) for c, (x, v) in zip(cfgs, inputs)])
    for k, c in enumerate(cfgs):
        apbf.apbf_set_camera_at(batch, k, c.eye)
    apbf.apbf_step(batch, 1)
    got = apbf.apbf_read_state(batch, pos=True, vel=True, n_iter=True)
    offs = np.concatenate([[0], np.cumsum([c.n for c in cfgs])])
    sizes = np.array([c.n for c in cfgs])
    picks = sorted({int(sizes.argmin()), int(sizes.argmax()), 17, 200})
    for k in picks:
        c = cfgs[k]
        x, v = inputs[k]
        p = oracle.make_params(c, rho0=r0, eye=c.eye)
        st = oracle.step(p, x, v)
        inv = np.argsort(st.ids)
        a, b = offs[k], offs[k + 1]
        assert np.abs(got["pos"][a:b] - st.x[inv]).max() <= 1e-5 * c.h, k
        assert np.abs(got["vel"][a:b] - st.v[inv]).max() <= 1e-5 * c.h / c.dt, k
        lv, _ = oracle.lod_levels(p, x)
        assert np.array_equal(got["n_iter"][a:b].astype(np.int32), lv), k
    apbf.apbf_destroy_scene(batch)


def test_batch_graph_replay_equals_eager_and_density_aggregates():
    cfgs = _batch_configs(5, 3)
    r0 = rest_density(cfgs[0])
    descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0) for c in cfgs]
    eager_descs = [apbf.desc_from_config(c, *scenes.make_scene(c), r0, flags=apbf.APBF_FLAG_NO_GRAPH) for c in cfgs]
    g = apbf.apbf_create_batch(descs)
    e = apbf.apbf_create_batch(eager_descs)
    for s in (g, e):
        for k, c in enumerate(cfgs):
            _drive(s, k, c, 0, index=k)
        apbf.apbf_step(s, 3)
    a = apbf.apbf_read_state(g, pos=True, vel=True)
    b = apbf.apbf_read_state(e, pos=True, vel=True)
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["vel"], b["vel"])
    # aggregate density statistics equal the oracle's over all scenes' positions
    stats = apbf.apbf_density_stats(g)
    rhos, off = [], 0
    for c in cfgs:
        p = oracle.make_params(c, rho0=r0)
        _, rho = oracle.density_stats(p, a["pos"][off:off + c.n], want_rho=True)
        rhos.append(rho)
        off += c.n
    e_all = np.concatenate(rhos) / np.float32(r0) - 1.0
    ref = [np.abs(e_all).mean(), np.abs(e_all).max(), e_all.mean(), np.maximum(e_all, 0).mean()]
    assert np.allclose(stats, ref, rtol=1e-5, atol=1e-6), (stats, ref)


def test_tuning_choices_do_not_change_results_and_autotune_restores_the_state():
    cfg = scenes.config_dam_break_131k(n_min=3, n_max=9).replace(lattice=(40, 24, 16))
    x, v = scenes.make_scene(cfg)
    r0 = rest_density(cfg)
    ref = None
    for block, thr in ((256, 2.0), (128, 2.0), (256, 0.0), (128, 0.6), (256, 0.85)):
        s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
        apbf.apbf_set_camera(s, cfg.eye)
        apbf.apbf_set_tuning(s, block, thr)
        apbf.apbf_step(s, 4)
        got = apbf.apbf_read_state(s, pos=True, vel=True, rho=True)
        if ref is None:
            ref = got
        for f in ref:
            assert np.array_equal(got[f], ref[f]), (block, thr, f)
    s = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, r0))
    apbf.apbf_set_camera(s, cfg.eye)
    res = apbf.apbf_autotune(s, 2)
    assert len(res["trials"]) == 10 and res["block"] in (128, 256)
    assert res["ms_per_step"] == min(t[2] for t in res["trials"])
    apbf.apbf_step(s, 4)
    got = apbf.apbf_read_state(s, pos=True, vel=True, rho=True)
    for f in ref:
        assert np.array_equal(got[f], ref[f]), f
