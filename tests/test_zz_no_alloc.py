"""apbf_density_stats_static: the density diagnostic for callers that may not
allocate GPU memory while they run (for example a frame loop in which a
cudaMalloc would synchronise the device and stall the frame). Its scratch is
one static device array shared by all calls, so each check runs it twice in a
row and compares every result with the oracle's density statistics and with
the scene's own apbf_density_stats, at a small size and at exactly the
documented maxima (65,536 particles, 262,144 cells)."""
import numpy as np
import pytest

import oracle
from paper_1608_04721_gb300 import apbf, build, scenes

pytestmark = pytest.mark.gpu

# the tolerance of the other GPU-vs-oracle density diagnostic checks: FP32
# density sums against FP64 (|rho/rho0 - 1| carries ~1e-6 absolute rounding)
RTOL, ATOL = 1e-5, 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    apbf.lib()


def _run_twice(cfg, grid_lo, grid_hi, step_counts):
    import torch

    x, v = scenes.make_scene(cfg)
    rho0 = float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))
    scene = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, rho0))
    p = oracle.make_params(cfg, rho0=rho0, grid_lo=grid_lo, grid_hi=grid_hi)
    stats_dev = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    for k, steps in enumerate(step_counts):
        apbf.apbf_step(scene, steps)
        ref = apbf.apbf_density_stats(scene)
        pos = apbf.apbf_read_state(scene, pos=True, vel=False)["pos"]
        pos_dev = torch.from_numpy(pos).cuda().contiguous()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        apbf.apbf_density_stats_static(pos_dev, cfg.n, cfg.h, cfg.mass, rho0, grid_lo, grid_hi, stats_dev)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        got = stats_dev.cpu().numpy()
        orc = oracle.density_stats(p, pos)
        assert ref[0] > 0
        assert np.allclose(got, orc, rtol=RTOL, atol=ATOL), (got, orc)
        assert np.allclose(got, ref, rtol=RTOL, atol=ATOL), (got, ref)
        if k > 0:
            # after the first call (which loads the module), a call reserves no device memory
            assert free_after == free_before, (free_before, free_after)
        stats_dev.fill_(-1.0)


def test_static_density_stats_match_the_oracle_twice():
    cfg = scenes.config_dam_break_4k()
    _run_twice(cfg, cfg.box_lo, cfg.box_hi, (4, 3))


def test_static_density_stats_at_the_maximum_sizes():
    """65,536 particles (the particle maximum) on a grid of 64^3 = 262,144
    cells (the cell maximum): dims = floor((6.35 - 0) / 0.1) + 1 = 64 per axis."""
    lo, hi = (0.0, 0.0, 0.0), (6.35, 6.35, 6.35)
    cfg = scenes.config_dam_break_4k().replace(lattice=(64, 32, 32), box_lo=lo, box_hi=hi)
    assert cfg.n == apbf.APBF_STATIC_MAX_PARTICLES
    dims = [int(np.floor(np.float32(np.float32(b - a) * np.float32(1.0 / np.float32(cfg.h))))) + 1
            for a, b in zip(lo, hi)]
    assert np.prod(dims) == apbf.APBF_STATIC_MAX_CELLS, dims
    _run_twice(cfg, lo, hi, (2, 2))



def test_a_warm_call_captures_into_a_cuda_graph():
    """After the first call (which loads the module and its static array), a
    call only enqueues stream work: it captures into a CUDA graph in global
    capture mode, where an allocation or a synchronising call would end the
    capture with an error, and each replay of the graph gives the oracle's
    statistics."""
    import torch

    cfg = scenes.config_dam_break_4k()
    x, _ = scenes.make_scene(cfg)
    x = np.ascontiguousarray(x, dtype=np.float32)
    rho0 = float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))
    p = oracle.make_params(cfg, rho0=rho0, grid_lo=cfg.box_lo, grid_hi=cfg.box_hi)
    orc = oracle.density_stats(p, x)
    pos_dev = torch.from_numpy(x).cuda().contiguous()
    stats_dev = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    args = (pos_dev, cfg.n, cfg.h, cfg.mass, rho0, cfg.box_lo, cfg.box_hi, stats_dev)
    apbf.apbf_density_stats_static(*args)  # the first call: module load
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="global"):
        apbf.apbf_density_stats_static(*args)
    for _ in range(2):
        stats_dev.fill_(-1.0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        got = stats_dev.cpu().numpy()
        assert np.allclose(got, orc, rtol=RTOL, atol=ATOL), (got, orc)


def test_sizes_beyond_the_static_maximum_are_rejected():
    import torch

    stats_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    pos_dev = torch.zeros(3, dtype=torch.float32, device="cuda")
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_density_stats_static(pos_dev, apbf.APBF_STATIC_MAX_PARTICLES + 1, 0.1, 1.0, 8078.2,
                                       (0, 0, 0), (1, 1, 1), stats_dev)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG and "maximum" in apbf.apbf_last_error()
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_density_stats_static(pos_dev, 1, 0.1, 1.0, 8078.2, (0, 0, 0), (100, 100, 100), stats_dev)
    # one more row of cells than the maximum grid above: 65 x 64 x 64
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_density_stats_static(pos_dev, 1, 0.1, 1.0, 8078.2, (0, 0, 0), (6.45, 6.35, 6.35), stats_dev)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG and "cells" in apbf.apbf_last_error()
    # a subnormal h: 1/h is not finite
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_density_stats_static(pos_dev, 1, 1e-40, 1.0, 8078.2, (0, 0, 0), (0, 0, 0), stats_dev)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
