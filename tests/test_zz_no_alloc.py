"""apbf_density_stats_static: the density diagnostic for callers that may not
allocate GPU memory while they run (for example a frame loop in which a
cudaMalloc would synchronise the device and stall the frame). Its scratch is
one static device array shared by all calls, so the check runs it twice in a
row and compares each result with the scene's own apbf_density_stats."""
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


def test_static_density_stats_match_the_scene_entry_point_twice():
    import torch

    cfg = scenes.config_dam_break_4k()
    x, v = scenes.make_scene(cfg)
    rho0 = float(np.float32(oracle.rest_density(cfg.h, cfg.mass, cfg.spacing)))
    scene = apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, rho0))
    stats_dev = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    for steps in (4, 3):
        apbf.apbf_step(scene, steps)
        ref = apbf.apbf_density_stats(scene)
        pos = apbf.apbf_read_state(scene, pos=True, vel=False)["pos"]
        pos_dev = torch.from_numpy(pos).cuda().contiguous()
        apbf.apbf_density_stats_static(pos_dev, cfg.n, cfg.h, cfg.mass, rho0, cfg.box_lo, cfg.box_hi, stats_dev)
        torch.cuda.synchronize()
        got = stats_dev.cpu().numpy()
        assert ref[0] > 0
        assert np.allclose(got, ref, rtol=1e-5, atol=1e-6), (got, ref)


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
