"""The debug build (libapbf_debug.so, device-side invariant checks compiled in)
on small scenes: no check fails on valid input, the checks change no result
bit (the same steps through the release library give the same state), the
stage-wise parity with the oracle holds under it, and a planted neighbour
entry past the padding record is caught and reported (APBF_ERR_CHECK_FAILED)
instead of being read. The debug library runs in a child process selected by
APBF_LIBRARY=debug, so this process keeps the release library."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1608_04721_gb300 import apbf, build, scenes
from tests.test_gpu_parity import make, rest_density

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1608_04721_gb300 import apbf, scenes
import tests.test_gpu_parity as T
assert apbf.apbf_debug_checks_enabled(), apbf.LIB_PATH
for name in ("pbf_4096", "apbf_ragged_1000_user_range"):
    cfg, kw = T.SMALL[name]()
    scene, p, x, v = T.make(cfg, **kw)
    st = T.check_stages(cfg, scene, p, x, v)
    T.check_final(cfg, scene, p, st)
cfg, kw = T.SMALL["apbf_5200"]()
scene, p, x, v = T.make(cfg, **kw)
apbf.apbf_step(scene, 3)
out = apbf.apbf_read_state(scene, pos=True, vel=True, n_iter=True)
np.savez(sys.argv[2], **out)
bad, p, x, v = T.make(cfg, **kw)
apbf.apbf_debug_plant(bad, 1)
apbf.apbf_step(bad, 1)
try:
    apbf.apbf_read_state(bad, pos=True)
    print("PLANT NOT CAUGHT")
except apbf.ApbfError as e:
    print("PLANT CAUGHT", e.status, apbf.apbf_last_error(bad))
'''


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    apbf.lib()


def test_debug_build_checks_pass_match_release_and_catch_a_planted_entry(tmp_path):
    out = tmp_path / "debug_state.npz"
    env = dict(os.environ, APBF_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "PLANT CAUGHT" in r.stdout, r.stdout
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("PLANT CAUGHT")][0]
    assert f" {apbf.APBF_ERR_CHECK_FAILED} " in line and "debug check 5" in line, line
    # the same three steps through the release library: the same bits
    assert not apbf.apbf_debug_checks_enabled()
    cfg, kw = __import__("tests.test_gpu_parity", fromlist=["SMALL"]).SMALL["apbf_5200"]()
    scene, p, x, v = make(cfg, **kw)
    apbf.apbf_step(scene, 3)
    rel = apbf.apbf_read_state(scene, pos=True, vel=True, n_iter=True)
    dbg = np.load(out)
    for k in rel:
        assert np.array_equal(rel[k], dbg[k]), k
    # the release build has no plant
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_debug_plant(scene, 1)
    assert e.value.status == apbf.APBF_ERR_NOT_SUPPORTED
