"""The C-ABI library loads and exports every entry point include/apbf.h
declares; host-only calls (no GPU) behave as documented."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1608_04721_gb300 import apbf, build, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "apbf.h")).read()
    return sorted(set(re.findall(r"APBF_API\s+[\w\s\*]+?\b(apbf_\w+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) == 38
    for path in (apbf.LIB_PATH, build.LIB_DEBUG):   # the release and the debug-check library
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                             check=True).stdout
        exported = set(re.findall(r"\bT\s+(apbf_\w+)", out))
        assert set(names) <= exported, path
        assert exported <= set(names), f"{path} exports symbols the header does not declare"
    assert sorted(apbf.EXPORTS) == names
    L = apbf.lib()
    for nm in names:
        assert getattr(L, nm) is not None


def test_rest_density_matches_closed_form():
    rho = apbf.apbf_rest_density(0.1, 1.0, 0.05)
    # FP32 h and spacing: compare with the lattice shell closed form at those values
    h, s = float(np.float32(0.1)), float(np.float32(0.05))
    closed = 315 / (64 * math.pi * h ** 9) * sum(
        m * (h * h - q * s * s) ** 3 for m, q in ((1, 0), (6, 1), (12, 2), (8, 3)))
    assert abs(rho - closed) / closed < 1e-12
    assert abs(rho - 8078.2013351575) / 8078.2 < 1e-6
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_rest_density(-1.0, 1.0, 0.05)


def _desc(**over):
    cfg = scenes.config_dam_break_4k().replace(lattice=(4, 4, 4))
    x, v = scenes.make_scene(cfg)
    kw = dict(rho0=8078.2)
    kw.update(over)
    return apbf.desc_from_config(cfg, over.pop("pos", x), v, **kw)


def test_scene_bytes_scale_with_particles():
    b1 = apbf.apbf_scene_bytes(_desc())
    cfg = scenes.config_ocean_1m()
    x = np.zeros((1048576, 3), np.float32) + 1.0
    d = apbf.desc_from_config(cfg, x, None, 8078.2)
    b2 = apbf.apbf_scene_bytes(d)
    assert b1 > 0 and b2 > 100 * b1
    # about 0.6 kB per particle with 128 neighbour slots, well inside 280 GB
    assert 400 * 1048576 < b2 < 1200 * 1048576


@pytest.mark.parametrize("over,status", [
    (dict(h=0.0), apbf.APBF_ERR_INVALID_ARG),
    (dict(dt=-1.0), apbf.APBF_ERR_INVALID_ARG),
    (dict(rho0=0.0), apbf.APBF_ERR_INVALID_ARG),
    (dict(n_min=0), apbf.APBF_ERR_INVALID_ARG),
    (dict(n_min=5, n_max=4), apbf.APBF_ERR_INVALID_ARG),
    (dict(n_max=256), apbf.APBF_ERR_INVALID_ARG),
    (dict(lod_mode=9), apbf.APBF_ERR_INVALID_ARG),
    (dict(stabil_s=9, stabil_iters=2), apbf.APBF_ERR_INVALID_ARG),
    (dict(stabil_s=2, stabil_iters=65), apbf.APBF_ERR_INVALID_ARG),
    (dict(max_neighbors=300), apbf.APBF_ERR_INVALID_ARG),
    (dict(box_lo=(-1.0, 0.0, 0.0)), apbf.APBF_ERR_INVALID_ARG),
    (dict(scorr_dq=0.2), apbf.APBF_ERR_INVALID_ARG),
    (dict(flags=8), apbf.APBF_ERR_INVALID_ARG),
])
def test_invalid_descriptions_are_rejected_on_the_host(over, status):
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_scene(_desc(**over), stream=0, device_arena=None)
    assert e.value.status == status
    assert apbf.apbf_last_error()


def test_non_finite_or_outside_positions_are_rejected():
    cfg = scenes.config_dam_break_4k().replace(lattice=(4, 4, 4))
    x, v = scenes.make_scene(cfg)
    x[3, 1] = np.nan
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, 8078.2), stream=0, device_arena=None)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG
    x[3, 1] = 5.0  # outside the 1.6 m grid
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_scene(apbf.desc_from_config(cfg, x, v, 8078.2), stream=0, device_arena=None)
    assert "outside" in apbf.apbf_last_error()


def test_status_strings():
    assert apbf.apbf_status_string(0) == "ok"
    assert "overflow" in apbf.apbf_status_string(apbf.APBF_ERR_NEIGHBOR_OVERFLOW)


def test_batch_validation_on_the_host():
    cfg = scenes.config_dam_break_4k().replace(lattice=(4, 4, 4))
    x, v = scenes.make_scene(cfg)
    a = apbf.desc_from_config(cfg, x, v, 8078.2)
    b = apbf.desc_from_config(cfg, x, v, 8078.2, eps=50.0)
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_create_batch([a, b], stream=0, device_arena=None)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG and "scene 1" in apbf.apbf_last_error()
    c = apbf.desc_from_config(cfg.replace(box_hi=(2.0, 1.6, 1.6)), x, v, 8078.2)
    assert apbf.apbf_batch_bytes([a, c]) > apbf.apbf_batch_bytes([a])
    with pytest.raises(apbf.ApbfError):
        apbf.apbf_create_batch([], stream=0, device_arena=None)


def test_server_capacity_from_budget():
    phys = _desc()
    b_small, n_small, c_small = apbf.apbf_server_bytes(phys, budget_bytes=1 << 30)
    b_big, n_big, c_big = apbf.apbf_server_bytes(phys, budget_bytes=150 * 10**9)
    # the largest particle capacity that fits: one more particle no longer fits
    assert b_small <= 1 << 30 and n_small > 0 and c_small == 4 * n_small
    over, _, _ = apbf.apbf_server_bytes(phys, max_particles=n_small + 1)
    assert over > 1 << 30
    # the whole 150 GB budget is usable (about 200 M particles): one more particle no longer fits
    assert n_big > 150 * 10**6 and b_big <= 150 * 10**9 and b_big > 149 * 10**9
    assert apbf.apbf_server_bytes(phys, max_particles=n_big + 1)[0] > 150 * 10**9
    # explicit capacities; bytes grow with each of them
    b1, n1, c1 = apbf.apbf_server_bytes(phys, max_particles=100000, max_cells=50000, max_scenes=16)
    assert (n1, c1) == (100000, 50000)
    assert apbf.apbf_server_bytes(phys, max_particles=200000, max_cells=50000, max_scenes=16)[0] > b1
    assert apbf.apbf_server_bytes(phys, max_particles=100000, max_cells=90000, max_scenes=16)[0] > b1


@pytest.mark.parametrize("kw,status", [
    (dict(), apbf.APBF_ERR_INVALID_ARG),                                   # neither capacity nor budget
    (dict(budget_bytes=1000), apbf.APBF_ERR_OUT_OF_MEMORY),                # not even one particle
    (dict(max_particles=(1 << 31) - 1), apbf.APBF_ERR_INVALID_ARG),        # beyond the slot space
    (dict(max_particles=1000, max_scenes=70000), apbf.APBF_ERR_INVALID_ARG),
    (dict(max_particles=10**7, budget_bytes=10**6), apbf.APBF_ERR_OUT_OF_MEMORY),
])
def test_server_bytes_rejects(kw, status):
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_server_bytes(_desc(), **kw)
    assert e.value.status == status


def test_server_bytes_rejects_bad_physics():
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_server_bytes(_desc(h=0.0), max_particles=1000)
    assert e.value.status == apbf.APBF_ERR_INVALID_ARG


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of include/apbf.h, compiled by the host C compiler, has the
    size and field offsets of its ctypes mirror in the binding."""
    import ctypes
    import subprocess

    structs = [apbf.apbf_scene_desc, apbf.apbf_step_info, apbf.apbf_obstacle, apbf.apbf_tune_result,
               apbf.apbf_server_desc, apbf.apbf_request, apbf.apbf_tick_info, apbf.apbf_request_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "apbf.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                    check=True).stdout.splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(st, f).offset, (name, f)


def test_a_long_grid_steps_alone_but_not_in_a_batch():
    """A grid spanning 8e8 or more fixed-point units on an axis (here 30 m at
    h = 0.1, 1.0e9 units of 2^-25 m) takes a coarser unit when the scene is
    alone; a batch shares the unit its h gives, so such a scene is refused
    there (host-only sizing calls, no GPU)."""
    cfg = scenes.config_dam_break_4k().replace(lattice=(4, 4, 4))
    x, v = scenes.make_scene(cfg)
    a = apbf.desc_from_config(cfg, x, v, 8078.2)
    long_cfg = cfg.replace(box_hi=(30.0, 1.6, 1.6))
    b = apbf.desc_from_config(long_cfg, x, v, 8078.2)
    assert apbf.apbf_scene_bytes(b) > 0
    assert apbf.apbf_batch_bytes([b]) > 0          # a batch of one is the scene alone
    with pytest.raises(apbf.ApbfError) as e:
        apbf.apbf_batch_bytes([a, b])
    assert e.value.status == apbf.APBF_ERR_NOT_SUPPORTED and "scene 1" in apbf.apbf_last_error()
    # 23.8 m (7.99e8 units) still shares the unit
    ok = apbf.desc_from_config(cfg.replace(box_hi=(23.8, 1.6, 1.6)), x, v, 8078.2)
    assert apbf.apbf_batch_bytes([a, ok]) > 0
