"""Input generator (seeded, deterministic, shaped like the workloads) and the
Table 1 performance-improvement metric."""
import math
import os

import numpy as np

from paper_1608_04721_gb300 import metrics, scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def test_splitmix64_reference_values():
    # splitmix64 with state 0: the first outputs of the published generator
    # (state advanced by the golden gamma before mixing).
    out = S.splitmix64(np.arange(1, 4, dtype=np.uint64) * S.GOLDEN)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lattice_shape_order_and_jitter():
    cfg = S.config_dam_break_4k()
    x, v = S.make_scene(cfg)
    assert x.shape == (4096, 3) and x.dtype == np.float32 and not v.any()
    ideal = np.stack(np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij"), -1)
    ideal = ideal[..., ::-1].reshape(-1, 3) * 0.05 + 0.025    # x fastest
    dev = x.astype(np.float64) - ideal
    assert np.abs(dev).max() <= 0.001 + 1e-6 and np.abs(dev).max() > 0.0009
    assert abs(dev.mean()) < 1e-4
    x2, _ = S.make_scene(cfg)
    assert np.array_equal(x, x2)
    x3, _ = S.make_scene(cfg.replace(seed=7))
    assert not np.array_equal(x, x3)


def test_workload_sizes():
    assert S.config_dam_break_4k().n == 4096
    assert S.config_dam_break_131k().n == 131072
    assert S.config_ocean_1m().n == 1048576
    c = S.config_ocean_1m()
    x = S.lattice_positions(c.replace(lattice=(4, 4, 4)))
    assert np.all(x >= 0)


def test_scene_drivers():
    c = S.config_ocean_1m()
    lo0, hi0 = S.box_at(c, 0)
    assert lo0[0] == 0.0 and hi0[0] == np.float32(9.6)
    lo_half, _ = S.box_at(c, int(round(1.0 / c.dt)))   # t = 1 s = T/2: wall fully in
    assert abs(lo_half[0] - 1.0) < 1e-3
    eyes = np.array([S.camera_at(c, s)[0] for s in range(0, c.steps, 7)])
    assert np.all((eyes[:, 2] > 3.5) & (eyes[:, 2] < 5.3))
    e0, d0 = S.camera_at(c, 0)
    assert abs(np.linalg.norm(d0) - 1) < 1e-6
    assert np.allclose(S.camera_at(c, c.steps)[0], e0)


def test_table1_improvement_definition():
    """Every printed improvement of Table 1 equals T_PBF(N_max)/T_APBF - 1 in
    percent, rounded half up."""
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    checked = 0
    for scen in {r[0] for r in rows}:
        rs = [r for r in rows if r[0] == scen]
        pbf_max = max((r for r in rs if r[2] == "PBF"), key=lambda r: int(r[3]))
        for r in rs:
            if r[2].startswith("APBF"):
                for col, icol in ((4, 6), (5, 7)):
                    imp = metrics.improvement(float(pbf_max[col]), float(r[col]))
                    assert math.floor(100 * imp + 0.5) == int(r[icol]), (scen, r)
                    checked += 1
    assert checked == 12


def test_traffic_capture_digest_ignores_comments_only():
    """bench.py keeps a committed ncu traffic figure only while the kernel code
    is the code it was taken on: comments and blank lines do not count, a
    change to any statement does."""
    import bench

    src = "// header\n__global__ void k(float *x)\n{\n    x[0] = 1.0f;  /* one */\n}\n"
    base = bench.kernel_source_digest(src)
    assert bench.kernel_source_digest(src.replace("// header", "// another header\n\n")) == base
    assert bench.kernel_source_digest(src.replace("/* one */", "/* a longer\n comment */")) == base
    assert bench.kernel_source_digest(src.replace("1.0f", "2.0f")) != base
    assert bench.kernel_source_digest(src.replace("x[0]", "x[1]")) != base



def test_traffic_from_a_stale_or_missing_capture_is_null(tmp_path, monkeypatch):
    """A traffic figure counts only for the kernel source it was captured on:
    a capture of other code, or none at all, reads as traffic null."""
    import bench

    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1608_04721_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_1608_04721_gb300" / "csrc" / "kernels.cu").write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic("lambda_kernel", "w") is None
    digest = bench.kernel_source_digest()
    (tmp_path / "profiles" / "traffic_w.txt").write_text(
        f"# header\nlambda_kernel dram_bytes_per_launch=123 source={digest}\n"
        "deltap_kernel dram_bytes_per_launch=456 source=0000000000000000\n")
    assert bench.read_traffic("lambda_kernel", "w") == 123.0
    assert bench.read_traffic("deltap_kernel", "w") is None


def test_reference_arm_runs_the_whole_workload_with_the_same_config():
    """bench.py --impl reference times the oracle on every particle of the
    workload (no extrapolation when W + K steps fit its budget) and reports
    the CUDA arm's config dict."""
    import json
    import subprocess
    import sys

    import bench

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "dam_break_4k",
                          "--steps", "2", "--warmup", "3"], cwd=root, capture_output=True, text=True, timeout=600,
                         check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    cfg = bench.workload("dam_break_4k", "apbf")
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["config"] == bench.workload_config(cfg, bench.workload("dam_break_4k", "pbf").n_max, 1)
    assert "whole workload" in line["cpu_baseline"]["sample"] and "x " not in line["cpu_baseline"]["sample"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["value"] > 0
    assert line["e2e"]["value"] == line["value"]


def test_claimed_launches_per_step_match_the_committed_launch_list():
    """bench.py's gpu_launches (kernels per step x steps) agrees with the ncu
    launch list of the benchmark's DTC step committed under profiles/."""
    import re

    import bench

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "profiles", "launches_apbf_ocean_1048576.md"), encoding="utf-8").read()
    m = re.search(r"### DTC: (\d+) steps, (\d+) launches", text)
    assert m, "no DTC launch table in the committed launch list"
    steps, launches = int(m.group(1)), int(m.group(2))
    assert bench.kernels_per_step(bench.workload("ocean_1m", "apbf")) * steps == launches


def test_stage_roofline_units_and_default_steps():
    """The HBM stage figures use each stage's own unit (particles, cells or
    (level bin, tile) entries), and each workload times its own length by
    default."""
    import bench

    cfg = bench.workload("ocean_1m", "apbf")
    k = cfg.n_max - cfg.n_min + 1
    entries = bench.level_entries(cfg)
    assert entries == k * (((cfg.n + 255) // 256 + 3) // 4 * 4) and entries % (4 * k) == 0
    assert bench.level_entries(bench.workload("ocean_1m", "pbf")) == 0
    r = bench.stage_roofline({"predict": 0.010, "scan": 0.005, "levels": 0.002}, cfg.n, 1000, None, entries)
    st = r["stages"]
    assert st["predict"]["units"] == cfg.n and st["scan"]["units"] == 1000 and st["levels"]["units"] == entries
    assert abs(st["predict"]["achieved_gbs"] - 40 * cfg.n / 10e-6 / 1e9) < 1e-6 * st["predict"]["achieved_gbs"]
    assert "copy_us" not in st["predict"]  # no device copy timed without torch
    assert {w: bench.default_steps(w) for w in ("ocean_1m", "dam_break_131k", "dam_break_4k", "batch_256")} == {
        "ocean_1m": 600, "dam_break_131k": 300, "dam_break_4k": 20, "batch_256": 100}
