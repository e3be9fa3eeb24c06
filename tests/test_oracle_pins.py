"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here re-types an oracle formula: each check is a closed form derived
independently, an invariant, a special case that reduces to a textbook
result, or brute force. What pins each oracle function:

  orc_poly6            normalisation (quadrature), second moment 3h^2/11, W(0)
  orc_spiky            normalisation (quadrature)
  orc_spiky_grad       finite differences of orc_spiky; zero at r = h and r = 0
  orc_rest_density     lattice shell closed form 315/(64 pi h^3) * 5.15625
  orc_constraint       rho = rho0 and lambda = 0 inside a jitter-free lattice;
                       gradients vs finite differences of C; lambda makes the
                       linearised constraint vanish (Eq. 2-4) when eps = 0
  orc_delta_p          sum_i dp_i = 0 (pairwise antisymmetry); equals Eq. 3
                       summed over the constraints; tensile term at r = dq
  orc_xsph             uniform field unchanged; momentum conserved; damping
  orc_neighbors        O(N^2) brute force (FP32 predicate) on <= 512 particles
  orc_cell_keys        each particle lies in its cell's box; key range
  orc_counting_sort    equals a stable argsort; cell starts = searchsorted
  orc_lod_levels       end points, monotonicity, equal-width bins, constant
                       level when n_min = n_max
  orc_view_basis, orc_pixel_ray, orc_depth_image, orc_dtvs_distance and the
                       DTVS levels: tests/test_oracle_dtvs_pins.py (pinhole and
                       sphere geometry in float64, occlusion, culling = brute force)
  orc_predict/orc_step isolated particle in free fall (closed form); clamp
                       keeps the box; APBF with every N_i = N_max is PBF;
                       nested active sets; finished particles stay fixed;
                       interior of a jitter-free lattice unchanged; a
                       finished neighbour enters Eq. 7 with its last lambda
                       (two-particle closed form that also tells the zero
                       and recompute-all options apart)
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_1608_04721_gb300 import scenes as S

H = 0.1


# ------------------------------------------------------------------ kernels

def test_poly6_normalisation_and_moments():
    norm, _ = integrate.quad(lambda r: 4 * math.pi * r * r * O.poly6(r * r, H), 0, H, epsabs=1e-14)
    assert abs(norm - 1.0) < 1e-10
    # second moment of (h^2 - r^2)^3 normalised: int r^2 W dV = 3 h^2 / 11
    m2, _ = integrate.quad(lambda r: 4 * math.pi * r ** 4 * O.poly6(r * r, H), 0, H, epsabs=1e-16)
    assert abs(m2 - 3 * H * H / 11) < 1e-12
    # value at the origin, 315 / (64 pi h^3)
    assert abs(O.poly6(0.0, H) - 1566.6814710608) < 1e-9
    assert O.poly6(H * H, H) == 0.0 and O.poly6(2 * H * H, H) == 0.0


def test_spiky_normalisation():
    norm, _ = integrate.quad(lambda r: 4 * math.pi * r * r * O.spiky(r, H), 0, H, epsabs=1e-14)
    assert abs(norm - 1.0) < 1e-10


def test_spiky_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = d * rng.uniform(0.05 * H, 0.95 * H)
        g = O.spiky_grad(r, H)
        fd = np.zeros(3)
        e = 1e-7
        for a in range(3):
            rp, rm = r.copy(), r.copy()
            rp[a] += e
            rm[a] -= e
            fd[a] = (O.spiky(np.linalg.norm(rp), H) - O.spiky(np.linalg.norm(rm), H)) / (2 * e)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-3)
    assert np.all(O.spiky_grad(np.array([H, 0, 0]), H) == 0)
    assert np.all(O.spiky_grad(np.zeros(3), H) == 0)
    # magnitude next to the origin: 45 / (pi h^6) * h^2
    g = O.spiky_grad(np.array([1e-12, 0, 0]), H)
    assert abs(-g[0] - 45 / (math.pi * H ** 6) * H * H) / (45 / (math.pi * H ** 4)) < 1e-9


def test_rest_density_closed_form(rho0_lattice):
    # neighbours of a lattice point with spacing s = h/2 strictly inside h sit
    # at |offset|^2 in {0, 1, 2, 3} s^2 with multiplicities 1, 6, 12, 8.
    closed = 315 / (64 * math.pi * H ** 3) * (1 + 6 * 0.75 ** 3 + 12 * 0.5 ** 3 + 8 * 0.25 ** 3)
    assert abs(closed - 8078.2013351575) < 1e-8
    assert abs(rho0_lattice - closed) < 1e-8


# ------------------------------------------------------- constraint, lambda

def _params(**kw):
    base = dict(h=H, dt=1 / 60, mass=1.0, eps=100.0, scorr_k=0.001, scorr_dq=0.02, xsph_c=0.01,
                scorr_n=4, gravity=(0, 0, 0), grid_lo=(-1, -1, -1), grid_hi=(3, 3, 3), n_min=1,
                n_max=1, lod_mode=O.ORC_LOD_FIXED)
    rho0 = kw.pop("rho0", O.rest_density(H, 1.0, 0.05))
    base.update(kw)
    return O.make_params(None, rho0=rho0, **base)


def _cluster(n=60, seed=0, spread=0.12):
    rng = np.random.default_rng(seed)
    return (1.0 + rng.uniform(-spread, spread, size=(n, 3))).astype(np.float32)


def test_interior_lattice_particle_at_rest_density(rho0_lattice):
    g = np.arange(9) * 0.05 + 0.5
    z, y, xx = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([xx.ravel(), y.ravel(), z.ravel()], 1)       # exact FP64 lattice
    p = _params()
    off, idx = O.neighbors(p, x.astype(np.float32))
    centre = 4 + 9 * (4 + 9 * 4)
    rho, C, _, lam = O.constraint(p, x, off, idx, centre)
    # the solver's h is the FP32 value of 0.1
    ref = 315 / (64 * math.pi * p.h ** 9) * sum(
        m * (p.h ** 2 - q * 0.0025) ** 3 for m, q in ((1, 0), (6, 1), (12, 2), (8, 3)))
    assert abs(rho - ref) / ref < 1e-12 and abs(ref - rho0_lattice) / ref < 1e-7
    # rho0 reaches the solver as FP32, so C carries its rounding (~3e-8)
    assert abs(C) < 1e-7 and abs(lam) < 1e-9


def _spiky_constraint(p, x, off, idx, i):
    """C_i evaluated with the spiky kernel (the kernel whose gradient Eq. 4 and
    Eq. 7 use, following PBF): sum_j m spiky(|x_i - x_j|) / rho0 over the
    fixed neighbour set plus the self term, minus 1."""
    s = O.spiky(0.0, p.h)
    for j in idx[off[i]:off[i + 1]]:
        s += O.spiky(float(np.linalg.norm(x[i] - x[j])), p.h)
    return p.mass * s / p.rho0 - 1.0


def test_constraint_gradient_matches_finite_differences():
    """grad_k C_i is the exact gradient of the spiky-kernel density constraint
    (PBF evaluates rho with poly6 and its gradient with spiky)."""
    x = _cluster().astype(np.float64)
    p = _params()
    off, idx = O.neighbors(p, x.astype(np.float32))
    checked = 0
    e = 1e-7
    for i in range(0, len(x), 7):
        _, _, grad, _ = O.constraint(p, x, off, idx, i)
        members = [i] + list(idx[off[i]:off[i + 1]])
        for slot, k in enumerate(members[:6]):
            for a in range(3):
                xp, xm = x.copy(), x.copy()
                xp[k, a] += e
                xm[k, a] -= e
                fd = (_spiky_constraint(p, xp, off, idx, i) - _spiky_constraint(p, xm, off, idx, i)) / (2 * e)
                assert abs(grad[slot, a] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, k, a)
                checked += 1
    assert checked > 100


def test_lambda_zeroes_the_linearised_constraint():
    """Eq. 2-4: moving every particle k by lambda_i w grad_k C_i changes the
    linearised constraint by -C_i when eps = 0 (the slope is measured on the
    constraint whose gradient is used, the spiky one)."""
    x = _cluster(seed=5).astype(np.float64)
    p = _params(eps=0.0)
    off, idx = O.neighbors(p, x.astype(np.float32))
    for i in (0, 11, 23, 42):
        _, C, grad, lam = O.constraint(p, x, off, idx, i)
        members = [i] + list(idx[off[i]:off[i + 1]])
        step = np.zeros_like(x)
        for slot, k in enumerate(members):
            step[k] += lam * (1.0 / p.mass) * grad[slot]
        s = 1e-4
        c0 = _spiky_constraint(p, x, off, idx, i)
        c1 = _spiky_constraint(p, x + s * step, off, idx, i)
        c2 = _spiky_constraint(p, x + 2 * s * step, off, idx, i)
        slope = (4 * (c1 - c0) - (c2 - c0)) / (2 * s)  # Richardson, O(s^2)
        assert abs(slope + C) <= 1e-6 * max(abs(C), 1e-3), (i, slope, C)


def test_delta_p_sums_to_zero():
    x = _cluster(n=120, seed=9).astype(np.float64)
    p = _params(scorr_k=0.001)
    off, idx = O.neighbors(p, x.astype(np.float32))
    lam = np.random.default_rng(1).uniform(-2e-3, 5e-3, size=len(x))
    dp = O.delta_p(p, x, lam, off, idx)
    scale = np.abs(dp).sum()
    assert scale > 0
    assert np.all(np.abs(dp.sum(axis=0)) <= 1e-12 * scale)


def test_delta_p_equals_eq3_summed_over_constraints():
    """dp_i = w sum_c lambda_c grad_i C_c (Eq. 3 for every density constraint c)."""
    x = _cluster(n=80, seed=2).astype(np.float64)
    p = _params(scorr_k=0.0)
    off, idx = O.neighbors(p, x.astype(np.float32))
    lam = np.random.default_rng(4).uniform(-2e-3, 5e-3, size=len(x))
    dp = O.delta_p(p, x, lam, off, idx)
    ref = np.zeros_like(x)
    for c in range(len(x)):
        _, _, grad, _ = O.constraint(p, x, off, idx, c)
        members = [c] + list(idx[off[c]:off[c + 1]])
        for slot, k in enumerate(members):
            ref[k] += lam[c] * (1.0 / p.mass) * grad[slot]
    assert np.allclose(dp, ref, rtol=1e-10, atol=1e-15)


def test_tensile_term_at_dq():
    """Two particles at distance dq with lambda = 0: the tensile term equals
    -k and pushes them apart by k |grad W(dq)| / rho0 each."""
    p = _params(scorr_k=0.001, scorr_n=4, scorr_dq=0.02)
    x = np.array([[1.0, 1.0, 1.0], [1.02, 1.0, 1.0]])
    off = np.array([0, 1, 2], np.int32)
    idx = np.array([1, 0], np.int32)
    dp = O.delta_p(p, x, np.zeros(2), off, idx)
    g = O.spiky_grad(x[0] - x[1], H)
    expect = 0.001 * np.linalg.norm(g) / p.rho0
    assert dp[0, 0] < 0 and dp[1, 0] > 0
    assert abs(abs(dp[0, 0]) - expect) <= 1e-6 * expect
    assert np.allclose(dp[0], -dp[1])


def test_xsph_invariants():
    x = _cluster(n=70, seed=7).astype(np.float64)
    p = _params()
    off, idx = O.neighbors(p, x.astype(np.float32))
    u = np.tile([0.3, -1.2, 2.0], (len(x), 1))
    assert np.allclose(O.xsph(p, x, u, off, idx), u, atol=1e-15)
    v = np.random.default_rng(8).normal(size=x.shape)
    out = O.xsph(p, x, v, off, idx)
    assert np.allclose(out.sum(axis=0), v.sum(axis=0), atol=1e-12)
    # damping: for two approaching particles the relative speed shrinks
    x2 = np.array([[1.0, 1.0, 1.0], [1.05, 1.0, 1.0]])
    v2 = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    o2 = O.xsph(p, x2, v2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))
    assert 0 < o2[0, 0] < 1.0 and -1.0 < o2[1, 0] < 0


# ---------------------------------------------------- grid, sort, neighbours

def _brute_neighbors(x: np.ndarray, h: float):
    x = x.astype(np.float32)
    h2 = np.float32(h) * np.float32(h)
    d = x[:, None, :] - x[None, :, :]          # float32 ops
    r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]
    r2 = r2 + d[..., 2] * d[..., 2]
    m = r2 < h2
    np.fill_diagonal(m, False)
    return [np.nonzero(m[i])[0] for i in range(len(x))]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_neighbors_equal_brute_force(seed):
    cfg = S.config_dam_break_4k().replace(lattice=(8, 8, 8), seed=seed)
    x, _ = S.make_scene(cfg)          # 512 particles, many pairs within 0.01h of r = h
    x = x + np.float32(0.013 * seed)
    p = _params(grid_lo=(0, 0, 0), grid_hi=(1.6, 1.6, 1.6))
    off, idx = O.neighbors(p, x)
    ref = _brute_neighbors(x, H)
    near = 0
    for i in range(len(x)):
        got = idx[off[i]:off[i + 1]]
        assert np.array_equal(got, ref[i]), i
        near += np.sum(np.abs(np.linalg.norm(x[got] - x[i], axis=1) - H) < 1e-3)
    assert near > 100


def test_cell_keys_geometry():
    cfg = S.config_dam_break_4k()
    x, _ = S.make_scene(cfg)
    p = _params(grid_lo=(0, 0, 0), grid_hi=(1.6, 1.6, 1.6))
    dims = O.grid_dims(p)
    keys = O.cell_keys(p, x).astype(np.int64)
    assert keys.max() < dims.prod()
    cx = keys % dims[0]
    cy = (keys // dims[0]) % dims[1]
    cz = keys // (dims[0] * dims[1])
    c = np.stack([cx, cy, cz], 1).astype(np.float64)
    lo = np.asarray(p.grid_lo[:], np.float64)
    xd = x.astype(np.float64)
    slack = 1e-6
    assert np.all(xd >= lo + c * H - slack) and np.all(xd < lo + (c + 1) * H + slack)


def test_counting_sort_is_stable_argsort():
    rng = np.random.default_rng(0)
    keys = rng.integers(0, 50, size=2000).astype(np.uint32)
    order, start = O.counting_sort(keys, 50)
    assert np.array_equal(order, np.argsort(keys, kind="stable"))
    assert np.array_equal(start, np.searchsorted(np.sort(keys), np.arange(51)).astype(np.uint32))
    assert start[-1] == len(keys)


# ------------------------------------------------------------------ LOD

def test_lod_levels_bins():
    n = 1000
    x = np.zeros((n, 3), np.float32)
    x[:, 0] = np.linspace(1.0, 5.0, n, dtype=np.float32)
    p = _params(lod_mode=O.ORC_LOD_DTC, n_min=3, n_max=15, eye=(0, 0, 0))
    lv, rng = O.lod_levels(p, x)
    assert lv[0] == 15 and lv[-1] == 3
    assert np.all(np.diff(lv) <= 0)
    counts = np.bincount(lv, minlength=16)[3:16]
    assert counts.min() >= n // 13 - 2 and counts.max() <= n // 13 + 2
    assert abs(rng[0] - 1.0) < 1e-6 and abs(rng[1] - 5.0) < 1e-6
    # n_min == n_max: constant; fixed mode: n_max
    lv2, _ = O.lod_levels(_params(lod_mode=O.ORC_LOD_DTC, n_min=7, n_max=7), x)
    assert np.all(lv2 == 7)
    lv3, _ = O.lod_levels(_params(lod_mode=O.ORC_LOD_FIXED, n_min=2, n_max=9), x)
    assert np.all(lv3 == 9)
    # user range: closer than d_near -> n_max, farther than d_far -> n_min
    lv4, _ = O.lod_levels(_params(lod_mode=O.ORC_LOD_DTC, n_min=3, n_max=15, d_near=2.0, d_far=3.0), x)
    assert np.all(lv4[x[:, 0] < 2.0] == 15) and np.all(lv4[x[:, 0] > 3.0] == 3)


# ------------------------------------------------------------------ step

def test_isolated_particle_free_fall():
    p = _params(gravity=(0, 0, -9.81), n_max=4)
    x = np.array([[1.0, 1.0, 1.5]], np.float32)
    v = np.array([[0.5, 0.0, -1.0]], np.float32)
    st = O.step(p, x, v, want_final64=True)
    dt = np.float32(1 / 60)
    vz = np.float32(-1.0) + dt * np.float32(-9.81)
    xz = np.float32(1.5) + dt * vz
    xx = np.float32(1.0) + dt * np.float32(0.5)
    assert st.x[0, 2] == xz and st.x[0, 0] == xx
    assert abs(st.v_final[0, 2] - (float(xz) - 1.5) / float(dt)) < 1e-12
    assert abs(st.v[0, 2] - float(vz)) < 1e-5


def test_clamp_keeps_particles_in_the_box():
    cfg = S.config_dam_break_4k().replace(lattice=(8, 8, 8))
    x, v = S.make_scene(cfg)
    v[:] = np.float32(-20.0)
    p = O.make_params(cfg, rho0=O.rest_density(H, 1, 0.05), box_lo=(0.1, 0, 0))
    st = O.step(p, x, v)
    assert np.all(st.x >= np.asarray(p.box_lo[:], np.float32)) and np.all(st.x <= np.asarray(p.box_hi[:], np.float32))


def test_apbf_with_all_levels_at_nmax_is_pbf(rho0_lattice):
    cfg = S.config_dam_break_4k().replace(lattice=(10, 10, 10))
    x, v = S.make_scene(cfg)
    pf = O.make_params(cfg, rho0=rho0_lattice, n_min=6, n_max=6, lod_mode=O.ORC_LOD_FIXED)
    pa = O.make_params(cfg, rho0=rho0_lattice, n_min=6, n_max=6, lod_mode=O.ORC_LOD_DTC, eye=(-2, 0.5, 0.5))
    a = O.step(pf, x, v, want_final64=True)
    b = O.step(pa, x, v, want_final64=True)
    assert np.array_equal(a.x_final, b.x_final) and np.array_equal(a.v_final, b.v_final)
    assert np.array_equal(a.ids, b.ids)


def test_active_sets_nested_and_finished_particles_fixed(rho0_lattice):
    cfg = S.config_dam_break_4k().replace(lattice=(12, 12, 12))
    x, v = S.make_scene(cfg)
    p = O.make_params(cfg, rho0=rho0_lattice, n_min=2, n_max=7, lod_mode=O.ORC_LOD_DTC, eye=(-1.0, 0.3, 0.3))
    st = O.step(p, x, v, record=True, rec_iters=7)
    ac = st.active_count
    assert ac[0] == ac[1] == len(x) and np.all(np.diff(ac[1:]) <= 0) and ac[-1] == 0
    lvl = st.level_presort[st.order]
    assert len(np.unique(lvl)) == 6
    for L in range(2, 7):
        sel = lvl == L
        for l in range(L, 7):
            assert np.array_equal(st.xs[l][sel], st.xs[L - 1][sel])
        # and they did move while active
        assert not np.array_equal(st.xs[L - 1][sel], st.xs[L - 2][sel])


def test_zero_gravity_lattice_interior_unchanged(rho0_lattice):
    """Jitter-free lattice, no gravity, one iteration: lambda is nonzero only
    within 2 spacings of the surface, so dp is nonzero only within 4; the
    tensile and XSPH terms cancel by symmetry in the interior."""
    # h = 1/8 and spacing 1/16 make every FP32 lattice coordinate exact, so the
    # lattice is exactly symmetric
    cfg = S.config_dam_break_4k().replace(jitter=0.0, gravity=(0, 0, 0), block_lo=(0.25, 0.25, 0.25),
                                          box_hi=(2.5, 2.5, 2.5), h=0.125, spacing=0.0625, scorr_dq=0.025)
    x, v = S.make_scene(cfg)
    p = O.make_params(cfg, rho0=O.rest_density(0.125, 1.0, 0.0625), n_min=1, n_max=1)
    st = O.step(p, x, v, want_final64=True)
    x0 = x[st.ids].astype(np.float64)
    lat = np.rint((x0 - 0.25) / 0.0625 - 0.5).astype(int)
    depth = np.minimum(lat, 15 - lat).min(axis=1)
    inner = depth >= 4
    assert inner.sum() == 8 ** 3
    assert np.abs(st.x_final[inner] - x0[inner]).max() < 1e-12
    assert np.abs(st.x_final[depth == 0] - x0[depth == 0]).max() > 1e-4
    assert np.abs(st.v_final[depth >= 6]).max() < 1e-9


# ------------------------------------------- lambda of finished neighbours

def _two_particle_step(p, xa: float, xb: float, lam_b_second: str):
    """Closed form of one step of two particles on the x axis, particle a of
    level 2 and b of level 1, written out from Eq. 4-7 for the scalar case
    (no gravity, no velocity, box far away). Returns (x_a, x_b) after the step.

    lam_b_second says which lambda of b enters a's correction in iteration 2,
    where b is no longer active: 'stale' (b's lambda of iteration 1, the
    reading the compensation of Sec. 4.2 / Fig. 5 needs), 'zero', or
    'recompute' (b's lambda at the positions of iteration 2)."""
    h = float(p.h)
    m = float(p.mass)
    w = 1.0 / m
    rho0 = float(p.rho0)
    eps = float(p.eps)
    k = float(p.scorr_k)
    n = int(p.scorr_n)
    dq = float(p.scorr_dq)
    c_poly6 = 315.0 / (64.0 * math.pi * h ** 9)
    c_spiky = 45.0 / (math.pi * h ** 6)

    def W(r):
        return c_poly6 * (h * h - r * r) ** 3 if r < h else 0.0

    def lam_of(r):
        # rho = m (W(0) + W(r)); |grad_a C| = |grad_b C| = (m / rho0) |grad W(r)|
        C = m * (W(0.0) + W(r)) / rho0 - 1.0
        g = m / rho0 * c_spiky * (h - r) ** 2
        return -C / (w * 2.0 * g * g + eps)

    def dxa(r, lam_a, lam_b):
        # Eq. 7 for a: (w m / rho0) (lam_a + lam_b + s_corr) grad W(x_a - x_b), and
        # grad W(x_a - x_b) points from a to b (x_a < x_b) with magnitude c (h - r)^2
        scorr = -k * (W(r) / W(dq)) ** n
        return w * m / rho0 * (lam_a + lam_b + scorr) * c_spiky * (h - r) ** 2

    r1 = xb - xa
    lam1 = lam_of(r1)
    d1 = dxa(r1, lam1, lam1)
    xa, xb = xa + d1, xb - d1                 # iteration 1: both move, b opposite to a
    r2 = xb - xa
    lam_a2 = lam_of(r2)
    lam_b = {"stale": lam1, "zero": 0.0, "recompute": lam_a2}[lam_b_second]
    xa = xa + dxa(r2, lam_a2, lam_b)          # iteration 2: only a moves
    return xa, xb


@pytest.mark.parametrize("mode,name", [(O.ORC_LAMBDA_STALE, "stale"), (O.ORC_LAMBDA_ZERO, "zero"),
                                       (O.ORC_LAMBDA_RECOMPUTE, "recompute")])
def test_finished_neighbour_enters_with_its_last_lambda(mode, name):
    """Particle b finishes after iteration 1 (level 1), a takes part in
    iteration 2 (level 2, nearer the camera). In iteration 2 a's correction
    uses b's lambda from iteration 1 (stale reading); the zero and
    recompute-all options of the oracle give their own closed forms, and the
    three differ by far more than the tolerance."""
    xa0, xb0 = np.float32(1.0), np.float32(1.06)
    x = np.array([[xa0, 1.0, 1.0], [xb0, 1.0, 1.0]], np.float32)
    v = np.zeros_like(x)
    h = np.float32(H)
    w0 = 315.0 / (64.0 * math.pi * float(h) ** 3)          # W(0)
    # rest density 5 % above the pair's own density: a small, well-conditioned correction
    rho_pair = w0 * (1.0 + (1.0 - (float(xb0) - float(xa0)) ** 2 / float(h) ** 2) ** 3)
    p = _params(rho0=1.05 * rho_pair, n_min=1, n_max=2, lod_mode=O.ORC_LOD_DTC, eye=(0.0, 1.0, 1.0),
                lambda_mode=mode)
    lv, _ = O.lod_levels(p, x)
    assert list(lv) == [2, 1]
    st = O.step(p, x, v, want_final64=True)
    got = st.x_final[np.argsort(st.ids)]
    expect = {nm: _two_particle_step(p, float(xa0), float(xb0), nm) for nm in ("stale", "zero", "recompute")}
    ea, eb = expect[name]
    assert abs(got[0, 0] - ea) < 1e-12 and abs(got[1, 0] - eb) < 1e-12, (got[:, 0], ea, eb)
    assert np.all(got[:, 1:] == 1.0)
    others = [expect[nm][0] for nm in expect if nm != name]
    # the readings are told apart by far more than the 1e-5 h position tolerance
    assert min(abs(ea - o) for o in others) > 1e-5 * H


def test_thread_count_does_not_change_any_bit():
    """The per-particle loops run on OpenMP threads; every particle's own sums
    keep their order, so a step, the neighbour lists and the density
    statistics are bit-identical at any thread count."""
    cfg = S.config_dam_break_4k().replace(lattice=(14, 12, 10), lod_mode=S.LOD_DTC, n_min=2, n_max=6,
                                          camera="fixed", eye=(-1.0, 0.3, 0.3))
    x, v = S.make_scene(cfg)
    p = O.make_params(cfg, rho0=O.rest_density(H, 1.0, 0.05), eye=cfg.eye)
    before = O.set_threads(0)
    try:
        out = []
        for t in (1, 4):
            O.set_threads(t)
            st = O.step(p, x, v, record=True, rec_iters=6, want_final64=True)
            stats, rho = O.density_stats(p, st.x, want_rho=True)
            out.append((st, stats, rho, O.neighbors(p, st.x)))
        (a, sa, ra, na), (b, sb, rb, nb) = out
        for k in ("x", "v", "ids", "lam", "rho", "xs", "x_final", "v_final", "nbr_off", "nbr_idx"):
            assert np.array_equal(getattr(a, k), getattr(b, k), equal_nan=True), k
        assert np.array_equal(sa, sb) and np.array_equal(ra, rb)
        assert np.array_equal(na[0], nb[0]) and np.array_equal(na[1], nb[1])
    finally:
        O.set_threads(before)
