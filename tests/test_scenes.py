"""Properties of the seeded scene generators that the workloads rely on.

The generators hold none of the method's arithmetic; these tests use the oracle
only to evaluate forces on the generated inputs.
"""
import numpy as np

import oracle
from paper_2101_12408_gb300 import scenes


def test_film_flat_sheet_exerts_no_tangential_force_on_free_nodes():
    """Surface energy of a flat sheet with constant coefficient (section
    "Surface Tension"): its gradient at rest must vanish on every node whose
    tangential velocity is free, so that only a varying coefficient moves the
    film. The edge pull has to land on the slip node layers instead."""
    for spc in (1, 2, 4):
        sc = scenes.film(nx=20, ny=16, nz=12, height_cells=3, seed=3, surf_per_cell=spc)
        sc.params.gamma_law = scenes.GAMMA_CONST
        sc.params.gamma_lg = 1.0
        sc.params.gravity = (0.0, 0.0, 0.0)
        sc.params.lambda_l = 0.0
        sc.params.mu_l = 0.0
        sc.params.thermal = False
        sim = oracle.OracleSim(sc)
        sim.resample()
        sim.p2g()
        st = sim.newton_state()
        f = st.gradient(np.zeros_like(st.vn))
        g = np.stack(np.unravel_index(np.arange(st.G), sc.n, order="F"), -1)
        scale = sc.params.dt * sc.dx          # dt * gamma * (edge length dx)
        for ax in (0, 1):
            free = (g[:, ax] >= 2) & (g[:, ax] <= sc.n[ax] - 3)
            assert np.max(np.abs(f[free, ax])) <= 1e-12 * scale
            z1 = 2 + 3                        # the sheet's height, between node rows z1-1 and z1
            wall = (g[:, ax] <= 1) & (g[:, 2] >= z1 - 1) & (g[:, 2] <= z1)
            # the two edges' pull, gamma/2 per unit length on each wall layer
            assert np.max(np.abs(f[wall, ax])) > 0.1 * scale
        assert np.isclose(np.sum(np.abs(sc.dA[:, 2])), (sc.n[0] - 2) * (sc.n[1] - 2) * sc.dx ** 2)


def test_film_steps_converge_and_stay_slow():
    """The film at its default (SI water) parameters: Newton converges within a
    few iterations each step and the flow stays far below a cell per step."""
    sc = scenes.film(nx=24, ny=24, nz=12, height_cells=4, seed=41)
    sim = oracle.OracleSim(sc)
    for _ in range(3):
        sim.step()
        assert 0 < sim.stats["newton"] <= 5 and not sim.stats.get("stalled", False)
        assert sim.stats["residual"][-1] <= sc.params.newton_tol * sim.stats["residual"][0]
    vmax = np.abs(sim.sc.v).max()
    assert vmax * sc.params.dt < 0.01 * sc.dx


def test_benchmark_inputs_have_the_documented_sizes():
    """The seeded generators give the particle and sample counts the input
    recipe states, so every measurement refers to the same inputs."""
    d = scenes.config(0)
    assert (d.n_particles, d.n_surface) == (17184, 1608)
    f = scenes.config(1)
    assert (f.n_particles, f.n_surface) == (738048, 31752)
    assert f.params.rho == 1000.0 and f.params.lambda_l == 1e6


def test_batch_workload_follows_its_recipe():
    """The batched workload: 64 independent scenes with grid edges in [32, 96] and
    particle counts in [5k, 300k] (both drawn log-uniform, so the smallest and the
    largest tenth of each range are both represented), droplets and films and
    constant and temperature-dependent gamma mixed, 5 439 405 particles in all."""
    b = scenes.batch()
    assert len(b) == 64
    ns = np.array([s.n[0] for s in b])
    cnt = np.array([s.n_particles for s in b])
    assert ns.min() >= 32 and ns.max() <= 96
    assert cnt.min() >= 5e3 * 0.9 and cnt.max() <= 3e5 * 1.1
    assert int(cnt.sum()) == 5439405
    # log-uniform: about half of the scenes below the geometric mean of each range
    assert 20 <= np.sum(ns < np.sqrt(32 * 96)) <= 44
    assert 20 <= np.sum(cnt < np.sqrt(5e3 * 3e5)) <= 44
    drops = np.array(["droplet" in s.name for s in b])
    thermal = np.array([s.params.thermal for s in b])
    assert 20 <= drops.sum() <= 44 and 20 <= thermal.sum() <= 44
    for s in b:
        assert s.params.rho == 1000.0 and s.params.lambda_l == 1e6
        lo = np.floor(s.x / s.dx).min(0)
        hi = np.floor(s.x / s.dx).max(0)
        assert np.all(lo >= 1) and np.all(hi <= np.asarray(s.n) - 2)   # every stencil on the grid


def test_inclined_plane_workload_follows_its_recipe():
    """The 8M-particle workload: 40 droplets with radii uniform in [9.3, 24.8]
    cells on a 256^3 grid, disjoint and above a 30-degree slip plane through
    (0.5, 0.2, 0.5) with gaps of 0.5 to 120 cells, gravity -9.8 along y, water in
    SI units, samples on each droplet's sphere with the solid-liquid kind within
    dx of the plane."""
    sc = scenes.incline()
    assert (sc.n_particles, sc.n_surface) == (8272476, 317603)
    c, r = sc.meta["centers"], sc.meta["radii"] / sc.dx
    assert len(r) == 40 and r.min() >= 9.3 and r.max() <= 24.8
    gaps = np.linalg.norm(c[:, None] - c[None], axis=-1) - (r[:, None] + r[None]) * sc.dx
    assert np.all(gaps[~np.eye(40, dtype=bool)] > 0.0)
    nrm = np.asarray(sc.plane_n)
    assert np.allclose(nrm, [-0.5, np.sqrt(3) / 2, 0.0]) and np.isclose(sc.plane_d, nrm @ [0.5, 0.2, 0.5])
    assert np.all(sc.x @ nrm - sc.plane_d > 0.0)
    assert sc.params.gravity == (0.0, -9.8, 0.0) and sc.params.rho == 1000.0 and sc.params.lambda_l == 1e6
    # each droplet starts between 0.5 and 120 cells above the plane
    gap = (c @ nrm - sc.plane_d) / sc.dx - r
    assert gap.min() >= 0.5 and gap.max() <= 120.0
    d = sc.s @ nrm - sc.plane_d
    np.testing.assert_array_equal(sc.kind, (d < sc.dx).astype(np.uint8))


def test_wax_workload_follows_its_recipe():
    """The melting-wax workload: a 96^3-cell solid cube at 8 particles per cell
    (7 077 888) resting on the sticky floor of a 256x256x128 grid at T0, samples on
    its five free faces with outward area vectors (none on the face on the floor),
    the -x face heated at b = 50, Robin convection h = 0.5 towards T0 everywhere,
    E(T) from 1e4 at 298 to 0 at the melting point 303, phase change on."""
    sc = scenes.wax()
    assert sc.n == (256, 256, 128) and sc.n_particles == 96 ** 3 * 8
    lo, hi = sc.x.min(0) / sc.dx, sc.x.max(0) / sc.dx
    assert np.all(hi - lo < 96) and np.all(hi - lo > 95.5) and lo[2] < 2.5
    assert np.all(sc.phase == scenes.PHASE_SOLID) and np.all(sc.T == 298.0)
    p = sc.params
    assert (p.E0, p.T0, p.T_melt, p.h) == (1e4, 298.0, 303.0, 0.5) and p.phase_change and p.thermal
    nrm = sc.dA / np.linalg.norm(sc.dA, axis=1, keepdims=True)
    faces = {tuple(v) for v in np.round(nrm, 12)}
    assert faces == {(-1.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)}
    minus_x = np.isclose(nrm[:, 0], -1.0)
    np.testing.assert_array_equal(sc.b, np.where(minus_x, 50.0, 0.0))
    assert np.all(sc.Tbar == 298.0)
    # outward: every sample lies on the side of the cube its area vector points to
    centre = 0.5 * (sc.x.min(0) + sc.x.max(0))
    assert np.all(np.sum((sc.s - centre) * nrm, 1) > 0.0)


def test_film_workload_follows_its_recipe():
    """The Marangoni film: a 6-cell liquid layer over the sticky floor of a
    128x128x32 grid with slip side walls and an open top, samples on the top face
    only (reaching the side walls' node layers, reading R26), a Gaussian hot spot
    of sigma = 10 cells and Delta T = 1 at the centre, gamma(T) = 1 - 0.5 (T - T0)
    clamped at 0, Robin convection h = 5 towards T0, rho c_p = 1, K = 0.1, dt = 5e-4."""
    sc = scenes.config(1)
    assert sc.n == (128, 128, 32)
    assert sc.walls == (scenes.WALL_SLIP,) * 4 + (scenes.WALL_STICKY, scenes.WALL_NONE)
    lo, hi = sc.x.min(0) / sc.dx, sc.x.max(0) / sc.dx
    assert np.all(lo > 2.0) and lo[2] < 2.25 and hi[2] < 8.0 and hi[2] > 7.75 and np.all(hi[:2] < 126.0)
    assert np.all(sc.s[:, 2] == 8.0 * sc.dx) and np.all(sc.dA[:, :2] == 0.0) and np.all(sc.dA[:, 2] > 0.0)
    assert sc.s[:, 0].min() < 2.0 * sc.dx and sc.s[:, 0].max() > 126.0 * sc.dx
    p = sc.params
    r2 = np.sum((sc.x[:, :2] / sc.dx - 64.0) ** 2, 1)
    np.testing.assert_allclose(sc.T, p.T0 + np.exp(-r2 / (2.0 * 10.0 ** 2)), atol=0.02)
    assert sc.T.max() > p.T0 + 0.99
    assert p.gamma_law == scenes.GAMMA_LINEAR and p.gamma_p[:3] == (1.0, -0.5, 0.0) and p.gamma_p[3] >= 1e30
    assert (p.h, p.K, p.dt) == (5.0, 0.1, 5e-4) and np.isclose(p.rho * p.cp, 1.0) and np.all(sc.Tbar == p.T0)
