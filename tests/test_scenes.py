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
