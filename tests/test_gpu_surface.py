"""Device surface-sample generation (section "Surface Particle Sampling")
against the FP64 oracle, through the C ABI: the samples themselves, and whole
steps that regenerate the surface before resampling."""
import numpy as np
import pytest

import oracle
from oracle import surface as osurf
from paper_2101_12408_gb300 import scenes

pytestmark = pytest.mark.gpu

mpm = pytest.importorskip("paper_2101_12408_gb300.mpm")


def relerr(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _droplet():
    return scenes.droplet(n=32, r_cells=6.0, seed=5)


def _incline():
    return scenes.incline(n=48, n_drops=2, r_range=(3.0, 5.0), seed=43, gap_cells=(0.0, 0.5))


@pytest.mark.parametrize("make", [_droplet, _incline])
def test_generated_samples_match_oracle(make):
    sc = make()
    ctx = mpm.Context(sc, surface_capacity_factor=3.0)
    ctx.load_scene(0)
    for seed in (77, 78):
        cnt = ctx.generate_surface(seed, 2.0)
        plane = (sc.plane_n, sc.plane_d) if sc.plane_mode else None
        s, dA, kind, _ = osurf.generate(sc.x, sc.n, sc.dx, seed, 2.0, plane)
        assert int(cnt[0]) == s.shape[0] > 0
        got = ctx.get_surface(0)
        # the same float64 formulas in the same order: equal up to the last bits
        assert np.max(np.abs(got["s"] - s)) <= 1e-14
        assert relerr(got["dA"], dA) <= 1e-13
        np.testing.assert_array_equal(got["kind"], kind)
    ctx.close()


def test_steps_with_generated_surface_match_oracle():
    sc = _droplet()
    sc.params.newton_tol = 1e-10
    sc.params.cg_rtol = 1e-6
    ctx = mpm.Context(sc, precision=mpm.PREC_FP64, surface_capacity_factor=3.0)
    ctx.load_scene(0)
    sim = oracle.OracleSim(sc)
    for seed in (11, 12):
        ctx.generate_surface(seed)
        sim.generate_surface(seed)
        ctx.resample()
        ctx.p2g()
        ctx.newton_step()
        sim.resample()
        sim.p2g()
        sim.grid_update()
        np.testing.assert_array_equal(ctx.get_surface(0)["parent"], sim.parent)
        # Both sides stop Newton at a 1e-10 relative residual. The end-of-step
        # velocity v - r/m (reading R17 of the final force evaluation) carries
        # the leftover residual divided by the node mass, so nodes with little
        # mass (balance particles just outside the surface) hold the largest
        # differences, ~1e-8 of the largest velocity; weighted by mass they are
        # a few 1e-9 (measured 2.9e-9)
        vg, vo = ctx.get_grid(0, mpm.FIELD_VHAT), sim.vhat
        assert relerr(vg, vo) < 3e-8
        m = sim.grid["m"][:, None]
        assert np.sum(m * np.abs(vg - vo)) <= 1e-8 * np.sum(m * np.abs(vo))
        ctx.g2p()
        sim.g2p()
    # Balance particles put small masses on nodes just outside the surface; the
    # Newton stop (1e-10 relative residual) leaves velocity errors ~ residual / m
    # there, which G2P passes to the particles' velocities: ~1e-7 here, still two
    # orders below the 1e-5 bound on one step's grid velocity
    p = ctx.get_particles(0)
    assert relerr(p["v"], sim.sc.v) < 2e-6
    ctx.close()


def test_momentum_conserved_with_generated_surface():
    sc = scenes.droplet(n=32, r_cells=6.0, seed=12, v0=(0.3, -0.1, 0.2), spin=1.5, lambda_l=100.0)
    ctx = mpm.Context(sc, precision=mpm.PREC_FP32_FP64RED, surface_capacity_factor=3.0)
    ctx.load_scene(0)
    m0 = np.sum(sc.m[:, None] * sc.v, 0)
    for seed in range(3):
        ctx.generate_surface(100 + seed)
        ctx.step()
    p = ctx.get_particles(0)
    np.testing.assert_allclose(np.sum(sc.m[:, None] * p["v"], 0), m0, rtol=0, atol=1e-10 * np.abs(m0).max())
    ctx.close()


@pytest.mark.parametrize("make", [_droplet, _incline])
def test_marching_cubes_samples_match_oracle(make):
    """The same through marching cubes (the paper's isocontour method): the
    device's loops, decider and fans against the oracle's, sample for sample."""
    sc = make()
    ctx = mpm.Context(sc, surface_capacity_factor=3.0)
    ctx.load_scene(0)
    plane = (sc.plane_n, sc.plane_d) if sc.plane_mode else None
    for seed in (77, 78):
        cnt = ctx.generate_surface(seed, 2.0, method="cubes")
        s, dA, kind, _ = osurf.generate(sc.x, sc.n, sc.dx, seed, 2.0, plane, method="cubes")
        assert int(cnt[0]) == s.shape[0] > 0
        got = ctx.get_surface(0)
        assert np.max(np.abs(got["s"] - s)) <= 1e-14
        assert relerr(got["dA"], dA) <= 1e-13
        np.testing.assert_array_equal(got["kind"], kind)
    # the tetrahedral surface again from the same context: the two methods share its buffers
    cnt = ctx.generate_surface(77, 2.0)
    s, _, _, _ = osurf.generate(sc.x, sc.n, sc.dx, 77, 2.0, plane)
    assert int(cnt[0]) == s.shape[0]
    assert np.max(np.abs(ctx.get_surface(0)["s"] - s)) <= 1e-14
    ctx.close()
