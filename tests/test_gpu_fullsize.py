"""Parity at the benchmark's full size: the inclined-plane workload (40 drops,
8.27M particles, 256^3 grid), in the float32 operator form and the launch
configuration the bench times.

The oracle cannot run the whole workload. Instead it computes sampled outputs
one by one: closest parents of sampled samples, and P2G sums at sampled nodes
from the GPU's own particle state after a full step. Everything else is
checked through properties that hold at any size: the operator is symmetric
and positive, and G2P hands the grid's momentum to the particles exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2101_12408_gb300 import mpm, scenes

from _sampled import hessvec_at_nodes, nearest_parents, p2g_at_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def incline():
    sc = scenes.incline(n_drops=40)
    ctx = mpm.Context(sc, precision=mpm.PREC_FP32_FP64RED, surface_capacity_factor=2.0)
    ctx.load_scene(0)
    ctx.step()
    # the state after one step, resampled and transferred again
    ctx.resample()
    ctx.p2g()
    p = ctx.get_particles(0)
    srf = ctx.get_surface(0)
    return sc, ctx, p, srf


def test_fullsize_closest_parents_at_sampled_samples(incline):
    sc, ctx, p, srf = incline
    rng = np.random.default_rng(5)
    which = rng.choice(len(srf["s"]), 150, replace=False)
    np.testing.assert_array_equal(srf["parent"][which], nearest_parents(p["x"], srf["s"], which, sc.dx, sc.n))


def test_fullsize_p2g_at_sampled_nodes(incline):
    sc, ctx, p, srf = incline
    m = ctx.get_grid(0, mpm.FIELD_MASS)
    mv = ctx.get_grid(0, mpm.FIELD_MOMENTUM)
    rng = np.random.default_rng(6)
    act = np.flatnonzero(m > 0)
    # random active nodes, and the centre nodes of some samples' stencils
    st = oracle.Stencil(srf["s"][rng.choice(len(srf["s"]), 16, replace=False)], sc.dx, sc.n)
    nodes = np.unique(np.concatenate([rng.choice(act, 24, replace=False), st.node[:, 13]]))
    mo, mvo = p2g_at_nodes(sc.n, sc.dx, p["x"], p["v"], p["A"], sc.m, srf["s"], srf["b"], srf["parent"], nodes)
    assert np.all(mo > 0)
    # float64 transfers: sums in another order only
    np.testing.assert_allclose(m[nodes], mo, rtol=1e-12, atol=0)
    np.testing.assert_allclose(mv[nodes], mvo, rtol=1e-10, atol=1e-12 * np.abs(mvo).max())


def test_fullsize_operator_is_symmetric_and_positive(incline):
    sc, ctx, p, srf = incline
    act = ctx.get_grid(0, mpm.FIELD_MASS) > 0
    ctx.set_velocity(0, ctx.get_grid(0, mpm.FIELD_VN))
    rng = np.random.default_rng(7)
    d1 = rng.standard_normal((act.size, 3)) * act[:, None]
    d2 = rng.standard_normal((act.size, 3)) * act[:, None]
    u1 = ctx.apply_hessian(0, d1).astype(np.float64)
    u2 = ctx.apply_hessian(0, d2).astype(np.float64)
    d1 = d1.astype(np.float32).astype(np.float64)
    d2 = d2.astype(np.float32).astype(np.float64)
    a11, a22 = float(np.sum(d1 * u1)), float(np.sum(d2 * u2))
    a12, a21 = float(np.sum(d1 * u2)), float(np.sum(d2 * u1))
    assert a11 > 0 and a22 > 0
    # float32 operator arithmetic, float64 dots
    assert abs(a12 - a21) <= 1e-4 * np.sqrt(a11 * a22)


@pytest.mark.parametrize("mode", [mpm.HESS_PROJECTED, mpm.HESS_EXACT])
def test_fullsize_operator_at_sampled_nodes(incline, mode):
    """mpm_apply_hessian at ~40 sampled free nodes against the oracle's
    per-particle definition, evaluated one node at a time from the particles and
    samples that reach it. The direction vanishes on the Dirichlet and massless
    nodes, so P dv = dv, and the sampled nodes are free, so P acts as the
    identity on their rows."""
    sc, ctx, p, srf = incline
    n = sc.n
    m = ctx.get_grid(0, mpm.FIELD_MASS)
    vn = ctx.get_grid(0, mpm.FIELD_VN)
    ctx.set_velocity(0, vn)
    xi = oracle.node_positions(n, sc.dx)
    g = np.stack(np.unravel_index(np.arange(m.size), tuple(n), order="F"), -1)
    inner = np.all((g >= 2) & (g <= np.array(n) - 3), axis=1)
    free = inner & (xi @ np.asarray(sc.plane_n) - sc.plane_d >= 0.0) & (m > 0)
    rng = np.random.default_rng(8)
    dv = rng.standard_normal((m.size, 3)) * free[:, None]
    dv = dv.astype(np.float32).astype(np.float64)
    # free nodes in the bulk, next to surface samples, and next to the plane
    st = oracle.Stencil(srf["s"][rng.choice(len(srf["s"]), 16, replace=False)], sc.dx, n)
    plane_phi = xi @ np.asarray(sc.plane_n) - sc.plane_d
    near_plane = np.flatnonzero(free & (plane_phi < 2 * sc.dx))
    nodes = np.concatenate([rng.choice(np.flatnonzero(free), 16, replace=False), st.node[:, 13],
                            rng.choice(near_plane, 8, replace=False)])
    nodes = np.unique(nodes[free[nodes]])
    assert nodes.size >= 30
    # the surface coefficient by interface kind (solid-liquid within dx of the plane)
    kind_sl = srf["s"] @ np.asarray(sc.plane_n) - sc.plane_d < sc.dx
    gamma = np.where(kind_sl, sc.params.gamma_sl, sc.params.gamma_lg)
    full, stiff = hessvec_at_nodes(n, sc.dx, sc.params.dt, p["x"], sc.V0, p["J"], sc.params.lambda_l, srf["s"],
                                   srf["dA"], gamma, vn, dv, m, nodes,
                                   oracle.energy.HESS_PROJECTED if mode == mpm.HESS_PROJECTED
                                   else oracle.energy.HESS_EXACT)
    out = ctx.apply_hessian(0, dv.astype(np.float32), mode=mode).astype(np.float64)
    got = out[nodes]
    assert np.max(np.abs(got - full)) <= 2e-5 * np.max(np.abs(full))
    got_stiff = got - m[nodes, None] * dv[nodes]
    assert np.max(np.abs(got_stiff - stiff)) <= 1e-4 * np.max(np.abs(stiff))
    assert np.max(np.abs(stiff)) > 0


def test_fullsize_step_hands_grid_momentum_to_particles(incline):
    sc, ctx, p, srf = incline
    m = ctx.get_grid(0, mpm.FIELD_MASS)
    stats = ctx.newton_step()[0]
    assert stats["residual"] <= sc.params.newton_tol * max(stats["residual0"], 1e-12)
    vhat = ctx.get_grid(0, mpm.FIELD_VHAT)
    ctx.g2p()
    v = ctx.get_particles(0)["v"]
    grid = np.sum(m[:, None] * vhat, 0)
    part = np.sum(sc.m[:, None] * v, 0)
    scale = np.sum(sc.m[:, None] * np.abs(v))
    np.testing.assert_allclose(part, grid, rtol=0, atol=1e-10 * scale)
