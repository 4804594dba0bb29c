"""The one-by-one oracle helpers used at the full benchmark size agree with the
oracle's whole-grid results on a workload small enough to run whole."""
import numpy as np

import oracle
from paper_2101_12408_gb300 import scenes

from _sampled import nearest_parents, p2g_at_nodes


def test_sampled_p2g_and_parents_match_the_whole_grid_oracle():
    sc = scenes.droplet(n=16, r_cells=4.0, seed=13, v0=(0.2, 0.1, -0.3), spin=0.5)
    rng = np.random.default_rng(2)
    sc.A = rng.standard_normal(sc.A.shape)
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    act = np.flatnonzero(sim.grid["m"] > 0)
    # random active nodes, plus nodes reached by samples and balance particles
    st = oracle.Stencil(np.concatenate([sc.s[:10], sim.bpos[:10]]), sc.dx, sc.n)
    nodes = np.unique(np.concatenate([rng.choice(act, 30, replace=False), st.node[:, 13]]))
    m, mv = p2g_at_nodes(sc.n, sc.dx, sc.x, sc.v, sc.A, sc.m, sc.s, sim.bpos, sim.parent, nodes)
    np.testing.assert_allclose(m, sim.grid["m"][nodes], rtol=1e-13, atol=0)
    np.testing.assert_allclose(mv, sim.grid["mv"][nodes], rtol=1e-12, atol=1e-15 * np.abs(sim.grid["mv"]).max())
    which = rng.choice(sc.n_surface, 40, replace=False)
    np.testing.assert_array_equal(nearest_parents(sc.x, sc.s, which, sc.dx, sc.n), sim.parent[which])


def test_sampled_hessvec_matches_the_whole_grid_oracle():
    """hessvec_at_nodes (one node at a time, on a window around it) against the
    oracle's whole-grid Hessian-vector product, in both modes, at bulk nodes and
    nodes reached by surface samples."""
    from oracle.energy import HESS_EXACT, HESS_PROJECTED
    from _sampled import hessvec_at_nodes
    sc = scenes.droplet(n=20, r_cells=5.0, seed=14, lambda_l=70.0)
    rng = np.random.default_rng(3)
    sc.J = rng.uniform(0.9, 1.1, sc.J.shape)
    sc.params.dt = 0.02
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    st = sim.newton_state()
    act = st.active
    v = (st.vn + 0.5 * rng.standard_normal(st.vn.shape)) * act[:, None]
    dv = rng.standard_normal(v.shape) * act[:, None]
    ss = oracle.Stencil(sc.s[:12], sc.dx, sc.n)
    nodes = np.unique(np.concatenate([rng.choice(np.flatnonzero(act), 20, replace=False), ss.node[:, 13]]))
    for mode in (HESS_PROJECTED, HESS_EXACT):
        ref = st.hessvec(v, dv, mode)
        full, stiff = hessvec_at_nodes(sc.n, sc.dx, sc.params.dt, sc.x, sc.V0, sc.J, sc.params.lambda_l, sc.s,
                                       sc.dA, st.gamma, v, dv, st.m, nodes, mode)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(full, ref[nodes], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(stiff, ref[nodes] - st.m[nodes, None] * dv[nodes], rtol=0, atol=1e-12 * scale)


def test_hessvec_with_only_surface_samples_near_the_node():
    """A node whose mass comes from samples alone: the particle set of its window
    is empty, and the row is the mass term plus the samples' terms."""
    from oracle.energy import HESS_EXACT, HESS_PROJECTED
    n, dx = (8, 8, 8), 1.0 / 8
    m = np.zeros(512)
    m[4 + 8 * (4 + 8 * 4)] = 0.3
    s = np.array([[0.55, 0.55, 0.55]])
    st = oracle.NewtonState(n, dx, 0.01, np.zeros(3), m, np.zeros((512, 3)), np.zeros((0, 3)), np.zeros(0),
                            np.zeros(0), np.zeros((0, 3, 3)), np.zeros(0, np.int64), 50.0, 0.0, np.zeros(0),
                            np.zeros(0), s, np.array([[0.0, 0.0, 0.01]]), np.array([1.0]))
    dv = np.random.default_rng(1).standard_normal((512, 3))
    for mode in (HESS_PROJECTED, HESS_EXACT):
        out = st.hessvec(np.zeros((512, 3)), dv, mode)
        assert np.all(np.isfinite(out)) and np.any(out != 0.0)
