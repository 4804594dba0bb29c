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
