"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(B-spline moments, ellipsoid area, rigid/affine motions), textbook or library
routines (cofactor = det * inverse^T, SVD), conservation laws the paper claims
(split, P2G, merge), finite differences of the energy, brute-force symmetry and
definiteness, and special cases with known answers.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import constitutive as cst
from oracle.energy import HESS_EXACT, HESS_PROJECTED
from paper_2101_12408_gb300 import scenes

RNG = np.random.default_rng(7)


# ----------------------------------------------------------------------------
# B-spline (section "Transfer: P2G": quadratic B-splines, nodes at cell centres)
# ----------------------------------------------------------------------------

def _bspline_1d(d):
    """Textbook quadratic B-spline, written piecewise in the distance."""
    d = np.abs(d)
    return np.where(d < 0.5, 0.75 - d * d, np.where(d < 1.5, 0.5 * (1.5 - d) ** 2, 0.0))


def test_spline_matches_piecewise_definition():
    n = (10, 10, 10)
    dx = 0.1
    X = RNG.uniform(1.0, 9.0, size=(200, 3)) * dx
    st = oracle.Stencil(X, dx, n)
    # brute force over every node of the grid
    xi = oracle.node_positions(n, dx)
    for p in range(0, 200, 17):
        d = (X[p] - xi) / dx
        w = np.prod(_bspline_1d(d), -1)
        dense = np.zeros(xi.shape[0])
        dense[st.node[p]] = st.N[p]
        np.testing.assert_allclose(dense, w, atol=1e-15)
        # gradient by central differences of the piecewise definition
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (np.prod(_bspline_1d((X[p] + e - xi) / dx), -1) - np.prod(_bspline_1d((X[p] - e - xi) / dx), -1)) / (2 * h)
            g = np.zeros(xi.shape[0])
            g[st.node[p]] = st.dN[p, :, a]
            np.testing.assert_allclose(g, fd, atol=1e-6 / dx)


def test_spline_moment_identities():
    n = (12, 12, 12)
    dx = 1.0 / 12
    X = RNG.uniform(1.0, 11.0, size=(500, 3)) * dx
    st = oracle.Stencil(X, dx, n)
    r = st.xi - X[:, None, :]
    np.testing.assert_allclose(st.N.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.einsum("pq,pqa->pa", st.N, r), 0.0, atol=1e-15)
    D = np.einsum("pq,pqa,pqb->pab", st.N, r, r)
    # second moment dx^2/4 I (the constant APIC inertia the paper's merge relies on)
    np.testing.assert_allclose(D, np.broadcast_to(np.eye(3) * dx * dx / 4, D.shape), atol=1e-15)
    np.testing.assert_allclose(st.dN.sum(1), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.einsum("pqa,pqb->pab", st.xi, st.dN), np.broadcast_to(np.eye(3), D.shape), atol=1e-12)


# ----------------------------------------------------------------------------
# cofactor, polar SVD, fixed corotated (section "Constitutive Models")
# ----------------------------------------------------------------------------

def test_cofactor_is_det_inverse_transpose():
    F = np.eye(3) + 0.3 * RNG.standard_normal((50, 3, 3))
    C = cst.cof(F)
    ref = np.linalg.det(F)[:, None, None] * np.swapaxes(np.linalg.inv(F), 1, 2)
    np.testing.assert_allclose(C, ref, rtol=1e-11, atol=1e-12)
    dF = RNG.standard_normal((50, 3, 3))
    h = 1e-6
    fd = (cst.cof(F + h * dF) - cst.cof(F - h * dF)) / (2 * h)
    np.testing.assert_allclose(cst.dcof(F, dF), fd, atol=1e-8)


def test_polar_and_fixed_corotated():
    F = np.eye(3) + 0.25 * RNG.standard_normal((40, 3, 3))
    F[:5] = F[:5] * np.array([1, 1, -1])[None, :, None]  # a few inverted
    R, S, sig = cst.polar(F)
    np.testing.assert_allclose(np.einsum("pka,pkb->pab", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    np.testing.assert_allclose(S, np.swapaxes(S, 1, 2), atol=1e-12)
    np.testing.assert_allclose(R @ S, F, atol=1e-12)
    # singular values: |sigma| equal numpy's, sign of the product = sign det F
    np.testing.assert_allclose(np.sort(np.abs(sig), 1), np.sort(np.linalg.svd(F, compute_uv=False), 1), atol=1e-12)
    np.testing.assert_allclose(np.prod(sig, 1), np.linalg.det(F), rtol=1e-10)
    mu = RNG.uniform(1, 3, 40)
    lam = RNG.uniform(1, 3, 40)
    h = 1e-6
    dF = RNG.standard_normal((40, 3, 3))
    P = cst.fcr_P(F, mu, lam)
    fd = (cst.fcr_energy(F + h * dF, mu, lam) - cst.fcr_energy(F - h * dF, mu, lam)) / (2 * h)
    np.testing.assert_allclose(np.einsum("pab,pab->p", P, dF), fd, rtol=1e-6, atol=1e-7)
    ok = np.abs(np.linalg.det(F)) > 0.2  # away from degenerate polar
    fdP = (cst.fcr_P(F + h * dF, mu, lam) - cst.fcr_P(F - h * dF, mu, lam)) / (2 * h)
    np.testing.assert_allclose(cst.fcr_dP(F, dF, mu, lam)[ok], fdP[ok], rtol=1e-5, atol=1e-6)


# ----------------------------------------------------------------------------
# split (Eq. pbal, Eq. cons_mom), P2G and merge conservation
# ----------------------------------------------------------------------------

def _moving_droplet(**kw):
    sc = scenes.droplet(n=16, r_cells=4.0, seed=11, **kw)
    rng = np.random.default_rng(3)
    sc.v = rng.standard_normal(sc.v.shape)
    sc.A = rng.standard_normal(sc.A.shape) * 3.0
    return sc


def _angular(x, m, v, A, dx):
    # APIC angular momentum of a particle: x x m v + m dx^2/4 eps_abg A_gb
    return np.sum(np.cross(x, m[:, None] * v), 0) + dx * dx / 4 * np.einsum("abg,p,pgb->a", cst.EPS, m, A)


def test_nearest_parent_against_kdtree_distance():
    from scipy.spatial import cKDTree
    sc = _moving_droplet()
    parent, best = oracle.nearest_parent(sc.x, sc.s)
    d, _ = cKDTree(sc.x).query(sc.s)
    np.testing.assert_allclose(np.sqrt(best), d, rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(sc.x[parent] - sc.s, axis=1), d, rtol=1e-12)


def test_split_conserves_mass_momentum_com():
    sc = _moving_droplet()
    parent, count, mt, b = oracle.split(sc.x, sc.m, sc.s)
    assert np.all(count[parent] >= 1)
    # mass: every group member carries m~, 2|Pi|+1 members
    np.testing.assert_allclose(np.sum(mt * (2 * count + 1)), np.sum(sc.m), rtol=1e-14)
    # centre of mass of each group is x_p (Eq. cons_mom)
    com = mt[:, None] * sc.x
    np.add.at(com, parent, mt[parent][:, None] * (sc.s + b))
    np.testing.assert_allclose(com / sc.m[:, None], sc.x, rtol=1e-13, atol=1e-15)
    # linear and angular momentum of the split collection
    allx = np.concatenate([sc.x, sc.s, b])
    allm = np.concatenate([mt, mt[parent], mt[parent]])
    allv = np.concatenate([sc.v, sc.v[parent], sc.v[parent]])
    allA = np.concatenate([sc.A, sc.A[parent], sc.A[parent]])
    np.testing.assert_allclose(np.sum(allm[:, None] * allv, 0), np.sum(sc.m[:, None] * sc.v, 0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(_angular(allx, allm, allv, allA, sc.dx), _angular(sc.x, sc.m, sc.v, sc.A, sc.dx),
                               rtol=1e-12, atol=1e-14)


def test_p2g_conserves_and_preserves_affine():
    sc = _moving_droplet()
    parent, count, mt, b = oracle.split(sc.x, sc.m, sc.s)
    g = oracle.p2g(sc.n, sc.dx, sc.x, sc.v, sc.A, mt, sc.s, b, parent)
    xi = oracle.node_positions(sc.n, sc.dx)
    np.testing.assert_allclose(g["m"].sum(), sc.m.sum(), rtol=1e-13)
    np.testing.assert_allclose(g["mv"].sum(0), np.sum(sc.m[:, None] * sc.v, 0), rtol=1e-12, atol=1e-14)
    Lg = np.sum(np.cross(xi, g["mv"]), 0)
    np.testing.assert_allclose(Lg, _angular(sc.x, sc.m, sc.v, sc.A, sc.dx), rtol=1e-11, atol=1e-13)
    # affine field v = a + B x with A = B transfers exactly (plain APIC, no split:
    # split members carry the parent's v_p, not the field at their own position)
    a = np.array([0.3, -0.2, 0.1])
    B = RNG.standard_normal((3, 3))
    v = a + sc.x @ B.T
    A = np.broadcast_to(B, sc.A.shape).copy()
    g = oracle.p2g(sc.n, sc.dx, sc.x, v, A, sc.m)
    vi = oracle.grid_velocity(g["m"], g["mv"])
    act = g["m"] > 0
    np.testing.assert_allclose(vi[act], a + xi[act] @ B.T, atol=1e-12)


def test_g2p_merge_conserves():
    sc = _moving_droplet()
    parent, count, mt, b = oracle.split(sc.x, sc.m, sc.s)
    g = oracle.p2g(sc.n, sc.dx, sc.x, sc.v, sc.A, mt, sc.s, b, parent)
    act = g["m"] > 0
    vhat = np.zeros((g["m"].size, 3))
    vhat[act] = RNG.standard_normal((act.sum(), 3))
    out = oracle.g2p(sc.n, sc.dx, vhat, sc.x, sc.m, mt, sc.s, b, parent)
    xi = oracle.node_positions(sc.n, sc.dx)
    np.testing.assert_allclose(np.sum(sc.m[:, None] * out["v"], 0), np.sum(g["m"][:, None] * vhat, 0), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(_angular(sc.x, sc.m, out["v"], out["A"], sc.dx),
                               np.sum(np.cross(xi, g["m"][:, None] * vhat), 0), rtol=1e-11, atol=1e-13)
    # unsplit particles reproduce an affine grid field exactly (APIC)
    a = np.array([0.1, 0.2, -0.3])
    B = RNG.standard_normal((3, 3))
    vhat = np.where(act[:, None], a + xi @ B.T, 0.0)
    out = oracle.g2p(sc.n, sc.dx, vhat, sc.x, sc.m, mt, sc.s, b, parent)
    free = count == 0
    np.testing.assert_allclose(out["v"][free], a + sc.x[free] @ B.T, atol=1e-12)
    np.testing.assert_allclose(out["A"][free], np.broadcast_to(B, out["A"][free].shape), atol=1e-10)


# ----------------------------------------------------------------------------
# energy (section "Momentum Update")
# ----------------------------------------------------------------------------

def _state(sc, v=None):
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    st = sim.newton_state()
    return sim, st


def _affine_grid_velocity(sc, B, a=np.zeros(3)):
    xi = oracle.node_positions(sc.n, sc.dx)
    return a + xi @ B.T


def _ellipsoid_area(a, b, c):
    a, b, c = sorted([a, b, c], reverse=True)
    phi = math.acos(c / a)
    m = (a * a * (b * b - c * c)) / (b * b * (a * a - c * c))
    return 2 * math.pi * c * c + 2 * math.pi * a * b / math.sin(phi) * (
        special.ellipeinc(phi, m) * math.sin(phi) ** 2 + special.ellipkinc(phi, m) * math.cos(phi) ** 2)


def test_surface_energy_sphere_scaling_and_ellipsoid():
    sc = scenes.droplet(n=32, r_cells=8.0, seed=5, surf_per_cell=6.0, gamma=0.7)
    sc.params.lambda_l = 0.0
    sim, st = _state(sc)
    dt = sc.params.dt
    r = 0.25
    e_surf = lambda v: st.energy(v) - (0.5 * np.sum(st.m[st.active] * np.sum((v - st.vn)[st.active] ** 2, -1)))
    # at rest: gamma 4 pi r^2
    np.testing.assert_allclose(e_surf(np.zeros((st.G, 3))), 0.7 * 4 * math.pi * r * r, rtol=1e-12)
    # uniform scaling F^ = s I: gamma s^2 4 pi r^2
    s_fac = 1.3
    v = _affine_grid_velocity(sc, (s_fac - 1.0) / dt * np.eye(3))
    np.testing.assert_allclose(e_surf(v), 0.7 * s_fac ** 2 * 4 * math.pi * r * r, rtol=1e-11)
    # general affine map: area of the image ellipsoid (exact elliptic-integral formula)
    Fm = np.array([[1.2, 0.1, 0.0], [0.05, 0.9, 0.2], [0.0, -0.1, 1.1]])
    v = _affine_grid_velocity(sc, (Fm - np.eye(3)) / dt)
    sv = np.linalg.svd(Fm, compute_uv=False) * r
    np.testing.assert_allclose(e_surf(v), 0.7 * _ellipsoid_area(*sv), rtol=2e-4)


def test_liquid_energy_affine_closed_form():
    sc = _moving_droplet()
    sc.params.gamma_lg = 0.0
    sc.params.lambda_l = 37.0
    sc.J = RNG.uniform(0.9, 1.1, sc.J.shape)
    sim, st = _state(sc)
    B = 5.0 * RNG.standard_normal((3, 3))
    v = _affine_grid_velocity(sc, B)
    J = (1.0 + sc.params.dt * np.trace(B)) * sc.J
    kin = 0.5 * np.sum(st.m[st.active] * np.sum((v - st.vn)[st.active] ** 2, -1))
    np.testing.assert_allclose(st.energy(v) - kin, np.sum(0.5 * 37.0 * (J - 1) ** 2 * sc.V0), rtol=1e-11)


def _mixed_scene():
    """Tiny scene with liquid + solid particles, viscosity, gravity and surface."""
    sc = scenes.droplet(n=10, r_cells=2.6, seed=9, gravity=(0.0, -3.0, 0.5), mu_l=0.05, lambda_l=40.0)
    rng = np.random.default_rng(1)
    half = sc.x[:, 0] > 0.5
    sc.phase[half] = scenes.PHASE_SOLID
    sc.F[half] = np.eye(3) + 0.05 * rng.standard_normal((half.sum(), 3, 3))
    sc.J = rng.uniform(0.95, 1.05, sc.J.shape)
    sc.params.E0 = 30.0
    sc.params.T_melt = 10.0
    sc.T = rng.uniform(0.0, 5.0, sc.T.shape)
    sc.v = rng.standard_normal(sc.v.shape) * 0.3
    sc.params.dt = 0.02
    sc.params.gamma_lg = 0.8
    return sc


def test_gradient_and_exact_hessian_match_finite_differences():
    sc = _mixed_scene()
    sim, st = _state(sc)
    act = st.active[:, None]
    rng = np.random.default_rng(2)
    v = (st.vn + 0.5 * rng.standard_normal(st.vn.shape)) * act
    for _ in range(3):
        d = rng.standard_normal(v.shape) * act
        h = 1e-5
        fd = (st.energy(v + h * d) - st.energy(v - h * d)) / (2 * h)
        an = np.sum(st.gradient(v) * d)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8), (fd, an)
        fdg = (st.gradient(v + h * d) - st.gradient(v - h * d)) / (2 * h)
        hv = st.hessvec(v, d, HESS_EXACT)
        assert np.max(np.abs(fdg - hv)) <= 1e-6 * np.max(np.abs(hv))


def test_hessian_symmetric_and_projected_psd():
    sc = scenes.droplet(n=8, r_cells=1.6, seed=4, mu_l=0.1, lambda_l=50.0)
    sc.params.dt = 0.05
    sc.params.gamma_lg = 2.0
    sim, st = _state(sc)
    rng = np.random.default_rng(5)
    v = (st.vn + rng.standard_normal(st.vn.shape)) * st.active[:, None]
    idx = np.flatnonzero(st.active)
    ncol = idx.size * 3
    for mode in (HESS_EXACT, HESS_PROJECTED):
        H = np.zeros((ncol, ncol))
        for c in range(ncol):
            e = np.zeros((st.G, 3))
            e[idx[c // 3], c % 3] = 1.0
            H[:, c] = st.hessvec(v, e, mode)[idx].ravel()
        np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
        if mode == HESS_PROJECTED:
            ev = np.linalg.eigvalsh(0.5 * (H + H.T))
            # M + (PSD terms): no eigenvalue below the smallest node mass (up to round-off)
            assert ev.min() >= st.m[idx].min() - 1e-12 * np.abs(ev).max()


def test_internal_forces_sum_to_zero():
    sc = _mixed_scene()
    sc.params.gravity = (0.0, 0.0, 0.0)
    sim, st = _state(sc)
    rng = np.random.default_rng(8)
    v = (st.vn + rng.standard_normal(st.vn.shape)) * st.active[:, None]
    r = st.gradient(v) - st.m[:, None] * (v - st.vn) * st.active[:, None]
    # translation invariance of e: sum_i de/dy_i = 0
    assert np.max(np.abs(r.sum(0))) <= 1e-12 * np.max(np.abs(r))
    d = rng.standard_normal(v.shape) * st.active[:, None]
    hv = st.hessvec(v, d) - st.m[:, None] * d
    assert np.max(np.abs(hv.sum(0))) <= 1e-12 * np.max(np.abs(hv))


# ----------------------------------------------------------------------------
# Newton (special cases with known answers)
# ----------------------------------------------------------------------------

def test_newton_zero_forces_is_free_fall():
    sc = _moving_droplet(gravity=(0.0, -9.8, 1.0))
    sc.params.lambda_l = 0.0
    sc.params.gamma_lg = 0.0
    sim = oracle.OracleSim(sc)
    sim.resample(); sim.p2g(); sim.grid_update()
    act = sim.grid["m"] > 0
    np.testing.assert_allclose(sim.vhat[act], sim.vn[act] + sc.params.dt * np.array([0.0, -9.8, 1.0]), atol=1e-14)
    # the initial guess P(v^n + dt g) already solves it: no Newton iteration
    assert sim.stats["newton"] == 0


def test_armijo_takes_the_first_sufficient_decrease():
    """Backtracking over alpha = 1, 1/2, ...: the first trial whose decrease is at
    least c alpha |slope| (c = 1e-4); an increase, however small, is never taken."""
    from oracle.solver import armijo
    # phi(alpha) = (alpha - 0.3)^2 - 0.09 has slope -0.6 at 0: alpha = 1 rises, 1/2 falls enough
    assert armijo(lambda a: (a - 0.3) ** 2 - 0.09, 0.0, -0.6, 12) == 0.5
    # a quadratic with its minimum at 1 takes the full step
    assert armijo(lambda a: (a - 1.0) ** 2 - 1.0, 0.0, -2.0, 12) == 1.0
    # a tiny rise along the direction: no trial passes
    assert armijo(lambda a: 1e-5 * a, 0.0, -1.0, 12) is None
    # a decrease smaller than c alpha |slope| is not sufficient
    assert armijo(lambda a: -0.5e-4 * a, 0.0, -1.0, 3) is None
    # the number of trials bounds the search: 1, 1/2, 1/4 only
    assert armijo(lambda a: 0.0 if a < 0.2 else 1.0, 0.0, -1e-9, 3) is None
    assert armijo(lambda a: -1.0 if a < 0.2 else 1.0, 0.0, -1.0, 4) == 0.125


def test_newton_pure_liquid_is_one_step():
    sc = _moving_droplet()
    sc.params.gamma_lg = 0.0
    sc.params.lambda_l = 2000.0
    sc.params.cg_rtol = 1e-13
    sc.params.max_cg = 5000
    sim = oracle.OracleSim(sc)
    sim.resample(); sim.p2g(); sim.grid_update()
    assert sim.stats["newton"] == 1
    assert sim.stats["residual"][-1] <= 1e-10 * sim.stats["residual"][0]


# ----------------------------------------------------------------------------
# heat (section "Temperature Update")
# ----------------------------------------------------------------------------

def _thermal_scene():
    sc = scenes.droplet(n=12, r_cells=3.0, seed=21, thermal=True)
    rng = np.random.default_rng(4)
    sc.T = rng.uniform(0.0, 2.0, sc.T.shape)
    sc.gradT = rng.standard_normal(sc.gradT.shape)
    sc.params.h = 3.0
    sc.params.H = 0.7
    sc.params.K = 0.2
    sc.b = rng.uniform(0, 1, sc.n_surface)
    sc.Tbar = rng.uniform(0, 1, sc.n_surface)
    return sc


def test_temperature_transfers_are_exact_for_affine_fields():
    """Temperature P2G with the gradient term and G2P of T and grad T (section
    "Transfer: P2G" and the G2P of section "Discretization") reproduce an affine
    field T = a + g.x exactly: the B-spline weights sum to one and have zero
    first moment about the particle."""
    sc = scenes.droplet(n=12, r_cells=3.0, seed=22, thermal=True)
    a, g = 0.4, np.array([1.5, -0.7, 0.3])
    sc.T = a + sc.x @ g
    sc.gradT = np.broadcast_to(g, sc.gradT.shape).copy()
    out = oracle.p2g(sc.n, sc.dx, sc.x, sc.v, sc.A, sc.m, m=sc.m, T=sc.T, gradT=sc.gradT)
    xi = oracle.node_positions(sc.n, sc.dx)
    act = out["mT"] > 0
    np.testing.assert_allclose(out["mTT"][act] / out["mT"][act], a + xi[act] @ g, atol=1e-13)
    That = a + xi @ g
    back = oracle.g2p(sc.n, sc.dx, np.zeros((xi.shape[0], 3)), sc.x, sc.m, sc.m, That=That)
    np.testing.assert_allclose(back["T"], sc.T, atol=1e-13)
    np.testing.assert_allclose(back["gradT"], sc.gradT, atol=1e-11)


def test_gamma_reads_the_affine_grid_temperature_at_the_samples():
    """gamma(T) of each sample from the renormalised interpolation of the grid
    temperature T^n (reading R9): exact for an affine field wherever all of the
    sample's stencil nodes carry thermal mass, then the linear law."""
    sc = scenes.droplet(n=12, r_cells=4.0, seed=23, thermal=True)
    a, g = 0.2, np.array([0.5, 1.0, -0.8])
    sc.T = a + sc.x @ g
    sc.gradT = np.broadcast_to(g, sc.gradT.shape).copy()
    rng = np.random.default_rng(9)
    c = np.full(3, 0.5)
    d = rng.standard_normal((40, 3))
    sc.s = c + d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0.0, 1.5, (40, 1)) * sc.dx
    sc.dA = np.tile([0.0, 0.0, sc.dx ** 2], (40, 1))
    sc.kind = np.zeros(40, np.uint8)
    sc.b = np.zeros(40)
    sc.Tbar = np.zeros(40)
    sc.params.gamma_law = scenes.GAMMA_LINEAR
    sc.params.gamma_p = (1.0, -0.3, 0.2, 1.1)
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    st = oracle.Stencil(sc.s, sc.dx, sc.n)
    full = np.all(sim.grid["mT"][st.node] > 0, axis=1)
    assert full.sum() >= 30
    Ts = a + sc.s @ g
    np.testing.assert_allclose(sim.Tr[full], Ts[full], atol=1e-12)
    np.testing.assert_allclose(sim.gamma[full], np.clip(1.0 - 0.3 * (Ts[full] - sc.params.T0), 0.2, 1.1), atol=1e-12)


def test_uniform_heat_source_raises_temperature_by_dt_H_over_rho_cp():
    """The source term sum_p N_i(x_p) H V^n_p of section "Temperature Update"
    (reading R4) with no conduction and no boundary flux: every node with
    thermal mass warms by dt H / (rho c_p)."""
    sc = scenes.droplet(n=12, r_cells=3.0, seed=24, thermal=True, rho=2.0)
    sc.T[:] = 0.3
    sc.gradT[:] = 0.0
    sc.params.K = 0.0
    sc.params.h = 0.0
    sc.b[:] = 0.0
    sc.params.H = 5.0
    sc.params.cp = 0.8
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    hs = sim.heat_system()
    T, _ = oracle.heat_solve(hs, 1e-14, 5000)
    rise = sc.params.dt * sc.params.H / (2.0 * sc.params.cp)
    np.testing.assert_allclose(T[hs.unknown], 0.3 + rise, rtol=1e-12)


@pytest.mark.parametrize("phase,scale", [(scenes.PHASE_LIQUID, 0.8), (scenes.PHASE_SOLID, 1.1)])
def test_heat_source_acts_on_the_current_volume(phase, scale):
    """The source is a power per unit current volume, V^n_p = J V^0_p (liquid J,
    solid det F): a uniformly compressed liquid (J = 0.8) or stretched solid
    (F = 1.1 I) warms by dt H J / (rho c_p) at every node with thermal mass."""
    sc = scenes.droplet(n=12, r_cells=3.0, seed=24, thermal=True, rho=2.0)
    sc.T[:] = 0.3
    sc.gradT[:] = 0.0
    sc.params.K = 0.0
    sc.params.h = 0.0
    sc.b[:] = 0.0
    sc.params.H = 5.0
    sc.params.cp = 0.8
    sc.phase[:] = phase
    if phase == scenes.PHASE_LIQUID:
        sc.J[:] = scale
        J = scale
    else:
        sc.F[:] = scale * np.eye(3)
        J = scale ** 3
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    hs = sim.heat_system()
    T, _ = oracle.heat_solve(hs, 1e-14, 5000)
    np.testing.assert_allclose(T[hs.unknown], 0.3 + sc.params.dt * sc.params.H * J / (2.0 * sc.params.cp),
                               rtol=1e-12)


def test_sticky_plane_holds_what_lies_in_its_solid():
    """A sticky plane (reading R14) fixes every node on its solid side: particles
    deep in it stay where they are under gravity, while the nodes on the open
    side keep all three components."""
    from oracle.boundary import projector
    n, dx = (16, 16, 16), 1.0 / 16
    nrm = np.array([0.5, 0.8660254037844386, 0.0])
    d = float(nrm @ np.array([0.5, 0.7, 0.5]))
    walls = (scenes.WALL_NONE,) * 6
    P = projector(n, dx, walls, tuple(nrm), d, scenes.WALL_STICKY)
    below = oracle.node_positions(n, dx) @ nrm - d < 0
    assert 0 < below.sum() < below.size
    np.testing.assert_array_equal(P[below], 0.0)
    np.testing.assert_array_equal(P[~below], np.broadcast_to(np.eye(3), P[~below].shape))
    sc = scenes.droplet(n=16, r_cells=1.5, seed=26, gravity=(0.0, -9.8, 0.0), lambda_l=10.0, gamma=0.0,
                        center=(0.5, 0.35, 0.5))
    sc.plane_n, sc.plane_d, sc.plane_mode = tuple(nrm), d, scenes.WALL_STICKY
    x0 = sc.x.copy()
    assert np.all(x0 @ nrm - d < -3 * dx)
    sim = oracle.OracleSim(sc)
    sim.step()
    np.testing.assert_array_equal(sim.sc.x, x0)
    np.testing.assert_array_equal(sim.sc.v, 0.0)


def test_affine_grid_motion_moves_particles_and_carries_samples_exactly():
    """Under an affine grid velocity a + B x the end of a step is a closed form:
    particles move to x + dt (a + B x), liquids scale J by 1 + dt tr B and solids
    map F to (I + dt B) F (reading R11); carried samples move the same way and
    their area vectors follow Nanson's formula det(F) F^-T dA with F = I + dt B
    (the updated-Lagrangian area map of Eq. pestul, reading R16)."""
    sc = _mixed_scene()
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    rng = np.random.default_rng(17)
    a = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    xi = oracle.node_positions(sc.n, sc.dx)
    sim.vhat = a + xi @ B.T
    sim.That = None
    x0, s0, dA0, J0, F0 = sc.x.copy(), sc.s.copy(), sc.dA.copy(), sc.J.copy(), sc.F.copy()
    sim.prm.phase_change = False
    sim.g2p()
    out = sim.sc
    dt = sc.params.dt
    Fm = np.eye(3) + dt * B
    free = sim.count == 0
    np.testing.assert_allclose(out.x[free], x0[free] + dt * (a + x0[free] @ B.T), atol=1e-13)
    liq = free & (sc.phase == 0)
    sol = free & (sc.phase == 1)
    np.testing.assert_allclose(out.J[liq], (1 + dt * np.trace(B)) * J0[liq], rtol=1e-12)
    np.testing.assert_allclose(out.F[sol], np.einsum("ab,pbc->pac", Fm, F0[sol]), atol=1e-12)
    np.testing.assert_allclose(out.s, s0 + dt * (a + s0 @ B.T), atol=1e-13)
    nanson = np.linalg.det(Fm) * np.linalg.inv(Fm).T
    np.testing.assert_allclose(out.dA, dA0 @ nanson.T, atol=1e-14 * np.abs(dA0).max() + 1e-15)


def test_heat_operator_symmetric_spd_and_balance():
    sc = _thermal_scene()
    sim = oracle.OracleSim(sc)
    sim.resample(); sim.p2g()
    hs = sim.heat_system()
    idx = np.flatnonzero(hs.unknown)
    A = np.zeros((idx.size, idx.size))
    for c in range(idx.size):
        e = np.zeros(hs.G)
        e[idx[c]] = 1.0
        A[:, c] = hs.apply(e)[idx]
    np.testing.assert_allclose(A, A.T, atol=1e-13 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    # balance: summing all rows, the Laplacian cancels
    T, _ = oracle.heat_solve(hs, 1e-12, 5000)
    lhs = np.sum(hs.diag * (T - hs.Tn))
    # Robin flux of each sample: interpolate T over the stencil nodes that carry
    # thermal mass with renormalised weights
    w = hs.ss.N * hs.unknown[hs.ss.node]
    w = w / w.sum(1, keepdims=True)
    Ts = np.sum(w * T[hs.ss.node], 1)
    rhs = (-np.sum(sc.params.h * hs.area * Ts) + np.sum((sc.params.h * sc.Tbar + sc.b) * hs.area)
           + np.sum(sc.params.H * hs.Vn))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9)


def test_heat_conduction_term_is_minus_k_laplacian_on_a_regular_lattice():
    """Away from the particles' boundary the conduction rows are a weak form of
    -div(K grad T) (section "Temperature Update"): sum_p K V_p gradN_i(x_p) .
    grad T(x_p) = -int N_i K lap T = -K lap T V_i for a quadratic T, whose
    quadratic B-spline interpolant has the exact gradient. On a regular lattice of
    particles (two per cell and axis) the particle quadrature of it is exact, so
    the rows equal -K lap T V_i with V_i = sum_p N_i(x_p) V_p; for T = cos(k x)
    they approach K k^2 T_i V_i at second order in k dx."""
    from oracle.spline import scatter
    n, dx, K = (24, 12, 12), 1.0 / 24, 0.2
    rng = np.random.default_rng(3)
    x = scenes.lattice_in(lambda p: np.ones(p.shape[:-1], bool), np.array([2, 2, 2]), np.array([22, 10, 10]),
                          dx, rng, 2, jitter=0.0)
    V = np.full(x.shape[0], dx ** 3 / 8)
    G = int(np.prod(n))
    st = oracle.Stencil(x, dx, n)
    mT = scatter(G, st.node, st.N)
    no = np.zeros((0, 3))
    hs = oracle.HeatSystem(n, dx, 1e-3, 1.0, K, 0.0, 0.0, mT, np.zeros(G), x, V, no, no, np.zeros(0), np.zeros(0))
    Vi = scatter(G, st.node, st.N * V[:, None])
    xi = oracle.node_positions(n, dx)
    g = np.stack(np.unravel_index(np.arange(G), n, order="F"), -1)
    inner = np.all((g >= [4, 4, 4]) & (g <= [19, 7, 7]), 1)
    for T, lap in ((xi[:, 0] ** 2, 2.0), (xi[:, 1] ** 2 + xi[:, 2] ** 2, 4.0), (xi[:, 0] * xi[:, 2], 0.0)):
        L = hs.apply(T) - hs.diag * np.where(hs.unknown, T, 0.0)
        np.testing.assert_allclose(L[inner], -K * lap * Vi[inner], atol=1e-6 * K * 2.0 * Vi[inner].max())
    errs = []
    for period in (8, 16):
        k = 2.0 * np.pi / (period * dx)
        T = np.cos(k * xi[:, 0])
        L = hs.apply(T) - hs.diag * np.where(hs.unknown, T, 0.0)
        big = inner & (np.abs(T) > 0.5)
        errs.append(np.max(np.abs(L[big] / (K * k * k * T[big] * Vi[big]) - 1.0)))
    assert errs[1] < 0.05 and 3.0 < errs[0] / errs[1] < 5.0


def test_heat_uniform_ambient_is_fixed_point():
    sc = _thermal_scene()
    sc.T[:] = 1.5
    sc.gradT[:] = 0.0
    sc.Tbar[:] = 1.5
    sc.b[:] = 0.0
    sc.params.H = 0.0
    sim = oracle.OracleSim(sc)
    sim.resample(); sim.p2g()
    hs = sim.heat_system()
    T, _ = oracle.heat_solve(hs, 1e-13, 5000)
    np.testing.assert_allclose(T[hs.unknown], 1.5, rtol=1e-10)


# ----------------------------------------------------------------------------
# whole step (section "Conservation" example: explicit steps conserve exactly)
# ----------------------------------------------------------------------------

def test_explicit_step_conserves_momentum_and_angular_momentum():
    sc = scenes.droplet(n=16, r_cells=4.0, seed=31, spin=2.0, v0=(0.1, 0.0, -0.2), lambda_l=20.0)
    sc.params.gamma_lg = 0.2
    sc.params.dt = 1e-4
    m0 = np.sum(sc.m[:, None] * sc.v, 0)
    L0 = _angular(sc.x, sc.m, sc.v, sc.A, sc.dx)
    sim = oracle.OracleSim(sc, explicit=True)
    for _ in range(2):
        sim.step()
    s = sim.sc
    np.testing.assert_allclose(np.sum(s.m[:, None] * s.v, 0), m0, atol=1e-13 * np.abs(m0).max())
    np.testing.assert_allclose(_angular(s.x, s.m, s.v, s.A, s.dx), L0, atol=1e-12 * np.abs(L0).max())


def test_implicit_step_conserves_linear_momentum():
    sc = scenes.droplet(n=16, r_cells=4.0, seed=32, v0=(0.3, -0.1, 0.2), spin=1.0, lambda_l=50.0)
    m0 = np.sum(sc.m[:, None] * sc.v, 0)
    sim = oracle.OracleSim(sc)
    sim.step()
    s = sim.sc
    np.testing.assert_allclose(np.sum(s.m[:, None] * s.v, 0), m0, atol=1e-10 * np.abs(m0).max())


@pytest.mark.parametrize("method", ["tetra", "cubes"])
def test_step_with_a_generated_surface_conserves_momentum(method):
    """Section "Conservation": with samples generated on the particles' surface
    (either triangulation), split, P2G, the implicit solve with its final force
    evaluation, and the merge keep the particles' linear momentum."""
    sc = scenes.droplet(n=16, r_cells=4.0, seed=33, v0=(0.2, 0.1, -0.3), spin=1.5, lambda_l=50.0)
    m0 = np.sum(sc.m[:, None] * sc.v, 0)
    sim = oracle.OracleSim(sc)
    assert sim.generate_surface(9, 2.0, method) > 100
    sim.step()
    s = sim.sc
    np.testing.assert_allclose(np.sum(s.m[:, None] * s.v, 0), m0, atol=1e-10 * np.abs(m0).max())


def _analytic_fcr_hessian(F, mu, lam):
    """The 9x9 Hessian of the fixed-corotated energy from the analytic eigensystem of
    isotropic energies: with the signed SVD F = U diag(s) V^T, each pair (x, y)
    (third index z) has eigenvalue (psi_x - psi_y) / (s_x - s_y) on U sym(e_x e_y) V^T
    and (psi_x + psi_y) / (s_x + s_y) on U skew(e_x e_y) V^T, and the scaling modes
    U diag(q) V^T carry the eigen-pairs of d^2 psi / ds^2."""
    U, s, Vt = np.linalg.svd(F)
    s = s.copy()
    if np.linalg.det(U) < 0:
        U[:, 2] *= -1
        s[2] *= -1
    if np.linalg.det(Vt) < 0:
        Vt[2, :] *= -1
        s[2] *= -1
    J = s.prod()
    modes = []
    Hs = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            pi = np.prod([s[a] for a in range(3) if a != i])
            pj = np.prod([s[a] for a in range(3) if a != j])
            Hs[i, j] = (2 * mu if i == j else 0.0) + lam * pi * pj + (lam * (J - 1) * s[3 - i - j] if i != j else 0.0)
    w, q = np.linalg.eigh(Hs)
    for t in range(3):
        modes.append((w[t], U @ np.diag(q[:, t]) @ Vt))
    for x, y in ((0, 1), (0, 2), (1, 2)):
        z = 3 - x - y
        L = np.zeros((3, 3))
        L[x, y] = L[y, x] = 1 / math.sqrt(2)
        T = np.zeros((3, 3))
        T[x, y], T[y, x] = 1 / math.sqrt(2), -1 / math.sqrt(2)
        modes.append((2 * mu - lam * (J - 1) * s[z], U @ L @ Vt))
        modes.append((2 * mu - 4 * mu / (s[x] + s[y]) + lam * (J - 1) * s[z], U @ T @ Vt))
    return sum(lv * np.outer(Q.ravel(), Q.ravel()) for lv, Q in modes), modes


def test_solid_hessian_matches_analytic_eigensystem_and_projection_is_psd():
    from oracle.energy import NewtonState
    rng = np.random.default_rng(11)
    F = np.eye(3) + 0.45 * rng.standard_normal((6, 3, 3))
    F[0] = np.eye(3)
    F[1] = np.diag([0.5, 0.8, 1.4])                       # compressed: indefinite twist modes
    F[2] = np.diag([1.0, 1.0, -0.3])                      # inverted
    mu = np.full(6, 2.0)
    lam = np.full(6, 5.0)
    Hp = NewtonState.solid_hessian_psd(F, mu, lam)
    for p in range(6):
        H = np.zeros((9, 9))
        for l in range(9):
            E = np.zeros((1, 3, 3))
            E.reshape(9)[l] = 1.0
            H[:, l] = oracle.constitutive.fcr_dP(F[p:p + 1], E, mu[p:p + 1], lam[p:p + 1]).reshape(9)
        Ha, modes = _analytic_fcr_hessian(F[p], 2.0, 5.0)
        # the exact dP, applied to the nine unit directions, is the analytic Hessian
        np.testing.assert_allclose(H, Ha, atol=1e-12 * np.abs(Ha).max())
        # the projection clamps exactly the negative analytic eigenvalues
        Hplus = sum(max(lv, 0.0) * np.outer(Q.ravel(), Q.ravel()) for lv, Q in modes)
        np.testing.assert_allclose(Hp[p], Hplus, atol=1e-12 * np.abs(Ha).max())
        assert np.linalg.eigvalsh(Hp[p]).min() >= -1e-12 * np.abs(Ha).max()
    # at rest psi is convex: projected = exact
    assert min(lv for lv, _ in _analytic_fcr_hessian(F[0], 2.0, 5.0)[1]) >= -1e-14
    # the compressed state has negative (twist) eigenvalues, which the projection removes
    assert min(lv for lv, _ in _analytic_fcr_hessian(F[1], 2.0, 5.0)[1]) < 0.0


def test_projected_operator_psd_with_deformed_solids():
    sc = _mixed_scene()
    rng = np.random.default_rng(7)
    sol = sc.phase == scenes.PHASE_SOLID
    sc.F[sol] = np.diag([0.55, 0.8, 1.3]) + 0.1 * rng.standard_normal((sol.sum(), 3, 3))
    sc.params.E0 = 3000.0
    sc.params.gamma_lg = 0.0
    sim, st = _state(sc)
    v = st.vn * st.active[:, None]
    idx = np.flatnonzero(st.active)
    ncol = idx.size * 3
    g = np.stack(np.unravel_index(idx, sc.n, order="F"), -1)
    colour = (g % 5) @ np.array([1, 5, 25])
    ev = {}
    for mode in (HESS_EXACT, HESS_PROJECTED):
        # nodes of one colour are 5 apart, farther than any two nodes sharing a
        # particle (2), so one application per colour and component fills their columns
        H = np.zeros((ncol, ncol))
        for col in np.unique(colour):
            members = np.flatnonzero(colour == col)
            for q in range(3):
                e = np.zeros((st.G, 3))
                e[idx[members], q] = 1.0
                he = st.hessvec(v, e, mode)
                for j in members:
                    near = np.flatnonzero(np.all(np.abs(g - g[j]) <= 2, axis=1))
                    H[(3 * near[:, None] + np.arange(3)).ravel(), 3 * j + q] = he[idx[near]].ravel()
        np.testing.assert_allclose(H, H.T, atol=1e-10 * np.abs(H).max())
        ev[mode] = np.linalg.eigvalsh(0.5 * (H + H.T))
    mmin = st.m[idx].min()
    assert ev[HESS_EXACT].min() < mmin                     # the exact operator is indefinite here
    assert ev[HESS_PROJECTED].min() >= mmin - 1e-10 * np.abs(ev[HESS_PROJECTED]).max()


# ----------------------------------------------------------------------------
# Coulomb friction of the slip plane (section "Examples": drops on ramps with a
# friction coefficient) and the massless-sample variant (section "Surface
# Particle Sampling")
# ----------------------------------------------------------------------------

def _block_below_incline(theta_deg, mu):
    """A few particles deep inside the solid side of a slip plane: every node of
    their stencils is a plane node, so they move like a block on an incline."""
    sc = scenes.droplet(n=16, r_cells=1.0, seed=21, gravity=(0.0, -9.8, 0.0), lambda_l=0.0, gamma=0.0)
    a = math.radians(theta_deg)
    nrm = np.array([-math.sin(a), math.cos(a), 0.0])
    sc.plane_n = tuple(nrm)
    sc.plane_d = float(nrm @ np.array([0.5, 0.8, 0.5]))
    sc.plane_mode = scenes.WALL_SLIP
    sc.params.friction = mu
    rng = np.random.default_rng(4)
    x = np.array([0.5, 0.3, 0.5]) + rng.uniform(-1.0, 1.0, (12, 3)) * sc.dx
    assert np.all(x @ nrm - sc.plane_d < -4 * sc.dx)
    P = scenes._particles(x, 1.0, sc.dx, 8, rng)
    for k, val in P.items():
        setattr(sc, k, val)
    sc.s = np.zeros((0, 3))
    sc.dA = np.zeros((0, 3))
    sc.kind = np.zeros(0, np.uint8)
    sc.b = np.zeros(0)
    sc.Tbar = np.zeros(0)
    return sc, nrm


@pytest.mark.parametrize("theta,mu", [(30.0, 0.2), (30.0, 0.0), (30.0, 0.7), (10.0, 0.2)])
def test_friction_block_on_incline_matches_textbook(theta, mu):
    """From rest, one step: the block slides down the slope with acceleration
    g (sin theta - mu cos theta) when tan theta > mu, and stays at rest otherwise."""
    sc, nrm = _block_below_incline(theta, mu)
    sim = oracle.OracleSim(sc)
    sim.step()
    g = np.array(sc.params.gravity)
    down = g - (g @ nrm) * nrm
    down /= np.linalg.norm(down)
    a = math.radians(theta)
    acc = max(0.0, 9.8 * (math.sin(a) - mu * math.cos(a)))
    expect = sc.params.dt * acc * down
    np.testing.assert_allclose(sim.sc.v, np.broadcast_to(expect, sim.sc.v.shape), atol=1e-14)


def test_friction_never_adds_energy_and_reduces_to_slip():
    from oracle.boundary import coulomb_plane
    rng = np.random.default_rng(6)
    nrm = np.array([0.3, 0.9, -0.2])
    nrm /= np.linalg.norm(nrm)
    v = rng.standard_normal((500, 3))
    nodes = rng.uniform(size=500) < 0.8
    slip = v - np.outer(v @ nrm, nrm)
    np.testing.assert_allclose(coulomb_plane(v, nodes, nrm, 0.0), v, rtol=0, atol=1e-15)
    for mu in (0.1, 0.5, 3.0):
        out = coulomb_plane(v, nodes, nrm, mu)
        proj = out - np.outer(out @ nrm, nrm)
        # tangential speed never grows, direction kept, untouched away from the plane
        # or where the node leaves the plane
        assert np.all(np.linalg.norm(proj, axis=1) <= np.linalg.norm(slip, axis=1) + 1e-15)
        assert np.all(np.einsum("ga,ga->g", proj, slip) >= -1e-15)
        keep = ~nodes | (v @ nrm >= 0)
        np.testing.assert_array_equal(out[keep], v[keep])
        # the normal part is left for the projection
        np.testing.assert_allclose(out @ nrm, v @ nrm, rtol=0, atol=1e-15)


def _one_sided_droplet(massless):
    """Zero-gravity droplet whose samples on one side sit a cell outside the
    particles, so their stencils reach nodes that no particle touches."""
    sc = scenes.droplet(n=16, r_cells=4.0, seed=23, lambda_l=50.0, gamma=1.0)
    c = np.array([0.5, 0.5, 0.5])
    up = sc.s[:, 2] > c[2]
    rel = sc.s[up] - c
    r = np.linalg.norm(rel, axis=1, keepdims=True)
    sc.s[up] = c + rel * (r + sc.dx) / r
    sc.params.massless_surface = massless
    return sc


def test_massless_samples_lose_momentum_only_through_massless_nodes():
    """The paper's point: with massless samples, surface forces that land on nodes
    without mass are dropped, so the step no longer conserves momentum; the
    split-mass samples with balance particles conserve it. Explicit steps, as in
    the paper's conservation example."""
    out = {}
    for massless in (False, True):
        sc = _one_sided_droplet(massless)
        sim = oracle.OracleSim(sc, explicit=True)
        sim.resample()
        sim.p2g()
        m_grid = sim.grid["m"]
        np.testing.assert_allclose(m_grid.sum(), sc.m.sum(), rtol=1e-13)
        sim.grid_update()
        st = sim.state
        # force scale: at v = v^n without gravity the gradient is dt times the internal forces
        scale = np.abs(st.gradient(st.vn)).sum()
        mom = np.sum(m_grid[:, None] * sim.vhat, 0)
        out[massless] = (np.abs(mom).max() / scale, m_grid)
    # conservative variant: momentum of the grid stays zero to round-off
    assert out[False][0] < 1e-12
    # massless variant: the nodes touched only by the outer samples carry forces but no mass
    assert out[True][0] > 1e-4
    assert np.any((out[True][1] == 0) & (out[False][1] > 0))


# ----------------------------------------------------------------------------
# Dirichlet conditions (section "Conservation of Mass and Momentum", Eq. vbc:
# v . n = 0 on slip boundaries, v = 0 on sticky ones) as a per-node projection
# ----------------------------------------------------------------------------

def test_projector_is_the_orthogonal_projection_onto_admissible_velocities():
    from oracle.boundary import projector, slip_plane_nodes
    n = (9, 8, 10)
    dx = 1.0 / 10
    walls = (scenes.WALL_SLIP, scenes.WALL_STICKY, scenes.WALL_SLIP, scenes.WALL_NONE,
             scenes.WALL_NONE, scenes.WALL_SLIP)
    nrm = np.array([0.3, 0.9, 0.2])
    nrm /= np.linalg.norm(nrm)
    d = float(nrm @ np.array([0.45, 0.25, 0.5]))
    P = projector(n, dx, walls, tuple(nrm), d, scenes.WALL_SLIP)
    # symmetric and idempotent at every node
    np.testing.assert_allclose(P, np.swapaxes(P, 1, 2), atol=1e-15)
    np.testing.assert_allclose(np.einsum("gab,gbc->gac", P, P), P, atol=1e-14)
    g = np.stack(np.unravel_index(np.arange(P.shape[0]), n, order="F"), -1)
    xi = oracle.node_positions(n, dx)
    below = xi @ nrm - d < 0
    slip_x = g[:, 0] <= 1
    sticky = g[:, 0] >= n[0] - 2
    slip_y = g[:, 1] <= 1
    slip_z = g[:, 2] >= n[2] - 2
    e = np.eye(3)
    for k in range(P.shape[0]):
        walls_here = [a for a, on in enumerate((slip_x[k], slip_y[k], slip_z[k])) if on]
        if sticky[k] or (below[k] and walls_here) or len(walls_here) == 3:
            expect = np.zeros((3, 3))
        elif below[k]:
            expect = e - np.outer(nrm, nrm)
        else:
            expect = e.copy()
            for a in walls_here:
                expect[a, a] = 0.0
        np.testing.assert_allclose(P[k], expect, atol=1e-15)
    # the friction nodes are exactly the nodes projected by the plane alone
    plane_only = np.array([np.allclose(P[k], e - np.outer(nrm, nrm)) for k in range(P.shape[0])])
    np.testing.assert_array_equal(slip_plane_nodes(n, dx, walls, tuple(nrm), d, scenes.WALL_SLIP), plane_only)


# ----------------------------------------------------------------------------
# Contact angle (section "Contact Angle"): Young's law as the minimum of the
# surface energy of a resting drop
# ----------------------------------------------------------------------------

def _cap_energy(theta_deg, volume, k_sl, n, ncap=4000, nbase=2000):
    """Surface energy at rest (F = I) of a spherical cap of the given volume that
    meets a horizontal slip plane at theta: liquid-gas samples on the cap, and
    samples on the wetted disk with area vectors into the plane, classified and
    weighted by the oracle (reading R13: within dx of the plane is solid-liquid)."""
    th = math.radians(theta_deg)
    R = (volume / ((1 - math.cos(th)) ** 2 * (2 + math.cos(th)) * math.pi / 3)) ** (1 / 3)
    h, a, z0 = R * (1 - math.cos(th)), R * math.sin(th), 0.3
    c = np.array([0.5, 0.5, z0 - R * math.cos(th)])
    sc = scenes.droplet(n=n, r_cells=2.0, seed=1, gamma=1.0, lambda_l=0.0)
    sc.params.gamma_sl = k_sl
    sc.plane_n, sc.plane_d, sc.plane_mode = (0.0, 0.0, 1.0), z0, scenes.WALL_SLIP
    gold = math.pi * (3 - math.sqrt(5))
    k = np.arange(ncap) + 0.5
    zr = (z0 + k / ncap * h - c[2]) / R          # heights uniform in [z0, top]: uniform area
    rr = np.sqrt(np.maximum(0.0, 1 - zr * zr))
    nrm = np.stack([rr * np.cos(k * gold), rr * np.sin(k * gold), zr], -1)
    kb = np.arange(nbase) + 0.5
    rb = a * np.sqrt(kb / nbase)
    base = np.stack([0.5 + rb * np.cos(kb * gold), 0.5 + rb * np.sin(kb * gold), np.full(nbase, z0)], -1)
    sc.s = np.concatenate([c + R * nrm, base])
    sc.dA = np.concatenate([nrm * (2 * math.pi * R * h / ncap), np.tile([0.0, 0.0, -math.pi * a * a / nbase], (nbase, 1))])
    ns = sc.s.shape[0]
    sc.kind, sc.b, sc.Tbar = np.zeros(ns, np.uint8), np.zeros(ns), np.zeros(ns)
    rng = np.random.default_rng(0)
    x = np.array([0.5, 0.5, z0 + 0.5 * h]) + rng.uniform(-0.2, 0.2, (20, 3)) * min(R, h)
    for key, val in scenes._particles(x, 1.0, sc.dx, 8, rng).items():
        setattr(sc, key, val)
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    st = sim.newton_state()
    return st.energy(np.zeros_like(st.vn))      # at rest only the surface term remains


@pytest.mark.parametrize("k_sl", [0.5, 0.0])
def test_static_contact_angle_converges_to_youngs_law(k_sl):
    """At fixed volume, gamma_LG A_cap + k_SL,eff A_wet is smallest where
    cos theta = -k_SL,eff / gamma_LG. The oracle's discrete energy (samples,
    interface kinds, coefficients) has its minimum there up to the width of the
    solid-liquid band, which shrinks with dx: under 3 degrees at 17 cells of
    radius. A flipped sign of the solid-liquid coefficient would put it at the
    supplementary angle."""
    young = math.degrees(math.acos(-k_sl))
    volume = 2.0 / 3.0 * math.pi * (10 / 64) ** 3
    errs = []
    for n in (64, 128):
        ths = young + np.arange(-10.0, 10.5, 5.0)
        es = np.array([_cap_energy(t, volume, k_sl, n) for t in ths])
        assert np.argmin(es) in (1, 2, 3)
        q = np.polyfit(ths, es, 2)
        errs.append(abs(-q[1] / (2 * q[0]) - young))
    assert errs[1] < 3.0
    assert errs[1] <= errs[0] + 0.1


# ----------------------------------------------------------------------------
# Curved solids (the glass of section "Examples"): a spherical level set
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("outside", [True, False])
def test_sphere_projector_removes_the_local_normal(outside):
    from oracle.boundary import projector, sphere_phi_normal
    n, dx = (12, 12, 12), 1.0 / 12
    sphere = (0.5, 0.52, 0.47, 0.31, outside)
    walls = (scenes.WALL_SLIP,) + (scenes.WALL_NONE,) * 5
    P = projector(n, dx, walls, sphere=sphere, sphere_mode=scenes.WALL_SLIP)
    xi = oracle.node_positions(n, dx)
    phi, nrm = sphere_phi_normal(xi, sphere)
    g = np.stack(np.unravel_index(np.arange(P.shape[0]), n, order="F"), -1)
    # the normal is the unit gradient of phi (central differences of the distance)
    h = 1e-6
    fd = np.stack([(sphere_phi_normal(xi + h * e, sphere)[0] - sphere_phi_normal(xi - h * e, sphere)[0]) / (2 * h)
                   for e in np.eye(3)], -1)
    np.testing.assert_allclose(fd, nrm, atol=1e-6)
    solid = phi < 0
    wall = g[:, 0] <= 1
    assert solid.sum() > 50 and (~solid).sum() > 50
    np.testing.assert_allclose(P, np.swapaxes(P, 1, 2), atol=1e-15)
    np.testing.assert_allclose(np.einsum("gab,gbc->gac", P, P), P, atol=1e-14)
    s = solid & ~wall
    np.testing.assert_allclose(P[s], np.eye(3) - np.einsum("ga,gb->gab", nrm[s], nrm[s]), atol=1e-15)
    np.testing.assert_array_equal(P[solid & wall], 0.0)
    np.testing.assert_allclose(P[~solid & ~wall], np.broadcast_to(np.eye(3), P[~solid & ~wall].shape), atol=0)


def _block_in_bowl(r_cells, mu, alpha_deg=30.0):
    """A few particles inside a spherical bowl's wall, at polar angle alpha from
    its lowest point, deep enough that every node of their stencils is solid."""
    n = 64
    dx = 1.0 / n
    c = np.array([0.5, 0.5, 0.55])
    R = r_cells * dx
    sc = scenes.droplet(n=n, r_cells=1.0, seed=25, gravity=(0.0, 0.0, -9.8), lambda_l=0.0, gamma=0.0)
    sc.sphere, sc.sphere_mode = (c[0], c[1], c[2], R, True), scenes.WALL_SLIP
    sc.params.friction = mu
    a = math.radians(alpha_deg)
    p0 = c + (R + 4.0 * dx) * np.array([math.sin(a), 0.0, -math.cos(a)])
    rng = np.random.default_rng(8)
    x = p0 + rng.uniform(-0.3, 0.3, (8, 3)) * dx
    for key, val in scenes._particles(x, 1.0, dx, 8, rng).items():
        setattr(sc, key, val)
    sc.s, sc.dA = np.zeros((0, 3)), np.zeros((0, 3))
    sc.kind, sc.b, sc.Tbar = np.zeros(0, np.uint8), np.zeros(0), np.zeros(0)
    return sc


@pytest.mark.parametrize("mu", [0.0, 0.2])
def test_block_in_a_bowl_slides_as_on_its_tangent_plane(mu):
    """One step from rest: each particle moves as a block on the incline tangent
    to the bowl at its own position, a = g (sin alpha - mu cos alpha) down the
    slope. The node normals vary over the stencil, but their first-order
    variation cancels (the weights have zero first moment about the particle),
    so the error falls with the square of dx / R."""
    from oracle.boundary import sphere_phi_normal
    err = []
    for r_cells in (10.0, 20.0):
        sc = _block_in_bowl(r_cells, mu)
        sim = oracle.OracleSim(sc)
        sim.step()
        g = np.array(sc.params.gravity)
        _, nrm = sphere_phi_normal(sc.x, sc.sphere)
        gn = nrm @ g
        gt = g - gn[:, None] * nrm
        lt = np.linalg.norm(gt, axis=1)
        expect = sc.params.dt * np.maximum(0.0, 1.0 - mu * np.abs(gn) / lt)[:, None] * gt
        err.append(np.abs(sim.sc.v - expect).max() / (sc.params.dt * 9.8))
    # the particles sit 4 cells into the wall: radii of curvature 14 and 24 cells, so
    # second order gives a ratio (14/24)^2 = 0.34 (first order would give 0.58)
    assert err[1] < 2e-3
    assert err[1] < 0.45 * err[0]


def test_sphere_sticky_nodes_and_solid_liquid_samples():
    """A sticky sphere fixes its solid nodes; samples within dx of the sphere's
    solid are solid-liquid and take the effective coefficient (reading R13 with
    the sphere's signed distance)."""
    from oracle.boundary import projector, sphere_phi_normal
    n, dx = (16, 16, 16), 1.0 / 16
    sphere = (0.5, 0.5, 0.5, 0.35, True)
    P = projector(n, dx, (scenes.WALL_NONE,) * 6, sphere=sphere, sphere_mode=scenes.WALL_STICKY)
    phi, _ = sphere_phi_normal(oracle.node_positions(n, dx), sphere)
    np.testing.assert_array_equal(P[phi < 0], 0.0)
    np.testing.assert_array_equal(P[phi >= 0], np.broadcast_to(np.eye(3), P[phi >= 0].shape))
    sc = scenes.droplet(n=16, r_cells=4.0, seed=26, gamma=1.0)
    sc.params.gamma_sl = 0.4
    sc.sphere, sc.sphere_mode = (0.5 + 1.0 / 16, 0.5, 0.5, 5.0 / 16, True), scenes.WALL_SLIP
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    near = sphere_phi_normal(sc.s, sc.sphere)[0] < sc.dx
    assert near.any() and (~near).any()
    np.testing.assert_array_equal(sim.sc.kind, near.astype(np.uint8))
    np.testing.assert_allclose(sim.gamma, np.where(near, 0.4, 1.0))


# ----------------------------------------------------------------------------
# The surface part of the definiteness fix (section "Momentum Update": the
# projected Hessian keeps the Gauss-Newton term and the positive, conformal part
# of the cofactor curvature). The split into conformal and anti-conformal parts
# depends on the relative orientation of the frames of n and a: the pins below fail
# if one frame is flipped, if the anti-conformal combination is kept, or if the
# positive part is scaled wrongly (each checked by planting it in the oracle).
# ----------------------------------------------------------------------------

def _cof_apply(X, a):
    """cof(X) a written as (X u) x (X w) for any u, w with u x w = a (no epsilon
    tensor, no inverse, so it also holds for singular X)."""
    an = np.linalg.norm(a)
    u = np.cross(a, [1.0, 0.3, -0.2])
    u /= np.linalg.norm(u)
    w = np.cross(a / an, u) * an          # u x w = u x (a x u) |a|/|a| = a (u unit, u . a = 0)
    return np.cross(X @ u, X @ w), u, w


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def _one_sample_state(Fh, a, gamma, dt=0.01):
    """A NewtonState with one surface sample whose iterate gives F^ = Fh, and one
    particle with no stiffness (so only the sample acts; the nodes carry no mass)."""
    n, dx = (8, 8, 8), 1.0 / 8
    s = np.array([[0.43, 0.51, 0.47]])
    x = np.array([[0.5, 0.5, 0.5]])
    one = np.ones(1)
    st = oracle.NewtonState(n, dx, dt, np.zeros(3), np.zeros(512), np.zeros((512, 3)), x, one * dx ** 3,
                            one, np.eye(3)[None], np.zeros(1, np.int64), 0.0, 0.0, np.zeros(1), np.zeros(1),
                            s, a[None], np.array([gamma]))
    xi = oracle.node_positions(n, dx)
    v = (xi - s) @ ((Fh - np.eye(3)) / dt).T     # affine: F^ = I + dt L(s) = Fh exactly
    return st, v, xi, s[0]


def _sample_map(st, v, xi, s, X, mode):
    """The sample's dG for dF^ = X: an affine direction dv_i = X (x_i - s) has
    dF^ = X exactly, and sum_i out_i (x_i - s)^T = dt^2 dG because
    sum_i gradN_i (x_i - s)^T = I (spline moment identity)."""
    dv = (xi - s) @ X.T
    out = st.hessvec(v, dv, mode)
    return out.T @ (xi - s) / st.dt ** 2


def test_conformal_frames_reproduce_the_cofactor_curvature():
    """n . cof(X) a = |a| det[t_i . X s_j] with the oracle's right-handed frames."""
    from oracle.energy import _frame
    rng = np.random.default_rng(31)
    for _ in range(50):
        X = rng.standard_normal((3, 3))
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        a = rng.standard_normal(3) * rng.uniform(0.1, 3.0)
        lhs = nrm @ _cof_apply(X, a)[0]
        t1, t2 = _frame(nrm[None])
        s1, s2 = _frame((a / np.linalg.norm(a))[None])
        x = np.array([[t[0] @ X @ sv[0] for sv in (s1, s2)] for t in (t1, t2)])
        assert abs(lhs - np.linalg.norm(a) * np.linalg.det(x)) <= 1e-12 * max(1.0, abs(lhs))


def test_projected_surface_term_keeps_the_conformal_and_drops_the_anticonformal_curvature():
    rng = np.random.default_rng(32)
    for trial in range(6):
        Fh = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        a = rng.standard_normal(3) * 0.02
        gamma = rng.uniform(0.2, 2.0)
        st, v, xi, s = _one_sample_state(Fh, a, gamma)
        c = _cof_apply(Fh, a)[0]
        nrm = c / np.linalg.norm(c)
        # tangential frames of n and a/|a|, built here from a random rotation (the
        # conformal span does not depend on the in-plane angle, only on handedness)
        R1, R2 = _rotation(rng), _rotation(rng)
        t1 = np.cross(nrm, R1[0]); t1 /= np.linalg.norm(t1); t2 = np.cross(nrm, t1)
        ah = a / np.linalg.norm(a)
        s1 = np.cross(ah, R2[0]); s1 /= np.linalg.norm(s1); s2 = np.cross(ah, s1)
        conf = [np.outer(t1, s1) + np.outer(t2, s2), np.outer(t1, s2) - np.outer(t2, s1)]
        anti = [np.outer(t1, s1) - np.outer(t2, s2), np.outer(t1, s2) + np.outer(t2, s1)]
        al, be = rng.standard_normal(2)
        Xc = al * conf[0] + be * conf[1]
        Xa = al * anti[0] + be * anti[1]
        scale = gamma * np.linalg.norm(a) * np.linalg.norm(Xc)
        # conformal directions: projected == exact
        mE = _sample_map(st, v, xi, s, Xc, HESS_EXACT)
        mP = _sample_map(st, v, xi, s, Xc, HESS_PROJECTED)
        np.testing.assert_allclose(mP, mE, atol=1e-10 * scale)
        # anti-conformal directions: projected == exact minus the whole curvature,
        # gamma K[X] with K[X] = grad_X (n . cof(X) a) = ((X w) x n) u^T + (n x (X u)) w^T
        _, u, w = _cof_apply(Xa, a)
        K = np.outer(np.cross(Xa @ w, nrm), u) + np.outer(np.cross(nrm, Xa @ u), w)
        mE = _sample_map(st, v, xi, s, Xa, HESS_EXACT)
        mP = _sample_map(st, v, xi, s, Xa, HESS_PROJECTED)
        np.testing.assert_allclose(mE - mP, gamma * K, atol=1e-10 * scale)
        # ... and what remains is the Gauss-Newton form gamma |(I - n n^T) dc|^2 / |c|,
        # dc = (X u) x (F^ w) + (F^ u) x (X w)
        _, u, w = _cof_apply(Fh, a)
        dc = np.cross(Xa @ u, Fh @ w) + np.cross(Fh @ u, Xa @ w)
        dcp = dc - nrm * (nrm @ dc)
        np.testing.assert_allclose(np.sum(Xa * mP), gamma * dcp @ dcp / np.linalg.norm(c),
                                   rtol=1e-10, atol=1e-12 * scale * np.linalg.norm(Xa))


def test_exact_minus_projected_surface_term_is_negative_semidefinite():
    """Per sample, in dF^ space: exact - projected = -gamma |a| times the projector on
    the anti-conformal plane, so two eigenvalues -gamma |a| and seven zeros."""
    rng = np.random.default_rng(33)
    for trial in range(4):
        Fh = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        a = rng.standard_normal(3) * 0.05
        gamma = rng.uniform(0.2, 2.0)
        st, v, xi, s = _one_sample_state(Fh, a, gamma)
        D = np.zeros((9, 9))
        for k in range(9):
            E = np.zeros(9)
            E[k] = 1.0
            E = E.reshape(3, 3)
            D[:, k] = (_sample_map(st, v, xi, s, E, HESS_EXACT) - _sample_map(st, v, xi, s, E, HESS_PROJECTED)).ravel()
        ga = gamma * np.linalg.norm(a)
        np.testing.assert_allclose(D, D.T, atol=1e-10 * ga)
        ev = np.sort(np.linalg.eigvalsh(0.5 * (D + D.T)))
        np.testing.assert_allclose(ev, [-ga, -ga] + [0.0] * 7, atol=1e-9 * ga)


def test_solid_at_the_melting_point_stores_the_liquids_energy():
    """Reading of section "Thermomechanical Material Dependence and Phase Change"
    with the candle example's single bulk modulus for both phases: E(T) reaches 0
    at T_melt and sets the shear modulus only, so a solid at the melting point with
    F = c I has the liquid's energy lambda_l/2 (J - 1)^2 and force at J = c^3 (at
    the step's start, v = 0, where the liquid's J and the solid's det F agree)."""
    base = scenes.droplet(n=12, r_cells=3.0, seed=31, lambda_l=70.0, gamma=0.0)
    base.params.E0 = 500.0
    base.params.T0, base.params.T_melt = 0.0, 10.0
    c = 0.97
    liq = base.copy()
    liq.J = np.full(liq.J.shape, c ** 3)
    sol = base.copy()
    sol.phase[:] = scenes.PHASE_SOLID
    sol.F = np.broadcast_to(c * np.eye(3), sol.F.shape).copy()
    sol.T = np.full(sol.T.shape, 10.0)       # at the melting point: E = 0
    st = []
    for sc in (liq, sol):
        sim, s = _state(sc)
        st.append(s)
    v0 = np.zeros((st[0].G, 3))
    e_liq, e_sol = st[0].energy(v0), st[1].energy(v0)
    assert e_liq > 0
    np.testing.assert_allclose(e_sol, e_liq, rtol=1e-12)
    g_liq, g_sol = st[0].gradient(v0), st[1].gradient(v0)
    np.testing.assert_allclose(g_sol, g_liq, rtol=0, atol=1e-12 * np.abs(g_liq).max())
    # below the melting point the shear modulus adds energy for a sheared F
    sol2 = sol.copy()
    sol2.T = np.full(sol.T.shape, 5.0)
    sol2.F = np.broadcast_to(np.array([[1.0, 0.1, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]), sol.F.shape).copy()
    _, s2 = _state(sol2)
    assert s2.energy(v0) > 0


# ----------------------------------------------------------------------------
# Pins added where a planted mistake in the oracle went unnoticed by the others
# ----------------------------------------------------------------------------

def test_gamma_reads_a_uniform_temperature_exactly_at_every_sample():
    """The renormalised interpolation of reading R9 returns a uniform grid
    temperature unchanged at every sample, also where only part of the sample's
    stencil carries thermal mass (samples on and just outside the surface)."""
    sc = scenes.droplet(n=12, r_cells=3.0, seed=24, thermal=True)
    sc.T[:] = 1.7
    sc.gradT[:] = 0.0
    rng = np.random.default_rng(5)
    d = rng.standard_normal((60, 3))
    r = (3.0 + rng.uniform(-0.5, 1.2, (60, 1))) * sc.dx
    sc.s = np.full(3, 0.5) + d / np.linalg.norm(d, axis=1, keepdims=True) * r
    sc.dA = np.tile([0.0, 0.0, sc.dx ** 2], (60, 1))
    sc.kind, sc.b, sc.Tbar = np.zeros(60, np.uint8), np.zeros(60), np.zeros(60)
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    st = oracle.Stencil(sc.s, sc.dx, sc.n)
    has = sim.grid["mT"][st.node] > 0
    partial = has.any(1) & ~has.all(1)
    assert partial.sum() >= 20
    np.testing.assert_allclose(sim.Tr[has.any(1)], 1.7, rtol=1e-13)


@pytest.mark.parametrize("T,frac", [(298.0, 1.0), (299.25, 0.75), (300.5, 0.5), (303.0, 0.0), (320.0, 0.0)])
def test_solid_shear_modulus_follows_youngs_modulus_of_temperature(T, frac):
    """Section "Thermomechanical Material Dependence": the wax's Young's modulus
    falls linearly from E0 at T0 to zero at the melting point, and the shear
    modulus of isotropic elasticity is E / (2 (1 + nu)). Measured from the
    fixed-corotated energy of a small simple shear (J = 1, so only the shear
    modulus acts): psi = mu gamma^2 / 2 + O(gamma^4)."""
    from oracle.step import solid_lame
    prm = scenes.wax(nx=16, ny=16, nz=16, cube_cells=4).params
    assert (prm.T0, prm.T_melt, prm.E0, prm.nu) == (298.0, 303.0, 1e4, 0.3)
    mu, lam = solid_lame(np.array([T]), prm)
    g = 1e-4
    F = np.eye(3)[None].copy()
    F[0, 0, 1] = g
    psi = cst.fcr_energy(F, mu, lam)[0]
    assert 2.0 * psi / g ** 2 == pytest.approx(frac * 1e4 / (2.0 * 1.3), rel=1e-7, abs=1e-9)


def test_generated_kinds_are_the_resample_classification():
    """Samples made on the particles' surface carry the interface kind that
    resampling assigns (reading R13: solid-liquid within dx of the plane), so
    both sides of the pipeline classify a generated sample alike."""
    sc = scenes.incline(n=48, n_drops=2, r_range=(3.0, 5.0), seed=43, gap_cells=(0.0, 0.5))
    sim = oracle.OracleSim(sc)
    sim.generate_surface(5)
    k0 = sim.sc.kind.copy()
    d = sim.sc.s @ np.asarray(sc.plane_n) - sc.plane_d
    assert np.sum((d > 0.5 * sc.dx) & (d < sc.dx)) > 10     # samples in the outer half of the band
    sim.resample()
    np.testing.assert_array_equal(k0, sim.sc.kind)
    assert 0 < int(k0.sum()) < k0.size


def test_viscous_term_weighs_the_current_volume():
    """Eq. disc_force's viscous term integrates over the current volume V^n = J^n V^0:
    for an affine grid velocity v = B x its energy is dt mu / 2 |sym B|^2 sum J^n V^0."""
    sc = _moving_droplet(mu_l=0.3, lambda_l=0.0, gamma=0.0)
    sc.J = RNG.uniform(0.4, 0.6, sc.J.shape)
    sim, st = _state(sc)
    B = RNG.standard_normal((3, 3))
    v = _affine_grid_velocity(sc, B)
    kin = 0.5 * np.sum(st.m[st.active] * np.sum((v - st.vn)[st.active] ** 2, -1))
    S = 0.5 * (B + B.T)
    expect = sc.params.dt * 0.3 / 2.0 * np.sum(S * S) * np.sum(sc.J * sc.V0)
    np.testing.assert_allclose(st.energy(v) - kin, expect, rtol=1e-11)


def test_closest_parent_ties_go_to_the_smaller_index():
    """Reading R12: equal squared distances go to the smaller particle index
    (exact ties by construction: offsets of powers of two)."""
    from oracle.resample import nearest_parent
    c = np.array([0.5, 0.5, 0.5])
    h = 2.0 ** -6
    offs = np.array([[h, 0, 0], [-h, 0, 0], [0, h, 0], [0, 0, -h]])
    for perm in ([0, 1, 2, 3], [3, 2, 1, 0], [2, 0, 3, 1]):
        x = np.vstack([c + 3 * h, c + offs[perm]])
        p, best = nearest_parent(x, c[None])
        assert p[0] == 1 and best[0] == h * h
    # a particle a few ulps closer wins over the smaller index
    x = np.vstack([c + [h, 0, 0], c + [h - 2.0 ** -48, 0, 0]])
    assert x[1, 0] - c[0] < x[0, 0] - c[0]
    assert nearest_parent(x, c[None])[0][0] == 1


@pytest.mark.parametrize("start,T,end", [(scenes.PHASE_SOLID, 303.4, scenes.PHASE_LIQUID),
                                         (scenes.PHASE_LIQUID, 302.6, scenes.PHASE_SOLID),
                                         (scenes.PHASE_SOLID, 302.6, scenes.PHASE_SOLID),
                                         (scenes.PHASE_LIQUID, 303.4, scenes.PHASE_LIQUID)])
def test_phase_change_at_the_melting_point(start, T, end):
    """Section "Thermomechanical Material Dependence and Phase Change": a particle
    whose temperature after the step lies above the melting point is liquid, one
    below it solid, and a particle that changes phase starts from its rest state
    (J = 1, F = I). A uniform temperature with no heat flow stays uniform through
    the transfers, so every particle ends at T."""
    sc = scenes.wax(nx=16, ny=16, nz=16, cube_cells=4)
    sc.phase[:] = start
    sc.T[:] = T
    sc.gradT[:] = 0.0
    sc.params.K = 0.0
    sc.params.h = 0.0
    sc.params.H = 0.0
    sc.b[:] = 0.0
    sc.params.gamma_p = (0.0, 0.0, 0.0, 0.0)
    sc.params.gravity = (0.0, 0.0, 0.0)
    sc.J[:] = 0.97
    sc.F[:] = 1.01 * np.eye(3)
    sim = oracle.OracleSim(sc)
    sim.step()
    np.testing.assert_allclose(sim.sc.T, T, rtol=1e-12)
    np.testing.assert_array_equal(sim.sc.phase, end)
    if end != start:
        np.testing.assert_array_equal(sim.sc.J, 1.0)
        np.testing.assert_array_equal(sim.sc.F, np.broadcast_to(np.eye(3), sim.sc.F.shape))


def test_gamma_law_stays_in_its_range():
    """The wax's gamma(T) = 0.1 - 0.01 (T - T0) is clamped to [0, 0.1] (reading R9):
    below T0 it keeps 0.1, past T0 + 10 it is zero, never negative."""
    from oracle.step import gamma_of
    prm = scenes.wax(nx=16, ny=16, nz=16, cube_cells=4).params
    T = np.array([prm.T0 - 5.0, prm.T0, prm.T0 + 5.0, prm.T0 + 10.0, prm.T0 + 50.0])
    g = gamma_of(T, np.zeros(5, np.uint8), prm)
    np.testing.assert_allclose(g, [0.1, 0.1, 0.05, 0.0, 0.0], atol=1e-15)
