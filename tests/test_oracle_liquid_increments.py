"""The liquid energy is exactly quadratic in the grid velocity (J is affine in v,
section "Momentum Update", Eq. fe), so its gradient changes by exactly H_l dv.
This is what lets a Newton solve carry the liquid gradient as one float64
evaluation at the initial guess plus float32 operator increments alpha H_l d
(float32 arithmetic and float32 node sums emulated here in numpy), reaching the
1e-6 residual as the float64 solve does, while a float32 liquid gradient stalls
near 1e-4 (the residual of a resting drop is a small difference of large
hydrostatic forces)."""
import copy

import numpy as np

import oracle
from oracle.boundary import apply_projector
from oracle.energy import HESS_EXACT, HESS_PROJECTED
from oracle.solver import armijo, pcg
from paper_2101_12408_gb300 import scenes


def _liquid_hessvec32(state, d):
    st, liq = state.st, state.liq
    dN = st.dN.astype(np.float32)
    tr = np.einsum("pqa,pqa->p", d.astype(np.float32)[st.node], dN)
    kap = (state.dt ** 2 * state.lam_l * state.Jn ** 2 * state.V0 * liq).astype(np.float32)
    out = np.zeros((state.G, 3), np.float32)
    np.add.at(out, st.node, (kap * tr)[:, None, None] * dN)
    return out.astype(np.float64)


def _liquid_gradient32(state, v):
    st, liq = state.st, state.liq
    dN = st.dN.astype(np.float32)
    tr = np.einsum("pqa,pqa->p", v.astype(np.float32)[st.node], dN)
    J = (np.float32(1) + np.float32(state.dt) * tr) * state.Jn.astype(np.float32)
    k = (state.dt * state.lam_l * state.Jn * state.V0 * liq).astype(np.float32)
    out = np.zeros((state.G, 3), np.float32)
    np.add.at(out, st.node, (k * (J - np.float32(1)))[:, None, None] * dN)
    return out.astype(np.float64)


def _solve(state, P, prm, form, max_newton):
    """Newton-CG as the oracle's solver, with the liquid gradient in one of three
    forms; returns the true float64 relative residual per iterate."""
    rest = copy.copy(state)
    rest.lam_l = 0.0
    act = state.active
    inv_m = np.where(act, 1.0 / np.where(act, state.m, 1.0), 0.0)

    def proj(u):
        return apply_projector(P, u) * act[:, None]

    v = proj(state.vn + prm.dt * state.g)
    g0 = state.gradient(v) - rest.gradient(v)
    acc = np.zeros_like(v)
    true, r0 = [], None
    for _ in range(max_newton):
        if form == "fp64":
            g = state.gradient(v)
        elif form == "increments":
            g = rest.gradient(v) + g0 + acc
        else:
            g = rest.gradient(v) + _liquid_gradient32(state, v)
        r = proj(g)
        rt = proj(state.gradient(v))
        true.append(float(np.sqrt(np.sum(rt * rt))))
        rn = float(np.sqrt(np.sum(r * r)))
        r0 = rn if r0 is None else r0
        if rn <= 1e-6 * r0:
            break
        d, _ = pcg(lambda u: proj(state.hessvec(v, proj(u), HESS_PROJECTED)), -r,
                   lambda u: proj(u * inv_m[:, None]), 1e-3, 1000)
        alpha = armijo(lambda a: state.energy(v + a * d), state.energy(v), float(np.sum(r * d)), 12)
        if alpha is None:
            break
        v = v + alpha * d
        acc = acc + alpha * _liquid_hessvec32(state, d)
    return np.array(true) / true[0]


def _state():
    sc = scenes.incline(n=48, n_drops=2, r_range=(3.0, 5.0), seed=43, gap_cells=(0.0, 0.5))
    sim = oracle.OracleSim(sc)
    sim.resample()
    sim.p2g()
    return sim, sim.newton_state()


def test_liquid_gradient_changes_by_exactly_its_hessian():
    sim, st = _state()
    rest = copy.copy(st)
    rest.lam_l = 0.0
    rng = np.random.default_rng(8)
    v = rng.standard_normal(st.vn.shape) * st.active[:, None]
    dv = rng.standard_normal(st.vn.shape) * st.active[:, None]
    gl = lambda u: st.gradient(u) - rest.gradient(u)  # noqa: E731
    hl = st.hessvec(v, dv, HESS_EXACT) - rest.hessvec(v, dv, HESS_EXACT)
    diff = gl(v + dv) - gl(v)
    np.testing.assert_allclose(diff, hl, atol=1e-10 * np.abs(hl).max())


def test_float32_increments_reach_the_newton_tolerance():
    sim, st = _state()
    fp64 = _solve(st, sim.P, sim.prm, "fp64", 30)
    inc = _solve(st, sim.P, sim.prm, "increments", 30)
    f32 = _solve(st, sim.P, sim.prm, "fp32", 4)
    assert fp64[-1] <= 1e-6 and inc[-1] <= 1e-6
    assert len(inc) == len(fp64)
    assert f32[-1] > 1e-5
