"""Newton-Krylov solve of the backward-Euler momentum system, and the heat CG.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

The paper solves the nonlinear system with Newton's method (section "Momentum
Update", last paragraph) and leaves the linear solver and globalisation to
earlier work. Readings used here:
* unknowns: nodes with mass, under the Dirichlet projection P (symmetric);
* initial guess v = P (v^n + dt g);
* direction: Jacobi-preconditioned CG (preconditioner 1/m_i) on P H P d = -P r,
  relative tolerance cg_rtol on the residual 2-norm; on non-positive curvature
  CG stops with the current iterate (or the preconditioned steepest descent
  direction if that happens on the first iteration);
* Armijo backtracking on Phi (c = 1e-4, halving, at most max_ls trials); when no
  trial decreases Phi the iterate is kept and Newton stops;
* stop when |P r|_2 <= tol * max(|P r_0|_2, 1e-12);
* the step ends with one explicit evaluation of the grid forces at the
  converged iterate, v = P (v - r(v)/m) = P (v^n + dt g + dt f(x + dt v)/m), so the
  total grid momentum changes by exactly dt sum_i (f_i + m_i g) (the internal
  forces sum to zero) instead of by the leftover Newton residual;
* with a slip plane and a friction coefficient, Coulomb friction acts on that
  end-of-step velocity at the plane's nodes before the projection (the paper
  gives only the coefficient, section "Examples"; see boundary.coulomb_plane).
Heat: CG with the same preconditioner form (diagonal c_p m^T/dt) on the SPD
heat operator, initial guess T^n.
"""
import numpy as np

from .boundary import apply_projector, coulomb
from .energy import HESS_PROJECTED


def pcg(apply, b, precond, rtol, maxit, neg_curv_exit=True):
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.sqrt(np.sum(b * b))
    if bnorm == 0.0:
        return x, 0
    z = precond(r)
    p = z.copy()
    rz = np.sum(r * z)
    it = 0
    for it in range(1, maxit + 1):
        q = apply(p)
        pq = np.sum(p * q)
        if neg_curv_exit and pq <= 0.0:
            if it == 1:
                x = p
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        if np.sqrt(np.sum(r * r)) <= rtol * bnorm:
            break
        z = precond(r)
        rz_new = np.sum(r * z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def armijo(phi, phi0, slope, max_ls, c=1e-4):
    """Backtracking line search: the first of alpha = 1, 1/2, 1/4, ... (max_ls
    trials) with phi(alpha) <= phi0 + c alpha slope (sufficient decrease along a
    descent direction, slope < 0), or None when no trial passes."""
    alpha = 1.0
    for _ in range(max_ls):
        if phi(alpha) <= phi0 + c * alpha * slope:
            return alpha
        alpha *= 0.5
    return None


def newton_solve(state, P, prm, hess_mode=HESS_PROJECTED, explicit=False, friction=None):
    """Returns the end-of-step grid velocity and a stats dict.

    friction: None, or (solid nodes (G,) bool, their unit normals (G, 3), mu) for
    the slip solids' Coulomb friction on the end-of-step velocity before the
    projection.
    """
    m = state.m
    act = state.active
    inv_m = np.where(act, 1.0 / np.where(act, m, 1.0), 0.0)

    def proj(u):
        return apply_projector(P, u) * act[:, None]

    v = proj(state.vn + prm.dt * state.g)
    stats = dict(newton=0, cg=[], residual=[], alpha=[])
    if not explicit:
        r0 = None
        for k in range(prm.max_newton):
            r = proj(state.gradient(v))
            rn = float(np.sqrt(np.sum(r * r)))
            stats["residual"].append(rn)
            if r0 is None:
                r0 = rn
            if rn <= prm.newton_tol * max(r0, 1e-12):
                break
            d, its = pcg(lambda u: proj(state.hessvec(v, proj(u), hess_mode)), -r,
                         lambda u: proj(u * inv_m[:, None]), prm.cg_rtol, prm.max_cg)
            stats["cg"].append(its)
            phi0 = state.energy(v)
            slope = float(np.sum(r * d))
            alpha = armijo(lambda a: state.energy(v + a * d), phi0, slope, prm.max_ls)
            stats["newton"] = k + 1
            if alpha is None:
                # no trial decreases Phi (round-off floor, or a CG direction that
                # lost its meaning): keep the iterate and stop
                stats["alpha"].append(0.0)
                stats["stalled"] = True
                break
            stats["alpha"].append(alpha)
            v = v + alpha * d
    else:
        # explicit step (q = 0 in Eq. disc_force): forces at the unmoved nodes,
        # i.e. the objective's gradient at v = 0 gives -m v^n - dt m g - dt f(x)
        v = np.zeros_like(state.vn)
    # explicit force evaluation at the final iterate
    r = state.gradient(v)
    v = v - r * inv_m[:, None]
    if friction is not None:
        nodes, normals, mu = friction
        v = coulomb(v, nodes & act, normals, mu)
    v = proj(v)
    return v, stats


def heat_solve(system, rtol, maxit):
    """Solves A T = rhs on the unknown nodes, initial guess T^n."""
    u = system.unknown
    inv_d = np.where(u, 1.0 / np.where(u, system.diag, 1.0), 0.0)
    T0 = np.where(u, system.Tn, 0.0)
    b = system.rhs() - system.apply(T0)
    dT, its = pcg(system.apply, b, lambda r: r * inv_d, rtol * np.sqrt(np.sum(system.rhs() ** 2)) /
                  max(np.sqrt(np.sum(b * b)), 1e-300), maxit, neg_curv_exit=False)
    return T0 + dT, its
