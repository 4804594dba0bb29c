"""Backward-Euler momentum objective, its gradient and Hessian-vector products.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

Paper, section "Momentum Update" (Eq. disc_force, the discrete energy e(y) and
Eq. fe). With y = x + dt v (the grid nodes moved by the new velocity) the
backward-Euler equations m (v - v^n)/dt = f(x + dt v) + m g are the stationarity
conditions of

  Phi(v) = sum_i 1/2 m_i |v_i - v^n_i|^2 - dt sum_i m_i g.v_i + e(x + dt v)
           + dt mu/2 sum_p V^n_p |eps(v; x_p)|^2,

e(y) = sum_p [psi^h(F_p) + lambda/2 (J_p - 1)^2] V^0_p + sum_r k_r |cof(F^_r) dA_r|,

with, at a point z, L(z) = sum_i v_i gradN_i(z)^T (so sum_i y_i gradN_i^T = I + dt L):
  liquid  J_p = (1 + dt tr L(x_p)) J^n_p        (the paper's (1 - d + y.gradN) J^n)
  solid   F_p = (I + dt L(x_p)) F^n_p
  surface F^_r = I + dt L(s_r), the surface term |J^ F^-T dA| = |cof(F^) dA|
  viscous eps = sym L(x_p), weight V^n_p = J^n_p V^0_p (the paper's V^n approximation).
Reading: Eq. fe evaluates the surface term's gradN at x_p; the surface samples
are the quadrature points of the surface integral, so it is evaluated at s_r.

Hessian-vector products (the linearisation the paper defers to earlier work):
  kinetic   m_i dv_i
  liquid    dt^2 lambda (J^n)^2 V^0 gradN_i (sum_j gradN_j . dv_j)     (rank one, PSD)
  viscous   dt mu V^n sym(dL) gradN_i                                  (PSD)
  solid     dt^2 V^0 dP(F; dL F^n) F^nT gradN_i                         EXACT
            the same with dP = H+ : dF, H+ the particle's 9x9 Hessian
            d^2 psi / dF^2 with its negative eigenvalues set to zero         PROJECTED
  surface   dt^2 dG gradN_i(s_r) with, for c = cof(F^) a, n = c/|c|, C = dc/dF^,
            dc = C : dF, dn = (I - n n^T) dc / |c|,
            dG_gd = k (dn_a C_agd + n_a dC_agd)         EXACT
            dG_gd = k (dn_a C_agd + Q+[dF^])             PROJECTED
  Reading of the paper's deferred "definiteness fix": the exact surface Hessian
  is the Gauss-Newton term k dc^T (I - n n^T) dc / |c| (PSD) plus the curvature of
  the cofactor, n . cof(dF) a, which does not depend on F^. In right-handed frames
  (t1, t2, n) and (s1, s2, a/|a|) it equals |a| det of the 2x2 tangential block
  x_ij = t_i . dF s_j, an indefinite form with eigenvalues +|a| on the conformal
  directions (x11 + x22, x12 - x21) and -|a| on the anti-conformal ones. The
  projected Hessian keeps the Gauss-Newton term and the positive (conformal)
  part Q+, so it stays PSD and keeps the surface's stiffness against in-plane
  dilation (dropping the whole curvature term loses it and stalls Newton).
  For solids the paper's "definiteness fix" is read as the usual per-particle
  projection: eigen-decompose the particle's symmetric 9x9 Hessian of psi(F)
  (formed here by applying the exact dP to the nine unit directions) and clamp
  its negative eigenvalues to zero. Where psi is convex at F (e.g. near rest)
  PROJECTED equals EXACT.
"""
import numpy as np

from .constitutive import EPS, cof, fcr_energy, fcr_P, fcr_dP
from .spline import Stencil, scatter

HESS_EXACT, HESS_PROJECTED = 0, 1


def _L(st, v):
    return np.einsum("pqa,pqb->pab", v[st.node], st.dN)


def _frame(u):
    """Unit vectors t1, t2 with (t1, t2, u) right-handed, for unit rows u."""
    # helper axis: the coordinate axis least aligned with u
    k = np.argmin(np.abs(u), axis=1)
    e = np.zeros_like(u)
    e[np.arange(u.shape[0]), k] = 1.0
    t1 = e - u * np.sum(e * u, 1, keepdims=True)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(u, t1)
    return t1, t2


class NewtonState:
    """Everything fixed during one backward-Euler solve."""

    def __init__(self, n, dx, dt, gravity, m, vn, x, V0, Jn, Fn, phase, lam_l, mu_l,
                 mu_h, lam_h, s, dA, gamma):
        self.n, self.dx, self.dt = tuple(n), dx, dt
        self.G = int(np.prod(n))
        self.g = np.asarray(gravity, float)
        self.m = m
        self.active = m > 0
        self.vn = vn
        self.st = Stencil(x, dx, n)
        self.ss = Stencil(s, dx, n)
        self.V0 = V0
        self.Jn = Jn
        self.Fn = Fn
        self.liq = phase == 0
        self.sol = phase == 1
        self.lam_l, self.mu_l = lam_l, mu_l
        self.mu_h, self.lam_h = mu_h, lam_h
        self.dA = dA
        self.gamma = gamma
        detF = np.linalg.det(Fn)
        self.Vn = np.where(self.liq, Jn, detF) * V0

    # ---- per-particle kinematics at the iterate v ----
    def kinematics(self, v):
        dt = self.dt
        Lp = _L(self.st, v)
        J = (1.0 + dt * np.trace(Lp, axis1=1, axis2=2)) * self.Jn
        F = np.einsum("pab,pbc->pac", np.eye(3) + dt * Lp, self.Fn)
        Fh = np.eye(3) + dt * _L(self.ss, v)
        c = np.einsum("rab,rb->ra", cof(Fh), self.dA)
        return Lp, J, F, Fh, c

    def energy(self, v):
        dt = self.dt
        a = self.active
        dv = v - self.vn
        kin = 0.5 * np.sum(self.m[a] * np.sum(dv[a] ** 2, -1)) - dt * np.sum(self.m[a] * (v[a] @ self.g))
        Lp, J, F, Fh, c = self.kinematics(v)
        liq = self.liq
        e = np.sum(0.5 * self.lam_l * (J[liq] - 1.0) ** 2 * self.V0[liq])
        eps = 0.5 * (Lp + np.swapaxes(Lp, 1, 2))
        e_visc = dt * 0.5 * self.mu_l * np.sum(self.Vn[liq] * np.sum(eps[liq] ** 2, (1, 2)))
        sol = self.sol
        e_sol = 0.0
        if np.any(sol):
            e_sol = np.sum(fcr_energy(F[sol], self.mu_h[sol], self.lam_h[sol]) * self.V0[sol])
        e_surf = np.sum(self.gamma * np.linalg.norm(c, axis=1))
        return kin + e + e_visc + e_sol + e_surf

    def _conformal_part(self, nrm, X):
        """Positive part of the cofactor curvature n . cof(X) a (see module doc).

        With right-handed frames (t1, t2, n) and (s1, s2, a/|a|) and x_ij = t_i . X s_j,
        n . cof(X) a = |a| (x11 x22 - x12 x21); its positive part as a quadratic form
        is |a|/2 [(x11 + x22)^2 + (x12 - x21)^2], whose Hessian-vector product is
        |a|/2 [(x11 + x22) (t1 s1^T + t2 s2^T) + (x12 - x21) (t1 s2^T - t2 s1^T)].
        """
        a = self.dA
        an = np.linalg.norm(a, axis=1)
        t1, t2 = _frame(nrm)
        s1, s2 = _frame(a / an[:, None])
        x = lambda t, s: np.einsum("ra,rab,rb->r", t, X, s)
        x11, x22, x12, x21 = x(t1, s1), x(t2, s2), x(t1, s2), x(t2, s1)
        out = ((x11 + x22)[:, None, None] * (np.einsum("ra,rb->rab", t1, s1) + np.einsum("ra,rb->rab", t2, s2))
               + (x12 - x21)[:, None, None] * (np.einsum("ra,rb->rab", t1, s2) - np.einsum("ra,rb->rab", t2, s1)))
        return 0.5 * an[:, None, None] * out

    def _surface_C(self, Fh):
        # C_agd = dc_a / dF_gd = eps_agk eps_bdl a_b F_kl
        return np.einsum("agk,bdl,rb,rkl->ragd", EPS, EPS, self.dA, Fh)

    def gradient(self, v):
        """dPhi/dv on every node (G, 3); zero on massless nodes."""
        dt = self.dt
        G = self.G
        out = np.zeros((G, 3))
        a = self.active
        out[a] = self.m[a, None] * (v[a] - self.vn[a]) - dt * self.m[a, None] * self.g
        Lp, J, F, Fh, c = self.kinematics(v)
        st = self.st
        liq = self.liq.astype(float)
        sol = self.sol
        # liquid pressure and viscosity: sum a stress-like 3x3 per particle, then scatter M gradN
        M = ((dt * self.lam_l * (J - 1.0) * self.Jn * self.V0) * liq)[:, None, None] * np.eye(3)
        eps = 0.5 * (Lp + np.swapaxes(Lp, 1, 2))
        M = M + (dt * self.mu_l * self.Vn * liq)[:, None, None] * eps
        if np.any(sol):
            Ps = np.zeros((st.count, 3, 3))
            Ps[sol] = fcr_P(F[sol], self.mu_h[sol], self.lam_h[sol])
            M = M + (dt * self.V0)[:, None, None] * np.einsum("pab,pcb->pac", Ps, self.Fn)
        out += scatter(G, st.node, np.einsum("pab,pqb->pqa", M, st.dN))
        # surface
        if self.ss.count:
            nrm = c / np.linalg.norm(c, axis=1, keepdims=True)
            Gs = self.gamma[:, None, None] * np.einsum("ra,ragd->rgd", nrm, self._surface_C(Fh))
            out += scatter(G, self.ss.node, dt * np.einsum("rgd,rqd->rqg", Gs, self.ss.dN))
        return out

    @staticmethod
    def solid_hessian_psd(F, mu, lam):
        """Per particle: d^2 psi / dF^2 as a 9x9 matrix (row-major dF), with its
        negative eigenvalues set to zero."""
        n = F.shape[0]
        H = np.zeros((n, 9, 9))
        for l in range(9):
            E = np.zeros((n, 9))
            E[:, l] = 1.0
            H[:, :, l] = fcr_dP(F, E.reshape(n, 3, 3), mu, lam).reshape(n, 9)
        H = 0.5 * (H + np.swapaxes(H, 1, 2))
        w, Q = np.linalg.eigh(H)
        return np.einsum("pak,pk,pbk->pab", Q, np.maximum(w, 0.0), Q)

    def hessvec(self, v, dv, mode=HESS_PROJECTED):
        """(d^2 Phi / dv^2) dv on every node (G, 3)."""
        dt = self.dt
        G = self.G
        out = np.zeros((G, 3))
        a = self.active
        out[a] = self.m[a, None] * dv[a]
        Lp, J, F, Fh, c = self.kinematics(v)
        st = self.st
        dL = _L(st, dv)
        liq = self.liq.astype(float)
        sol = self.sol
        M = ((dt * dt * self.lam_l * self.Jn ** 2 * self.V0 * np.trace(dL, axis1=1, axis2=2)) * liq)[:, None, None] * np.eye(3)
        M = M + (dt * self.mu_l * self.Vn * liq)[:, None, None] * 0.5 * (dL + np.swapaxes(dL, 1, 2))
        if np.any(sol):
            dF = np.einsum("pab,pbc->pac", dL[sol], self.Fn[sol])
            dP = np.zeros((st.count, 3, 3))
            if mode == HESS_EXACT:
                dP[sol] = fcr_dP(F[sol], dF, self.mu_h[sol], self.lam_h[sol])
            else:
                Hp = self.solid_hessian_psd(F[sol], self.mu_h[sol], self.lam_h[sol])
                dP[sol] = np.einsum("pab,pb->pa", Hp, dF.reshape(-1, 9)).reshape(-1, 3, 3)
            M = M + (dt * dt * self.V0)[:, None, None] * np.einsum("pab,pcb->pac", dP, self.Fn)
        out += scatter(G, st.node, np.einsum("pab,pqb->pqa", M, st.dN))
        if self.ss.count:
            ss = self.ss
            dFh = _L(ss, dv)
            C = self._surface_C(Fh)
            cn = np.linalg.norm(c, axis=1)
            nrm = c / cn[:, None]
            dc = np.einsum("ragd,rgd->ra", C, dFh)
            dn = (dc - nrm * np.sum(nrm * dc, 1, keepdims=True)) / cn[:, None]
            dG = np.einsum("ra,ragd->rgd", dn, C)
            if mode == HESS_EXACT:
                dC = np.einsum("agk,bdl,rb,rkl->ragd", EPS, EPS, self.dA, dFh)
                dG = dG + np.einsum("ra,ragd->rgd", nrm, dC)
            else:
                dG = dG + self._conformal_part(nrm, dFh)
            dG = self.gamma[:, None, None] * dG
            out += scatter(G, ss.node, dt * dt * np.einsum("rgd,rqd->rqg", dG, ss.dN))
        return out
