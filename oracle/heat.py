"""Implicit heat system with the particle-based Robin boundary term.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

Paper, section "Temperature Update" (discretising Eq. energy_weak):

  c_p m_i (T_i^{n+1} - T_i^n)/dt = - sum_p K gradN_i(x_p) . (sum_j T_j gradN_j(x_p)) V^n_p
                                   - sum_r h N_i(s_r) (sum_j T_j N_j(s_r)) |dA_r|
                                   + sum_r N_i(s_r) (h Tbar_r + b_r) |dA_r|
                                   + sum_p N_i(x_p) H V^n_p.
Readings:
* m_i is the thermal mass m^T_i = sum_p m_p N_i(x_p) of the temperature P2G;
* the printed source term carries a stray h; it is sum_p N_i(x_p) H V^n_p;
* the unknowns are nodes with m^T_i > 0. A surface sample's weights are
  restricted to those nodes and renormalised, w_ri = N_i(s_r) [m^T_i > 0] /
  sum_j N_j(s_r) [m^T_j > 0] (samples with no such node are ignored), so the
  Robin operator h |dA_r| w_r w_r^T stays symmetric, the whole boundary flux
  enters the unknowns and T = Tbar is an exact steady state.
"""
import numpy as np

from .spline import Stencil, scatter


class HeatSystem:
    def __init__(self, n, dx, dt, cp, K, h, H, mT, Tn, x, Vn, s, dA, b, Tbar):
        self.G = int(np.prod(n))
        self.unknown = mT > 0
        self.diag = cp * mT / dt
        self.Tn = Tn
        self.st = Stencil(x, dx, n)
        self.ss = Stencil(s, dx, n)
        self.K, self.h, self.H = K, h, H
        self.Vn = Vn
        self.area = np.linalg.norm(dA, axis=1)
        self.b, self.Tbar = b, Tbar
        if self.ss.count:
            w = self.ss.N * self.unknown[self.ss.node]
            tot = w.sum(1, keepdims=True)
            self.wS = np.where(tot > 0, w / np.where(tot > 0, tot, 1.0), 0.0)

    def apply(self, T):
        T = np.where(self.unknown, T, 0.0)
        st, ss = self.st, self.ss
        gradT = np.einsum("pq,pqa->pa", T[st.node], st.dN)
        out = self.diag * T
        out += scatter(self.G, st.node, (self.K * self.Vn)[:, None] * np.einsum("pqa,pa->pq", st.dN, gradT))
        if ss.count:
            Ts = np.einsum("rq,rq->r", T[ss.node], self.wS)
            out += scatter(self.G, ss.node, (self.h * self.area * Ts)[:, None] * self.wS)
        return np.where(self.unknown, out, 0.0)

    def rhs(self):
        st, ss = self.st, self.ss
        out = self.diag * self.Tn
        if ss.count:
            out += scatter(self.G, ss.node, ((self.h * self.Tbar + self.b) * self.area)[:, None] * self.wS)
        out += scatter(self.G, st.node, (self.H * self.Vn)[:, None] * st.N)
        return np.where(self.unknown, out, 0.0)
