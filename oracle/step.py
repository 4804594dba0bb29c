"""One full time step in the paper's order, on a Scene's arrays.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

Paper, section "Discretization", the four steps: (1) resample the surface
(surface and balance particles, split), (2) P2G of momentum and temperature,
(3) grid momentum and temperature update, (4) G2P with merge. Also section
"Thermomechanical Material Dependence and Phase Change" (phase flip with
J = 1 / F = I reset) and "Contact Angle" (interface-dependent coefficients).

Readings:
* gamma(T): the surface coefficient of sample r is the scene's law evaluated
  at T_r = sum_i N_i(s_r) T^n_i over nodes with thermal mass, divided by the sum
  of those weights (the grid temperature before the heat solve, so gamma is
  frozen over the step); solid-liquid samples take the effective coefficient
  gamma_sl = k_SL - k_SG;
* solid-liquid samples: with a solid plane, s_r is solid-liquid when its signed
  distance to the plane is below dx;
* the heat solve and the momentum solve are independent within a step;
* E(T) = E0 max(0, (T_melt - T)/(T_melt - T0)) per particle from T^n_p and the
  shear Lame coefficient mu = E / (2 (1 + nu)); the volumetric coefficient of the
  solid is the scene's bulk modulus lambda_l at every temperature (the paper's
  candle example gives one bulk modulus for the liquid and solid phases), so a
  solid at the melting point (E = 0) stores the liquid's energy lambda_l/2 (J-1)^2;
* without surface regeneration, the surface samples of the next step are the
  current ones carried by the grid velocity: s <- s + dt sum_i N_i(s) v_i and
  dA <- cof(I + dt sum_i v_i gradN_i(s)^T) dA (the updated-Lagrangian area map
  of Eq. pestul);
* particles move with their new velocity, x <- x + dt v_p; liquids update
  J <- (1 + dt tr grad v) J, solids F <- (I + dt grad v) F;
* Coulomb friction of a slip plane (section "Examples", liquid drops on ramps
  with friction coefficient 0.2; no formula is given): applied at the plane's
  nodes to the end-of-step velocity of the final force evaluation, before the
  projection (see boundary.coulomb_plane);
* the massless-sample variant the paper compares against (section "Surface
  Particle Sampling"): samples carry no mass and have no balance particles, so
  P2G and G2P see the interior particles alone with their whole mass, while the
  surface energy still acts through the samples.
"""
import numpy as np

from .boundary import projector, slip_plane_nodes, slip_sphere_nodes, sphere_phi_normal
from .constitutive import cof
from .energy import NewtonState, HESS_PROJECTED
from .heat import HeatSystem
from .resample import split
from .solver import newton_solve, heat_solve
from .spline import Stencil, node_positions
from .surface import generate
from .transfer import p2g, g2p, grid_velocity


def solid_lame(T, prm):
    """Lame coefficients (mu, lambda) of the solid at temperatures T."""
    return youngs(T, prm) / (2.0 * (1.0 + prm.nu)), np.full(np.shape(T), float(prm.lambda_l))


def youngs(T, prm):
    if prm.E0 == 0.0:
        return np.zeros_like(T)
    return prm.E0 * np.maximum(0.0, (prm.T_melt - T) / (prm.T_melt - prm.T0))


def gamma_of(T, kind, prm):
    if prm.gamma_law == 0:
        g = np.full(T.shape, prm.gamma_lg)
    else:
        g0, g1, gmin, gmax = prm.gamma_p
        g = np.clip(g0 + g1 * (T - prm.T0), gmin, gmax)
    return np.where(kind == 1, prm.gamma_sl, g)


class OracleSim:
    """Holds one scene's particle state and advances it step by step."""

    def __init__(self, scene, hess_mode=HESS_PROJECTED, explicit=False):
        self.sc = scene.copy()
        self.prm = self.sc.params
        self.hess_mode = hess_mode
        self.explicit = explicit
        sc = self.sc
        solid = (sc.plane_n, sc.plane_d, sc.plane_mode, sc.sphere, sc.sphere_mode)
        self.P = projector(sc.n, sc.dx, sc.walls, *solid)
        self.G = int(np.prod(sc.n))
        self.friction = None
        if self.prm.friction > 0.0 and (sc.plane_mode == 1 or sc.sphere_mode == 1):
            on_p = slip_plane_nodes(sc.n, sc.dx, sc.walls, *solid)
            on_s = slip_sphere_nodes(sc.n, sc.dx, sc.walls, *solid)
            normals = np.zeros((self.G, 3))
            if sc.plane_mode == 1:
                nn = np.asarray(sc.plane_n, float)
                normals[on_p] = nn / np.linalg.norm(nn)
            if sc.sphere_mode == 1:
                normals[on_s] = sphere_phi_normal(node_positions(sc.n, sc.dx)[on_s], sc.sphere)[1]
            self.friction = (on_p | on_s, normals, self.prm.friction)
        # the massless-sample variant: samples carry no mass, no balance particles
        self.massless = bool(self.prm.massless_surface)

    # (0) surface samples generated on the particles' union-of-spheres surface
    def generate_surface(self, seed, per_cell_area=2.0, method="tetra"):
        sc = self.sc
        plane = (sc.plane_n, sc.plane_d) if sc.plane_mode else None
        s, dA, kind, _ = generate(sc.x, sc.n, sc.dx, seed, per_cell_area, plane, method)
        sc.s, sc.dA, sc.kind = s, dA, kind
        sc.b = np.zeros(s.shape[0])
        sc.Tbar = np.full(s.shape[0], self.prm.T0)
        return s.shape[0]

    # (1) resample
    def resample(self):
        sc = self.sc
        if sc.plane_mode or sc.sphere_mode:
            near = np.zeros(sc.s.shape[0], bool)
            if sc.plane_mode:
                near |= sc.s @ np.asarray(sc.plane_n) - sc.plane_d < sc.dx
            if sc.sphere_mode:
                near |= sphere_phi_normal(sc.s, sc.sphere)[0] < sc.dx
            sc.kind = near.astype(np.uint8)
        self.parent, self.count, self.mt, self.bpos = split(sc.x, sc.m, sc.s)
        if self.massless:
            self.mt = sc.m.copy()

    # (2) P2G
    def p2g(self):
        sc = self.sc
        thermal = self.prm.thermal
        group = (None, None, None) if self.massless else (sc.s, self.bpos, self.parent)
        out = p2g(sc.n, sc.dx, sc.x, sc.v, sc.A, self.mt, *group,
                  m=sc.m, T=sc.T if thermal else None, gradT=sc.gradT if thermal else None)
        self.grid = out
        self.vn = grid_velocity(out["m"], out["mv"])
        if thermal:
            mT = out["mT"]
            self.Tn = np.where(mT > 0, out["mTT"] / np.where(mT > 0, mT, 1.0), 0.0)
        # gamma per surface sample
        if thermal:
            ss = Stencil(sc.s, sc.dx, sc.n)
            has = (out["mT"][ss.node] > 0).astype(float)
            wsum = np.sum(ss.N * has, 1)
            Tr = np.where(wsum > 0, np.sum(ss.N * has * self.Tn[ss.node], 1) / np.where(wsum > 0, wsum, 1.0),
                          self.prm.T0)
        else:
            Tr = np.full(sc.n_surface, self.prm.T0)
        self.Tr = Tr
        self.gamma = gamma_of(Tr, sc.kind, self.prm)

    def newton_state(self):
        sc, prm = self.sc, self.prm
        mu_h, lam_h = solid_lame(sc.T, prm)
        return NewtonState(sc.n, sc.dx, prm.dt, prm.gravity, self.grid["m"], self.vn, sc.x, sc.V0,
                           sc.J, sc.F, sc.phase, prm.lambda_l, prm.mu_l, mu_h, lam_h,
                           sc.s, sc.dA, self.gamma)

    def heat_system(self):
        sc, prm = self.sc, self.prm
        Vn = np.where(sc.phase == 0, sc.J, np.linalg.det(sc.F)) * sc.V0
        return HeatSystem(sc.n, sc.dx, prm.dt, prm.cp, prm.K, prm.h, prm.H, self.grid["mT"], self.Tn,
                          sc.x, Vn, sc.s, sc.dA, sc.b, sc.Tbar)

    # (3) grid update
    def grid_update(self):
        prm = self.prm
        self.That = None
        self.heat_its = 0
        if prm.thermal:
            # solved to 1e-13 relative to |rhs| (near round-off), tighter than any GPU tolerance
            self.That, self.heat_its = heat_solve(self.heat_system(), 1e-13, 20000)
        self.state = self.newton_state()
        self.vhat, self.stats = newton_solve(self.state, self.P, prm, self.hess_mode, self.explicit,
                                             friction=self.friction)

    # (4) G2P
    def g2p(self):
        sc, prm = self.sc, self.prm
        group = (None, None, None) if self.massless else (sc.s, self.bpos, self.parent)
        out = g2p(sc.n, sc.dx, self.vhat, sc.x, sc.m, self.mt, *group, self.That)
        dt = prm.dt
        Lg = out["grad_v"]
        liq = sc.phase == 0
        sc.J = np.where(liq, (1.0 + dt * np.trace(Lg, axis1=1, axis2=2)) * sc.J, sc.J)
        Fnew = np.einsum("pab,pbc->pac", np.eye(3) + dt * Lg, sc.F)
        sc.F = np.where(liq[:, None, None], sc.F, Fnew)
        sc.v = out["v"]
        sc.A = out["A"]
        if prm.thermal:
            sc.T = out["T"]
            sc.gradT = out["gradT"]
        # carry the surface samples
        ss = Stencil(sc.s, sc.dx, sc.n)
        vs = np.einsum("rq,rqa->ra", ss.N, self.vhat[ss.node])
        Ls = np.einsum("rqa,rqb->rab", self.vhat[ss.node], ss.dN)
        sc.dA = np.einsum("rab,rb->ra", cof(np.eye(3) + dt * Ls), sc.dA)
        sc.s = sc.s + dt * vs
        sc.x = sc.x + dt * sc.v
        if prm.phase_change:
            melt = (sc.phase == 1) & (sc.T > prm.T_melt)
            freeze = (sc.phase == 0) & (sc.T < prm.T_melt)
            sc.phase = np.where(melt, 0, np.where(freeze, 1, sc.phase)).astype(np.uint8)
            flip = melt | freeze
            sc.J = np.where(flip, 1.0, sc.J)
            sc.F = np.where(flip[:, None, None], np.eye(3), sc.F)

    def step(self):
        self.resample()
        self.p2g()
        self.grid_update()
        self.g2p()
