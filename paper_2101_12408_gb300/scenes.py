"""Seeded synthetic scenes: particle sets, surface quadrature samples and parameters.

This module only *generates inputs*. It holds none of the method's arithmetic
(no spline weights, transfers, energies or solves), so both the CPU oracle's
tests and the CUDA path consume exactly the same arrays from here.

Every generator takes a seed and draws from ``numpy.random.default_rng(seed)``.
Shapes follow the paper's workloads (Examples section: droplets, thin films,
melting wax blocks) at the sizes of the benchmark configurations:

* ``droplet``   -- unit cube, n^3 grid, one sphere, 8 particles per cell on a
  jittered 2x2x2 sub-cell lattice, surface samples on the analytic sphere
  (Fibonacci lattice, area-weighted normals summing to 4 pi r^2).
* ``film``      -- thin liquid layer over a sticky floor, surface samples on the
  top face, Gaussian hot spot in temperature (Marangoni film).
* ``incline``   -- many droplets above a 30-degree slip plane, gravity, interface
  dependent surface coefficients (liquid-gas vs solid-liquid).
* ``wax``       -- a solid fixed-corotated cube on a sticky floor, heated on one
  face, temperature-dependent Young's modulus and surface coefficient.
* ``batch``     -- many small droplet/film scenes with log-uniform sizes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Wall modes per face (x-, x+, y-, y+, z-, z+): the outer two node layers.
WALL_NONE, WALL_SLIP, WALL_STICKY = 0, 1, 2
# Surface sample kinds: liquid-gas or solid-liquid interface.
KIND_LG, KIND_SL = 0, 1
# Surface-coefficient laws.
GAMMA_CONST, GAMMA_LINEAR = 0, 1
# Particle phases.
PHASE_LIQUID, PHASE_SOLID = 0, 1


@dataclasses.dataclass
class Params:
    dt: float = 1e-3
    gravity: tuple = (0.0, 0.0, 0.0)
    rho: float = 1.0
    lambda_l: float = 100.0          # liquid bulk modulus
    mu_l: float = 0.0                # liquid viscosity
    E0: float = 0.0                  # solid Young's modulus at T <= T0
    nu: float = 0.3                  # solid Poisson ratio
    T0: float = 0.0                  # reference temperature
    T_melt: float = 1e30             # melting point (phase change when enabled)
    cp: float = 1.0
    K: float = 0.1                   # thermal diffusivity
    h: float = 0.0                   # Robin convection coefficient
    H: float = 0.0                   # volumetric heat source
    gamma_law: int = GAMMA_CONST
    gamma_p: tuple = (1.0, 0.0, 0.0, 1e30)  # linear law: g0 + g1 (T - T0), clamped to [gmin, gmax]
    gamma_lg: float = 1.0
    gamma_sl: float = 0.0            # effective solid-liquid coefficient (k_SL - k_SG)
    newton_tol: float = 1e-6
    cg_rtol: float = 1e-3
    heat_rtol: float = 1e-6
    max_newton: int = 30
    max_cg: int = 1000
    max_ls: int = 12
    thermal: bool = False            # run the heat solve and gamma(T)
    phase_change: bool = False
    friction: float = 0.0            # Coulomb coefficient at nodes of a slip plane (0: frictionless)
    massless_surface: bool = False   # samples carry no mass and have no balance particles


@dataclasses.dataclass
class Scene:
    name: str
    n: tuple                          # grid nodes per axis (= cells per axis)
    dx: float
    params: Params
    walls: tuple = (WALL_NONE,) * 6
    plane_n: tuple = (0.0, 1.0, 0.0)  # solid plane phi(x) = n.x - d (solid where phi < 0)
    plane_d: float = 0.0
    plane_mode: int = WALL_NONE
    # spherical solid (cx, cy, cz, R, solid_outside): a bowl when solid_outside, else a ball;
    # the oracle takes it, the device path does not yet
    sphere: tuple = None
    sphere_mode: int = WALL_NONE
    # particles (float64)
    x: np.ndarray = None
    v: np.ndarray = None
    A: np.ndarray = None
    m: np.ndarray = None
    V0: np.ndarray = None
    J: np.ndarray = None
    F: np.ndarray = None
    T: np.ndarray = None
    gradT: np.ndarray = None
    phase: np.ndarray = None
    # surface quadrature samples
    s: np.ndarray = None
    dA: np.ndarray = None
    kind: np.ndarray = None
    b: np.ndarray = None              # boundary heating rate per sample
    Tbar: np.ndarray = None           # ambient temperature per sample
    meta: dict = dataclasses.field(default_factory=dict)   # generator bookkeeping (droplet centres, radii)

    @property
    def n_particles(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_surface(self) -> int:
        return int(self.s.shape[0])

    def copy(self) -> "Scene":
        out = dataclasses.replace(self)
        for f in dataclasses.fields(self):
            val = getattr(self, f.name)
            if isinstance(val, np.ndarray):
                setattr(out, f.name, val.copy())
        out.params = dataclasses.replace(self.params)
        return out


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------

def lattice_in(inside, lo_cell, hi_cell, dx, rng, ppc_axis=2, jitter=0.25):
    """Jittered sub-cell lattice: ppc_axis^3 samples per cell in cells [lo, hi).

    Each sample sits at its sub-cell centre plus a uniform offset of +-jitter
    sub-cells, so it never leaves its sub-cell; samples with inside(x) False are
    dropped.
    """
    lo = np.asarray(lo_cell, np.int64)
    hi = np.asarray(hi_cell, np.int64)
    h = 1.0 / ppc_axis
    sub = (np.arange(ppc_axis) + 0.5) * h
    out = []
    # iterate over z slabs to bound memory
    for cz in range(lo[2], hi[2]):
        cx, cy = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]), indexing="ij")
        cx = cx.ravel(); cy = cy.ravel()
        sx, sy, sz = np.meshgrid(sub, sub, sub, indexing="ij")
        sx = sx.ravel(); sy = sy.ravel(); sz = sz.ravel()
        px = (cx[:, None] + sx[None, :]).ravel()
        py = (cy[:, None] + sy[None, :]).ravel()
        pz = (cz + np.broadcast_to(sz[None, :], (cx.size, sz.size))).ravel()
        p = np.stack([px, py, pz], -1)
        p = p + rng.uniform(-jitter * h, jitter * h, size=p.shape)
        p = p * dx
        keep = inside(p)
        out.append(p[keep])
    if not out:
        return np.zeros((0, 3))
    return np.concatenate(out, 0)


def fibonacci_sphere(center, r, count):
    """count points on a sphere (Fibonacci lattice) and equal-area normals."""
    k = np.arange(count) + 0.5
    z = 1.0 - 2.0 * k / count
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    nrm = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], -1)
    pts = np.asarray(center)[None, :] + r * nrm
    dA = nrm * (4.0 * math.pi * r * r / count)
    return pts, dA


def _particles(x, rho, dx, ppc, rng, phase=PHASE_LIQUID, T=None):
    n = x.shape[0]
    V0 = np.full(n, dx ** 3 / ppc)
    m = rho * V0
    out = dict(
        x=x.astype(np.float64),
        v=np.zeros((n, 3)),
        A=np.zeros((n, 3, 3)),
        m=m,
        V0=V0,
        J=np.ones(n),
        F=np.broadcast_to(np.eye(3), (n, 3, 3)).copy(),
        T=np.zeros(n) if T is None else T,
        gradT=np.zeros((n, 3)),
        phase=np.full(n, phase, np.uint8),
    )
    return out


def _surface(s, dA, kind=None, b=None, Tbar=None):
    ns = s.shape[0]
    return dict(
        s=s.astype(np.float64),
        dA=dA.astype(np.float64),
        kind=np.zeros(ns, np.uint8) if kind is None else kind.astype(np.uint8),
        b=np.zeros(ns) if b is None else b,
        Tbar=np.zeros(ns) if Tbar is None else Tbar,
    )


def _surface_count_sphere(r, dx, per_cell_area=2.0):
    # about `per_cell_area` samples per dx^2 of surface
    return max(8, int(round(per_cell_area * 4.0 * math.pi * r * r / (dx * dx))))


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def droplet(n=32, r_cells=8.0, seed=1001, ppc_axis=2, surf_per_cell=2.0,
            gamma=1.0, lambda_l=100.0, mu_l=0.0, rho=1.0, dt=1e-3,
            gravity=(0.0, 0.0, 0.0), v0=(0.0, 0.0, 0.0), spin=0.0,
            walls=(WALL_NONE,) * 6, center=None, thermal=False) -> Scene:
    """Single droplet in a unit cube (the small parity workload).

    Default: 32^3, dx = 1/32, r = 0.25 centred, 8 ppc, ~1.6k surface samples,
    gamma = 1, rho = 1, bulk modulus 100, no gravity, dt = 1e-3.
    ``v0`` adds a uniform velocity and ``spin`` a rigid rotation about z
    (used by conservation tests).
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    r = r_cells * dx
    c = np.array([0.5, 0.5, 0.5]) if center is None else np.asarray(center, float)
    lo = np.floor((c - r) / dx).astype(int) - 1
    hi = np.ceil((c + r) / dx).astype(int) + 1
    x = lattice_in(lambda p: np.sum((p - c) ** 2, -1) < r * r, lo, hi, dx, rng, ppc_axis)
    ppc = ppc_axis ** 3
    P = _particles(x, rho, dx, ppc, rng)
    P["v"][:] = np.asarray(v0, float)
    if spin != 0.0:
        rel = x - c
        P["v"][:, 0] += -spin * rel[:, 1]
        P["v"][:, 1] += spin * rel[:, 0]
        Wm = np.array([[0.0, -spin, 0.0], [spin, 0.0, 0.0], [0.0, 0.0, 0.0]])
        P["A"][:] = Wm
    s, dA = fibonacci_sphere(c, r, _surface_count_sphere(r, dx, surf_per_cell))
    S = _surface(s, dA)
    prm = Params(dt=dt, gravity=tuple(gravity), rho=rho, lambda_l=lambda_l, mu_l=mu_l,
                 gamma_law=GAMMA_CONST, gamma_lg=gamma, thermal=thermal)
    return Scene(name=f"droplet{n}", n=(n, n, n), dx=dx, params=prm, walls=tuple(walls), **P, **S)


def film(nx=128, ny=128, nz=32, height_cells=6, seed=1002, ppc_axis=2, surf_per_cell=2,
         T0=0.0, dT=1.0, sigma_cells=10.0, h=5.0, K=0.1, cp=1e-3, lambda_l=1e6,
         mu_l=1e-3, rho=1000.0, dt=5e-4, gravity=(0.0, 0.0, -9.8)) -> Scene:
    """Marangoni thin film: a liquid layer `height_cells` thick over a sticky floor.

    Slip side walls; surface samples on the top face only; linear
    gamma(T) = 1 - 0.5 (T - T0) clamped at 0; Gaussian hot spot
    T = T0 + dT exp(-rho^2 / (2 sigma^2)) with rho in cells from the centre;
    Robin convection h with ambient T0 on the top face.

    Water in SI units (rho = 1000, bulk modulus 1e6, viscosity 1e-3), as for the
    inclined droplets. The heat problem per unit volume is rho c_p = 1 with
    conductivity K = 0.1 and h = 5. With rho = 1 the Marangoni stress
    accelerates the top node row at ~800 m/s^2 at dx = 1/128. The surface flow
    then reaches metres per second within 15 steps and converges at the walls,
    where the carried samples outrun their particles.

    The top sheet is a regular lattice of `surf_per_cell` (1, 2 or 4) samples
    per face cell that is point-symmetric about every node centre, and it runs
    over cells 1..n-2 in x and y, i.e. onto the slip node layers. A flat sheet
    of constant gamma then exerts no tangential force on any free node: the
    interior dipoles cancel by the symmetry, and the edge's pull
    (gamma N_i(x_edge) per unit length) lands on the wall nodes, whose normal
    velocity is zeroed. Only gamma's variation (the Marangoni stress) drives the
    surface. A sheet that ends at the liquid's edge (x = 2 dx) instead pulls the
    first free node row inward with gamma/2 per unit length, an acceleration of
    order gamma / (rho dx^2) at the light top nodes that grows 16-fold from
    dx = 1/32 to 1/128; jittered samples add forces of the same order at every
    top node.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / nx
    z0, z1 = 2, 2 + height_cells
    lo = (2, 2, z0)
    hi = (nx - 2, ny - 2, z1)
    x = lattice_in(lambda p: np.ones(p.shape[0], bool), lo, hi, dx, rng, ppc_axis)
    ppc = ppc_axis ** 3
    cxy = np.array([nx / 2.0, ny / 2.0]) * dx

    def temp(p):
        rr = np.sum(((p[:, :2] - cxy) / dx) ** 2, -1)
        return T0 + dT * np.exp(-rr / (2.0 * sigma_cells ** 2))

    P = _particles(x, rho, dx, ppc, rng, T=temp(x))
    # top-face samples: a regular lattice over face cells 1..n-2 (onto the wall layers)
    offs = {1: [(0.5, 0.5)], 2: [(0.25, 0.25), (0.75, 0.75)],
            4: [(0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)]}[surf_per_cell]
    fx, fy = np.meshgrid(np.arange(1, nx - 1), np.arange(1, ny - 1), indexing="ij")
    sxy = (np.stack([fx.ravel(), fy.ravel()], -1)[:, None, :] + np.asarray(offs)[None]).reshape(-1, 2)
    s = np.concatenate([sxy * dx, np.full((sxy.shape[0], 1), z1 * dx)], -1)
    dA = np.zeros_like(s)
    dA[:, 2] = dx * dx / surf_per_cell
    S = _surface(s, dA, b=np.zeros(s.shape[0]), Tbar=np.full(s.shape[0], T0))
    prm = Params(dt=dt, gravity=tuple(gravity), rho=rho, lambda_l=lambda_l, mu_l=mu_l,
                 T0=T0, cp=cp, K=K, h=h, gamma_law=GAMMA_LINEAR,
                 gamma_p=(1.0, -0.5, 0.0, 1e30), thermal=True)
    walls = (WALL_SLIP, WALL_SLIP, WALL_SLIP, WALL_SLIP, WALL_STICKY, WALL_NONE)
    return Scene(name=f"film{nx}x{ny}x{nz}", n=(nx, ny, nz), dx=dx, params=prm, walls=walls, **P, **S)


def incline(n=256, n_drops=40, r_range=(9.3, 24.8), seed=1003, ppc_axis=2, surf_per_cell=2.0,
            gamma_lg=1.0, gamma_sl=0.5, lambda_l=1e6, mu_l=0.0, rho=1000.0, dt=1e-3,
            angle_deg=30.0, gap_cells=(0.5, 120.0)) -> Scene:
    """Droplets above a 30-degree inclined slip plane, gravity -9.8 in y.

    The plane passes through (0.5, 0.2, 0.5) with normal (-sin a, cos a, 0).
    Radii are drawn uniform in `r_range` cells; centres are rejection-sampled so
    droplets do not overlap and sit `gap` cells above the plane. The effective
    solid-liquid coefficient 0.5 with gamma_LG = 1 targets a 120-degree contact
    angle (Young: cos theta = -k_SL_eff / k_LG).
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    a = math.radians(angle_deg)
    nrm = np.array([-math.sin(a), math.cos(a), 0.0])
    p0 = np.array([0.5, 0.2, 0.5])
    d = float(nrm @ p0)
    centers, radii = [], []
    tries = 0
    margin = 4 * dx
    r = rng.uniform(*r_range) * dx
    while len(centers) < n_drops and tries < 100000:
        tries += 1
        if tries % 2000 == 0:  # a radius that does not fit is redrawn (rarely)
            r = rng.uniform(*r_range) * dx
        gap = rng.uniform(*gap_cells) * dx
        x0 = rng.uniform(r + margin, 1.0 - r - margin)
        z0 = rng.uniform(r + margin, 1.0 - r - margin)
        # phi(c) = n.c - d = r + gap  ->  solve for y
        y0 = (r + gap + d - nrm[0] * x0) / nrm[1]
        c = np.array([x0, y0, z0])
        if np.any(c - r < margin) or np.any(c + r > 1.0 - margin):
            continue
        if any(np.linalg.norm(c - cc) < r + rr + 2 * dx for cc, rr in zip(centers, radii)):
            continue
        centers.append(c)
        radii.append(r)
        r = rng.uniform(*r_range) * dx
    xs, ss, dAs = [], [], []
    for c, r in zip(centers, radii):
        lo = np.floor((c - r) / dx).astype(int) - 1
        hi = np.ceil((c + r) / dx).astype(int) + 1
        xs.append(lattice_in(lambda p, c=c, r=r: np.sum((p - c) ** 2, -1) < r * r, lo, hi, dx, rng, ppc_axis))
        s, dA = fibonacci_sphere(c, r, _surface_count_sphere(r, dx, surf_per_cell))
        ss.append(s)
        dAs.append(dA)
    x = np.concatenate(xs, 0)
    P = _particles(x, rho, dx, ppc_axis ** 3, rng)
    s = np.concatenate(ss, 0)
    dA = np.concatenate(dAs, 0)
    phi = s @ nrm - d
    kind = np.where(phi < dx, KIND_SL, KIND_LG).astype(np.uint8)
    S = _surface(s, dA, kind=kind)
    prm = Params(dt=dt, gravity=(0.0, -9.8, 0.0), rho=rho, lambda_l=lambda_l, mu_l=mu_l,
                 gamma_law=GAMMA_CONST, gamma_lg=gamma_lg, gamma_sl=gamma_sl)
    walls = (WALL_STICKY,) * 6
    return Scene(name=f"incline{n}", n=(n, n, n), dx=dx, params=prm, walls=walls,
                 plane_n=tuple(nrm), plane_d=d, plane_mode=WALL_SLIP,
                 meta=dict(centers=np.array(centers), radii=np.array(radii)), **P, **S)


def wax(nx=256, ny=256, nz=128, cube_cells=96, seed=1004, ppc_axis=2, surf_per_cell=2,
        E0=1e4, nu=0.3, T0=298.0, T_melt=303.0, rho=1.0, dt=1e-3, h=0.5, b_heat=50.0,
        K=0.1, cp=1.0, mu_l=1e-3) -> Scene:
    """Melting wax block: a fixed-corotated cube on a sticky floor, heated on -x.

    E(T) falls linearly from E0 at T0 to 0 at T_melt and sets the solid's shear
    modulus; the bulk modulus E0 / (3 (1 - 2 nu)) serves the liquid and the solid
    phases; gamma(T) = clamp(0.1 - 0.01 (T - T0), 0, 0.1).
    Surface samples cover the five free faces; the -x face carries the heating
    rate b, every face Robin convection h towards T0.
    """
    rng = np.random.default_rng(seed)
    dx = 1.0 / nx
    L = cube_cells
    lo = np.array([(nx - L) // 2, (ny - L) // 2, 2])
    hi = lo + L
    x = lattice_in(lambda p: np.ones(p.shape[0], bool), lo, hi, dx, rng, ppc_axis)
    P = _particles(x, rho, dx, ppc_axis ** 3, rng, phase=PHASE_SOLID, T=np.full(x.shape[0], T0))
    ss, dAs, bs = [], [], []
    for axis in range(3):
        for side in (0, 1):
            if axis == 2 and side == 0:
                continue  # bottom face rests on the floor
            o = [a for a in range(3) if a != axis]
            u, w = np.meshgrid(np.arange(lo[o[0]], hi[o[0]]), np.arange(lo[o[1]], hi[o[1]]), indexing="ij")
            u = np.repeat(u.ravel(), surf_per_cell)
            w = np.repeat(w.ravel(), surf_per_cell)
            jit = rng.uniform(0.0, 1.0, size=(u.size, 2))
            p = np.zeros((u.size, 3))
            p[:, o[0]] = (u + jit[:, 0]) * dx
            p[:, o[1]] = (w + jit[:, 1]) * dx
            p[:, axis] = (hi[axis] if side else lo[axis]) * dx
            nrm = np.zeros(3)
            nrm[axis] = 1.0 if side else -1.0
            dA = np.broadcast_to(nrm * dx * dx / surf_per_cell, p.shape).copy()
            ss.append(p)
            dAs.append(dA)
            bs.append(np.full(u.size, b_heat if (axis == 0 and side == 0) else 0.0))
    s = np.concatenate(ss, 0)
    S = _surface(s, np.concatenate(dAs, 0), b=np.concatenate(bs, 0), Tbar=np.full(s.shape[0], T0))
    prm = Params(dt=dt, gravity=(0.0, 0.0, -9.8), rho=rho, lambda_l=E0 / (3.0 * (1.0 - 2.0 * nu)),
                 mu_l=mu_l, E0=E0, nu=nu, T0=T0, T_melt=T_melt, cp=cp, K=K, h=h,
                 gamma_law=GAMMA_LINEAR, gamma_p=(0.1, -0.01, 0.0, 0.1), thermal=True, phase_change=True)
    walls = (WALL_STICKY,) * 6
    return Scene(name=f"wax{nx}x{ny}x{nz}", n=(nx, ny, nz), dx=dx, params=prm, walls=walls, **P, **S)


def batch(n_scenes=64, seed=2000, n_range=(32, 96), count_range=(5e3, 3e5), dt=1e-3):
    """Many independent scenes: droplet or film (50/50), constant or linear gamma(T).

    The droplets are water in SI units (rho = 1000, bulk modulus 1e6), as the
    inclined droplets: with the small droplet's rho = 1 the capillary stiffness
    dt^2 gamma / (rho dx^3) reaches 0.88 on a 96^3 grid, and droplets on grids
    finer than 80^3 diverged within 14 steps."""
    out = []
    for k in range(n_scenes):
        rng = np.random.default_rng(seed + k)
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        count = math.exp(rng.uniform(math.log(count_range[0]), math.log(count_range[1])))
        thermal = bool(rng.integers(0, 2))
        if rng.integers(0, 2) == 0:
            # droplet with `count` particles at 8 ppc: r^3 = 3 count / (32 pi) cells^3
            r_cells = (3.0 * count / (8.0 * 4.0 * math.pi)) ** (1.0 / 3.0)
            r_cells = min(r_cells, 0.5 * n - 4)
            sc = droplet(n=n, r_cells=r_cells, seed=seed + k, dt=dt, thermal=thermal, rho=1000.0, lambda_l=1e6)
            if thermal:
                sc.T = 0.5 * np.clip((sc.x[:, 0] - 0.5) / (r_cells / n), -1.0, 1.0) + 0.5
                sc.params.gamma_law = GAMMA_LINEAR
                sc.params.gamma_p = (1.0, -0.5, 0.0, 1e30)
                sc.params.h = 1.0
                sc.Tbar = np.zeros(sc.n_surface)
        else:
            nz = max(16, n // 4)
            height = int(max(2, min(nz - 6, round(count / (8.0 * (n - 4) ** 2)))))
            sc = film(nx=n, ny=n, nz=nz, height_cells=height, seed=seed + k, dt=dt)
            if not thermal:
                sc.params.thermal = False
                sc.params.gamma_law = GAMMA_CONST
        sc.name = f"batch{k}_{sc.name}"
        out.append(sc)
    return out


def config(index: int, **kw):
    """The five benchmark workloads by index (0-based)."""
    if index == 0:
        return droplet(seed=1000 + 1, **kw)
    if index == 1:
        return film(seed=1000 + 2, **kw)
    if index == 2:
        return incline(seed=1000 + 3, **kw)
    if index == 3:
        return wax(seed=1000 + 4, **kw)
    if index == 4:
        return batch(**kw)
    raise ValueError(index)


def window(sc: Scene, center, size_cells: int, name=None) -> Scene:
    """Sub-box of a scene: particles and samples within `size_cells` cells around
    `center`, shifted into a grid of that size with the same dx and parameters
    (a bounded sample of a large workload; droplets are independent within a step)."""
    dx = sc.dx
    c_cell = np.floor(np.asarray(center) / dx).astype(int)
    lo = c_cell - size_cells // 2
    lo = np.clip(lo, 0, np.asarray(sc.n) - size_cells)
    shift = lo * dx
    hi = shift + size_cells * dx
    inside = np.all((sc.x >= shift + 2 * dx) & (sc.x < hi - 2 * dx), 1)
    sin = np.all((sc.s >= shift + 2 * dx) & (sc.s < hi - 2 * dx), 1)
    out = sc.copy()
    out.name = name or f"{sc.name}_window{size_cells}"
    out.n = (size_cells,) * 3
    for f in ("x", "v", "A", "m", "V0", "J", "F", "T", "gradT", "phase"):
        setattr(out, f, getattr(sc, f)[inside].copy())
    out.x = out.x - shift
    for f in ("s", "dA", "kind", "b", "Tbar"):
        setattr(out, f, getattr(sc, f)[sin].copy())
    out.s = out.s - shift
    if sc.plane_mode:
        out.plane_d = sc.plane_d - float(np.asarray(sc.plane_n) @ shift)
    return out
