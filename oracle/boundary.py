"""Dirichlet velocity conditions on grid nodes as a symmetric projection.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

The paper states velocity conditions v.n = v_bc on the Dirichlet boundary
(section "Conservation of Mass and Momentum", Eq. vbc) without a grid recipe.
Reading used here:
* the outer two node layers of each face are Dirichlet when that face's wall
  mode is slip (normal component zeroed) or sticky (all components zeroed);
* nodes where a solid plane's signed distance n.x_i - d < 0 get the plane's
  mode;
* a node with a sticky condition, or with the plane plus any wall, or with slip
  walls on every axis, is fully fixed; slip walls on one or two axes zero those
  components (orthogonal normals, so that is a projection).
The result is one 3x3 symmetric projection P_i per node.
"""
import numpy as np

from .spline import node_positions


def sphere_phi_normal(pos, sphere):
    """Signed distance to a spherical solid and its unit normal into the liquid.

    sphere = (cx, cy, cz, R, solid_outside): with solid_outside the solid is the
    region |x - c| > R (a bowl holding the liquid), otherwise the ball
    |x - c| < R. phi < 0 in the solid; the normal is grad phi.
    """
    c = np.asarray(sphere[:3], float)
    R, outside = float(sphere[3]), bool(sphere[4])
    d = np.asarray(pos, float) - c
    r = np.linalg.norm(d, axis=-1)
    u = np.where(r[..., None] > 1e-300, d / np.where(r > 1e-300, r, 1.0)[..., None], np.array([0.0, 0.0, 1.0]))
    return (R - r, -u) if outside else (r - R, u)


def _node_classes(n, dx, walls, plane_n, plane_d, plane_mode, sphere=None, sphere_mode=0):
    """Fully fixed nodes (G,), slip axes (G, 3), nodes below the plane (G,) and
    nodes inside the spherical solid (G,)."""
    n = tuple(int(v) for v in n)
    G = n[0] * n[1] * n[2]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = [i.ravel(), j.ravel(), k.ravel()]
    sticky = np.zeros(G, bool)
    slip_axis = np.zeros((G, 3), bool)
    for face in range(6):
        axis, side = face // 2, face % 2
        mode = walls[face]
        if mode == 0:
            continue
        on = (idx[axis] <= 1) if side == 0 else (idx[axis] >= n[axis] - 2)
        if mode == 2:
            sticky |= on
        else:
            slip_axis[on, axis] = True
    on_plane = np.zeros(G, bool)
    if plane_mode:
        phi = node_positions(n, dx) @ np.asarray(plane_n, float) - plane_d
        on_plane = phi < 0
        if plane_mode == 2:
            sticky |= on_plane
    on_sphere = np.zeros(G, bool)
    if sphere_mode:
        phi_s, _ = sphere_phi_normal(node_positions(n, dx), sphere)
        on_sphere = phi_s < 0
        if sphere_mode == 2:
            sticky |= on_sphere
    nslip = slip_axis.sum(1)
    # two independent solid normals at one node fix it (plane and sphere, or a solid and a wall)
    full = (sticky | (on_plane & (nslip > 0)) | (on_sphere & (nslip > 0)) | (on_plane & on_sphere)
            | (nslip == 3))
    return full, slip_axis, on_plane, on_sphere


def projector(n, dx, walls, plane_n=(0.0, 1.0, 0.0), plane_d=0.0, plane_mode=0, sphere=None, sphere_mode=0):
    """Per-node projection matrices (G, 3, 3)."""
    full, slip_axis, on_plane, on_sphere = _node_classes(n, dx, walls, plane_n, plane_d, plane_mode,
                                                         sphere, sphere_mode)
    G = full.shape[0]
    P = np.broadcast_to(np.eye(3), (G, 3, 3)).copy()
    for a in range(3):
        P[slip_axis[:, a], a, :] = 0.0
        P[slip_axis[:, a], :, a] = 0.0
    if plane_mode == 1:
        nn = np.asarray(plane_n, float)
        nn = nn / np.linalg.norm(nn)
        sel = on_plane & ~full
        P[sel] = np.eye(3) - np.outer(nn, nn)
    if sphere_mode == 1:
        sel = on_sphere & ~full
        _, nrm = sphere_phi_normal(node_positions(n, dx)[sel], sphere)
        P[sel] = np.eye(3) - np.einsum("ga,gb->gab", nrm, nrm)
    P[full] = 0.0
    return P


def apply_projector(P, v):
    return np.einsum("gab,gb->ga", P, v)


def slip_plane_nodes(n, dx, walls, plane_n=(0.0, 1.0, 0.0), plane_d=0.0, plane_mode=0, sphere=None,
                     sphere_mode=0):
    """Nodes whose projection is the slip plane's, I - n n^T (G,) bool."""
    full, _, on_plane, _ = _node_classes(n, dx, walls, plane_n, plane_d, plane_mode, sphere, sphere_mode)
    return on_plane & ~full if plane_mode == 1 else np.zeros_like(full)


def slip_sphere_nodes(n, dx, walls, plane_n=(0.0, 1.0, 0.0), plane_d=0.0, plane_mode=0, sphere=None,
                      sphere_mode=0):
    """Nodes whose projection is the spherical solid's, I - n_i n_i^T (G,) bool."""
    full, _, _, on_sphere = _node_classes(n, dx, walls, plane_n, plane_d, plane_mode, sphere, sphere_mode)
    return on_sphere & ~full if sphere_mode == 1 else np.zeros_like(full)


def coulomb_plane(v, nodes, plane_n, mu):
    """Coulomb friction of the slip plane on end-of-step node velocities (G, 3).

    At a plane node whose velocity presses into the plane, v_n = v . n < 0, the
    plane's normal impulse m |v_n| bounds the tangential impulse by mu m |v_n|:
    the tangential part t = v - v_n n keeps its direction and loses mu |v_n| of
    its length, or stops when |t| <= mu |v_n|. The normal part is left for the
    projection. Other nodes are returned unchanged.
    """
    nn = np.asarray(plane_n, float)
    return coulomb(v, nodes, np.broadcast_to(nn / np.linalg.norm(nn), v.shape), mu)


def coulomb(v, nodes, normals, mu):
    """The same Coulomb rule with one unit solid normal per node (G, 3); the
    normals of nodes outside `nodes` are not read."""
    out = v.copy()
    vn = np.zeros(v.shape[0])
    vn[nodes] = np.einsum("ga,ga->g", v[nodes], normals[nodes])
    sel = nodes & (vn < 0.0)
    nsel = normals[sel]
    t = v[sel] - vn[sel, None] * nsel
    tl = np.linalg.norm(t, axis=1)
    lim = -mu * vn[sel]
    s = np.where(tl > lim, 1.0 - lim / np.where(tl > 0, tl, 1.0), 0.0)
    out[sel] = s[:, None] * t + vn[sel, None] * nsel
    return out
