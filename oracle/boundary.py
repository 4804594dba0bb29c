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


def _node_classes(n, dx, walls, plane_n, plane_d, plane_mode):
    """Fully fixed nodes (G,), slip axes (G, 3) and nodes below the plane (G,)."""
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
    nslip = slip_axis.sum(1)
    full = sticky | (on_plane & (nslip > 0)) | (nslip == 3)
    return full, slip_axis, on_plane


def projector(n, dx, walls, plane_n=(0.0, 1.0, 0.0), plane_d=0.0, plane_mode=0):
    """Per-node projection matrices (G, 3, 3)."""
    full, slip_axis, on_plane = _node_classes(n, dx, walls, plane_n, plane_d, plane_mode)
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
    P[full] = 0.0
    return P


def apply_projector(P, v):
    return np.einsum("gab,gb->ga", P, v)


def slip_plane_nodes(n, dx, walls, plane_n=(0.0, 1.0, 0.0), plane_d=0.0, plane_mode=0):
    """Nodes whose projection is the slip plane's, I - n n^T (G,) bool."""
    full, _, on_plane = _node_classes(n, dx, walls, plane_n, plane_d, plane_mode)
    return on_plane & ~full if plane_mode == 1 else np.zeros_like(full)


def coulomb_plane(v, nodes, plane_n, mu):
    """Coulomb friction of the slip plane on end-of-step node velocities (G, 3).

    At a plane node whose velocity presses into the plane, v_n = v . n < 0, the
    plane's normal impulse m |v_n| bounds the tangential impulse by mu m |v_n|:
    the tangential part t = v - v_n n keeps its direction and loses mu |v_n| of
    its length, or stops when |t| <= mu |v_n|. The normal part is left for the
    projection. Other nodes are returned unchanged.
    """
    nn = np.asarray(plane_n, float)
    nn = nn / np.linalg.norm(nn)
    out = v.copy()
    vn = v @ nn
    sel = nodes & (vn < 0.0)
    t = v[sel] - vn[sel, None] * nn
    tl = np.linalg.norm(t, axis=1)
    lim = -mu * vn[sel]
    s = np.where(tl > lim, 1.0 - lim / np.where(tl > 0, tl, 1.0), 0.0)
    out[sel] = s[:, None] * t + vn[sel, None] * nn
    return out
