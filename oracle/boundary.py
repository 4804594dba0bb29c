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


def projector(n, dx, walls, plane_n=(0.0, 1.0, 0.0), plane_d=0.0, plane_mode=0):
    """Per-node projection matrices (G, 3, 3)."""
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
