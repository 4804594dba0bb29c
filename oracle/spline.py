"""Quadratic B-spline interpolation on a uniform grid with nodes at cell centres.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

Paper, section "Transfer: P2G": N_i(x) = N(x - x_i) are quadratic B-splines
over the uniform grid with x_i at cell centres. So node i sits at
(i + 1/2) dx, a point in cell c = floor(x / dx) touches nodes c-1 .. c+1 per axis,
and with f = x/dx - 1/2 - (c - 1) in [1/2, 3/2) the three 1-D weights are the
quadratic B-spline evaluated at the distances f, f - 1, f - 2:

    w0 = (3/2 - f)^2 / 2,   w1 = 3/4 - (f - 1)^2,   w2 = (f - 1/2)^2 / 2.

Node ids are flat: id = i + nx (j + ny k).
"""
import numpy as np

# 27 stencil offsets, a (x) fastest
OFFSETS = np.array([(a, b, c) for c in range(3) for b in range(3) for a in range(3)], dtype=np.int64)


def axis_weights(u):
    """u = x / dx (any shape). Returns base node index, weights and d/du of weights."""
    base = np.floor(u).astype(np.int64) - 1
    f = u - 0.5 - base
    w = np.stack([0.5 * (1.5 - f) ** 2, 0.75 - (f - 1.0) ** 2, 0.5 * (f - 0.5) ** 2], -1)
    dw = np.stack([-(1.5 - f), -2.0 * (f - 1.0), f - 0.5], -1)
    return base, w, dw


def node_positions(n, dx):
    """Positions of all nodes, flat order, shape (G, 3)."""
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return (np.stack([i.ravel(), j.ravel(), k.ravel()], -1) + 0.5) * dx


class Stencil:
    """Weights N_i(x_p), gradients dN_i/dx(x_p) and node ids for a set of points."""

    def __init__(self, X, dx, n):
        X = np.asarray(X, np.float64).reshape(-1, 3)
        self.count = X.shape[0]
        base, w, dw = axis_weights(X / dx)
        a, b, c = OFFSETS[:, 0], OFFSETS[:, 1], OFFSETS[:, 2]
        ix = base[:, 0:1] + a
        iy = base[:, 1:2] + b
        iz = base[:, 2:3] + c
        if X.shape[0] and (ix.min() < 0 or iy.min() < 0 or iz.min() < 0
                           or ix.max() >= n[0] or iy.max() >= n[1] or iz.max() >= n[2]):
            raise ValueError("stencil leaves the grid: points must lie in cells 1 .. n-2")
        self.node = ix + n[0] * (iy + n[1] * iz)
        wx, wy, wz = w[:, 0, a], w[:, 1, b], w[:, 2, c]
        self.N = wx * wy * wz
        self.dN = np.stack([dw[:, 0, a] * wy * wz, wx * dw[:, 1, b] * wz, wx * wy * dw[:, 2, c]], -1) / dx
        self.xi = (np.stack([ix, iy, iz], -1) + 0.5) * dx
        self.X = X


def scatter(G, node, vals):
    """Sum vals (P, 27, ...) into a (G, ...) array at node ids (P, 27)."""
    vals = np.asarray(vals, np.float64)
    tail = vals.shape[2:]
    if node.size == 0:   # no points: nothing lands on the grid
        return np.zeros((G,) + tail)
    flat = vals.reshape(node.size, -1)
    out = np.zeros((G, flat.shape[1]))
    idx = node.ravel()
    for k in range(flat.shape[1]):
        out[:, k] = np.bincount(idx, weights=flat[:, k], minlength=G)
    return out.reshape((G,) + tail)


def gather(field, node):
    """field (G, ...) at node ids (P, 27) -> (P, 27, ...)."""
    return field[node]
