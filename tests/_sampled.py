"""Oracle results at a few sampled outputs of a large workload, one by one.

At the full benchmark size the oracle cannot run the whole workload, but each
grid node's P2G sums and each sample's closest particle depend only on the
particles near it. These helpers pick those particles and hand them to the
oracle's own routines.
"""
import numpy as np

import oracle


class CellIndex:
    """Points sorted by their cell (x fastest), for the points in a box of cells."""

    def __init__(self, pos, dx, n):
        self.n = tuple(int(v) for v in n)
        c = np.clip(np.floor(np.asarray(pos) / dx).astype(np.int64), 0, np.array(self.n) - 1)
        key = c[:, 0] + self.n[0] * (c[:, 1] + self.n[1] * c[:, 2])
        self.order = np.argsort(key, kind="stable")
        self.skey = key[self.order]

    def box(self, c, r):
        """Indices of the points whose cell lies within r cells of cell c (per axis), ascending."""
        lo = np.maximum(np.asarray(c) - r, 0)
        hi = np.minimum(np.asarray(c) + r, np.array(self.n) - 1)
        parts = []
        for z in range(lo[2], hi[2] + 1):
            for y in range(lo[1], hi[1] + 1):
                base = self.n[0] * (y + self.n[1] * z)
                a = np.searchsorted(self.skey, base + lo[0], side="left")
                b = np.searchsorted(self.skey, base + hi[0], side="right")
                parts.append(self.order[a:b])
        return np.sort(np.concatenate(parts)) if parts else np.zeros(0, np.int64)


def p2g_at_nodes(n, dx, x, v, A, m, s, b, parent, nodes):
    """Grid mass and momentum at the linear node ids `nodes` (x fastest).

    A particle in cell c reaches nodes c-1..c+1 per axis, and so do the samples
    and balance particles by their own positions. The oracle's P2G runs on the
    particles and samples that reach any sampled node. The samples' parents
    come along for their velocity, affine matrix and split mass, and the split
    mass uses the parents' group sizes over the whole workload.
    """
    g = np.stack(np.unravel_index(np.asarray(nodes), tuple(n), order="F"), -1)
    ix, isx, ib = CellIndex(x, dx, n), CellIndex(s, dx, n), CellIndex(b, dx, n)
    near_x = np.unique(np.concatenate([ix.box(gi, 1) for gi in g]))
    near_r = np.unique(np.concatenate([isx.box(gi, 1) for gi in g] + [ib.box(gi, 1) for gi in g]))
    keep = np.zeros(len(x), bool)
    keep[near_x] = True
    # parents kept only for their samples are not near any sampled node, so their
    # own weights add nothing there
    keep[parent[near_r]] = True
    idx = np.flatnonzero(keep)
    remap = np.full(len(x), -1, np.int64)
    remap[idx] = np.arange(idx.size)
    count = np.bincount(parent, minlength=len(x))
    mt = m / (2.0 * count + 1.0)
    out = oracle.p2g(n, dx, x[idx], v[idx], A[idx], mt[idx], s[near_r], b[near_r], remap[parent[near_r]])
    return out["m"][nodes], out["mv"][nodes]


def nearest_parents(x, s, which, dx, n, reach_cells=3):
    """The oracle's closest particle to each sample in `which`, searched among
    the particles within `reach_cells` cells (a box that holds every particle
    within 2 dx of the sample); indices into x."""
    ix = CellIndex(x, dx, n)
    out = np.empty(len(which), np.int64)
    for k, r in enumerate(which):
        cand = ix.box(np.floor(s[r] / dx).astype(np.int64), reach_cells)
        local, _ = oracle.nearest_parent(x[cand], s[r][None, :])
        out[k] = cand[local[0]]
    return out


def hessvec_at_nodes(n, dx, dt, x, V0, Jn, lam, s, dA, gamma, v, dv, m, nodes, mode, half=4):
    """The oracle's Hessian-vector product (NewtonState.hessvec, liquid particles
    and surface samples) at the linear node ids `nodes`, one node at a time.

    A node's row gathers the particles and samples in the 27 cells around it;
    their stencils read v and dv on the nodes within 2 of it. Each node is
    evaluated on a (2 half)^3 window of the grid around it, with positions
    shifted by whole cells, and the window's nodes carrying v, dv and m. Returns
    the rows (len(nodes), 3) with the mass term m dv and without it."""
    n = tuple(int(q) for q in n)
    g = np.stack(np.unravel_index(np.asarray(nodes), n, order="F"), -1)
    ix, isx = CellIndex(x, dx, n), CellIndex(s, dx, n)
    w = 2 * half
    loc = half + w * (half + w * half)
    full = np.zeros((len(nodes), 3))
    stiff = np.zeros((len(nodes), 3))
    for k, gi in enumerate(g):
        lo = gi - half
        sel = ix.box(gi, 1)
        ssel = isx.box(gi, 1)
        win = np.stack(np.meshgrid(*[np.arange(lo[a], lo[a] + w) for a in range(3)], indexing="ij"), -1)
        ids = (win[..., 0] + n[0] * (win[..., 1] + n[1] * win[..., 2])).transpose(2, 1, 0).ravel()
        shift = lo * dx
        np_ = sel.size
        st = oracle.NewtonState((w, w, w), dx, dt, np.zeros(3), m[ids], np.zeros((w ** 3, 3)), x[sel] - shift,
                                V0[sel], Jn[sel], np.broadcast_to(np.eye(3), (np_, 3, 3)).copy(),
                                np.zeros(np_, np.int64), lam, 0.0, np.zeros(np_), np.zeros(np_),
                                s[ssel] - shift, dA[ssel], gamma[ssel])
        out = st.hessvec(v[ids], dv[ids], mode)
        full[k] = out[loc]
        stiff[k] = out[loc] - m[ids][loc] * dv[ids][loc]
    return full, stiff
