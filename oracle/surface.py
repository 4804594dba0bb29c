"""Surface-sample generation: union-of-spheres level set, isosurface
triangulation, per-triangle Poisson sampling.

TEST INFRASTRUCTURE ONLY (FP64 oracle).

Paper, section "Surface Particle Sampling": the level set enclosing the interior
particles is the union of spheres of radius 0.867 dx around them (3D), not
smoothed or shifted; its zero isocontour is triangulated and sampled triangle
by triangle, the sample count per triangle drawn from a Poisson distribution
(mean proportional to the triangle's area) and the points uniform in the
triangle (Osada's square-root construction); each sample's area-weighted
normal dA points along the triangle normal.

Readings (the paper leaves these open):
* The level set lives on the MPM nodes (cell centres (i + 1/2) dx) and is
  phi(i) = min(d_i, 1.5 dx) - 0.867 dx, d_i the distance to the nearest
  particle. Any particle closer than 1.5 dx lies in the 27 cells around the node,
  so this is exact wherever phi < 0.6 dx.
* The isocontour is extracted by marching tetrahedra: each cube of 8 nodes is
  cut into the 6 tetrahedra around its main diagonal (corner 000 to 111, one per
  ordering of the axes), which triangulates every cube consistently with its
  neighbours and has no ambiguous cases; inside is phi < 0. Edge points by
  linear interpolation. Triangles face outward (towards phi >= 0).
* Or by marching cubes, the paper's method (Chernyaev's): each cube's crossing
  edges are joined into closed loops face by face, ambiguous faces resolved by
  the asymptotic decider, and each loop is cut into a fan of triangles from its
  first point (cube_loops). Interior ambiguities (tunnels through the cube) are
  not formed: loops are built from face segments only.
* Enumeration order (it fixes the random counters): cubes by the block-major key
  of their lowest corner (4x4x4 blocks, as the grid), then tetrahedron, then
  triangle; for marching cubes, loop then fan triangle, triangle t of cube q
  taking counter slot 12 q + t.
* Random numbers: the SplitMix64 generator (Steele, Lea, Flood 2014) seeded with
  `seed`; the value for counter k is its (k+1)-th output, and triangle t of
  tetrahedron e of cube key q draws counters ((6 q + e) 2 + t) 64 + j,
  j = 0 for its count, 2i+1 and 2i+2 for sample i. A uniform is the top 53 bits
  times 2^-53. Counts are capped at 31.
* The samples' mean density is rho = `per_cell_area` samples per dx^2 of surface,
  and every sample carries |dA| = 1 / rho: with Poisson counts of mean rho A this
  makes sum |dA| an unbiased estimate of the area. (Area / count per triangle,
  read literally, drops the area of the triangles that draw no sample, and on a
  tetrahedral triangulation most triangles are far smaller than 1 / rho.)
* Kind: solid-liquid where the plane's signed distance is below dx (plane
  scenes), liquid-gas elsewhere.
"""
import math

import numpy as np
from scipy.spatial import cKDTree

R0_FACTOR = 0.867
CLAMP_FACTOR = 1.5
KMAX = 31
GOLDEN = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1

# the six tetrahedra of a cube: vertices 000, e_a, e_a + e_b, 111 for the axis orders (a, b, c)
_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _tet_corners():
    out = []
    for a, b, _ in _ORDERS:
        v1 = [0, 0, 0]
        v1[a] = 1
        v2 = list(v1)
        v2[b] = 1
        out.append(((0, 0, 0), tuple(v1), tuple(v2), (1, 1, 1)))
    return out


TETS = _tet_corners()


def splitmix64(seed, k):
    """(k+1)-th output of SplitMix64 started from `seed` (Python ints)."""
    z = (seed + (k + 1) * GOLDEN) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def uniform(seed, k):
    return (splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0)


def block_key(q, n):
    """Block-major key of node q (4x4x4 blocks, blocks x-fastest, x-fastest inside)."""
    nb = [(n[a] + 3) // 4 for a in range(3)]
    gb = q[0] // 4 + nb[0] * (q[1] // 4 + nb[1] * (q[2] // 4))
    return gb * 64 + (q[0] % 4) + 4 * (q[1] % 4) + 16 * (q[2] % 4)


def level_set(x, n, dx):
    """phi on the nodes of the particles' 3x3x3 stencils (dict node -> phi); every
    other node has phi = 1.5 dx - 0.867 dx."""
    r0 = R0_FACTOR * dx
    cells = np.floor(x / dx).astype(np.int64)
    offs = np.array([(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)])
    nodes = np.unique((cells[:, None, :] + offs[None, :, :]).reshape(-1, 3), axis=0)
    pos = (nodes + 0.5) * dx
    tree = cKDTree(x)
    dist, idx = tree.query(pos, k=1)
    # the distance itself is formed as the device forms it: sqrt((dx^2 + dy^2) + dz^2)
    d = pos - x[idx]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    dd = np.sqrt(d2)
    phi = np.minimum(dd, CLAMP_FACTOR * dx) - r0
    return {tuple(q): float(p) for q, p in zip(nodes.tolist(), phi)}, CLAMP_FACTOR * dx - r0


def _edge_point(qa, qb, pa, pb, dx):
    t = pa / (pa - pb)
    out = []
    for c in range(3):
        xa = (qa[c] + 0.5) * dx
        xb = (qb[c] + 0.5) * dx
        out.append(xa + t * (xb - xa))
    return out


def _sub(a, b):
    return [a[0] - b[0], a[1] - b[1], a[2] - b[2]]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def tet_triangles(qv, pv, dx):
    """Triangles of one tetrahedron (node indices qv, values pv), facing outward."""
    ins = [i for i in range(4) if pv[i] < 0.0]
    out = [i for i in range(4) if not pv[i] < 0.0]
    if len(ins) == 0 or len(ins) == 4:
        return []

    def e(i, j):
        return _edge_point(qv[i], qv[j], pv[i], pv[j], dx)

    if len(ins) == 1:
        i = ins[0]
        tris = [(e(i, out[0]), e(i, out[1]), e(i, out[2]))]
    elif len(ins) == 3:
        l = out[0]
        tris = [(e(ins[0], l), e(ins[1], l), e(ins[2], l))]
    else:
        i, j = ins
        k, l = out
        tris = [(e(i, k), e(i, l), e(j, l)), (e(i, k), e(j, l), e(j, k))]
    # outward: along (centroid of outside vertices) - (centroid of inside vertices)
    g = [0.0, 0.0, 0.0]
    for c in range(3):
        so = sum(float(qv[o][c]) for o in out) / len(out)
        si = sum(float(qv[i][c]) for i in ins) / len(ins)
        g[c] = so - si
    res = []
    for p0, p1, p2 in tris:
        nrm = _cross(_sub(p1, p0), _sub(p2, p0))
        if (nrm[0] * g[0] + nrm[1] * g[1]) + nrm[2] * g[2] < 0.0:
            p1, p2 = p2, p1
        res.append((p0, p1, p2))
    return res


# ---- marching cubes (the paper's isocontour method) ----
#
# Corner c = x + 2 y + 4 z of a cube. Edge 4 a + j + 2 k runs along axis a between
# the two corners whose other two axes (in increasing order) have bits (j, k).
# Face (w, s) is the face at coordinate s along axis w; its corners are listed
# counter-clockwise as seen from outside the cube (the right-hand rule about its
# outward normal), with in-face axes u = w + 1, v = w + 2 (mod 3), e_u x e_v = e_w.


def _corner_bits(c):
    return (c & 1, (c >> 1) & 1, (c >> 2) & 1)


def _edge_corners(e):
    a, jk = divmod(e, 4)
    b, c = [ax for ax in range(3) if ax != a]
    bits = [0, 0, 0]
    bits[b] = jk & 1
    bits[c] = jk >> 1
    c0 = bits[0] + 2 * bits[1] + 4 * bits[2]
    return c0, c0 + (1 << a)


def _edge_index(ca, cb):
    lo, hi = min(ca, cb), max(ca, cb)
    for e in range(12):
        if _edge_corners(e) == (lo, hi):
            return e
    raise ValueError("corners are not adjacent")


def _face_corners(w, s):
    u, v = (w + 1) % 3, (w + 2) % 3
    uv = ((0, 0), (1, 0), (1, 1), (0, 1)) if s == 1 else ((0, 0), (0, 1), (1, 1), (1, 0))
    out = []
    for iu, iv in uv:
        bits = [0, 0, 0]
        bits[w], bits[u], bits[v] = s, iu, iv
        out.append(bits[0] + 2 * bits[1] + 4 * bits[2])
    return out


FACES = [_face_corners(w, s) for w in range(3) for s in (0, 1)]


def cube_loops(cphi):
    """Closed loops of crossing edges of one cube (corner values cphi[8], inside
    phi < 0), each ordered so that the surface it bounds faces outward.

    On every face, walking its corners counter-clockwise from outside, a crossing
    edge is entering (outside corner to inside corner) or leaving. Each face
    segment runs from an entering crossing to a leaving one. A face with four
    crossings (diagonal corners inside) is ambiguous; it is resolved by the
    asymptotic decider (the sign of the bilinear interpolant at its saddle point,
    Chernyaev's face test): the inside corners a, c join across the face when
    phi_a phi_c > phi_b phi_d, and then each entering crossing pairs with the
    leaving crossing before it, else with the one after it. Both cubes sharing a
    face take the same decision from the same four values. Each crossing edge is
    entering on exactly one of its two faces, so following the segments visits
    disjoint closed loops; a loop starts at its smallest edge index."""
    inside = [p < 0.0 for p in cphi]
    nxt = {}
    for fc in FACES:
        cr = []   # (edge, entering?) in counter-clockwise order
        for k in range(4):
            a, b = fc[k], fc[(k + 1) % 4]
            if inside[a] != inside[b]:
                cr.append((_edge_index(a, b), inside[b]))
        if len(cr) == 2:
            ent = [e for e, en in cr if en][0]
            lea = [e for e, en in cr if not en][0]
            nxt[ent] = lea
        elif len(cr) == 4:
            ins = [c for c in fc if inside[c]]
            out = [c for c in fc if not inside[c]]
            joined = cphi[ins[0]] * cphi[ins[1]] > cphi[out[0]] * cphi[out[1]]
            for k in range(4):
                e, en = cr[k]
                if en:
                    nxt[e] = cr[(k - 1) % 4][0] if joined else cr[(k + 1) % 4][0]
    loops, seen = [], set()
    for e0 in sorted(nxt):
        if e0 in seen:
            continue
        loop, e = [], e0
        while e not in seen:
            seen.add(e)
            loop.append(e)
            e = nxt[e]
        assert e == e0, "face segments do not close"
        loops.append(loop)
    return loops


def cube_triangles(q, cphi, dx):
    """Marching-cubes triangles of the cube with lowest corner q: every loop of
    cube_loops as a fan from its first point. Edge points by linear interpolation
    from the inside corner to the outside one (the tetrahedral path's formula, so
    a shared edge gives the same point in every cube)."""
    tris = []
    for loop in cube_loops(cphi):
        pts = []
        for e in loop:
            ca, cb = _edge_corners(e)
            i, o = (ca, cb) if cphi[ca] < 0.0 else (cb, ca)
            qi = tuple(q[a] + _corner_bits(i)[a] for a in range(3))
            qo = tuple(q[a] + _corner_bits(o)[a] for a in range(3))
            pts.append(_edge_point(qi, qo, cphi[i], cphi[o], dx))
        for k in range(1, len(pts) - 1):
            tris.append((pts[0], pts[k], pts[k + 1]))
    return tris


def isosurface_cubes(phi_of, cubes, n, dx):
    """Marching-cubes triangles and their counter keys over the cubes (lowest
    corners) in block-major order: triangle t of the cube with key q has key
    12 q + t (the same twelve counter slots per cube as the tetrahedral path)."""
    tris, keys = [], []
    for q in sorted(cubes, key=lambda q: block_key(q, n)):
        key = block_key(q, n)
        cphi = [phi_of((q[0] + (c & 1), q[1] + ((c >> 1) & 1), q[2] + (c >> 2))) for c in range(8)]
        for t, tri in enumerate(cube_triangles(q, cphi, dx)):
            tris.append(tri)
            keys.append(12 * key + t)
    return tris, keys


def isosurface(phi_of, cubes, n, dx):
    """Triangles (list of (p0, p1, p2), keys) over the cubes (lowest corners), in the
    block-major order; phi_of(node) gives phi."""
    tris, keys = [], []
    for q in sorted(cubes, key=lambda q: block_key(q, n)):
        key = block_key(q, n)
        for e, corners in enumerate(TETS):
            qv = [(q[0] + c[0], q[1] + c[1], q[2] + c[2]) for c in corners]
            pv = [phi_of(v) for v in qv]
            for t, tri in enumerate(tet_triangles(qv, pv, dx)):
                tris.append(tri)
                keys.append((6 * key + e) * 2 + t)
    return tris, keys


def sample_triangles(tris, keys, seed, density):
    """Samples and their dA: count ~ Poisson(density * area) capped at KMAX, points by
    Osada's construction, dA = unit triangle normal / density."""
    s, dA = [], []
    for (p0, p1, p2), key in zip(tris, keys):
        nrm = _cross(_sub(p1, p0), _sub(p2, p0))
        nn = math.sqrt((nrm[0] * nrm[0] + nrm[1] * nrm[1]) + nrm[2] * nrm[2])
        area = 0.5 * nn
        lam = density * area
        base = key * 64
        u = uniform(seed, base)
        k = 0
        p = math.exp(-lam)
        F = p
        while u >= F and k < KMAX:
            k += 1
            p = p * lam / k
            F = F + p
        if k == 0:
            continue
        w = 1.0 / (nn * density)
        for i in range(k):
            r1 = uniform(seed, base + 2 * i + 1)
            r2 = uniform(seed, base + 2 * i + 2)
            a = math.sqrt(r1)
            b0 = 1.0 - a
            b1 = a * (1.0 - r2)
            b2 = a * r2
            s.append([(b0 * p0[c] + b1 * p1[c]) + b2 * p2[c] for c in range(3)])
            dA.append([nrm[c] * w for c in range(3)])
    return np.array(s, np.float64).reshape(-1, 3), np.array(dA, np.float64).reshape(-1, 3)


def generate(x, n, dx, seed, per_cell_area=2.0, plane=None, method="tetra"):
    """Surface samples of the particles x (origin 0): positions, dA, kind
    (0 liquid-gas, 1 solid-liquid), and the triangles they came from. method:
    "tetra" (marching tetrahedra) or "cubes" (marching cubes)."""
    if method not in ("tetra", "cubes"):
        raise ValueError(f"unknown isosurface method {method!r}")
    x = np.asarray(x, np.float64)
    phi, clamp = level_set(x, n, dx)

    def phi_of(q):
        return phi.get(q, clamp)

    cubes = set()
    for q, p in phi.items():
        if p < 0.0:
            for c in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)):
                m = (q[0] - c[0], q[1] - c[1], q[2] - c[2])
                if min(m) >= 0 and m[0] < n[0] - 1 and m[1] < n[1] - 1 and m[2] < n[2] - 1:
                    cubes.add(m)
    tris, keys = (isosurface_cubes if method == "cubes" else isosurface)(phi_of, cubes, n, dx)
    s, dA = sample_triangles(tris, keys, seed, per_cell_area / (dx * dx))
    kind = np.zeros(s.shape[0], np.uint8)
    if plane is not None and s.shape[0]:
        pn, pd = plane
        kind = np.where(s @ np.asarray(pn, np.float64) - pd < dx, 1, 0).astype(np.uint8)
    return s, dA, kind, tris
