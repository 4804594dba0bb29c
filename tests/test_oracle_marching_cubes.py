"""Pins of the oracle's marching cubes (section "Surface Particle Sampling": the
isocontour of the union-of-spheres level set by marching cubes, Chernyaev's
variant). The triangulation is built from face segments, not from a case table,
so it is pinned against facts that fix any marching-cubes surface: the triangle
counts of the fifteen classic corner configurations under every symmetry of the
cube, the asymptotic decider on ambiguous faces, a closed and consistently
oriented surface over random fields, the exact plane of a linear field, and
second-order convergence to a sphere's area and volume. It is then compared with
the tetrahedral triangulation the same level set gives."""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

from oracle import surface as S
from paper_2101_12408_gb300 import scenes

# the fifteen classic configurations (Lorensen and Cline, 1987) as sets of inside
# corners (corner c = x + 2 y + 4 z), with their triangle counts when every
# ambiguous face keeps its inside corners apart
CASES = [
    ((), 0),
    ((0,), 1),
    ((0, 1), 2),            # one edge
    ((0, 3), 2),            # face diagonal (ambiguous face)
    ((0, 7), 2),            # body diagonal
    ((0, 1, 2), 3),         # three corners of a face
    ((0, 1, 7), 3),         # an edge and the far corner of an adjacent face
    ((1, 2, 4), 3),         # three corners pairwise face-diagonal
    ((0, 1, 2, 3), 2),      # a whole face
    ((0, 1, 2, 4), 4),      # a corner with its three neighbours
    ((0, 1, 6, 7), 4),      # two opposite parallel edges
    ((0, 1, 3, 5), 4),      # a corner, two neighbours and one more: a hexagon
    ((0, 1, 2, 7), 4),      # three corners of a face and the opposite corner
    ((0, 3, 5, 6), 4),      # checkerboard
    ((0, 1, 3, 7), 4),      # a path of three edges along x, y, z
]


def _symmetries():
    """The 48 symmetries of the cube as corner permutations."""
    out = []
    for perm in itertools.permutations(range(3)):
        for flip in itertools.product((0, 1), repeat=3):
            m = []
            for c in range(8):
                b = S._corner_bits(c)
                nb = [b[perm[a]] ^ flip[a] for a in range(3)]
                m.append(nb[0] + 2 * nb[1] + 4 * nb[2])
            out.append(m)
    return out


def _values(inside, rng, in_mag=0.1):
    """Corner values: inside corners in (-2 in_mag, -in_mag], outside ones in [1, 2)."""
    return [(-in_mag * (1.0 + rng.random())) if c in inside else 1.0 + rng.random() for c in range(8)]


def test_classic_cases_triangle_counts_under_every_symmetry():
    rng = np.random.default_rng(7)
    syms = _symmetries()
    assert len({tuple(m) for m in syms}) == 48
    for inside, ntri in CASES:
        for m in syms:
            ins = {m[c] for c in inside}
            # separated: shallow inside corners, the decider keeps them apart
            vals = _values(ins, rng)
            tris = S.cube_triangles((0, 0, 0), vals, 1.0)
            assert len(tris) == ntri, (inside, m)
            # the complement with the values negated: its deep inside corners join
            # across every ambiguous face, which is the same surface around `ins`
            # facing the other way (the same count, the opposite vector area)
            neg = [-v for v in vals]
            tris_c = S.cube_triangles((0, 0, 0), neg, 1.0)
            assert len(tris_c) == ntri, (inside, m)
            va = sum(np.cross(np.subtract(p1, p0), np.subtract(p2, p0)) for p0, p1, p2 in tris) if tris else 0
            vc = sum(np.cross(np.subtract(p1, p0), np.subtract(p2, p0)) for p0, p1, p2 in tris_c) if tris_c else 0
            assert np.allclose(va, -vc, atol=1e-12)
    # every one of the 256 configurations is one of the fifteen up to symmetry and complement
    seen = set()
    for inside, _ in CASES:
        for m in syms:
            ins = frozenset(m[c] for c in inside)
            seen.add(ins)
            seen.add(frozenset(range(8)) - ins)
    assert len(seen) == 256


def test_asymptotic_decider_joins_deep_diagonal_corners():
    # face z = 0 with corners 0 and 3 inside: separated gives two corner triangles,
    # joined (the bilinear saddle inside) one band of four crossings
    cphi = [-0.1, 1.0, 1.0, -0.1, 1.0, 1.0, 1.0, 1.0]
    assert [len(l) for l in S.cube_loops(cphi)] == [3, 3]
    cphi = [-3.0, 1.0, 1.0, -3.0, 1.0, 1.0, 1.0, 1.0]     # 9 > 1: the saddle is inside
    assert [len(l) for l in S.cube_loops(cphi)] == [6]
    # the test is the sign of phi_a phi_c - phi_b phi_d, so it is the same from both
    # cubes that share the face, and a tie keeps the corners apart (phi = 0 is outside)
    cphi = [-1.0, 1.0, 1.0, -1.0, 1.0, 1.0, 1.0, 1.0]
    assert [len(l) for l in S.cube_loops(cphi)] == [3, 3]


def _directed_edges(tris):
    cnt = Counter()
    for tri in tris:
        k = [tuple(p) for p in tri]
        for a in range(3):
            cnt[(k[a], k[(a + 1) % 3])] += 1
    return cnt


def test_random_fields_give_closed_oriented_surfaces():
    """Every directed triangle edge is matched by the reverse edge, so the pieces
    of neighbouring cubes meet exactly (shared edge points, the same face
    decisions) and all face one way; the enclosed volume by the divergence
    theorem is positive (outward)."""
    rng = np.random.default_rng(3)
    n = (9, 8, 7)
    dx = 0.25
    for trial in range(6):
        vals = rng.normal(size=n)
        vals[[0, -1], :, :] = 1.0
        vals[:, [0, -1], :] = 1.0
        vals[:, :, [0, -1]] = 1.0
        if trial % 2:                     # deeper inside values join more ambiguous faces
            vals = np.where(vals < 0, 3.0 * vals, vals)

        def phi(q):
            return float(vals[q])

        cubes = [(i, j, k) for i in range(n[0] - 1) for j in range(n[1] - 1) for k in range(n[2] - 1)]
        tris, keys = S.isosurface_cubes(phi, cubes, n, dx)
        assert len(tris) > 50
        cnt = _directed_edges(tris)
        assert all(cnt[(b, a)] == v for (a, b), v in cnt.items())
        vol = sum(np.dot(p0, np.cross(p1, p2)) for p0, p1, p2 in tris) / 6.0
        assert vol > 0.0
        assert len(set(keys)) == len(keys)
        assert all(k % 12 < 11 for k in keys)


def test_isosurface_cubes_of_a_linear_field_is_the_plane():
    n, dx = (8, 8, 8), 1.0 / 8
    nrm = np.array([0.3, -0.2, 1.0])
    nrm /= np.linalg.norm(nrm)
    d0 = 3.37 * dx

    def phi(q):
        return float(np.dot((np.array(q) + 0.5) * dx, nrm) - d0)

    cubes = [(i, j, k) for i in range(7) for j in range(7) for k in range(7)]
    tris, _ = S.isosurface_cubes(phi, cubes, n, dx)
    vec = np.zeros(3)
    for p0, p1, p2 in tris:
        for p in (p0, p1, p2):
            assert abs(np.dot(p, nrm) - d0) < 1e-14
        vec += 0.5 * np.cross(np.subtract(p1, p0), np.subtract(p2, p0))
    # every facet lies in the plane and faces +nrm; the summed vector area is the
    # plane's section of the node box [dx/2, 7.5 dx]^3 projected on z
    assert np.allclose(vec / np.linalg.norm(vec), nrm, atol=1e-14)
    assert vec[2] == pytest.approx(7 * dx * 7 * dx, rel=1e-12)


def _sphere(r_cells, n, c, method):
    dx = 1.0 / n
    R = r_cells * dx

    def phi(q):
        return math.sqrt(sum(((q[a] + 0.5) * dx - c[a]) ** 2 for a in range(3))) - R

    lo = [max(0, int((c[a] - R) / dx) - 2) for a in range(3)]
    hi = [min(n - 1, int((c[a] + R) / dx) + 2) for a in range(3)]
    cubes = [(i, j, k) for i in range(lo[0], hi[0]) for j in range(lo[1], hi[1]) for k in range(lo[2], hi[2])]
    iso = S.isosurface_cubes if method == "cubes" else S.isosurface
    tris, keys = iso(phi, cubes, (n,) * 3, dx)
    area = sum(0.5 * np.linalg.norm(np.cross(np.subtract(p1, p0), np.subtract(p2, p0))) for p0, p1, p2 in tris)
    vol = sum(np.dot(np.subtract(p0, c), np.cross(np.subtract(p1, c), np.subtract(p2, c))) for p0, p1, p2 in tris) / 6.0
    return tris, keys, area, vol, R, dx


def test_marching_cubes_sphere_converges_at_second_order():
    c = (0.513, 0.479, 0.507)
    ea, ev = {}, {}
    for r_cells in (6.0, 12.0):
        tris, _, area, vol, R, _ = _sphere(r_cells, 32, c, "cubes")
        ea[r_cells] = area / (4.0 * math.pi * R * R) - 1.0
        ev[r_cells] = vol / (4.0 / 3.0 * math.pi * R ** 3) - 1.0
        # a sphere is one closed surface: V - E + F = 2 over the shared edge points
        verts = {tuple(p) for t in tris for p in t}
        edges = {frozenset((tuple(t[a]), tuple(t[(a + 1) % 3]))) for t in tris for a in range(3)}
        assert len(verts) - len(edges) + len(tris) == 2
    assert abs(ea[6.0]) < 0.02 and abs(ea[12.0]) < 0.005
    assert 3.0 < ea[6.0] / ea[12.0] < 5.5
    assert abs(ev[6.0]) < 0.02 and 3.0 < ev[6.0] / ev[12.0] < 5.5


def test_tetrahedra_and_cubes_sample_the_same_surface():
    """The tetrahedral triangulation (the default) and marching cubes of the same
    union-of-spheres level set: different triangles (marching cubes makes about a
    third as many), the same enclosed volume to 0.5%, the same shell of samples
    around the particles, and areas that differ by the facets' roughness only.
    The tetrahedra cut every cube along its diagonals as well, so their surface
    follows more of the bumps of the union of spheres (radial spread of the
    samples 0.080 dx against 0.059 dx) and is about 3% larger (measured 2.9% and
    3.0% on droplets of 6 and 10 cells)."""
    sc = scenes.droplet(n=32, r_cells=6.0, seed=5)
    c = sc.x.mean(0)
    out = {}
    for method in ("tetra", "cubes"):
        s, dA, kind, tris = S.generate(sc.x, sc.n, sc.dx, 41, 2.0, None, method)
        area = sum(0.5 * np.linalg.norm(np.cross(np.subtract(p1, p0), np.subtract(p2, p0))) for p0, p1, p2 in tris)
        vol = sum(np.dot(np.subtract(p0, c), np.cross(np.subtract(p1, c), np.subtract(p2, c)))
                  for p0, p1, p2 in tris) / 6.0
        out[method] = (s, dA, tris, area, vol)
    st, dAt, tt, at, vt = out["tetra"]
    sm, dAm, tm, am, vm = out["cubes"]
    assert len(tm) < 0.5 * len(tt)
    assert abs(vm / vt - 1.0) < 0.005
    assert 0.0 < 1.0 - am / at < 0.05
    for s, dA, area in ((st, dAt, at), (sm, dAm, am)):
        N = s.shape[0]
        assert abs(np.linalg.norm(dA, axis=1).sum() / area - 1.0) < 4.0 / math.sqrt(N)
    assert abs(sm.shape[0] / st.shape[0] - am / at) < 6.0 / math.sqrt(st.shape[0])
    # the same shell around the particles, the cubes' one the smoother
    rt, rm = np.linalg.norm(st - c, axis=1), np.linalg.norm(sm - c, axis=1)
    assert abs(rt.mean() - rm.mean()) < 0.05 * sc.dx
    assert rm.std() < rt.std() < 0.1 * sc.dx
    assert np.all(np.sum(dAm * (sm - c), axis=1) > 0.0)


def test_cube_triangles_per_cube_fit_the_counter_slots():
    """At most ten triangles per cube (twelve crossing edges, at least one loop of
    three or more), so the twelve counter slots per cube never overlap; checked
    over every configuration with random magnitudes."""
    rng = np.random.default_rng(11)
    worst = 0
    for m in range(256):
        for _ in range(20):
            ins = {c for c in range(8) if (m >> c) & 1}
            cphi = _values(ins, rng, in_mag=float(rng.choice([0.1, 3.0])))
            loops = S.cube_loops(cphi)
            assert sum(len(l) for l in loops) == sum(
                1 for e in range(12) if (cphi[S._edge_corners(e)[0]] < 0) != (cphi[S._edge_corners(e)[1]] < 0))
            assert all(len(l) >= 3 for l in loops)
            worst = max(worst, sum(len(l) - 2 for l in loops))
    assert worst <= 10
