"""Pins of the oracle's surface-sample generation (section "Surface Particle
Sampling"): the random generator's published outputs, exact isosurfaces of
linear fields, closed outward surfaces around particles, and the statistics of
the per-triangle Poisson / Osada sampling."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import surface as S  # noqa: E402
from paper_2101_12408_gb300 import scenes  # noqa: E402


def test_splitmix64_published_outputs():
    # SplitMix64 started from seed 0: its first three outputs
    assert S.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert S.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert S.splitmix64(0, 2) == 0x06C45D188009454F
    u = [S.uniform(12345, k) for k in range(20000)]
    assert min(u) >= 0.0 and max(u) < 1.0
    assert abs(np.mean(u) - 0.5) < 0.01 and abs(np.var(u) - 1.0 / 12.0) < 0.005


def test_isosurface_of_a_linear_field_is_the_plane():
    n, dx = (8, 8, 8), 1.0 / 8
    z0 = 3.37 * dx   # between node planes 2 and 3 ((i + 1/2) dx)

    def phi(q):  # inside below the plane
        return (q[2] + 0.5) * dx - z0

    cubes = [(i, j, k) for i in range(1, 5) for j in range(1, 4) for k in range(1, 5)]
    tris, _ = S.isosurface(phi, cubes, n, dx)
    area = 0.0
    for p0, p1, p2 in tris:
        for p in (p0, p1, p2):
            assert p[2] == pytest.approx(z0, abs=1e-15)
        nrm = S._cross(S._sub(p1, p0), S._sub(p2, p0))
        assert nrm[2] > 0 and abs(nrm[0]) < 1e-15 and abs(nrm[1]) < 1e-15   # outward = +z
        area += 0.5 * nrm[2]
    # the cubes cover x in [1.5, 5.5] dx and y in [1.5, 4.5] dx
    assert area == pytest.approx(4 * dx * 3 * dx, rel=1e-13)


def _edges(tris):
    from collections import Counter
    cnt = Counter()
    for tri in tris:
        keys = [tuple(round(c, 12) for c in p) for p in tri]
        for a in range(3):
            cnt[frozenset((keys[a], keys[(a + 1) % 3]))] += 1
    return cnt


def test_single_particle_gives_a_closed_outward_surface():
    n, dx = (8, 8, 8), 1.0 / 8
    xp = np.array([[3.3 * dx, 4.6 * dx, 3.9 * dx]])
    phi, clamp = S.level_set(xp, n, dx)
    assert min(phi.values()) < 0.0       # the radius 0.867 dx always reaches a node
    cubes = {(q[0] - a, q[1] - b, q[2] - c) for q, p in phi.items() if p < 0
             for a in (0, 1) for b in (0, 1) for c in (0, 1)}
    tris, _ = S.isosurface(lambda q: phi.get(q, clamp), cubes, n, dx)
    assert len(tris) > 0
    vec = np.zeros(3)
    for p0, p1, p2 in tris:
        nrm = np.array(S._cross(S._sub(p1, p0), S._sub(p2, p0)))
        vec += 0.5 * nrm
        c = (np.array(p0) + np.array(p1) + np.array(p2)) / 3.0
        assert np.dot(c - xp[0], nrm) > 0.0                  # outward
    area = sum(0.5 * np.linalg.norm(S._cross(S._sub(p1, p0), S._sub(p2, p0))) for p0, p1, p2 in tris)
    assert np.linalg.norm(vec) < 1e-12 * area                # closed: zero vector area
    assert all(v == 2 for v in _edges(tris).values())        # watertight


def test_droplet_surface_area_and_sample_weights():
    sc = scenes.droplet(n=32, r_cells=6.0, seed=5)
    dx = sc.dx
    s, dA, kind, tris = S.generate(sc.x, sc.n, dx, seed=77, per_cell_area=2.0)
    area = sum(0.5 * np.linalg.norm(S._cross(S._sub(p1, p0), S._sub(p2, p0))) for p0, p1, p2 in tris)
    R = 6.0 * dx
    # the union of spheres sits a fraction of a cell outside the particle cloud
    assert 4 * math.pi * R ** 2 < area < 4 * math.pi * (R + dx) ** 2
    assert all(v == 2 for v in _edges(tris).values())
    # each sample carries 1 / density: sum |dA| estimates the area (Poisson, ~1150
    # samples here), and the vector sum nearly closes
    tot = np.sum(np.linalg.norm(dA, axis=1))
    assert np.allclose(np.linalg.norm(dA, axis=1), dx * dx / 2.0, rtol=1e-12)
    assert abs(tot / area - 1.0) < 0.08
    assert np.linalg.norm(dA.sum(0)) < 0.1 * tot
    # samples lie on the surface: phi-distance to the cloud between r0 - dx and r0 + dx
    from scipy.spatial import cKDTree
    d, _ = cKDTree(sc.x).query(s)
    assert np.all(d > 0.867 * dx - dx) and np.all(d < 0.867 * dx + dx)


def test_osada_points_uniform_and_poisson_counts():
    p0, p1, p2 = [0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.0]
    s, dA = S.sample_triangles([(p0, p1, p2)] * 400, list(range(400)), seed=9, density=60.0)
    # barycentric coordinates of every point
    T = np.array([[p1[0] - p0[0], p2[0] - p0[0]], [p1[1] - p0[1], p2[1] - p0[1]]])
    lam = np.linalg.solve(T, s[:, :2].T).T
    bary = np.c_[1 - lam.sum(1), lam]
    assert np.all(bary > -1e-12) and np.all(np.abs(s[:, 2]) == 0.0)
    assert np.allclose(bary.mean(0), 1.0 / 3.0, atol=0.01)
    # area 0.45, density 60: Poisson mean 27 per triangle
    assert abs(s.shape[0] / 400.0 - 27.0) < 0.8
    assert np.allclose(dA[:, 2], 1.0 / 60.0, rtol=1e-12) and np.all(dA[:, :2] == 0.0)


def _sphere_isosurface(r_cells, n, c):
    """Triangles of phi = |x - c| - R sampled at the nodes of an n^3 grid."""
    dx = 1.0 / n
    R = r_cells * dx

    def phi(q):
        return math.sqrt(sum(((q[a] + 0.5) * dx - c[a]) ** 2 for a in range(3))) - R

    lo = [max(0, int((c[a] - R) / dx) - 2) for a in range(3)]
    hi = [min(n - 1, int((c[a] + R) / dx) + 2) for a in range(3)]
    cubes = set()
    for i in range(lo[0], hi[0]):
        for j in range(lo[1], hi[1]):
            for k in range(lo[2], hi[2]):
                v = [phi((i + a, j + b, k + e)) for a in (0, 1) for b in (0, 1) for e in (0, 1)]
                if min(v) < 0.0 <= max(v):
                    cubes.add((i, j, k))
    tris, keys = S.isosurface(phi, cubes, (n,) * 3, dx)
    area = sum(0.5 * np.linalg.norm(S._cross(S._sub(p1, p0), S._sub(p2, p0))) for p0, p1, p2 in tris)
    return tris, keys, area, R, dx


def test_tetrahedral_isosurface_of_a_sphere_area_and_sample_coverage():
    """The statistics that a marching-cubes surface of the same level set also
    meets, checked against the exact sphere instead (section "Surface Particle
    Sampling"): the triangulated area converges to 4 pi R^2 at second order in
    dx / R, and the per-triangle Poisson samples lie on the sphere, cover it
    uniformly (equal counts per octant, cos(polar angle) uniform, Archimedes) and
    carry |dA| summing to the area."""
    c = (0.513, 0.479, 0.507)   # off the node lattice
    err = {}
    for r_cells in (6.0, 12.0):
        tris, keys, area, R, dx = _sphere_isosurface(r_cells, 32, c)
        err[r_cells] = area / (4.0 * math.pi * R * R) - 1.0
    assert abs(err[6.0]) < 0.01 and abs(err[12.0]) < 0.003
    assert 3.0 < err[6.0] / err[12.0] < 5.5            # second order: halving dx / R quarters the error
    density = 2.0 / (dx * dx)
    s, dA = S.sample_triangles(tris, keys, seed=31, density=density)
    N = s.shape[0]
    assert abs(N / (density * area) - 1.0) < 4.0 / math.sqrt(density * area)
    rel = s - np.asarray(c)
    dist = np.linalg.norm(rel, axis=1)
    assert np.all(np.abs(dist - R) < 0.05 * dx)
    octant = (rel[:, 0] > 0) + 2 * (rel[:, 1] > 0) + 4 * (rel[:, 2] > 0)
    counts = np.bincount(octant, minlength=8)
    assert np.all(np.abs(counts - N / 8.0) < 5.0 * math.sqrt(N / 8.0))
    hist = np.histogram(rel[:, 2] / dist, bins=10, range=(-1.0, 1.0))[0]
    chi2 = float(np.sum((hist - N / 10.0) ** 2 / (N / 10.0)))
    assert chi2 < 33.7                                   # 9 degrees of freedom, p = 1e-4
    mag = np.linalg.norm(dA, axis=1)
    assert abs(mag.sum() / area - 1.0) < 4.0 / math.sqrt(N)
    # outward and normal to the sphere up to the facets' tilt
    assert np.all(np.sum(dA * rel, axis=1) > 0.0)
    assert np.mean(np.sum(dA * rel, axis=1) / (mag * dist)) > 0.99


@pytest.mark.parametrize("method", ["tetra", "cubes"])
def test_surface_reaches_the_first_node_layer(method):
    """Cubes whose lowest corner lies on the grid's first node layer belong to
    the lattice too: a particle in cell 1 has its sphere cut by the cubes between
    node layers 0 and 1, and the surface there is triangulated (it ends at the
    grid's edge, where the nodes end)."""
    n, dx = (10, 10, 10), 1.0 / 10
    xp = np.array([[1.3 * dx, 4.55 * dx, 5.4 * dx]])
    s, dA, kind, tris = S.generate(xp, n, dx, 3, 40.0, None, method)
    pts = np.array([p for t in tris for p in t])
    assert pts[:, 0].min() < 1.0 * dx          # between node layers 0 (0.5 dx) and 1 (1.5 dx)
    assert np.any(s[:, 0] < 1.0 * dx)
