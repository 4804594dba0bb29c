"""The device's marching-cubes routine (csrc/mcubes.cuh) built for the host with
the host C++ compiler, against the FP64 oracle's marching cubes (section
"Surface Particle Sampling"): the same triangles, bit for bit, for every corner
configuration and on a droplet's union-of-spheres level set. The routine rounds
every product and sum on its own, so without contraction the host build gives
the device's values; the device kernels around it are checked on the GPU."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import surface as S
from paper_2101_12408_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("mc") / "libmc_host.so")
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
           os.path.join(HERE, "host", "mc_host_shim.cpp"), "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    lib = ctypes.CDLL(out)
    lib.mc_host_cube.restype = ctypes.c_int
    lib.mc_host_cube.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    return lib


def _host(lib, q, cphi, dx):
    c = np.ascontiguousarray(cphi, np.float64)
    qq = np.ascontiguousarray(q, np.int32)
    out = np.zeros((12, 9))
    n = lib.mc_host_cube(c.ctypes.data, qq.ctypes.data, dx, out.ctypes.data)
    return out[:n]


def _oracle(q, cphi, dx):
    tris = S.cube_triangles(q, list(cphi), dx)
    return np.array([np.concatenate(t) for t in tris]).reshape(-1, 9)


def test_every_configuration_matches_the_oracle_bitwise(shim):
    rng = np.random.default_rng(5)
    dx = 1.0 / 37
    for m in range(256):
        for mag in (0.05, 1.0, 20.0):
            for _ in range(4):
                ins = [(m >> c) & 1 for c in range(8)]
                cphi = [(-mag if i else 1.0) * (0.5 + rng.random()) for i in ins]
                q = tuple(int(v) for v in rng.integers(0, 200, 3))
                got, ref = _host(shim, q, cphi, dx), _oracle(q, cphi, dx)
                assert got.shape == ref.shape, (m, cphi)
                assert np.array_equal(got, ref), (m, cphi)


def test_droplet_level_set_matches_the_oracle_bitwise(shim):
    sc = scenes.droplet(n=32, r_cells=6.0, seed=5)
    phi, clamp = S.level_set(sc.x, sc.n, sc.dx)

    def phi_of(q):
        return phi.get(q, clamp)

    cubes = {(q[0] - a, q[1] - b, q[2] - c) for q, p in phi.items() if p < 0.0
             for a in (0, 1) for b in (0, 1) for c in (0, 1)}
    ref, _ = S.isosurface_cubes(phi_of, cubes, sc.n, sc.dx)
    got = []
    for q in sorted(cubes, key=lambda q: S.block_key(q, sc.n)):
        cphi = [phi_of((q[0] + (c & 1), q[1] + ((c >> 1) & 1), q[2] + (c >> 2))) for c in range(8)]
        got.extend(_host(shim, q, cphi, sc.dx))
    ref = np.array([np.concatenate(t) for t in ref])
    assert len(ref) > 1000
    assert np.array_equal(np.array(got), ref)
