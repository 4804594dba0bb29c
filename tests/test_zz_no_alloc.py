"""The allocation-free closest-particle search against the context path.

mpm_nearest_parent_noalloc serves callers that cannot allocate device memory
(allocators that forbid cudaMalloc after start-up, fixed memory budgets), so
cannot create a context. Its parents must equal those mpm_resample finds, index
for index, on two calls in a row (the calls share one fixed scratch array in the
library), for samples on the analytic sphere and for samples generated on the
particles' union-of-spheres surface (some lie farther than dx from every
particle, so the search must reach 2 dx as mpm_resample's does).
Collected last, so a failure here does not hide the other tests' results.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2101_12408_gb300 import scenes

pytestmark = pytest.mark.gpu

mpm = pytest.importorskip("paper_2101_12408_gb300.mpm")
torch = pytest.importorskip("torch")


def _context_parents(sc):
    ctx = mpm.Context(sc, precision=mpm.PREC_FP64)
    ctx.load_scene(0)
    ctx.resample()
    out = ctx.get_surface(0)["parent"]
    ctx.close()
    return out


def test_noalloc_parents_match_resample_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    for seed, r_cells in ((21, 8.0), (22, 6.5)):
        sc = scenes.droplet(n=32, r_cells=r_cells, seed=seed)
        ref = _context_parents(sc)
        x = torch.tensor(sc.x, dtype=torch.float64, device=dev).contiguous()
        s = torch.tensor(sc.s, dtype=torch.float64, device=dev).contiguous()
        for _ in range(2):
            parent = torch.full((sc.n_surface,), -7, dtype=torch.int32, device=dev)
            status = mpm.nearest_parent_noalloc(sc, x, s, parent)
            assert status == mpm.MPM_OK
            np.testing.assert_array_equal(parent.cpu().numpy(), ref)


def test_noalloc_parents_match_resample_on_generated_surfaces():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    sc = scenes.droplet(n=32, r_cells=7.0, seed=23)
    ctx = mpm.Context(sc, precision=mpm.PREC_FP64, surface_capacity_factor=8.0)
    ctx.load_scene(0)
    ctx.generate_surface(seed=5)
    ctx.resample()
    surf = ctx.get_surface(0)
    ctx.close()
    ref, s_np = surf["parent"], surf["s"]
    # the generated samples do include ones beyond dx of every particle
    d = cKDTree(sc.x).query(s_np)[0]
    assert np.any(d > sc.dx) and np.all(d <= 2 * sc.dx)
    x = torch.tensor(sc.x, dtype=torch.float64, device=dev).contiguous()
    s = torch.tensor(s_np, dtype=torch.float64, device=dev).contiguous()
    for _ in range(2):
        parent = torch.full((s_np.shape[0],), -7, dtype=torch.int32, device=dev)
        assert mpm.nearest_parent_noalloc(sc, x, s, parent) == mpm.MPM_OK
        np.testing.assert_array_equal(parent.cpu().numpy(), ref)


def test_noalloc_wrapper_rejects_wrong_dtypes_and_shapes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    sc = scenes.droplet(n=16, r_cells=4.0, seed=24)
    x = torch.tensor(sc.x, dtype=torch.float64, device=dev)
    s = torch.tensor(sc.s, dtype=torch.float64, device=dev)
    parent = torch.empty((sc.n_surface,), dtype=torch.int32, device=dev)
    with pytest.raises(ValueError):
        mpm.nearest_parent_noalloc(sc, x.float(), s, parent)
    with pytest.raises(ValueError):
        mpm.nearest_parent_noalloc(sc, x, s, parent[:-1])
    with pytest.raises(ValueError):
        mpm.nearest_parent_noalloc(sc, x.t(), s, parent)
    with pytest.raises(ValueError):
        mpm.nearest_parent_noalloc(sc, x.cpu(), s, parent)


def test_noalloc_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = scenes.droplet(n=128, r_cells=4.0, seed=3)   # 128^3 cells > 2^20
    dev = torch.device("cuda", 0)
    x = torch.tensor(sc.x, dtype=torch.float64, device=dev)
    s = torch.tensor(sc.s, dtype=torch.float64, device=dev)
    parent = torch.empty((sc.n_surface,), dtype=torch.int32, device=dev)
    assert mpm.nearest_parent_noalloc(sc, x, s, parent) == mpm.MPM_ERR_CAPACITY
