"""The allocation-free closest-particle search against the context path.

mpm_nearest_parent_noalloc serves callers that cannot allocate device memory
(graph capture in progress, allocators that forbid cudaMalloc, fixed memory
budgets). Its parents must equal those mpm_resample finds, index for index, on
two calls in a row (the calls share one fixed scratch array in the library).
Collected last, so a failure here does not hide the other tests' results.
"""
import numpy as np
import pytest

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
        parent = torch.full((sc.n_surface,), -7, dtype=torch.int32, device=dev)
        status = mpm.nearest_parent_noalloc(sc, x, s, parent)
        assert status == mpm.MPM_OK
        np.testing.assert_array_equal(parent.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = scenes.droplet(n=128, r_cells=4.0, seed=3)   # 128^3 cells > 2^20
    dev = torch.device("cuda", 0)
    x = torch.tensor(sc.x, dtype=torch.float64, device=dev)
    s = torch.tensor(sc.s, dtype=torch.float64, device=dev)
    parent = torch.empty((sc.n_surface,), dtype=torch.int32, device=dev)
    assert mpm.nearest_parent_noalloc(sc, x, s, parent) == mpm.MPM_ERR_CAPACITY
