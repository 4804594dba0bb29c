"""The C-ABI library builds, loads without a GPU and exports every symbol the
public header declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mpm_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2101_12408_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for need in ("mpm_create", "mpm_resample", "mpm_p2g", "mpm_apply_hessian", "mpm_heat_apply",
                 "mpm_newton_step", "mpm_g2p"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_2101_12408_gb300 import mpm
    assert sorted(mpm.EXPORTED) == _declared()


def test_struct_sizes_match_c_layout(lib):
    from paper_2101_12408_gb300 import mpm
    # sizes follow the C rules for the header's field order (8-byte aligned doubles)
    assert ctypes.sizeof(mpm.GridDesc) == 152
    assert ctypes.sizeof(mpm.Params) == 232
    assert ctypes.sizeof(mpm.SceneDesc) == 408
    assert ctypes.sizeof(mpm.Stats) == 64


def test_struct_layout_matches_the_header_compiled(tmp_path):
    """Sizes and the offsets of the last fields, from the header compiled by the host C compiler."""
    import shutil
    import subprocess
    from paper_2101_12408_gb300 import mpm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "mpm.h"\n'
        'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mpm_params), sizeof(mpm_scene_desc),'
        ' offsetof(mpm_params, phase_change), offsetof(mpm_params, friction),'
        ' offsetof(mpm_params, massless_surface), sizeof(mpm_grid_desc), offsetof(mpm_grid_desc, sphere),'
        ' offsetof(mpm_grid_desc, sphere_mode)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(mpm.Params), ctypes.sizeof(mpm.SceneDesc), mpm.Params.phase_change.offset,
                   mpm.Params.friction.offset, mpm.Params.massless_surface.offset, ctypes.sizeof(mpm.GridDesc),
                   mpm.GridDesc.sphere.offset, mpm.GridDesc.sphere_mode.offset]


def test_profile_layout_matches_the_header_compiled(tmp_path):
    """The profile record the binding reads (the autotuner's choices at its end)."""
    import shutil
    import subprocess
    from paper_2101_12408_gb300 import mpm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "profile.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "mpm.h"\n'
        'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(mpm_profile), offsetof(mpm_profile, cg_ctas_per_sm),'
        ' offsetof(mpm_profile, cg_graph_error), offsetof(mpm_profile, op_rows_per_chunk)); return 0; }\n')
    exe = tmp_path / "profile"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(mpm.Profile), mpm.Profile.cg_ctas_per_sm.offset, mpm.Profile.cg_graph_error.offset,
                   mpm.Profile.op_rows_per_chunk.offset]


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2101_12408_gb300 import mpm
    out = ctypes.c_void_p()
    # no scenes: rejected before any CUDA call
    assert lib.mpm_create(None, 0, 1, None, ctypes.byref(out)) == mpm.MPM_ERR_INVALID_ARG
    assert lib.mpm_resample(None) == mpm.MPM_ERR_INVALID_ARG
    assert lib.mpm_destroy(None) == mpm.MPM_ERR_INVALID_ARG
    for method in (mpm.ISO_TETRAHEDRA, mpm.ISO_CUBES, 7):
        assert lib.mpm_generate_surface_method(None, ctypes.c_uint64(1), ctypes.c_double(2.0), ctypes.c_int32(method),
                                               None) == mpm.MPM_ERR_INVALID_ARG


def test_invalid_friction_and_massless_flag_rejected_without_gpu(lib):
    """mpm_create checks every scene's parameters before any CUDA call."""
    from paper_2101_12408_gb300 import mpm, scenes
    sc = scenes.droplet(n=8, r_cells=2.0, seed=1)
    for field, bad in (("friction", -0.1), ("friction", float("nan")), ("friction", float("inf")),
                       ("massless_surface", 2), ("massless_surface", -1)):
        d = mpm.scene_desc(sc)
        setattr(d.params, field, bad)
        out = ctypes.c_void_p()
        assert lib.mpm_create(ctypes.byref(d), 1, 1, None, ctypes.byref(out)) == mpm.MPM_ERR_INVALID_ARG, field
        assert not out.value


def test_spherical_solid_reaches_the_descriptor_and_bad_spheres_are_rejected(lib):
    """The binding passes the spherical solid to mpm_grid_desc; mpm_create rejects
    a non-positive or non-finite radius, a non-finite centre and an unknown mode
    before any CUDA call."""
    from paper_2101_12408_gb300 import mpm, scenes
    sc = scenes.droplet(n=8, r_cells=2.0, seed=1)
    sc.sphere, sc.sphere_mode = (0.5, 0.45, 0.55, 0.3, True), scenes.WALL_SLIP
    d = mpm.scene_desc(sc)
    assert list(d.grid.sphere) == [0.5, 0.45, 0.55, 0.3]
    assert d.grid.sphere_outside == 1 and d.grid.sphere_mode == scenes.WALL_SLIP
    for field, idx, bad in (("sphere", 3, 0.0), ("sphere", 3, -0.2), ("sphere", 3, float("nan")),
                            ("sphere", 0, float("inf")), ("sphere_mode", None, 3)):
        d = mpm.scene_desc(sc)
        if idx is None:
            setattr(d.grid, field, bad)
        else:
            getattr(d.grid, field)[idx] = bad
        out = ctypes.c_void_p()
        assert lib.mpm_create(ctypes.byref(d), 1, 1, None, ctypes.byref(out)) == mpm.MPM_ERR_INVALID_ARG, (field, bad)
        assert not out.value
