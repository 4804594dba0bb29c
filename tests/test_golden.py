"""Stored fixtures in tests/golden: values the paper prints, and oracle outputs
written by tests/golden/make_golden.py (which calls only the oracle)."""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

from oracle import surface as osurf

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _paper():
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        return json.load(f)


def _stored():
    with open(os.path.join(GOLDEN, "oracle_droplet_step.json")) as f:
        return json.load(f)


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_levelset_radius_is_the_papers_and_isolated_particles_cross_the_grid():
    r = _paper()["levelset_radius_factor_3d"]["value"]
    assert osurf.R0_FACTOR == r
    # the property the paper gives for its choice: just above sqrt(3)/2, so a
    # lone particle's sphere always contains the nearest node and its level set
    # has a zero crossing on the grid
    assert math.sqrt(3.0) / 2.0 < r
    rng = np.random.default_rng(12)
    n, dx = (8, 8, 8), 1.0 / 8
    for k in range(40):
        x = (rng.uniform(2.0, 6.0, (1, 3))) * dx
        s, dA, kind, tris = osurf.generate(x, n, dx, seed=k, per_cell_area=8.0)
        assert len(tris) > 0


def test_oracle_reproduces_its_stored_droplet_step():
    ref = _stored()
    now = _maker().droplet_step()
    assert now["nodes"] == ref["nodes"] and now["particles"] == ref["particles"]
    np.testing.assert_allclose(now["vhat"], ref["vhat"], rtol=0, atol=1e-12 * ref["vhat_absmax"])
    np.testing.assert_allclose(now["v"], ref["v"], rtol=0, atol=1e-12 * ref["v_absmax"])
    np.testing.assert_allclose(now["x"], ref["x"], rtol=0, atol=1e-14)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gpu_step_matches_stored_oracle_values(prec):
    from paper_2101_12408_gb300 import mpm
    ref = _stored()
    sc = _maker().droplet_scene()
    p = mpm.PREC_FP64 if prec == "fp64" else mpm.PREC_FP32_FP64RED
    if prec == "fp32":
        # the float32 form at the scene's default solver settings
        sc.params.newton_tol, sc.params.cg_rtol, sc.params.max_cg = 1e-6, 1e-3, 1000
    tol = 1e-8 if prec == "fp64" else 1e-5
    ctx = mpm.Context(sc, precision=p)
    ctx.load_scene(0)
    ctx.resample()
    ctx.p2g()
    ctx.newton_step()
    vh = ctx.get_grid(0, mpm.FIELD_VHAT)[ref["nodes"]]
    assert np.max(np.abs(vh - np.array(ref["vhat"]))) < tol * ref["vhat_absmax"]
    ctx.g2p()
    part = ctx.get_particles(0)
    assert np.max(np.abs(part["v"][ref["particles"]] - np.array(ref["v"]))) < max(tol, 1e-7) * ref["v_absmax"]


def test_wax_workload_uses_the_papers_candle_constants():
    """The melting-wax workload takes the candle examples' printed constants:
    ambient and melting temperatures, K, c_p, no internal source, the Robin h and
    the heating rate b on the heated face, and a surface coefficient at T0 among
    the compared ones."""
    from paper_2101_12408_gb300 import scenes
    v = {k: e["value"] for k, e in _paper().items()}
    sc = scenes.wax(nx=16, ny=16, nz=16, cube_cells=4)
    p = sc.params
    assert p.T0 == v["candle_ambient_temperature"] and p.T_melt == v["candle_melting_point"]
    assert p.K == v["candle_thermal_diffusivity"] and p.cp == v["candle_specific_heat"]
    assert p.H == v["candle_internal_heat_source"] and p.h == v["candle_robin_h"]
    assert set(np.unique(sc.b)) == {0.0, v["candle_robin_b"]}
    assert p.gamma_p[0] in v["candle_surface_coefficients"]
    assert np.all(sc.Tbar == v["candle_ambient_temperature"])


def test_papers_contact_angle_ratios_and_the_oracles_energy_minimum():
    """The paper's settling-droplet figure pairs k_SL / k_LG ratios with contact
    angles through Young's relation theta = arccos(-k_SL / k_LG). For the
    hydrophobic 135-degree case the oracle's surface energy of resting caps (the
    samples, interface kinds and coefficients of reading R13) is smallest within
    a degree of it at 10 and 20 cells of radius."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_pins import _cap_energy
    e = _paper()["contact_angle_ratios"]
    for ratio, angle in zip(e["value"], e["angles_deg"]):
        assert math.degrees(math.acos(-ratio)) == pytest.approx(angle, abs=1e-9)
    k_sl = e["value"][2]
    volume = 2.0 / 3.0 * math.pi * (10 / 64) ** 3
    for n in (64, 128):
        ths = 135.0 + np.arange(-10.0, 10.5, 5.0)
        es = np.array([_cap_energy(t, volume, k_sl, n) for t in ths])
        assert np.argmin(es) == 2
        q = np.polyfit(ths, es, 2)
        assert abs(-q[1] / (2 * q[0]) - 135.0) < 1.0
