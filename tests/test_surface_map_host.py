"""The device's per-sample projected surface Hessian map (the body of
k_surf_hess in csrc/newton.cu with its helpers surf_G, tangent_frame,
add_conformal, cross_mat and the 3x3 helpers of csrc/common.cuh), built for the
host from its source text, against the FP64 oracle's projected surface
Hessian-vector product (section "Momentum Update", Eq. fe linearised; the
definiteness fix read as the Gauss-Newton term plus the conformal part of the
cofactor curvature). The kernel stores only the upper triangle of the 9x9 map,
so the map must be symmetric; it must also be positive semi-definite."""
import ctypes
import os
import subprocess
import types

import numpy as np
import pytest

from oracle.constitutive import cof
from oracle.energy import NewtonState

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_12408_gb300", "csrc")

from tests.test_polar_host import _host_text, _template_function  # noqa: E402

SHIM = r"""
#include <cmath>
using std::fabs; using std::sqrt;
namespace mpm {
%s
template <typename R>
void surf_map(const R* Fh, const R* av, const R* nv, R ic, R k, R* out) {
%s
        for (int m = 0; m < 9; ++m) out[9 * m + l] = G[m];
    }
}
}
extern "C" void h_surf_map(const double* Fh, const double* a, const double* n, double ic, double k, double* out) {
    mpm::surf_map<double>(Fh, a, n, ic, k, out);
}
extern "C" void h_surf_mapf(const float* Fh, const float* a, const float* n, float ic, float k, float* out) {
    mpm::surf_map<float>(Fh, a, n, ic, k, out);
}
"""


def _kernel_loop(src):
    """The column loop of k_surf_hess up to (not including) its upper-triangle store."""
    k0 = src.index("__global__ void k_surf_hess(")
    i = src.index("for (int l = 0; l < 9; ++l) {", k0)
    j = src.index("for (int m = 0; m <= l; ++m)", i)
    return src[i:j]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    common = open(os.path.join(CSRC, "common.cuh")).read()
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    helpers = [_template_function(common, n) for n in ("dcofactor", "matmul3")]
    helpers += [_template_function(newton, n) for n in ("cross_mat", "surf_G", "tangent_frame", "add_conformal")]
    d = tmp_path_factory.mktemp("surfmap")
    cpp = d / "surf_map_host.cpp"
    cpp.write_text(SHIM % (_host_text("\n\n".join(helpers)), _host_text(_kernel_loop(newton))))
    so = str(d / "libsurfmap.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_surf_map.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_double] * 2 + [ctypes.c_void_p]
    L.h_surf_mapf.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_float] * 2 + [ctypes.c_void_p]
    return L


def _device_map(L, Fh, a, gamma, dt, dtype=np.float64):
    c = cof(Fh[None])[0] @ a
    cn = np.linalg.norm(c)
    Fh_ = np.ascontiguousarray(Fh, dtype)
    a_ = np.ascontiguousarray(a, dtype)
    n_ = np.ascontiguousarray(c / cn, dtype)
    out = np.zeros(81, dtype)
    fn = L.h_surf_map if dtype == np.float64 else L.h_surf_mapf
    fn(Fh_.ctypes.data, a_.ctypes.data, n_.ctypes.data, 1.0 / cn, gamma * dt * dt, out.ctypes.data)
    return out.reshape(9, 9).astype(np.float64)


def _oracle_map(Fh, a, gamma, dt):
    """Column l: dt^2 gamma (dn_a C_agd + conformal part) for dF^ = e_l, through
    the oracle's own surface derivative and conformal-part functions."""
    st = types.SimpleNamespace(dA=a[None])
    C = NewtonState._surface_C(st, Fh[None])[0]
    c = cof(Fh[None])[0] @ a
    cn = np.linalg.norm(c)
    n = c / cn
    K = np.zeros((9, 9))
    for l in range(9):
        X = np.zeros(9)
        X[l] = 1.0
        X = X.reshape(3, 3)
        dc = np.einsum("agd,gd->a", C, X)
        dn = (dc - n * np.dot(n, dc)) / cn
        dG = np.einsum("a,agd->gd", dn, C) + NewtonState._conformal_part(st, n[None], X[None])[0]
        K[:, l] = dt * dt * gamma * dG.reshape(9)
    return K


def _cases(rng):
    out = []
    for scale in (1e-3, 0.1, 0.6):
        for _ in range(40):
            Fh = np.eye(3) + scale * rng.normal(size=(3, 3))
            a = rng.normal(size=3) * rng.uniform(1e-4, 1e-1)
            out.append((Fh, a))
    # axis-aligned normals and area vectors (ties in the tangent-frame helper)
    for ax in np.eye(3):
        out.append((np.eye(3), 0.01 * ax))
        out.append((np.diag([1.1, 0.9, 1.0]), -0.02 * ax))
    out.append((np.eye(3), 0.01 * np.array([1.0, 1.0, 0.0]) / np.sqrt(2)))
    return out


def test_surface_map_matches_the_oracle_and_is_symmetric_psd(lib):
    rng = np.random.default_rng(9)
    gamma, dt = 0.7, 1e-3
    for Fh, a in _cases(rng):
        Kd = _device_map(lib, Fh, a, gamma, dt)
        Ko = _oracle_map(Fh, a, gamma, dt)
        scale = np.abs(Ko).max()
        assert np.allclose(Kd, Ko, atol=1e-12 * scale, rtol=0)
        # the kernel stores the upper triangle only: the map is symmetric
        assert np.allclose(Kd, Kd.T, atol=1e-12 * scale, rtol=0)
        w = np.linalg.eigvalsh(0.5 * (Kd + Kd.T))
        assert w.min() >= -1e-12 * scale


def test_float_surface_map_within_float_rounding(lib):
    rng = np.random.default_rng(10)
    gamma, dt = 1.0, 1e-3
    for Fh, a in _cases(rng)[:80]:
        Kf = _device_map(lib, Fh, a, gamma, dt, np.float32)
        Ko = _oracle_map(Fh, a, gamma, dt)
        scale = np.abs(Ko).max()
        assert np.allclose(Kf, Ko, atol=2e-6 * scale, rtol=0)
        assert np.allclose(Kf, Kf.T, atol=2e-6 * scale, rtol=0)


SAMPLE_G_SHIM = r"""
#include <cmath>
using std::fabs; using std::sqrt;
enum { MPM_HESS_EXACT = 0, MPM_HESS_PROJECTED = 1 };
namespace mpm {
template <typename R> struct Cols { const R* a[9]; };
template <typename R> struct ApplyArgs {   // the fields sample_G reads
    Cols<R> sF, sa, sn;
    const R* sg;
    const R* sic;
    int mode;
};
%s
}
// G (3x3) of one sample for a given dF^, in the exact or projected mode
extern "C" void h_sample_G(const double* Fh, const double* a, const double* n, double k, double ic, int mode,
                           const double* dFh, double dt, double* G) {
    mpm::ApplyArgs<double> args;
    for (int q = 0; q < 9; ++q) args.sF.a[q] = Fh + q;
    for (int q = 0; q < 3; ++q) { args.sa.a[q] = a + q; args.sn.a[q] = n + q; }
    args.sg = &k;
    args.sic = &ic;
    args.mode = mode;
    mpm::sample_G<double>(args, 0, dFh, dt, G);
}
"""


@pytest.fixture(scope="module")
def sample_lib(tmp_path_factory):
    common = open(os.path.join(CSRC, "common.cuh")).read()
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    helpers = [_template_function(common, n) for n in ("dcofactor", "matmul3")]
    helpers += [_template_function(newton, n) for n in ("cross_mat", "surf_G", "tangent_frame", "add_conformal",
                                                        "sample_G")]
    d = tmp_path_factory.mktemp("sampleG")
    cpp = d / "sample_G_host.cpp"
    cpp.write_text(SAMPLE_G_SHIM % _host_text("\n\n".join(helpers)))
    so = str(d / "libsampleG.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_sample_G.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_double] * 2 + [ctypes.c_int, ctypes.c_void_p,
                                                                             ctypes.c_double, ctypes.c_void_p]
    return L


def test_sample_term_in_both_modes_matches_the_oracle(sample_lib):
    """sample_G (the general kernel's surface term, exact and projected) against
    the oracle's exact term dn_a C_agd + n_a dC_agd and its projected term."""
    from oracle.constitutive import EPS
    rng = np.random.default_rng(13)
    gamma, dt = 0.8, 1e-3
    for Fh, a in _cases(rng):
        c = cof(Fh[None])[0] @ a
        cn = np.linalg.norm(c)
        n = c / cn
        st = types.SimpleNamespace(dA=a[None])
        C = NewtonState._surface_C(st, Fh[None])[0]
        X = rng.standard_normal((3, 3))
        dc = np.einsum("agd,gd->a", C, X)
        dn = (dc - n * np.dot(n, dc)) / cn
        exact = np.einsum("a,agd->gd", dn, C) + np.einsum("a,agk,bdl,b,kl->gd", n, EPS, EPS, a, X)
        proj = np.einsum("a,agd->gd", dn, C) + NewtonState._conformal_part(st, n[None], X[None])[0]
        for mode, ref in ((0, exact), (1, proj)):
            G = np.zeros(9)
            args = [np.ascontiguousarray(v, np.float64) for v in (Fh, a, n, X)]
            sample_lib.h_sample_G(args[0].ctypes.data, args[1].ctypes.data, args[2].ctypes.data, gamma, 1.0 / cn,
                                  mode, args[3].ctypes.data, dt, G.ctypes.data)
            want = gamma * dt * dt * ref
            np.testing.assert_allclose(G.reshape(3, 3), want, atol=1e-12 * np.abs(want).max(), rtol=0)
