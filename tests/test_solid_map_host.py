"""The device's per-particle projected solid Hessian map (the body of
k_solid_hess in csrc/newton.cu, with svd3 and jacobi_rot of csrc/polar.cuh and
the 3x3 helpers of csrc/common.cuh), built for the host from its source text,
against the FP64 oracle's definition: the 9x9 Hessian of the fixed-corotated
energy formed from the exact dP on the nine unit directions, its negative
eigenvalues clamped by a numerical eigendecomposition, composed with
dF = dL F^n and M = dt^2 V0 dP F^nT (section "Constitutive Models"; the
definiteness fix read as the per-particle projection). The device writes the
same map from the analytic eigensystem of isotropic energies; here on repeated
and nearly repeated singular values, inverted elements and strong stretches."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle.energy import NewtonState
from tests.test_polar_host import _host_text, _rot, _template_function

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_12408_gb300", "csrc")

SHIM = r"""
#include <cmath>
using std::fabs; using std::sqrt; using std::copysign;
namespace mpm {
constexpr int sym9(int m, int l) { return m * 9 - m * (m - 1) / 2 + (l - m); }
%s
template <typename R>
void solid_map(const R* F, const R* Fo, R mu, R lam, R scale, R* Kout) {
%s
    for (int k = 0; k < 45; ++k) Kout[k] = Kp[k];
}
}
extern "C" void h_solid_map(const double* F, const double* Fo, double mu, double lam, double scale, double* K) {
    mpm::solid_map<double>(F, Fo, mu, lam, scale, K);
}
"""


def _kernel_body(src):
    k0 = src.index("__global__ void k_solid_hess(")
    i = src.index("R u[3][3], V[9], s[3];", k0)
    j = src.index("for (int k = 0; k < 45; ++k) K.a[k][i] = Kp[k];", i)
    return src[i:j]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    common = open(os.path.join(CSRC, "common.cuh")).read()
    polar = open(os.path.join(CSRC, "polar.cuh")).read()
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    helpers = [_template_function(common, n) for n in ("matmul3", "matmul3_bt")]
    helpers += [_template_function(polar, n) for n in ("jacobi_rot", "swap_cols", "svd3")]
    d = tmp_path_factory.mktemp("solidmap")
    cpp = d / "solid_map_host.cpp"
    cpp.write_text(SHIM % (_host_text("\n\n".join(helpers)), _host_text(_kernel_body(newton))))
    so = str(d / "libsolidmap.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_solid_map.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_double] * 3 + [ctypes.c_void_p]
    return L


def _device_map(L, F, Fo, mu, lam, scale):
    F_ = np.ascontiguousarray(F, np.float64)
    Fo_ = np.ascontiguousarray(Fo, np.float64)
    Kp = np.zeros(45)
    L.h_solid_map(F_.ctypes.data, Fo_.ctypes.data, mu, lam, scale, Kp.ctypes.data)
    K = np.zeros((9, 9))
    k = 0
    for m in range(9):
        for l in range(m, 9):
            K[m, l] = K[l, m] = Kp[k]
            k += 1
    return K


def _oracle_map(F, Fo, mu, lam, scale):
    H = NewtonState.solid_hessian_psd(F[None], np.array([mu]), np.array([lam]))[0]
    K = np.zeros((9, 9))
    for l in range(9):
        dL = np.zeros(9)
        dL[l] = 1.0
        dF = dL.reshape(3, 3) @ Fo
        dP = (H @ dF.reshape(9)).reshape(3, 3)
        K[:, l] = (scale * dP @ Fo.T).reshape(9)
    return K


def _cases(rng):
    out = []
    for sv in ([1.0, 1.0, 1.0], [1.2, 1.2, 0.8], [1.1, 1.0, 1.0], [1.3, 0.9, 0.7], [1.0, 1.0 + 1e-9, 0.9],
               [2.0, 0.5, 0.25], [1.1, 0.9, -0.4], [1.0, 0.8, -0.8 + 0.05], [0.6, 0.6, 0.6], [3.0, 1.0, 0.3]):
        for _ in range(8):
            out.append(_rot(rng) @ np.diag(sv) @ _rot(rng).T)
    return out


@pytest.mark.parametrize("mu,lam", [(1.0, 3.0), (5.0, 0.5), (0.0, 2.0)])
def test_solid_map_matches_the_clamped_numerical_hessian(lib, mu, lam):
    rng = np.random.default_rng(12)
    scale = 1e-3 ** 2 * 2e-6
    for F in _cases(rng):
        Fo = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
        Kd = _device_map(lib, F, Fo, mu, lam, scale)
        Ko = _oracle_map(F, Fo, mu, lam, scale)
        tol = 1e-9 * np.abs(Ko).max()
        assert np.allclose(Kd, Ko, atol=tol, rtol=0), F
        assert np.linalg.eigvalsh(Kd).min() >= -tol
