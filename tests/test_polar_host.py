"""The device's 3x3 polar decomposition and fixed-corotated stress differential
(csrc/polar.cuh, with the 3x3 helpers of csrc/common.cuh), built for the host
from their source text and checked against the mathematics on inputs the
parity scenes rarely reach: rotations and repeated singular values, inverted
and nearly flat elements, rank-one and zero F (section "Constitutive Models",
fixed corotated elasticity; the polar SVD with the sign of det F on the
smallest singular value). The device compiles the same text with contraction
into fused multiply-adds, so the checks are of identities, not of bits."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_12408_gb300", "csrc")


def _template_function(src, name):
    """The text of `template <typename R> ... name(...) { ... }` in src."""
    m = re.search(r"template <typename R>\s*\n__device__[^\n]*\b" + name + r"\(", src)
    assert m, name
    i = src.index("{", m.end())
    depth = 0
    for j in range(i, len(src)):
        if src[j] == "{":
            depth += 1
        elif src[j] == "}":
            depth -= 1
            if depth == 0:
                return src[m.start():j + 1]
    raise AssertionError(name)


def _host_text(txt):
    txt = txt.replace("__device__ __forceinline__", "inline").replace("__device__", "inline")
    return re.sub(r"#pragma unroll\s*\n", "", txt)


SHIM = r"""
#include <cmath>
using std::fabs; using std::sqrt; using std::copysign;
namespace mpm {
%s
}
extern "C" {
void h_svd3(const double* F, double* U, double* V, double* sig) {
    double u[3][3];
    mpm::svd3<double>(F, u, V, sig);
    for (int k = 0; k < 3; ++k) for (int i = 0; i < 3; ++i) U[3 * i + k] = u[k][i];
}
void h_svd3f(const float* F, float* U, float* V, float* sig) {
    float u[3][3];
    mpm::svd3<float>(F, u, V, sig);
    for (int k = 0; k < 3; ++k) for (int i = 0; i < 3; ++i) U[3 * i + k] = u[k][i];
}
void h_polar3(const double* F, double* Rm, double* K, double* sig) { mpm::polar3<double>(F, Rm, K, sig); }
void h_dP(const double* F, double mu, double lam, const double* dF, double* dP) {
    double Rm[9], K[6], s[3];
    mpm::polar3<double>(F, Rm, K, s);
    mpm::fcr_dP<double>(F, Rm, K, mu, lam, dF, dP);
}
double h_psi(const double* F, double mu, double lam) { return mpm::fcr_psi<double>(F, mu, lam); }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    common = open(os.path.join(CSRC, "common.cuh")).read()
    polar = open(os.path.join(CSRC, "polar.cuh")).read()
    helpers = [_template_function(common, n) for n in ("cofactor", "dcofactor", "det3", "matmul3")]
    body = polar[polar.index("namespace mpm {") + len("namespace mpm {"):polar.rindex("}  // namespace mpm")]
    d = tmp_path_factory.mktemp("polar")
    cpp = d / "polar_host.cpp"
    cpp.write_text(SHIM % _host_text("\n\n".join(helpers) + "\n" + body))
    so = str(d / "libpolar_host.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    vp = ctypes.c_void_p
    for f in ("h_svd3", "h_svd3f", "h_polar3"):
        getattr(L, f).argtypes = [vp] * 4
    L.h_dP.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp]
    L.h_psi.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.h_psi.restype = ctypes.c_double
    return L


def _p(a):
    return a.ctypes.data


def svd(L, F, dtype=np.float64):
    F = np.ascontiguousarray(F, dtype)
    U, V, s = np.zeros((3, 3), dtype), np.zeros((3, 3), dtype), np.zeros(3, dtype)
    (L.h_svd3 if dtype == np.float64 else L.h_svd3f)(_p(F), _p(U), _p(V), _p(s))
    return U, V, s


def _rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _cases(rng):
    out = [np.eye(3), np.diag([2.0, 2.0, 2.0]), np.diag([1.5, 1.5, 0.5]), np.diag([2.0, 0.5, 0.5]),
           np.diag([1.0, 1.0, -1.0]), np.diag([2.0, 2.0, -1e-3]), np.diag([1.0, 1e-9, 1e-9]),
           np.outer([1.0, 2.0, 0.5], [0.3, -1.0, 2.0]), np.zeros((3, 3)), -np.eye(3)]
    for sv in ([1.2, 0.9, 0.7], [3.0, 1.0, 1.0], [1.0, 1.0, 1e-4], [2.0, 1.0, -0.3], [1.0, 0.999999, 0.5],
               [5.0, 1e-3, -1e-3], [1.0, 1.0, 1.0]):
        for _ in range(20):
            out.append(_rot(rng) @ np.diag(sv) @ _rot(rng).T)
    for _ in range(200):
        out.append(rng.normal(size=(3, 3)))
    return out


def test_signed_svd_identities(lib):
    rng = np.random.default_rng(1)
    for F in _cases(rng):
        U, V, s = svd(lib, F)
        assert np.all(np.isfinite(U)) and np.all(np.isfinite(V)) and np.all(np.isfinite(s))
        for Q in (U, V):
            assert np.allclose(Q.T @ Q, np.eye(3), atol=1e-12)
            assert np.linalg.det(Q) == pytest.approx(1.0, abs=1e-12)
        scale = max(np.abs(F).max(), 1e-300)
        assert np.allclose(U @ np.diag(s) @ V.T, F, atol=1e-11 * scale)
        # magnitudes descending; the first two non-negative; the last carries det F's sign
        assert s[0] >= s[1] - 1e-12 * scale and s[1] >= abs(s[2]) - 1e-12 * scale and s[1] >= -1e-12 * scale
        ref = np.linalg.svd(F, compute_uv=False)
        assert np.allclose(np.abs(s), ref, atol=1e-10 * scale)
        dF = np.linalg.det(F)
        if abs(dF) > 1e-9 * scale ** 3:
            assert np.sign(s[2]) == np.sign(dF)


def test_float_svd_on_moderate_deformations(lib):
    rng = np.random.default_rng(2)
    for _ in range(300):
        F = _rot(rng) @ np.diag(rng.uniform(0.5, 1.5, 3) * rng.choice([1, 1, 1, -1], 3)) @ _rot(rng).T
        U, V, s = svd(lib, F, np.float32)
        U, V, s = U.astype(float), V.astype(float), s.astype(float)
        assert np.allclose(U.T @ U, np.eye(3), atol=2e-6) and np.allclose(V.T @ V, np.eye(3), atol=2e-6)
        assert np.allclose(U @ np.diag(s) @ V.T, F, atol=5e-6)
        assert np.sign(s[2]) == np.sign(np.linalg.det(F))


def test_polar_rotation_and_rotation_differential(lib):
    """R = U V^T is the rotation of the polar decomposition (R^T F symmetric;
    the unique one with det R = +1 when s2 + s3 > 0), and Kinv inverts
    tr(S) I - S, the operator of the rotation differential."""
    rng = np.random.default_rng(3)
    for F in _cases(rng):
        F = np.ascontiguousarray(F)
        Rm, K, s = np.zeros(9), np.zeros(6), np.zeros(3)
        lib.h_polar3(_p(F), _p(Rm), _p(K), _p(s))
        Rm = Rm.reshape(3, 3)
        scale = max(np.abs(F).max(), 1e-300)
        assert np.allclose(Rm.T @ Rm, np.eye(3), atol=1e-12) and np.linalg.det(Rm) == pytest.approx(1.0, abs=1e-12)
        S = Rm.T @ F
        assert np.allclose(S, S.T, atol=1e-11 * scale)
        if abs(s[1] + s[2]) > 1e-6 * scale:
            Kinv = np.array([[K[0], K[3], K[4]], [K[3], K[1], K[5]], [K[4], K[5], K[2]]])
            assert np.allclose(Kinv @ (np.trace(S) * np.eye(3) - S), np.eye(3), atol=1e-8)


def _P(F, mu, lam):
    U, _, Vt = np.linalg.svd(F)
    if np.linalg.det(U @ Vt) < 0:
        U[:, 2] = -U[:, 2]
    R = U @ Vt
    J = np.linalg.det(F)
    cof = J * np.linalg.inv(F).T
    return 2 * mu * (F - R) + lam * (J - 1) * cof


def test_stress_differential_against_central_differences(lib):
    """fcr_dP is the directional derivative of P = 2 mu (F - R) + lambda (J - 1) cof F,
    including inverted F; fcr_psi is the energy whose derivative P is."""
    rng = np.random.default_rng(4)
    mu, lam = 3.0, 7.0
    for sv in ([1.2, 0.9, 0.7], [1.0, 1.0, 1.0], [1.3, 1.3, 0.8], [1.1, 0.9, -0.4], [2.0, 0.5, 0.25]):
        for _ in range(20):
            F = np.ascontiguousarray(_rot(rng) @ np.diag(sv) @ _rot(rng).T)
            D = np.ascontiguousarray(rng.normal(size=(3, 3)))
            dP = np.zeros(9)
            lib.h_dP(_p(F), mu, lam, _p(D), _p(dP))
            h = 1e-6
            fd = (_P(F + h * D, mu, lam) - _P(F - h * D, mu, lam)) / (2 * h)
            assert np.allclose(dP.reshape(3, 3), fd, atol=1e-6 * max(1.0, np.abs(fd).max()))
            # psi's derivative along D is P : D
            e = lambda G: lib.h_psi(_p(np.ascontiguousarray(G)), mu, lam)  # noqa: E731
            assert (e(F + h * D) - e(F - h * D)) / (2 * h) == pytest.approx(np.sum(_P(F, mu, lam) * D), rel=1e-6,
                                                                            abs=1e-6)


COF_SHIM = r"""
namespace mpm {
%s
}
extern "C" void h_cof(const double* F, double* C) { mpm::cofactor<double>(F, C); }
extern "C" void h_dcof(const double* F, const double* D, double* C) { mpm::dcofactor<double>(F, D, C); }
"""


def test_cofactor_is_quadratic_as_the_line_search_uses_it(tmp_path):
    """The line search forms cof(F + alpha D) a as c0 + alpha c1 + alpha^2 c2 with
    c0 = cof(F) a, c1 = dcof(F)[D] a and c2 = cof(D) a (the cofactor is a quadratic
    form in F), so its surface energy differences need no re-evaluation of cof per
    trial. The device's cofactor and its derivative (csrc/common.cuh), built for
    the host: cof(F) = det(F) F^-T, and the expansion holds for any alpha."""
    common = open(os.path.join(CSRC, "common.cuh")).read()
    cpp = tmp_path / "cof_host.cpp"
    cpp.write_text(COF_SHIM % _host_text("\n\n".join(_template_function(common, n) for n in ("cofactor", "dcofactor"))))
    so = str(tmp_path / "libcof.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_cof.argtypes = [ctypes.c_void_p] * 2
    L.h_dcof.argtypes = [ctypes.c_void_p] * 3
    rng = np.random.default_rng(5)

    def cof(F):
        F = np.ascontiguousarray(F, np.float64)
        C = np.zeros(9)
        L.h_cof(_p(F), _p(C))
        return C.reshape(3, 3)

    def dcof(F, D):
        F, D = np.ascontiguousarray(F, np.float64), np.ascontiguousarray(D, np.float64)
        C = np.zeros(9)
        L.h_dcof(_p(F), _p(D), _p(C))
        return C.reshape(3, 3)

    for _ in range(100):
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        D = rng.standard_normal((3, 3))
        a = rng.standard_normal(3)
        np.testing.assert_allclose(cof(F), np.linalg.det(F) * np.linalg.inv(F).T, atol=1e-12)
        for alpha in (1.0, 0.5, 0.125, 2.0 ** -11):
            lhs = cof(F + alpha * D) @ a
            rhs = cof(F) @ a + alpha * (dcof(F, D) @ a) + alpha * alpha * (cof(D) @ a)
            np.testing.assert_allclose(lhs, rhs, atol=1e-12 * (1 + np.abs(lhs).max()))
