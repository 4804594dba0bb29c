"""The per-cell polynomial form of the liquid operator (csrc/newton.cu:
cell_coefficients with the 1-D transforms wT and dT, used by the float64
liquid evaluation and the line-search curvature, and in paired form by the
Hessian operator), built for the host from its source text, against the FP64
oracle's per-particle definition tr L(x_p) = sum_i v_i . gradN_i(x_p) with
quadratic B-splines (section "Transfer: P2G" weights, Eq. fe's J). The 26
coefficients of a cell, evaluated at the particle's in-cell coordinate t, must
give the same trace for any node velocities and any t in the cell."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests.test_polar_host import _host_text, _template_function

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_12408_gb300", "csrc")

SHIM = r"""
namespace mpm {
constexpr int PY = 8, PZ = 52, PN = 312;
inline int pidx(int x, int y, int z) { return x + PY * y + PZ * z; }
%s
}
// trace of dL (without 1/dx) at in-cell coordinates t for the cell (lx, ly, lz) of the halo
extern "C" double h_cell_trace(const double* halo, int lx, int ly, int lz, double tx, double ty, double tz) {
    double ph[3][mpm::PN];
    for (int c = 0; c < 3; ++c) for (int k = 0; k < mpm::PN; ++k) ph[c][k] = halo[c * mpm::PN + k];
    double C[3][3][3] = {};
    mpm::cell_coefficients<double>(ph, lx, ly, lz, C);
    const double px[3] = {1.0, tx, tx * tx}, py[3] = {1.0, ty, ty * ty}, pz[3] = {1.0, tz, tz * tz};
    double tr = 0.0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k)
        tr += C[i][j][k] * px[i] * py[j] * pz[k];
    return tr;
}
extern "C" double h_c222(const double* halo, int lx, int ly, int lz) {
    double ph[3][mpm::PN];
    for (int c = 0; c < 3; ++c) for (int k = 0; k < mpm::PN; ++k) ph[c][k] = halo[c * mpm::PN + k];
    double C[3][3][3] = {};
    mpm::cell_coefficients<double>(ph, lx, ly, lz, C);
    return C[2][2][2];
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    funcs = [_template_function(newton, n) for n in ("wT", "dT", "cell_coefficients")]
    d = tmp_path_factory.mktemp("cellpoly")
    cpp = d / "cell_poly_host.cpp"
    cpp.write_text(SHIM % _host_text("\n\n".join(funcs)))
    so = str(d / "libcellpoly.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_cell_trace.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 3 + [ctypes.c_double] * 3
    L.h_cell_trace.restype = ctypes.c_double
    L.h_c222.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 3
    L.h_c222.restype = ctypes.c_double
    return L


def test_cell_polynomial_equals_the_per_particle_trace(lib):
    rng = np.random.default_rng(21)
    # one 4^3 block and its halo (halo index = node index 0..5), inside a 7^3 grid so
    # that a particle on the block's upper faces still has its stencil on the grid
    # (the extra node layer carries zero weight and gradient there)
    n = (7, 7, 7)
    dx = 1.0 / 7
    for trial in range(60):
        v = np.zeros((7, 7, 7, 3))
        v[:6, :6, :6] = rng.standard_normal((6, 6, 6, 3))
        halo = np.zeros((3, 312))
        for z in range(6):
            for y in range(6):
                for x in range(6):
                    halo[:, x + 8 * y + 52 * z] = v[x, y, z]
        v = v.transpose(2, 1, 0, 3).reshape(-1, 3)           # flat, x fastest
        halo = np.ascontiguousarray(halo)
        lc = rng.integers(0, 4, 3)          # cell (lx, ly, lz) of the block = grid cell lc + 1
        t = rng.uniform(0.0, 1.0, 3)
        if trial < 8:                        # cell faces and corners
            t = rng.integers(0, 2, 3).astype(float)
        xp = (lc + 1 + t) * dx
        st = oracle.Stencil(xp[None], dx, n)
        ref = float(np.einsum("qa,qa->", v[st.node[0]], st.dN[0]))
        got = lib.h_cell_trace(halo.ctypes.data, int(lc[0]), int(lc[1]), int(lc[2]), *t) / dx
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-12 * np.abs(v).max() / dx)
        # the x^2 y^2 z^2 coefficient vanishes: each term of the trace is at most linear along its own axis
        assert lib.h_c222(halo.ctypes.data, int(lc[0]), int(lc[1]), int(lc[2])) == 0.0


SCATTER_SHIM = r"""
namespace mpm {
constexpr int UN = 1;   // the capture below replaces the halo writes
static double g_cap[3][27];
template <typename R>
void rmw_phases(R* uq, const R (&N)[3][3][3], int, int, int, bool = true) {
    const int q = (int)uq[0];   // the stub halo row carries its component index
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
        g_cap[q][a + 3 * b + 9 * c] = N[a][b][c];
}
%s
}
// node values (without 1/dx) that the moment tensor of one particle of weight s
// at in-cell coordinates t scatters to its 27 nodes, per component
extern "C" void h_cell_scatter(double s, double tx, double ty, double tz, double* out) {
    double M[3][3][3] = {};
    const double px[3] = {1.0, tx, tx * tx}, py[3] = {1.0, ty, ty * ty}, pz[3] = {1.0, tz, tz * tz};
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k)
        if (!(i == 2 && j == 2 && k == 2)) M[i][j][k] = s * px[i] * py[j] * pz[k];
    double ua[3][1] = {{0.0}, {1.0}, {2.0}};
    mpm::cell_scatter_warp<double>(M, ua, 0, 0, 0);
    for (int q = 0; q < 3; ++q) for (int k = 0; k < 27; ++k) out[27 * q + k] = mpm::g_cap[q][k];
}
"""


@pytest.fixture(scope="module")
def scatter_lib(tmp_path_factory):
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    funcs = [_template_function(newton, n) for n in ("wN", "dN", "cell_scatter_warp")]
    d = tmp_path_factory.mktemp("cellscatter")
    cpp = d / "cell_scatter_host.cpp"
    cpp.write_text(SCATTER_SHIM % _host_text("\n\n".join(funcs)))
    so = str(d / "libcellscatter.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_cell_scatter.argtypes = [ctypes.c_double] * 4 + [ctypes.c_void_p]
    return L


def test_cell_moments_scatter_to_the_weight_gradients(scatter_lib):
    """The transposed map (cell_scatter_warp with wN and dN): the moments
    sum_p s_p t_p^ijk of a cell scatter to node values sum_p s_p dx gradN_i(x_p),
    the per-particle scatter of the liquid's gradient and Hessian product."""
    rng = np.random.default_rng(22)
    dx = 1.0 / 7
    n = (7, 7, 7)
    for trial in range(40):
        t = rng.uniform(0.0, 1.0, 3) if trial >= 8 else rng.integers(0, 2, 3).astype(float)
        s = rng.uniform(0.5, 2.0)
        out = np.zeros(81)
        scatter_lib.h_cell_scatter(s, *t, out.ctypes.data)
        xp = (np.array([2.0, 2.0, 2.0]) + t) * dx        # cell (2, 2, 2): nodes 1..3 per axis
        st = oracle.Stencil(xp[None], dx, n)
        g = np.stack(np.unravel_index(st.node[0], n, order="F"), -1) - 1   # offsets 0..2 (t = 1: one cell up)
        ref = np.zeros((3, 27))
        for q in range(27):
            a, b, c = g[q]
            if max(a, b, c) <= 2:
                ref[:, a + 3 * b + 9 * c] += s * dx * st.dN[0, q]
            else:                                         # only on a face, where the weight and its gradient vanish
                assert np.all(np.abs(st.dN[0, q]) < 1e-12)
        np.testing.assert_allclose(out.reshape(3, 27), ref, atol=1e-12 * s, rtol=0)


PAIR_SHIM = r"""
#include <cmath>
struct float2 { float x, y; };
struct double2 { double x, y; };
inline float2 make_float2(float a, float b) { return {a, b}; }
inline double2 make_double2(double a, double b) { return {a, b}; }
// the paired instructions, one rounding per element (fma for the fused form)
inline float2 vadd(float2 a, float2 b) { return {a.x + b.x, a.y + b.y}; }
inline float2 vmul(float2 a, float2 b) { return {a.x * b.x, a.y * b.y}; }
inline float2 vfma(float2 a, float2 b, float2 c) { return {std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
inline float2 vsub(float2 a, float2 b) { return {a.x - b.x, a.y - b.y}; }
inline double2 vadd(double2 a, double2 b) { return {a.x + b.x, a.y + b.y}; }
inline double2 vmul(double2 a, double2 b) { return {a.x * b.x, a.y * b.y}; }
inline double2 vfma(double2 a, double2 b, double2 c) { return {std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
inline double2 vsub(double2 a, double2 b) { return {a.x - b.x, a.y - b.y}; }
namespace mpm {
constexpr int PY = 8, PZ = 52, PN = 312;
inline int pidx(int x, int y, int z) { return x + PY * y + PZ * z; }
%s
}
template <typename R>
static void pair(const double* halo, int m, int ly, int lz, double* out) {
    alignas(16) R ph[3][mpm::PN];
    for (int c = 0; c < 3; ++c) for (int k = 0; k < mpm::PN; ++k) ph[c][k] = (R)halo[c * mpm::PN + k];
    typename mpm::VPair<R>::T C[3][3][3];
    mpm::pair_coefficients<R>(ph, m, ly, lz, C);
    for (int i = 0; i < 27; ++i) { out[i] = (&C[0][0][0])[i].x; out[27 + i] = (&C[0][0][0])[i].y; }
}
extern "C" void h_pair(const double* halo, int m, int ly, int lz, double* out) { pair<double>(halo, m, ly, lz, out); }
extern "C" void h_pairf(const double* halo, int m, int ly, int lz, double* out) { pair<float>(halo, m, ly, lz, out); }
extern "C" void h_cell(const double* halo, int lx, int ly, int lz, double* out) {
    double ph[3][mpm::PN];
    for (int c = 0; c < 3; ++c) for (int k = 0; k < mpm::PN; ++k) ph[c][k] = halo[c * mpm::PN + k];
    double C[3][3][3] = {};
    mpm::cell_coefficients<double>(ph, lx, ly, lz, C);
    for (int i = 0; i < 27; ++i) out[i] = (&C[0][0][0])[i];
}
"""


def _vpair_text(src):
    i = src.index("template <typename R> struct VPair;")
    j = src.index("// the scalar transforms (wT, dT, wN, dN) on pairs", i)
    return src[i:j]


@pytest.fixture(scope="module")
def pair_lib(tmp_path_factory):
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    text = _vpair_text(newton) + "\n\n".join(
        _template_function(newton, n) for n in ("wT", "dT", "cell_coefficients"))
    # the paired transforms (templates on the pair type) and the pair helpers,
    # whose signatures span lines
    for name in ("pwT", "pdT", "row_pairs", "pair_coefficients"):
        k = newton.index("__device__ __forceinline__ void " + name + "(")
        k = newton.rindex("template <", 0, k)
        i = newton.index("{", newton.index(")", newton.index(name + "(", k)))
        depth = 0
        for j in range(i, len(newton)):
            depth += newton[j] == "{"
            depth -= newton[j] == "}"
            if depth == 0:
                break
        text += "\n\n" + newton[k:j + 1]
    d = tmp_path_factory.mktemp("pairpoly")
    cpp = d / "pair_poly_host.cpp"
    cpp.write_text(PAIR_SHIM % _host_text(text))
    so = str(d / "libpairpoly.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    for f in ("h_pair", "h_pairf", "h_cell"):
        getattr(L, f).argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    return L


def test_paired_coefficients_equal_the_two_cells(pair_lib):
    """The operator's paired form (pair_coefficients: the cells 2m and 2m+1 of a
    row as one float pair, the middle node pair formed from two aligned pairs)
    gives each cell's own 26 coefficients, in float64 to rounding and in float32
    to float32 rounding."""
    rng = np.random.default_rng(23)
    for trial in range(30):
        halo = np.ascontiguousarray(rng.standard_normal((3, 312)))
        for m in (0, 1):
            ly, lz = int(rng.integers(0, 4)), int(rng.integers(0, 4))
            got = np.zeros(54)
            pair_lib.h_pair(halo.ctypes.data, m, ly, lz, got.ctypes.data)
            gotf = np.zeros(54)
            pair_lib.h_pairf(halo.ctypes.data, m, ly, lz, gotf.ctypes.data)
            for half, lx in ((0, 2 * m), (1, 2 * m + 1)):
                ref = np.zeros(27)
                pair_lib.h_cell(halo.ctypes.data, lx, ly, lz, ref.ctypes.data)
                scale = np.abs(halo).max()
                np.testing.assert_allclose(got[27 * half:27 * half + 27], ref, atol=1e-13 * scale, rtol=0)
                np.testing.assert_allclose(gotf[27 * half:27 * half + 27], ref, atol=2e-6 * scale, rtol=0)


PAIR_SCATTER_SHIM = r"""
#include <cmath>
struct float2 { float x, y; };
struct double2 { double x, y; };
inline float2 make_float2(float a, float b) { return {a, b}; }
inline double2 make_double2(double a, double b) { return {a, b}; }
inline double2 vadd(double2 a, double2 b) { return {a.x + b.x, a.y + b.y}; }
inline double2 vmul(double2 a, double2 b) { return {a.x * b.x, a.y * b.y}; }
inline double2 vfma(double2 a, double2 b, double2 c) { return {std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
inline double2 vsub(double2 a, double2 b) { return {a.x - b.x, a.y - b.y}; }
inline void __syncwarp() {}
namespace mpm {
constexpr int PY = 8, PZ = 52, PN = 312, UN = PZ * 8;
inline int pidx(int x, int y, int z) { return x + PY * y + PZ * z; }
%s
}
// one pair's node values: cells A = (2m, ly, z) and B = (2m+1, ly, z), one particle
// each (weights sA, sB at in-cell coordinates tA, tB), accumulated into a zeroed halo
extern "C" void h_pair_scatter(double sA, const double* tA, double sB, const double* tB, int m, int ly, int zb,
                               double* ua_out) {
    alignas(16) static double ua[3][mpm::UN];
    for (int q = 0; q < 3; ++q) for (int k = 0; k < mpm::UN; ++k) ua[q][k] = 0.0;
    double2 M[3][3][3];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k) {
        const bool skip = i == 2 && j == 2 && k == 2;
        const double a = skip ? 0.0 : sA * std::pow(tA[0], i) * std::pow(tA[1], j) * std::pow(tA[2], k);
        const double b = skip ? 0.0 : sB * std::pow(tB[0], i) * std::pow(tB[1], j) * std::pow(tB[2], k);
        M[i][j][k] = {a, b};
    }
    mpm::pair_scatter<double>(M, ua, m, ly, zb);
    for (int q = 0; q < 3; ++q) for (int k = 0; k < mpm::UN; ++k) ua_out[q * mpm::UN + k] = ua[q][k];
}
"""


def _extract(src, name):
    k = src.index("__device__ __forceinline__ void " + name + "(")
    k = src.rindex("template <", 0, k)
    i = src.index("{", src.index(")", src.index(name + "(", k)))
    depth = 0
    for j in range(i, len(src)):
        depth += src[j] == "{"
        depth -= src[j] == "}"
        if depth == 0:
            return src[k:j + 1]


def test_paired_scatter_sends_both_cells_weight_gradients(tmp_path):
    """The operator's paired output path (pair_scatter: paired transposed
    transforms, the two cells' shared x-nodes summed by pair_rows, then the
    read-add-write phases of pair_rmw3) puts sum_p s_p dx gradN_i(x_p) of both
    cells of the pair on their nodes, and nothing elsewhere."""
    newton = open(os.path.join(CSRC, "newton.cu")).read()
    text = _vpair_text(newton)
    for name in ("pwN", "pdN", "pair_rows", "pair_rmw3", "pair_scatter"):
        text += "\n\n" + _extract(newton, name)
    cpp = tmp_path / "pair_scatter_host.cpp"
    cpp.write_text(PAIR_SCATTER_SHIM % _host_text(text))
    so = str(tmp_path / "libpairscatter.so")
    res = subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", str(cpp), "-o", so],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    L = ctypes.CDLL(so)
    L.h_pair_scatter.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p] + \
        [ctypes.c_int] * 3 + [ctypes.c_void_p]
    rng = np.random.default_rng(24)
    dx = 1.0 / 7
    n = (7, 7, 7)
    UN = 52 * 8
    for trial in range(30):
        m, ly, zb = int(rng.integers(0, 2)), int(rng.integers(0, 4)), int(rng.integers(0, 4))
        tA, tB = np.ascontiguousarray(rng.uniform(0, 1, 3)), np.ascontiguousarray(rng.uniform(0, 1, 3))
        sA, sB = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        out = np.zeros(3 * UN)
        L.h_pair_scatter(sA, tA.ctypes.data, sB, tB.ctypes.data, m, ly, zb, out.ctypes.data)
        out = out.reshape(3, UN)
        ref = np.zeros((3, UN))
        for s, t, x0 in ((sA, tA, 2 * m), (sB, tB, 2 * m + 1)):
            st = oracle.Stencil(((np.array([2.0, 2.0, 2.0]) + t) * dx)[None], dx, n)
            g = np.stack(np.unravel_index(st.node[0], n, order="F"), -1) - 1
            for q in range(27):
                a, b, c = g[q]
                ref[:, (x0 + a) + 8 * (ly + b) + 52 * (zb + c)] += s * dx * st.dN[0, q]
        np.testing.assert_allclose(out, ref, atol=1e-12, rtol=0)
