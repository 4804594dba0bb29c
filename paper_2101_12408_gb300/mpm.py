"""ctypes binding of libmpm_gb300.so (include/mpm.h). Argument marshalling only.

Every call goes to the CUDA library; there is no Python or CPU implementation
behind any of these names. If the library is missing, importing this module
raises (build it with ``paper_2101_12408_gb300/build.py``).

Arrays may be numpy arrays (host memory) or torch CUDA tensors (device
memory); the library copies from / to either.
"""
import ctypes
import os

import numpy as np

from . import scenes as _scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpm_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run paper_2101_12408_gb300/build.py (nvcc, sm_103a)")
_lib = ctypes.CDLL(LIB_PATH)

MPM_OK, MPM_ERR_INVALID_ARG, MPM_ERR_CAPACITY, MPM_ERR_CUDA, MPM_ERR_NOT_CONVERGED, MPM_ERR_TIMEOUT, \
    MPM_ERR_NUMERIC, MPM_ERR_DOMAIN = range(8)
PREC_FP64, PREC_FP32_FP64RED = 0, 1
HESS_EXACT, HESS_PROJECTED = 0, 1
ISO_TETRAHEDRA, ISO_CUBES = 0, 1
ISO_METHODS = {"tetra": ISO_TETRAHEDRA, "cubes": ISO_CUBES}
FIELD_MASS, FIELD_MOMENTUM, FIELD_VN, FIELD_THERMAL_MASS, FIELD_TN, FIELD_VHAT, FIELD_THAT, FIELD_ITERATE = range(8)
FIELD_COMPS = {FIELD_MASS: 1, FIELD_MOMENTUM: 3, FIELD_VN: 3, FIELD_THERMAL_MASS: 1, FIELD_TN: 1, FIELD_VHAT: 3,
               FIELD_THAT: 1, FIELD_ITERATE: 3}

EXPORTED = ["mpm_create", "mpm_destroy", "mpm_last_error", "mpm_set_particles", "mpm_get_particles",
            "mpm_set_surface", "mpm_get_surface", "mpm_resample", "mpm_p2g", "mpm_get_grid", "mpm_set_velocity",
            "mpm_energy_gradient", "mpm_apply_hessian", "mpm_heat_apply", "mpm_newton_step", "mpm_g2p", "mpm_step",
            "mpm_sync", "mpm_counts", "mpm_profile_enable", "mpm_get_profile", "mpm_nearest_parent_noalloc",
            "mpm_generate_surface", "mpm_generate_surface_method", "mpm_profile_apply"]


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("dx", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("walls", ctypes.c_int32 * 6), ("plane_n", ctypes.c_double * 3), ("plane_d", ctypes.c_double),
                ("plane_mode", ctypes.c_int32), ("pad_", ctypes.c_int32), ("sphere", ctypes.c_double * 4),
                ("sphere_outside", ctypes.c_int32), ("sphere_mode", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("rho", ctypes.c_double),
                ("lambda_l", ctypes.c_double), ("mu_l", ctypes.c_double), ("E0", ctypes.c_double),
                ("nu", ctypes.c_double), ("T0", ctypes.c_double), ("T_melt", ctypes.c_double),
                ("cp", ctypes.c_double), ("K", ctypes.c_double), ("h", ctypes.c_double), ("H", ctypes.c_double),
                ("gamma_law", ctypes.c_int32), ("thermal", ctypes.c_int32), ("gamma_p", ctypes.c_double * 4),
                ("gamma_lg", ctypes.c_double), ("gamma_sl", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("cg_rtol", ctypes.c_double), ("heat_rtol", ctypes.c_double), ("max_newton", ctypes.c_int32),
                ("max_cg", ctypes.c_int32), ("max_ls", ctypes.c_int32), ("phase_change", ctypes.c_int32),
                ("friction", ctypes.c_double), ("massless_surface", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("grid", GridDesc), ("params", Params), ("max_particles", ctypes.c_int64),
                ("max_surface", ctypes.c_int64), ("max_blocks", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int32), ("cg_iters", ctypes.c_int32), ("heat_iters", ctypes.c_int32),
                ("status", ctypes.c_int32), ("residual0", ctypes.c_double), ("residual", ctypes.c_double),
                ("momentum", ctypes.c_double * 3), ("pad_", ctypes.c_double)]

    def as_dict(self):
        return dict(newton_iters=self.newton_iters, cg_iters=self.cg_iters, heat_iters=self.heat_iters,
                    status=self.status, residual0=self.residual0, residual=self.residual,
                    momentum=list(self.momentum))


class Profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("apply_launches", ctypes.c_int64), ("apply_ms", ctypes.c_double),
                ("heat_apply_launches", ctypes.c_int64), ("heat_apply_ms", ctypes.c_double),
                ("phase_ms", ctypes.c_double * 5), ("newton_iters", ctypes.c_int64), ("cg_iters", ctypes.c_int64),
                ("heat_iters", ctypes.c_int64), ("cg_ctas_per_sm", ctypes.c_int32), ("cg_chunk", ctypes.c_int32),
                ("cg_graphs", ctypes.c_int32), ("cg_graph_error", ctypes.c_int32),
                ("op_rows_per_chunk", ctypes.c_int32), ("reserved_", ctypes.c_int32)]

    def as_dict(self):
        return dict(kernel_launches=self.kernel_launches, apply_launches=self.apply_launches, apply_ms=self.apply_ms,
                    heat_apply_launches=self.heat_apply_launches, heat_apply_ms=self.heat_apply_ms,
                    phase_ms=dict(zip(("resample", "p2g", "heat", "newton", "g2p"), list(self.phase_ms))),
                    newton_iters=self.newton_iters, cg_iters=self.cg_iters, heat_iters=self.heat_iters,
                    cg_ctas_per_sm=self.cg_ctas_per_sm, cg_chunk=self.cg_chunk, cg_graphs=self.cg_graphs,
                    cg_graph_error=self.cg_graph_error, op_rows_per_chunk=self.op_rows_per_chunk)


_vp = ctypes.c_void_p
_lib.mpm_create.argtypes = [ctypes.POINTER(SceneDesc), ctypes.c_int32, ctypes.c_int32, _vp, ctypes.POINTER(_vp)]
_lib.mpm_destroy.argtypes = [_vp]
_lib.mpm_last_error.argtypes = [_vp]
_lib.mpm_last_error.restype = ctypes.c_char_p
_lib.mpm_set_particles.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64] + [_vp] * 10
_lib.mpm_get_particles.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64] + [_vp] * 8
_lib.mpm_set_surface.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64] + [_vp] * 5
_lib.mpm_get_surface.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64] + [_vp] * 6
_lib.mpm_resample.argtypes = [_vp]
_lib.mpm_generate_surface.argtypes = [_vp, ctypes.c_uint64, ctypes.c_double, _vp]
_lib.mpm_generate_surface_method.argtypes = [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_int32, _vp]
_lib.mpm_p2g.argtypes = [_vp]
_lib.mpm_get_grid.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp]
_lib.mpm_set_velocity.argtypes = [_vp, ctypes.c_int32, _vp]
_lib.mpm_energy_gradient.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
_lib.mpm_apply_hessian.argtypes = [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int32]
_lib.mpm_heat_apply.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
_lib.mpm_newton_step.argtypes = [_vp, _vp]
_lib.mpm_g2p.argtypes = [_vp]
_lib.mpm_step.argtypes = [_vp, _vp]
_lib.mpm_sync.argtypes = [_vp]
_lib.mpm_counts.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int64)] * 4
_lib.mpm_profile_enable.argtypes = [_vp, ctypes.c_int32]
_lib.mpm_get_profile.argtypes = [_vp, ctypes.POINTER(Profile)]
_lib.mpm_profile_apply.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
_lib.mpm_nearest_parent_noalloc.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int64, _vp, ctypes.c_int64, _vp, _vp,
                                            _vp]
for _name in EXPORTED:
    if _name != "mpm_last_error":
        getattr(_lib, _name).restype = ctypes.c_int


class MPMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mpm status {status}: {msg}")
        self.status = status


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def scene_desc(sc, max_particles=None, max_surface=None, max_blocks=0):
    p = sc.params
    d = SceneDesc()
    d.grid.n[:] = [int(v) for v in sc.n]
    d.grid.dx = sc.dx
    d.grid.origin[:] = [0.0, 0.0, 0.0]
    d.grid.walls[:] = [int(w) for w in sc.walls]
    d.grid.plane_n[:] = list(sc.plane_n)
    d.grid.plane_d = sc.plane_d
    d.grid.plane_mode = int(sc.plane_mode)
    d.grid.sphere_mode = int(getattr(sc, "sphere_mode", 0))
    if d.grid.sphere_mode:
        d.grid.sphere[:] = [float(v) for v in sc.sphere[:4]]
        d.grid.sphere_outside = int(bool(sc.sphere[4]))
    P = d.params
    P.dt = p.dt
    P.gravity[:] = list(p.gravity)
    P.rho = p.rho
    P.lambda_l = p.lambda_l
    P.mu_l = p.mu_l
    P.E0 = p.E0
    P.nu = p.nu
    P.T0 = p.T0
    P.T_melt = p.T_melt
    P.cp = p.cp
    P.K = p.K
    P.h = p.h
    P.H = p.H
    P.gamma_law = int(p.gamma_law)
    P.thermal = int(bool(p.thermal))
    P.gamma_p[:] = list(p.gamma_p)
    P.gamma_lg = p.gamma_lg
    P.gamma_sl = p.gamma_sl
    P.newton_tol = p.newton_tol
    P.cg_rtol = p.cg_rtol
    P.heat_rtol = p.heat_rtol
    P.max_newton = p.max_newton
    P.max_cg = p.max_cg
    P.max_ls = p.max_ls
    P.phase_change = int(bool(p.phase_change))
    P.friction = float(getattr(p, "friction", 0.0))
    P.massless_surface = int(bool(getattr(p, "massless_surface", False)))
    d.max_particles = int(max_particles if max_particles is not None else sc.n_particles)
    d.max_surface = int(max_surface if max_surface is not None else sc.n_surface)
    d.max_blocks = int(max_blocks)
    return d


class Context:
    """One library context holding one or more scenes."""

    def __init__(self, scene_list, precision=PREC_FP32_FP64RED, stream=None, capacity_factor=1.0, max_blocks=0,
                 surface_capacity_factor=None):
        # generated surfaces (generate_surface) need room beyond the initial samples
        sfac = capacity_factor if surface_capacity_factor is None else surface_capacity_factor
        if isinstance(scene_list, _scenes.Scene):
            scene_list = [scene_list]
        self.scenes = list(scene_list)
        self.precision = precision
        self.rdtype = np.float64 if precision == PREC_FP64 else np.float32
        descs = (SceneDesc * len(self.scenes))()
        for k, sc in enumerate(self.scenes):
            descs[k] = scene_desc(sc, int(sc.n_particles * capacity_factor) + 1, int(sc.n_surface * sfac) + 1,
                                  max_blocks)
        h = _vp()
        st = stream
        if st is None:
            try:
                import torch
                if torch.cuda.is_available():
                    st = torch.cuda.current_stream().cuda_stream
            except Exception:  # noqa: BLE001 - torch is optional for the binding
                st = None
        self._check(_lib.mpm_create(descs, len(self.scenes), precision, st, ctypes.byref(h)), None)
        self.h = h
        self.np = [0] * len(self.scenes)
        self.ns = [0] * len(self.scenes)

    def _check(self, status, h=-1):
        if status != MPM_OK:
            hh = self.h if h == -1 else h
            msg = _lib.mpm_last_error(hh).decode() if hh else ""
            raise MPMError(status, msg)
        return status

    def close(self):
        if getattr(self, "h", None):
            _lib.mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    # ---- state I/O ----
    def set_particles(self, k, x, m, V0, v=None, A=None, J=None, F=None, T=None, gradT=None, phase=None):
        x = _f64(x)
        n = x.shape[0]
        arrs = [x, _f64(v), _f64(A), _f64(m), _f64(V0), _f64(J), _f64(F), _f64(T), _f64(gradT)]
        ph = None if phase is None else np.ascontiguousarray(phase, dtype=np.uint8)
        self._check(_lib.mpm_set_particles(self.h, k, n, *[_ptr(a) for a in arrs], _ptr(ph)))
        self.np[k] = n

    def set_surface(self, k, s, dA, kind=None, b=None, Tbar=None):
        s = _f64(s)
        kd = None if kind is None else np.ascontiguousarray(kind, dtype=np.uint8)
        self._check(_lib.mpm_set_surface(self.h, k, s.shape[0], _ptr(s), _ptr(_f64(dA)), _ptr(kd), _ptr(_f64(b)),
                                         _ptr(_f64(Tbar))))
        self.ns[k] = s.shape[0]

    def load_scene(self, k, sc=None):
        sc = self.scenes[k] if sc is None else sc
        self.set_particles(k, sc.x, sc.m, sc.V0, v=sc.v, A=sc.A, J=sc.J, F=sc.F, T=sc.T, gradT=sc.gradT,
                           phase=sc.phase)
        self.set_surface(k, sc.s, sc.dA, kind=sc.kind, b=sc.b, Tbar=sc.Tbar)

    @staticmethod
    def _outputs(spec, out):
        """Fresh arrays, or the caller's (e.g. in pinned host memory), checked."""
        if out is None:
            return {f: np.zeros(shape, dt) for f, (shape, dt) in spec.items()}
        for f, (shape, dt) in spec.items():
            a = out[f]
            if a.shape != shape or a.dtype != dt or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
                raise ValueError(f"output {f}: need a writeable C-contiguous {np.dtype(dt).name} array {shape}")
        return out

    def get_particles(self, k, out=None):
        n = self.np[k]
        f8 = np.float64
        out = self._outputs(dict(x=((n, 3), f8), v=((n, 3), f8), A=((n, 3, 3), f8), J=((n,), f8), F=((n, 3, 3), f8),
                                 T=((n,), f8), gradT=((n, 3), f8), phase=((n,), np.uint8)), out)
        self._check(_lib.mpm_get_particles(self.h, k, n, *[_ptr(out[f]) for f in
                                                         ("x", "v", "A", "J", "F", "T", "gradT", "phase")]))
        return out

    def get_surface(self, k, out=None):
        n = self.ns[k]
        f8 = np.float64
        out = self._outputs(dict(s=((n, 3), f8), dA=((n, 3), f8), kind=((n,), np.uint8), gamma=((n,), f8),
                                 parent=((n,), np.int32), b=((n, 3), f8)), out)
        self._check(_lib.mpm_get_surface(self.h, k, n, *[_ptr(out[f]) for f in
                                                       ("s", "dA", "kind", "gamma", "parent", "b")]))
        return out

    # ---- phases ----
    def generate_surface(self, seed, per_cell_area=2.0, method="tetra"):
        """Replaces every scene's surface samples with ones generated on the
        particles' union-of-spheres surface, triangulated by marching tetrahedra
        (method "tetra") or marching cubes ("cubes"); returns the per-scene counts."""
        if method not in ISO_METHODS:
            raise ValueError(f"unknown isosurface method {method!r}")
        cnt = np.zeros(len(self.scenes), np.int64)
        seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        if method == "tetra":
            self._check(_lib.mpm_generate_surface(self.h, seed, float(per_cell_area), _ptr(cnt)))
        else:
            self._check(_lib.mpm_generate_surface_method(self.h, seed, float(per_cell_area), ISO_METHODS[method],
                                                         _ptr(cnt)))
        for k in range(len(self.scenes)):
            self.ns[k] = int(cnt[k])
        return cnt

    def resample(self):
        self._check(_lib.mpm_resample(self.h))

    def p2g(self):
        self._check(_lib.mpm_p2g(self.h))

    def newton_step(self, allow_not_converged=True):
        st = (Stats * len(self.scenes))()
        s = _lib.mpm_newton_step(self.h, st)
        if not (s == MPM_OK or (allow_not_converged and s == MPM_ERR_NOT_CONVERGED)):
            self._check(s)
        return [x.as_dict() for x in st]

    def g2p(self):
        self._check(_lib.mpm_g2p(self.h))

    def step(self, allow_not_converged=True):
        st = (Stats * len(self.scenes))()
        s = _lib.mpm_step(self.h, st)
        if not (s == MPM_OK or (allow_not_converged and s == MPM_ERR_NOT_CONVERGED)):
            self._check(s)
        return [x.as_dict() for x in st]

    def sync(self):
        self._check(_lib.mpm_sync(self.h))

    def counts(self):
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(_lib.mpm_counts(self.h, *[ctypes.byref(x) for x in v]))
        return dict(particles=v[0].value, surface=v[1].value, blocks=v[2].value, work_blocks=v[3].value)

    def profile_enable(self, on=True):
        self._check(_lib.mpm_profile_enable(self.h, 1 if on else 0))

    def profile(self):
        p = Profile()
        self._check(_lib.mpm_get_profile(self.h, ctypes.byref(p)))
        return p.as_dict()

    def profile_apply(self, n_applies=200, mode=HESS_PROJECTED):
        """Mean device ms of one Hessian-operator application on the frozen Newton
        state (after newton_step, before g2p)."""
        ms = ctypes.c_double()
        self._check(_lib.mpm_profile_apply(self.h, int(n_applies), int(mode), ctypes.byref(ms)))
        return ms.value

    # ---- grid access / operators ----
    def _nodes(self, k):
        n = self.scenes[k].n
        return int(n[0]) * int(n[1]) * int(n[2])

    def get_grid(self, k, field):
        comps = FIELD_COMPS[field]
        out = np.zeros((self._nodes(k), comps) if comps > 1 else self._nodes(k))
        self._check(_lib.mpm_get_grid(self.h, k, field, _ptr(out)))
        return out

    def set_velocity(self, k, v):
        v = _f64(v).reshape(self._nodes(k), 3)
        self._check(_lib.mpm_set_velocity(self.h, k, _ptr(v)))

    def energy_gradient(self, k):
        g = np.zeros((self._nodes(k), 3))
        e = ctypes.c_double()
        self._check(_lib.mpm_energy_gradient(self.h, k, _ptr(g), ctypes.byref(e)))
        return e.value, g

    def apply_hessian(self, k, dv, mode=HESS_PROJECTED, out=None):
        if hasattr(dv, "data_ptr"):
            if out is None:
                out = dv.new_zeros(dv.shape)
            self._check(_lib.mpm_apply_hessian(self.h, k, _ptr(dv), _ptr(out), mode))
            return out
        dv = np.ascontiguousarray(dv, dtype=self.rdtype).reshape(self._nodes(k), 3)
        out = np.zeros_like(dv)
        self._check(_lib.mpm_apply_hessian(self.h, k, _ptr(dv), _ptr(out), mode))
        return out

    def heat_apply(self, k, T):
        T = np.ascontiguousarray(T, dtype=self.rdtype).reshape(self._nodes(k))
        out = np.zeros_like(T)
        self._check(_lib.mpm_heat_apply(self.h, k, _ptr(T), _ptr(out)))
        return out


def nearest_parent_noalloc(grid, x, s, parent, stream=None):
    """Closest particle of each sample without any allocation (see include/mpm.h).

    grid: a GridDesc (or a Scene); x (N, 3) and s (M, 3) float64 and parent (M,)
    int32 torch tensors, contiguous, on the current CUDA device (the library looks
    up its fixed scratch array for the current device and cannot check where a
    pointer lives). Returns the status code.
    """
    import torch
    dev = torch.cuda.current_device()
    for name, a, dt, shape in (("x", x, torch.float64, (None, 3)), ("s", s, torch.float64, (None, 3)),
                               ("parent", parent, torch.int32, (s.shape[0] if hasattr(s, "shape") else None,))):
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"{name}: need a torch CUDA tensor")
        if a.dtype != dt or a.dim() != len(shape) or any(w is not None and a.shape[i] != w
                                                          for i, w in enumerate(shape)):
            raise ValueError(f"{name}: need a {dt} tensor of shape {shape}, got {a.dtype} {tuple(a.shape)}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if not a.is_cuda or a.device.index != dev:
            raise ValueError(f"{name}: tensor must be on the current CUDA device cuda:{dev}, got {a.device}")
    if isinstance(grid, _scenes.Scene):
        grid = scene_desc(grid).grid
    return _lib.mpm_nearest_parent_noalloc(ctypes.byref(grid), int(x.shape[0]), _ptr(x), int(s.shape[0]), _ptr(s),
                                           _ptr(parent), stream)


def exported_symbols():
    return [n for n in EXPORTED if hasattr(_lib, n)]
