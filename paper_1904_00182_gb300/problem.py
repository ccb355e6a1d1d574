"""Problem handle: one ctypes call per C entry point (argument marshalling only)."""

import ctypes

import numpy as np

from . import _abi
from ._abi import NC_OBJ_MEAN_T_HEATED, NC_PREC_FP64, NC_PREC_MIXED, Grid, Stats, check, default_params

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the supported environment
    torch = None


def _ptr(x):
    """Address of a contiguous float64 torch tensor (host or CUDA) or NumPy array."""
    if x is None:
        return None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("expected a torch.Tensor or numpy.ndarray, got %r" % type(x))


def _as_f64(x, like_device=None):
    if torch is not None and isinstance(x, torch.Tensor):
        return x.detach().to(dtype=torch.float64).contiguous()
    return np.ascontiguousarray(x, dtype=np.float64)


class Problem:
    """A state / adjoint problem on an nx x ny x nz grid of cubic Q1 elements.

    h defaults to 1/nz (unit height). Parameters are the fields of nc_params (see
    include/natconv.h); pass ``params`` or keyword overrides of the defaults. Outputs are float64
    CUDA tensors on ``device``.
    """

    def __init__(self, nx, ny, nz, h=None, params=None, stream=None, device="cuda", **overrides):
        self.lib = _abi.load_library()
        self.grid = Grid(int(nx), int(ny), int(nz), float(h if h is not None else 1.0 / nz))
        self.params = params if params is not None else default_params(**overrides)
        if params is not None:
            for k, v in overrides.items():
                setattr(self.params, k, v)
        self.device = device
        self.nn = (nx + 1) * (ny + 1) * (nz + 1)
        self.ne = nx * ny * nz
        handle = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream is not None else None
        dev_ctx = torch.cuda.device(torch.device(device)) if torch is not None else None
        if dev_ctx is not None:
            with dev_ctx:
                status = self.lib.nc_create_problem(ctypes.byref(self.grid), ctypes.byref(self.params), st,
                                                    ctypes.byref(handle))
        else:
            status = self.lib.nc_create_problem(ctypes.byref(self.grid), ctypes.byref(self.params), st,
                                                ctypes.byref(handle))
        check(status, None)
        self.h = handle

    # -- lifetime ---------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.nc_destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, status):
        check(status, self.h)

    def _empty(self, n):
        return torch.empty(n, dtype=torch.float64, device=self.device)

    def set_params(self, **overrides):
        """Change parameters in place (not precision, mg_levels or restart); needs a new design."""
        p = _abi.Params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(self.params), ctypes.sizeof(p))
        for k, v in overrides.items():
            if not hasattr(p, k):
                raise KeyError("unknown parameter %r" % k)
            setattr(p, k, v)
        self._check(self.lib.nc_set_params(self.h, ctypes.byref(p)))
        self.params = p

    # -- the path -----------------------------------------------------------------------------
    def set_design(self, rho):
        rho = _as_f64(rho)
        if rho.shape[0] != self.ne:
            raise ValueError("design must have %d entries" % self.ne)
        self._check(self.lib.nc_set_design(self.h, _ptr(rho)))

    def set_state(self, P, T):
        P, T = _as_f64(P), _as_f64(T)
        self._check(self.lib.nc_set_state(self.h, _ptr(P), _ptr(T)))

    def solve_state(self):
        st = Stats()
        self._check(self.lib.nc_solve_state(self.h, ctypes.byref(st)))
        return st.as_dict()

    def objective(self, objective=NC_OBJ_MEAN_T_HEATED):
        f = ctypes.c_double()
        self._check(self.lib.nc_objective(self.h, objective, ctypes.byref(f)))
        return f.value

    def solve_adjoint(self, objective=NC_OBJ_MEAN_T_HEATED):
        f = ctypes.c_double()
        st = Stats()
        self._check(self.lib.nc_solve_adjoint(self.h, objective, ctypes.byref(f), ctypes.byref(st)))
        return f.value, st.as_dict()

    def sensitivities(self, out=None):
        out = self._empty(self.ne) if out is None else out
        self._check(self.lib.nc_sensitivities(self.h, _ptr(out)))
        return out

    def get_fields(self, velocity=True):
        P, T = self._empty(self.nn), self._empty(self.nn)
        u = self._empty(3 * self.ne) if velocity else None
        self._check(self.lib.nc_get_fields(self.h, _ptr(P), _ptr(T), _ptr(u)))
        return P, T, (u.view(self.ne, 3) if velocity else None)

    def adjoint(self):
        """The adjoint solution lambda (2N, node-interleaved)."""
        lam = self._empty(2 * self.nn)
        self._check(self.lib.nc_get_adjoint(self.h, _ptr(lam)))
        return lam

    def permeabilities(self):
        """(kappa_f, kappa_s) as resolved by the library."""
        kf, ks = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.nc_get_permeabilities(self.h, ctypes.byref(kf), ctypes.byref(ks)))
        return kf.value, ks.value

    def design_fields(self):
        gt, kap, k = self._empty(self.ne), self._empty(self.ne), self._empty(self.ne)
        self._check(self.lib.nc_get_design_fields(self.h, _ptr(gt), _ptr(kap), _ptr(k)))
        return gt, kap, k

    # -- measurement ---------------------------------------------------------------------------
    def set_profiling(self, on=True, classes=None):
        """Time every kernel class (on=True), none (False), or only the named classes."""
        if classes is not None:
            mask = 0
            for c in classes:
                mask |= 1 << _abi.PROF_CLASSES.index(c)
        else:
            mask = -1 if on else 0
        self._check(self.lib.nc_set_profiling(self.h, mask))

    def profile(self):
        """{class: (ms, launches, algorithmic bytes, algorithmic flops)} since set_profiling(True)."""
        out = {}
        for cls, name in enumerate(_abi.PROF_CLASSES):
            ms, n, b, f = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.nc_get_profile(self.h, cls, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                                ctypes.byref(f)))
            out[name] = (ms.value, n.value, b.value, f.value)
        return out

    def counters(self):
        n, b = ctypes.c_longlong(), ctypes.c_double()
        self._check(self.lib.nc_counters(self.h, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value

    # -- operator-level entry points -----------------------------------------------------------
    def eval_residual(self, s):
        s = _as_f64(s)
        out = self._empty(2 * self.nn)
        n2 = ctypes.c_double()
        self._check(self.lib.nc_eval_residual(self.h, _ptr(s), _ptr(out), ctypes.byref(n2)))
        return out, n2.value

    def apply_jacobian(self, s, v, precision=NC_PREC_FP64):
        s, v = _as_f64(s), _as_f64(v)
        out = self._empty(2 * self.nn)
        self._check(self.lib.nc_apply_jacobian(self.h, _ptr(s), _ptr(v), _ptr(out), precision))
        return out

    def apply_picard(self, s, v, transpose=False):
        """The frozen-coefficient finest-level multigrid operator (FP32) at s applied to v (or its transpose)."""
        s, v = _as_f64(s), _as_f64(v)
        out = self._empty(2 * self.nn)
        self._check(self.lib.nc_apply_picard(self.h, _ptr(s), _ptr(v), _ptr(out), 1 if transpose else 0))
        return out

    def apply_jacobian_transpose(self, s, w):
        s, w = _as_f64(s), _as_f64(w)
        out = self._empty(2 * self.nn)
        self._check(self.lib.nc_apply_jacobian_transpose(self.h, _ptr(s), _ptr(w), _ptr(out)))
        return out
