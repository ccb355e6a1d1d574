"""ctypes declarations of include/natconv.h (argument marshalling only)."""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libnatconv.so")

NC_OK = 0
NC_PREC_MIXED = 0
NC_PREC_FP64 = 1
NC_ARITH_DF64 = 0
NC_ARITH_FP64 = 1
NC_BASIS_FP64 = 0
NC_BASIS_FP32 = 1
NC_OBJ_MEAN_T_HEATED = 0
NC_OBJ_SUPG_COMPLIANCE = 1
NC_BC_TOP = 0
NC_BC_CAVITY = 1
NC_REGION_BOX = 0
NC_REGION_CYLINDER = 1
NC_MGOP_EXACT = 0
NC_MGOP_PICARD = 1
NC_SMOOTH_BLOCK_JACOBI = 0
NC_SMOOTH_ZLINE = 1
NC_FILTER_SPECTRAL = 0
NC_FILTER_CHEBYSHEV = 1

STATUS_NAMES = {0: "NC_OK", 1: "NC_ERR_ARG", 2: "NC_ERR_OOM", 3: "NC_ERR_CUDA", 4: "NC_ERR_DIVERGED",
                5: "NC_ERR_MAXIT", 6: "NC_ERR_NAN", 7: "NC_ERR_TIMEOUT", 8: "NC_ERR_STATE"}

# Every exported symbol of include/natconv.h.
EXPORTS = ("nc_default_params", "nc_create_problem", "nc_destroy_problem", "nc_footprint_bytes", "nc_set_params",
           "nc_set_design", "nc_set_state", "nc_solve_state", "nc_objective", "nc_solve_adjoint",
           "nc_sensitivities", "nc_get_fields", "nc_get_adjoint", "nc_get_permeabilities", "nc_get_design_fields", "nc_eval_residual",
           "nc_apply_jacobian", "nc_apply_jacobian_transpose", "nc_apply_picard", "nc_set_profiling", "nc_get_profile",
           "nc_counters", "nc_norm2_free_noalloc", "nc_last_error")

PROF_CLASSES = ("residual", "outer_op64", "outer_op32", "mg_op0", "mg_stencil", "mg_setup_fine", "smooth",
                "krylov_vec", "filter", "sens", "other", "mg_setup_coarse", "coarse_factor", "coarse_solve",
                "mg_stencil_l1", "mg_tail", "adjoint_df64", "mg_op0_picard")


class NatConvError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__("%s: %s" % (self.status_name, message))


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("kappa_f", ctypes.c_double), ("tune_dT", ctypes.c_double),
        ("kappa_ratio", ctypes.c_double), ("k_f", ctypes.c_double), ("k_s", ctypes.c_double),
        ("q_c", ctypes.c_double), ("q_p", ctypes.c_double), ("Q", ctypes.c_double),
        ("heated_layers", ctypes.c_int),
        ("rho0", ctypes.c_double), ("mu", ctypes.c_double), ("cp", ctypes.c_double), ("g", ctypes.c_double),
        ("filter_radius", ctypes.c_double), ("newton_rtol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
        ("krylov_rtol", ctypes.c_double), ("krylov_maxit", ctypes.c_int), ("restart", ctypes.c_int),
        ("precision", ctypes.c_int), ("mg_levels", ctypes.c_int), ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int), ("omega", ctypes.c_double), ("filter_rtol", ctypes.c_double),
        ("timeout_s", ctypes.c_double), ("adjoint_rtol", ctypes.c_double), ("coarse_refactor", ctypes.c_int),
        ("krylov_eta_min", ctypes.c_double), ("adjoint_eta_first", ctypes.c_double),
        ("mg_tail_nodes", ctypes.c_int), ("mg_reuse_below", ctypes.c_double), ("outer_arith", ctypes.c_int),
        ("krylov_basis", ctypes.c_int), ("krylov_reorth", ctypes.c_double), ("adjoint_df64_steps", ctypes.c_int),
        ("bc", ctypes.c_int), ("heat_nx", ctypes.c_int), ("heat_ny", ctypes.c_int), ("design_nx", ctypes.c_int),
        ("design_ny", ctypes.c_int), ("design_nz", ctypes.c_int), ("region_shape", ctypes.c_int),
        ("heat_radius", ctypes.c_double), ("design_radius", ctypes.c_double), ("heat_z0", ctypes.c_int),
        ("mg_op0", ctypes.c_int), ("mg_tail_ctas", ctypes.c_int), ("elem_chunk", ctypes.c_int),
        ("mg_nu_coarse", ctypes.c_int), ("mg_nu_coarse_level", ctypes.c_int),
        ("mg_smoother", ctypes.c_int), ("filter_method", ctypes.c_int), ("mg_galerkin", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [
        ("newton_its", ctypes.c_int), ("krylov_its", ctypes.c_int), ("residual_evals", ctypes.c_int),
        ("ramped", ctypes.c_int), ("rel_residual", ctypes.c_double), ("res_hist", ctypes.c_double * 64),
        ("krylov_hist", ctypes.c_int * 64), ("t_setup_ms", ctypes.c_double), ("t_krylov_ms", ctypes.c_double),
        ("t_total_ms", ctypes.c_double), ("alg_bytes", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
        ("mg_setups", ctypes.c_int),
    ]

    def as_dict(self):
        n = min(self.newton_its, 64)
        return dict(newton_its=self.newton_its, krylov_its=self.krylov_its, residual_evals=self.residual_evals,
                    ramped=bool(self.ramped), rel_residual=self.rel_residual,
                    res_hist=list(self.res_hist[:n]), krylov_hist=list(self.krylov_hist[:n]),
                    t_setup_ms=self.t_setup_ms, t_krylov_ms=self.t_krylov_ms, t_total_ms=self.t_total_ms,
                    alg_bytes=self.alg_bytes, kernel_launches=self.kernel_launches, mg_setups=self.mg_setups)


_lib = None


def load_library(path=None):
    """Load libnatconv.so and declare the C signatures; raises ImportError if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("natconv CUDA library not built (%s missing): run "
                          "`python -m paper_1904_00182_gb300.build` on a machine with nvcc" % p)
    lib = ctypes.CDLL(p)
    vp, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    sig = {
        "nc_default_params": ([ctypes.POINTER(Params)], i),
        "nc_create_problem": ([ctypes.POINTER(Grid), ctypes.POINTER(Params), vp, ctypes.POINTER(vp)], i),
        "nc_destroy_problem": ([vp], i),
        "nc_footprint_bytes": ([ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)], i),
        "nc_set_params": ([vp, ctypes.POINTER(Params)], i),
        "nc_set_design": ([vp, vp], i),
        "nc_set_state": ([vp, vp, vp], i),
        "nc_solve_state": ([vp, ctypes.POINTER(Stats)], i),
        "nc_objective": ([vp, i, dp], i),
        "nc_solve_adjoint": ([vp, i, dp, ctypes.POINTER(Stats)], i),
        "nc_sensitivities": ([vp, vp], i),
        "nc_get_fields": ([vp, vp, vp, vp], i),
        "nc_get_adjoint": ([vp, vp], i),
        "nc_get_permeabilities": ([vp, dp, dp], i),
        "nc_get_design_fields": ([vp, vp, vp, vp], i),
        "nc_eval_residual": ([vp, vp, vp, dp], i),
        "nc_apply_jacobian": ([vp, vp, vp, vp, i], i),
        "nc_apply_jacobian_transpose": ([vp, vp, vp, vp], i),
        "nc_apply_picard": ([vp, vp, vp, vp, i], i),
        "nc_set_profiling": ([vp, i], i),
        "nc_get_profile": ([vp, i, dp, ctypes.POINTER(ctypes.c_longlong), dp, dp], i),
        "nc_counters": ([vp, ctypes.POINTER(ctypes.c_longlong), dp], i),
        "nc_norm2_free_noalloc": ([ctypes.POINTER(Grid), i, vp, vp, vp], i),
        "nc_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def check(status, handle=None):
    if status != NC_OK:
        msg = load_library().nc_last_error(handle)
        raise NatConvError(status, msg.decode() if msg else "")


def default_params(**overrides):
    p = Params()
    check(load_library().nc_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError("unknown parameter %r" % k)
        setattr(p, k, v)
    return p


def footprint_bytes(grid, params):
    out = ctypes.c_size_t()
    check(load_library().nc_footprint_bytes(ctypes.byref(grid), ctypes.byref(params), ctypes.byref(out)))
    return out.value
