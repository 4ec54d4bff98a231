"""ctypes binding of libdjtled.so (C ABI in include/dj_tled.h).

Argument marshalling only: every step of the DJ-TLED path runs in the CUDA
library.  Functions carry the C names; ``Mesh`` wraps a handle for convenience.
If the library has not been built the import of this module still works, but
any call raises ``RuntimeError`` (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdjtled.so")

DJ_OK = 0
STATUS = {0: "DJ_OK", 1: "DJ_ERR_INVALID_ARG", 2: "DJ_ERR_BAD_MESH", 3: "DJ_ERR_INVERTED_ELEMENT",
          4: "DJ_ERR_NOT_PRECOMPUTED", 5: "DJ_ERR_NONFINITE", 6: "DJ_ERR_NOT_CONVERGED",
          7: "DJ_ERR_CUDA", 8: "DJ_ERR_OOM", 9: "DJ_ERR_UNSUPPORTED"}
(DJ_ERR_INVALID_ARG, DJ_ERR_BAD_MESH, DJ_ERR_INVERTED_ELEMENT, DJ_ERR_NOT_PRECOMPUTED, DJ_ERR_NONFINITE,
 DJ_ERR_NOT_CONVERGED, DJ_ERR_CUDA, DJ_ERR_OOM, DJ_ERR_UNSUPPORTED) = range(1, 10)
DJ_TET4, DJ_HEX8 = 4, 8
DJ_NH, DJ_TI, DJ_OT, DJ_MR = 0, 1, 2, 3

# every exported entry point of include/dj_tled.h
EXPORTS = [
    "dj_params_default", "dj_mesh_create", "dj_mesh_set_materials", "dj_mesh_set_bcs",
    "dj_mesh_update_bc_targets", "dj_mesh_set_loads", "dj_precompute", "dj_step", "dj_run_n",
    "dj_run_n_profiled", "dj_sync", "dj_relax_to_tol", "dj_relax_adaptive", "dj_set_displacements",
    "dj_get_displacements", "dj_get_displacements_device", "dj_internal_forces",
    "dj_state_size", "dj_get_state", "dj_set_state", "dj_get_info", "dj_status_string",
    "dj_last_error", "dj_mesh_destroy", "dj_mesh_set_groups", "dj_get_group_info",
    "dj_batch_create", "dj_batch_precompute", "dj_batch_run_n", "dj_batch_sync",
    "dj_batch_relax_to_tol", "dj_batch_instance_info", "dj_batch_get_displacements",
    "dj_batch_set_displacements", "dj_batch_get_info", "dj_batch_last_error", "dj_batch_destroy",
    "dj_set_displacements_device", "dj_evaluate_field", "dj_batch_get_displacements_device",
    "dj_mlp_create", "dj_mlp_num_params", "dj_mlp_get_params", "dj_mlp_set_params",
    "dj_mlp_get_grads", "dj_mlp_forward", "dj_mlp_loss_grad", "dj_mlp_adam_step",
    "dj_mlp_last_error", "dj_mlp_destroy", "dj_pod_fit", "dj_pod_project", "dj_pod_expand",
    "dj_residual_norms_static", "dj_set_step", "dj_batch_set_step", "dj_autotune",
    "dj_batch_autotune", "dj_linear_fit", "dj_linear_apply", "dj_profile_kernels",
    "dj_autotune_cold", "dj_quad_features", "dj_symmetric_eigen", "dj_mlp_set_precision",
    "dj_ws_params_default", "dj_ws_train", "dj_ws_fit", "dj_ws_predict", "dj_ws_relax_to_tol",
    "dj_ws_save", "dj_ws_load", "dj_ws_get_info", "dj_ws_last_error", "dj_ws_destroy", "dj_step_host",
]

DJ_WS_MLP_ON_COEFFS, DJ_WS_MLP_ON_FEATURES = 0, 1
DJ_WS_PARTS_FITTED, DJ_WS_PARTS_POLYNOMIAL, DJ_WS_PARTS_MLP = 0, 1, 2
DJ_WS_ARM_REST, DJ_WS_ARM_POLYNOMIAL, DJ_WS_ARM_FITTED = 0, 1, 2


class dj_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("dt_scale", C.c_double), ("alpha", C.c_double),
                ("hg_coeff", C.c_double), ("ramp_steps", C.c_longlong), ("ramp_kind", C.c_int),
                ("relax_check_every", C.c_int), ("renumber", C.c_int), ("assembly", C.c_int),
                ("tile_size", C.c_int), ("precision", C.c_int), ("anp", C.c_int), ("graph_pdl", C.c_int),
                ("max_blocks", C.c_int)]


class dj_adr_params(C.Structure):
    """Options of dj_relax_adaptive (include/dj_tled.h)."""
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double), ("disp_tol", C.c_double)]


class dj_adr_report(C.Structure):
    """Estimates of the last check of dj_relax_adaptive (include/dj_tled.h)."""
    _fields_ = [("alpha", C.c_double), ("lambda_", C.c_double), ("rho", C.c_double),
                ("err_est", C.c_double), ("n_estimates", C.c_longlong)]


class dj_info(C.Structure):
    _fields_ = [("n_nodes", C.c_longlong), ("n_elems", C.c_longlong), ("n_bc_dofs", C.c_longlong),
                ("step", C.c_longlong), ("elem_type", C.c_int), ("model_flags", C.c_int),
                ("dt", C.c_double), ("dt_crit", C.c_double), ("total_mass", C.c_double),
                ("device_bytes", C.c_longlong), ("elem_table_bytes_per_elem", C.c_longlong),
                ("slot_bytes_per_elem", C.c_longlong), ("gather_index_bytes", C.c_longlong),
                ("node_bytes_per_node", C.c_longlong), ("n_parts", C.c_longlong),
                ("assembly", C.c_int), ("tile_size", C.c_int), ("n_consts", C.c_int),
                ("precision", C.c_int), ("grid", C.c_int), ("n_tiles", C.c_longlong)]


class dj_ws_params(C.Structure):
    """Options of the learned warm start (include/dj_tled.h)."""
    _fields_ = [("n_in", C.c_int), ("n_out", C.c_int), ("hidden", C.c_int * 4), ("epochs", C.c_int),
                ("batch", C.c_int), ("lr", C.c_double), ("lr_final", C.c_double), ("quadratic", C.c_int),
                ("mlp", C.c_int), ("mlp_input", C.c_int), ("mlp_bf16", C.c_int), ("holdout", C.c_double),
                ("seed", C.c_ulonglong), ("adaptive", C.c_int), ("bootstrap", C.c_int)]


class dj_ws_info(C.Structure):
    _fields_ = [("n_loads", C.c_int), ("n_kept", C.c_int), ("n_train", C.c_int), ("n_holdout", C.c_int),
                ("n_in", C.c_int), ("n_out", C.c_int), ("n_in_kept", C.c_int), ("n_out_kept", C.c_int),
                ("n_features", C.c_int), ("n_bc", C.c_int), ("n_dof", C.c_longlong),
                ("quadratic_used", C.c_int), ("mlp_used", C.c_int), ("mlp_params", C.c_longlong),
                ("mlp_iterations", C.c_longlong), ("val_loss_first_order", C.c_double),
                ("val_loss_second_order", C.c_double), ("val_loss_polynomial", C.c_double),
                ("val_loss_polynomial_mlp", C.c_double), ("final_train_loss", C.c_double),
                ("mean_training_steps", C.c_double), ("data_seconds", C.c_double),
                ("fit_seconds", C.c_double), ("fit_seconds_polynomial", C.c_double)]


class dj_ws_result(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("steps_warm_attempt", C.c_longlong), ("residual", C.c_double),
                ("started_warm", C.c_int), ("fallback", C.c_int), ("residual_predicted", C.c_double),
                ("residual_prescribed_only", C.c_double), ("predict_seconds", C.c_double),
                ("seconds", C.c_double)]


def _struct_dict(st):
    out = {}
    for f, _ in st._fields_:
        v = getattr(st, f)
        out[f] = list(v) if hasattr(v, "__len__") else v
    return out


class DJError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_LL = C.POINTER(C.c_longlong)


def lib():
    """Load libdjtled.so; raises RuntimeError if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} not built: run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    sig = {
        "dj_params_default": (None, [C.POINTER(dj_params)]),
        "dj_mesh_create": (C.c_int, [C.c_int, _D, C.c_longlong, C.POINTER(C.c_int), C.c_longlong,
                                     C.POINTER(_P)]),
        "dj_mesh_set_materials": (C.c_int, [_P, C.POINTER(C.c_ubyte), _D, _D, _D, _D, _D, _D, _D, _D]),
        "dj_mesh_set_bcs": (C.c_int, [_P, _LL, _D, C.c_longlong]),
        "dj_mesh_update_bc_targets": (C.c_int, [_P, _D]),
        "dj_mesh_set_loads": (C.c_int, [_P, _D]),
        "dj_precompute": (C.c_int, [_P, C.POINTER(dj_params), _D]),
        "dj_step": (C.c_int, [_P, _P]),
        "dj_run_n": (C.c_int, [_P, C.c_longlong, _P]),
        "dj_run_n_profiled": (C.c_int, [_P, C.c_longlong, _P, _D, _D]),
        "dj_sync": (C.c_int, [_P, _P]),
        "dj_relax_to_tol": (C.c_int, [_P, C.c_double, C.c_longlong, _LL, _D, _P]),
        "dj_relax_adaptive": (C.c_int, [_P, C.c_double, C.c_longlong, C.POINTER(dj_adr_params), _LL, _D,
                                        C.POINTER(dj_adr_report), _P]),
        "dj_set_displacements": (C.c_int, [_P, _D]),
        "dj_get_displacements": (C.c_int, [_P, _D]),
        "dj_get_displacements_device": (C.c_int, [_P, _P, _P]),
        "dj_internal_forces": (C.c_int, [_P, _D, _D]),
        "dj_state_size": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
        "dj_get_state": (C.c_int, [_P, _P, C.c_size_t]),
        "dj_set_state": (C.c_int, [_P, _P, C.c_size_t]),
        "dj_get_info": (C.c_int, [_P, C.POINTER(dj_info)]),
        "dj_status_string": (C.c_char_p, [C.c_int]),
        "dj_last_error": (C.c_char_p, [_P]),
        "dj_mesh_destroy": (None, [_P]),
        "dj_mesh_set_groups": (C.c_int, [_P, C.POINTER(C.c_int), C.c_int]),
        "dj_get_group_info": (C.c_int, [_P, C.POINTER(C.c_int), _D, _D, _D]),
        "dj_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P)]),
        "dj_batch_precompute": (C.c_int, [_P, C.POINTER(dj_params)]),
        "dj_batch_run_n": (C.c_int, [_P, C.c_longlong, _P]),
        "dj_batch_sync": (C.c_int, [_P, _P]),
        "dj_batch_relax_to_tol": (C.c_int, [_P, C.c_double, C.c_longlong, _LL, _D, _P]),
        "dj_batch_instance_info": (C.c_int, [_P, C.c_int, _LL, _LL, _D, _D]),
        "dj_batch_get_displacements": (C.c_int, [_P, C.c_int, _D]),
        "dj_batch_set_displacements": (C.c_int, [_P, C.c_int, _D]),
        "dj_batch_get_info": (C.c_int, [_P, C.POINTER(C.c_int), _LL, _LL, _LL, _LL]),
        "dj_batch_last_error": (C.c_char_p, [_P]),
        "dj_batch_destroy": (None, [_P]),
        "dj_set_displacements_device": (C.c_int, [_P, _P, _P]),
        "dj_evaluate_field": (C.c_int, [_P, _P, _D, C.POINTER(C.c_int), _P]),
        "dj_batch_get_displacements_device": (C.c_int, [_P, C.c_int, _P, _P]),
        "dj_mlp_create": (C.c_int, [C.POINTER(C.c_int), C.c_int, C.c_ulonglong, C.POINTER(_P)]),
        "dj_mlp_num_params": (C.c_longlong, [_P]),
        "dj_mlp_get_params": (C.c_int, [_P, C.POINTER(C.c_float), C.c_longlong]),
        "dj_mlp_set_params": (C.c_int, [_P, C.POINTER(C.c_float), C.c_longlong]),
        "dj_mlp_get_grads": (C.c_int, [_P, C.POINTER(C.c_float), C.c_longlong]),
        "dj_mlp_forward": (C.c_int, [_P, _P, C.c_int, _P, _P]),
        "dj_mlp_loss_grad": (C.c_int, [_P, _P, _P, _P, C.c_int, _D, _P]),
        "dj_mlp_adam_step": (C.c_int, [_P, C.c_float, C.c_float, C.c_float, C.c_float, _P]),
        "dj_mlp_last_error": (C.c_char_p, [_P]),
        "dj_mlp_destroy": (None, [_P]),
        "dj_pod_fit": (C.c_int, [_P, C.c_longlong, C.c_int, C.c_int, _P, _P, _D, _P]),
        "dj_pod_project": (C.c_int, [_P, _P, C.c_longlong, C.c_int, _P, C.c_int, _P, _P]),
        "dj_linear_fit": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_double, _P, _P]),
        "dj_profile_kernels": (C.c_int, [_P, C.c_int, _P, C.c_size_t, _P, _D, _D]),
        "dj_autotune_cold": (C.c_int, [_P, C.c_int, _P, C.c_size_t, _P, C.POINTER(dj_params), _D]),
        "dj_quad_features": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
        "dj_linear_apply": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, C.c_float, C.c_float, _P, _P]),
        "dj_pod_expand": (C.c_int, [_P, _P, C.c_longlong, C.c_int, _P, C.c_int, _P, _P]),
        "dj_residual_norms_static": (C.c_int, [_P, _P, C.c_longlong, _P, _P]),
        "dj_set_step": (C.c_int, [_P, C.c_longlong]),
        "dj_batch_set_step": (C.c_int, [_P, C.c_longlong]),
        "dj_autotune": (C.c_int, [_P, C.c_int, _P, C.POINTER(dj_params), _D]),
        "dj_batch_autotune": (C.c_int, [_P, C.c_int, _P]),
        "dj_symmetric_eigen": (C.c_int, [_D, C.c_int, _D, _D]),
        "dj_mlp_set_precision": (C.c_int, [_P, C.c_int]),
        "dj_step_host": (C.c_int, [_P, _P, _P, C.c_int, _P]),
        "dj_ws_params_default": (None, [C.POINTER(dj_ws_params)]),
        "dj_ws_train": (C.c_int, [_P, _D, C.c_int, C.c_double, C.c_longlong, C.POINTER(dj_ws_params),
                                  C.POINTER(_P), _P]),
        "dj_ws_fit": (C.c_int, [_LL, C.c_int, C.c_longlong, _P, _P, C.c_int, C.POINTER(dj_ws_params),
                                C.POINTER(_P), _P]),
        "dj_ws_predict": (C.c_int, [_P, _D, C.c_int, _P, _P]),
        "dj_ws_relax_to_tol": (C.c_int, [_P, _P, _D, C.c_int, C.c_double, C.c_longlong,
                                         C.POINTER(dj_ws_result), _P]),
        "dj_ws_save": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
        "dj_ws_load": (C.c_int, [_P, C.c_size_t, C.POINTER(_P)]),
        "dj_ws_get_info": (C.c_int, [_P, C.POINTER(dj_ws_info)]),
        "dj_ws_last_error": (C.c_char_p, [_P]),
        "dj_ws_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _dptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


def _check(st: int, where: str, handle=None):
    if st != DJ_OK:
        detail = ""
        if handle:
            msg = lib().dj_last_error(handle)
            detail = msg.decode() if msg else ""
        raise DJError(st, where, detail)


def default_params(**kw) -> dj_params:
    p = dj_params()
    lib().dj_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


# ----------------------------------------------------------------- C names --
def dj_mesh_create(elem_type: int, X, conn):
    X = _f64(X)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    h = _P()
    n_nodes = X.shape[0] if X.ndim == 2 else X.size // 3
    n_elems = conn.shape[0] if conn.ndim == 2 else conn.size // max(int(elem_type), 1)
    st = lib().dj_mesh_create(int(elem_type), _dptr(X), n_nodes,
                              conn.ctypes.data_as(C.POINTER(C.c_int)), n_elems, C.byref(h))
    _check(st, "dj_mesh_create")
    return h


def dj_mesh_set_materials(h, model, mu, kappa, rho, eta_a=None, eta_b=None, c01=None, a_dir=None,
                          b_dir=None):
    model = np.ascontiguousarray(model, dtype=np.uint8)
    arrs = [_f64(x) for x in (mu, kappa, rho, eta_a, eta_b, c01, a_dir, b_dir)]
    st = lib().dj_mesh_set_materials(h, model.ctypes.data_as(C.POINTER(C.c_ubyte)),
                                     *[_dptr(a) for a in arrs])
    _check(st, "dj_mesh_set_materials", h)


def dj_mesh_set_bcs(h, dof, target):
    dof = np.ascontiguousarray(dof, dtype=np.int64)
    target = _f64(target)
    st = lib().dj_mesh_set_bcs(h, dof.ctypes.data_as(_LL), _dptr(target), dof.size)
    _check(st, "dj_mesh_set_bcs", h)


def dj_mesh_update_bc_targets(h, target):
    target = _f64(target)
    _check(lib().dj_mesh_update_bc_targets(h, _dptr(target)), "dj_mesh_update_bc_targets", h)


def dj_mesh_set_loads(h, R):
    R = _f64(R)
    _check(lib().dj_mesh_set_loads(h, _dptr(R)), "dj_mesh_set_loads", h)


def dj_precompute(h, params: Optional[dj_params] = None) -> float:
    dt = C.c_double(0.0)
    st = lib().dj_precompute(h, C.byref(params) if params is not None else None, C.byref(dt))
    _check(st, "dj_precompute", h)
    return dt.value


def dj_step(h, stream=None):
    _check(lib().dj_step(h, _stream(stream)), "dj_step", h)


def dj_run_n(h, n: int, stream=None):
    _check(lib().dj_run_n(h, int(n), _stream(stream)), "dj_run_n", h)


def dj_run_n_profiled(h, n: int, stream=None):
    a, b = C.c_double(0), C.c_double(0)
    _check(lib().dj_run_n_profiled(h, int(n), _stream(stream), C.byref(a), C.byref(b)),
           "dj_run_n_profiled", h)
    return a.value, b.value


def dj_sync(h, stream=None):
    _check(lib().dj_sync(h, _stream(stream)), "dj_sync", h)


def dj_relax_to_tol(h, tol: float, max_steps: int, stream=None, raise_on_fail=True):
    steps, r = C.c_longlong(0), C.c_double(0)
    st = lib().dj_relax_to_tol(h, float(tol), int(max_steps), C.byref(steps), C.byref(r),
                               _stream(stream))
    if raise_on_fail:
        _check(st, "dj_relax_to_tol", h)
    return st, steps.value, r.value


def dj_relax_adaptive(h, tol: float, max_steps: int, alpha_min=0.0, alpha_max=0.0, disp_tol=0.0,
                      stream=None, raise_on_fail=True):
    """Adaptive dynamic relaxation; returns (status, steps, residual, report dict)."""
    o = dj_adr_params(float(alpha_min), float(alpha_max), float(disp_tol))
    rep = dj_adr_report()
    steps, r = C.c_longlong(0), C.c_double(0)
    st = lib().dj_relax_adaptive(h, float(tol), int(max_steps), C.byref(o), C.byref(steps), C.byref(r),
                                 C.byref(rep), _stream(stream))
    if raise_on_fail:
        _check(st, "dj_relax_adaptive", h)
    report = {f.rstrip("_"): getattr(rep, f) for f, _ in dj_adr_report._fields_}
    return st, steps.value, r.value, report


def dj_set_displacements(h, U0):
    U0 = _f64(U0)
    _check(lib().dj_set_displacements(h, _dptr(U0)), "dj_set_displacements", h)


def dj_get_displacements(h, n_nodes: int, out=None) -> np.ndarray:
    """U in caller order (n_nodes x 3 doubles); `out` may be a caller-owned
    C-contiguous float64 array (e.g. a view of pinned host memory)."""
    if out is None:
        out = np.empty((n_nodes, 3), dtype=np.float64)
    elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size != 3 * n_nodes:
        raise ValueError("out must be a C-contiguous float64 array of n_nodes x 3")
    _check(lib().dj_get_displacements(h, _dptr(out)), "dj_get_displacements", h)
    return out


def dj_get_displacements_device(h, d_ptr: int, stream=None):
    _check(lib().dj_get_displacements_device(h, d_ptr, _stream(stream)),
           "dj_get_displacements_device", h)


def dj_internal_forces(h, U) -> np.ndarray:
    U = _f64(U)
    out = np.empty(U.shape, dtype=np.float64)
    _check(lib().dj_internal_forces(h, _dptr(U), _dptr(out)), "dj_internal_forces", h)
    return out


def dj_state_size(h) -> int:
    n = C.c_size_t(0)
    _check(lib().dj_state_size(h, C.byref(n)), "dj_state_size", h)
    return n.value


def dj_get_state(h) -> bytes:
    n = dj_state_size(h)
    buf = C.create_string_buffer(n)
    _check(lib().dj_get_state(h, C.cast(buf, _P), n), "dj_get_state", h)
    return buf.raw


def dj_set_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().dj_set_state(h, C.cast(buf, _P), len(blob)), "dj_set_state", h)


def dj_get_info(h) -> dj_info:
    info = dj_info()
    _check(lib().dj_get_info(h, C.byref(info)), "dj_get_info", h)
    return info


def dj_status_string(s: int) -> str:
    return lib().dj_status_string(int(s)).decode()


def dj_last_error(h) -> str:
    r = lib().dj_last_error(h)
    return r.decode() if r else ""


def dj_mesh_destroy(h):
    lib().dj_mesh_destroy(h)


def dj_mesh_set_groups(h, elem_group, n_groups):
    g = np.ascontiguousarray(elem_group, dtype=np.int32)
    _check(lib().dj_mesh_set_groups(h, g.ctypes.data_as(C.POINTER(C.c_int)), int(n_groups)),
           "dj_mesh_set_groups", h)


def dj_get_group_info(h):
    n = C.c_int(0)
    _check(lib().dj_get_group_info(h, C.byref(n), None, None, None), "dj_get_group_info", h)
    dt, dtc, r = (np.empty(n.value) for _ in range(3))
    _check(lib().dj_get_group_info(h, C.byref(n), _dptr(dt), _dptr(dtc), _dptr(r)),
           "dj_get_group_info", h)
    return dt, dtc, r


def _bcheck(st, where, b):
    if st != DJ_OK:
        msg = lib().dj_batch_last_error(b) if b else b""
        raise DJError(st, where, msg.decode() if msg else "")


def dj_batch_create(handles):
    arr = (_P * len(handles))(*[h.value if isinstance(h, _P) else h for h in handles])
    b = _P()
    _bcheck(lib().dj_batch_create(arr, len(handles), C.byref(b)), "dj_batch_create", None)
    return b


def dj_batch_precompute(b, params=None):
    _bcheck(lib().dj_batch_precompute(b, C.byref(params) if params is not None else None),
            "dj_batch_precompute", b)


def dj_batch_run_n(b, n, stream=None):
    _bcheck(lib().dj_batch_run_n(b, int(n), _stream(stream)), "dj_batch_run_n", b)


def dj_batch_sync(b, stream=None):
    _bcheck(lib().dj_batch_sync(b, _stream(stream)), "dj_batch_sync", b)


def dj_batch_relax_to_tol(b, tol, max_steps, stream=None, raise_on_fail=True):
    steps, r = C.c_longlong(0), C.c_double(0)
    st = lib().dj_batch_relax_to_tol(b, float(tol), int(max_steps), C.byref(steps), C.byref(r),
                                     _stream(stream))
    if raise_on_fail:
        _bcheck(st, "dj_batch_relax_to_tol", b)
    return st, steps.value, r.value


def dj_batch_instance_info(b, i):
    nn, ne, dt, r = C.c_longlong(0), C.c_longlong(0), C.c_double(0), C.c_double(0)
    _bcheck(lib().dj_batch_instance_info(b, int(i), C.byref(nn), C.byref(ne), C.byref(dt), C.byref(r)),
            "dj_batch_instance_info", b)
    return nn.value, ne.value, dt.value, r.value


def dj_batch_get_displacements(b, i, n_nodes):
    out = np.empty((n_nodes, 3))
    _bcheck(lib().dj_batch_get_displacements(b, int(i), _dptr(out)), "dj_batch_get_displacements", b)
    return out


def dj_batch_set_displacements(b, i, U0):
    U0 = _f64(U0)
    _bcheck(lib().dj_batch_set_displacements(b, int(i), _dptr(U0)), "dj_batch_set_displacements", b)


def dj_batch_get_info(b):
    n = C.c_int(0)
    v = [C.c_longlong(0) for _ in range(4)]
    _bcheck(lib().dj_batch_get_info(b, C.byref(n), *[C.byref(x) for x in v]), "dj_batch_get_info", b)
    return (n.value,) + tuple(x.value for x in v)


def dj_batch_destroy(b):
    lib().dj_batch_destroy(b)


def dj_set_displacements_device(h, d_ptr, stream=None):
    _check(lib().dj_set_displacements_device(h, d_ptr, _stream(stream)), "dj_set_displacements_device", h)


def dj_autotune(h, steps=200, stream=None):
    p = dj_params()
    ms = C.c_double(0)
    _check(lib().dj_autotune(h, int(steps), _stream(stream), C.byref(p), C.byref(ms)), "dj_autotune", h)
    return p, ms.value


def dj_autotune_cold(h, steps=50, d_flush=None, flush_bytes=0, stream=None):
    p = dj_params()
    ms = C.c_double(0)
    _check(lib().dj_autotune_cold(h, int(steps), d_flush, int(flush_bytes), _stream(stream), C.byref(p),
                                  C.byref(ms)), "dj_autotune_cold", h)
    return p, ms.value


def dj_batch_autotune(b, steps=100, stream=None):
    _bcheck(lib().dj_batch_autotune(b, int(steps), _stream(stream)), "dj_batch_autotune", b)


def dj_set_step(h, step):
    _check(lib().dj_set_step(h, int(step)), "dj_set_step", h)


def dj_batch_set_step(b, step):
    _bcheck(lib().dj_batch_set_step(b, int(step)), "dj_batch_set_step", b)


def dj_evaluate_field(h, d_ptr, stream=None):
    r, inv = C.c_double(0), C.c_int(0)
    _check(lib().dj_evaluate_field(h, d_ptr, C.byref(r), C.byref(inv), _stream(stream)),
           "dj_evaluate_field", h)
    return r.value, bool(inv.value)


def dj_batch_get_displacements_device(b, i, d_ptr, stream=None):
    _bcheck(lib().dj_batch_get_displacements_device(b, int(i), d_ptr, _stream(stream)),
            "dj_batch_get_displacements_device", b)


def _mcheck(st, where, m):
    if st != DJ_OK:
        msg = lib().dj_mlp_last_error(m) if m else b""
        raise DJError(st, where, msg.decode() if msg else "")


def dj_mlp_create(widths, seed=0):
    w = (C.c_int * len(widths))(*widths)
    m = _P()
    _mcheck(lib().dj_mlp_create(w, len(widths) - 1, int(seed), C.byref(m)), "dj_mlp_create", None)
    return m


def dj_mlp_num_params(m):
    return int(lib().dj_mlp_num_params(m))


def dj_mlp_get_params(m):
    n = dj_mlp_num_params(m)
    out = np.empty(n, dtype=np.float32)
    _mcheck(lib().dj_mlp_get_params(m, out.ctypes.data_as(C.POINTER(C.c_float)), n), "dj_mlp_get_params", m)
    return out


def dj_mlp_set_params(m, p):
    p = np.ascontiguousarray(p, dtype=np.float32)
    _mcheck(lib().dj_mlp_set_params(m, p.ctypes.data_as(C.POINTER(C.c_float)), p.size), "dj_mlp_set_params", m)


def dj_mlp_get_grads(m):
    n = dj_mlp_num_params(m)
    out = np.empty(n, dtype=np.float32)
    _mcheck(lib().dj_mlp_get_grads(m, out.ctypes.data_as(C.POINTER(C.c_float)), n), "dj_mlp_get_grads", m)
    return out


def dj_mlp_forward(m, d_X, batch, d_Y, stream=None):
    _mcheck(lib().dj_mlp_forward(m, d_X, int(batch), d_Y, _stream(stream)), "dj_mlp_forward", m)


def dj_mlp_loss_grad(m, d_X, d_T, d_w, batch, stream=None, want_loss=True):
    loss = C.c_double(0)
    _mcheck(lib().dj_mlp_loss_grad(m, d_X, d_T, d_w, int(batch), C.byref(loss) if want_loss else None,
                                   _stream(stream)), "dj_mlp_loss_grad", m)
    return loss.value


def dj_mlp_adam_step(m, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _mcheck(lib().dj_mlp_adam_step(m, float(lr), float(beta1), float(beta2), float(eps), _stream(stream)),
            "dj_mlp_adam_step", m)


def dj_mlp_destroy(m):
    lib().dj_mlp_destroy(m)


def dj_residual_norms_static(d_F, d_prescribed, n_nodes, d_out, stream=None):
    """Allocation-free residual sums (see include/dj_tled.h); returns the status."""
    return int(lib().dj_residual_norms_static(d_F, d_prescribed, int(n_nodes), d_out, _stream(stream)))


def dj_pod_fit(d_Y, rows, cols, r, d_mean, d_modes, stream=None):
    sig = np.empty(r)
    st = lib().dj_pod_fit(d_Y, int(rows), int(cols), int(r), d_mean, d_modes, _dptr(sig), _stream(stream))
    _check(st, "dj_pod_fit")
    return sig


def dj_pod_project(d_modes, d_mean, rows, r, d_X, cols, d_Q, stream=None):
    _check(lib().dj_pod_project(d_modes, d_mean, int(rows), int(r), d_X, int(cols), d_Q, _stream(stream)),
           "dj_pod_project")


def dj_pod_expand(d_modes, d_mean, rows, r, d_Q, cols, d_X, stream=None):
    _check(lib().dj_pod_expand(d_modes, d_mean, int(rows), int(r), d_Q, int(cols), d_X, _stream(stream)),
           "dj_pod_expand")


def dj_profile_kernels(h, launches, d_flush=None, flush_bytes=0, stream=None):
    """(ms per force launch, ms per update launch), each launch timed alone
    after an L2 eviction when a flush buffer is given."""
    f, u = C.c_double(0), C.c_double(0)
    _check(lib().dj_profile_kernels(h, int(launches), d_flush, int(flush_bytes), _stream(stream),
                                    C.byref(f), C.byref(u)), "dj_profile_kernels", h)
    return f.value, u.value


def dj_linear_fit(d_X, d_Y, S, n_in, n_out, ridge, d_W, stream=None):
    _check(lib().dj_linear_fit(d_X, d_Y, int(S), int(n_in), int(n_out), float(ridge), d_W, _stream(stream)),
           "dj_linear_fit")


def dj_quad_features(d_X, S, ld, n, d_F, stream=None):
    _check(lib().dj_quad_features(d_X, int(S), int(ld), int(n), d_F, _stream(stream)), "dj_quad_features")


def dj_linear_apply(d_W, n_out, n_in, d_X, S, alpha, beta, d_Y, stream=None):
    _check(lib().dj_linear_apply(d_W, int(n_out), int(n_in), d_X, int(S), float(alpha), float(beta), d_Y,
                                 _stream(stream)), "dj_linear_apply")


# ------------------------------------------------------------- convenience --
class Mesh:
    """Owning wrapper of a dj_mesh handle built from a workloads.Problem."""

    def __init__(self, problem, params: Optional[dj_params] = None, precompute: bool = True,
                 **param_kw):
        p = problem
        self.problem = p
        self.n_nodes = p.n_nodes
        self.h = dj_mesh_create(p.elem_type, p.X, p.conn)
        try:
            dj_mesh_set_materials(self.h, p.model, p.mu, p.kappa, p.rho, p.eta_a, p.eta_b, p.c01,
                                  p.a_dir, p.b_dir)
            dj_mesh_set_bcs(self.h, p.bc_dof, p.bc_target)
            if params is None:
                kw = dict(dt=p.dt, dt_scale=p.dt_scale, alpha=p.alpha, hg_coeff=p.hg_coeff,
                          ramp_steps=p.ramp_steps, ramp_kind=p.ramp_kind)
                if getattr(p, "anp", False):  # average nodal pressure runs on the bulk-copy tiles
                    kw.update(anp=1, assembly=2)
                kw.update(param_kw)
                params = default_params(**kw)
            self.params = params
            self.dt = dj_precompute(self.h, params) if precompute else None
        except Exception:
            dj_mesh_destroy(self.h)
            self.h = None
            raise

    def step(self, stream=None):
        dj_step(self.h, stream)

    def run(self, n, stream=None):
        dj_run_n(self.h, n, stream)

    def sync(self, stream=None):
        dj_sync(self.h, stream)

    def displacements(self) -> np.ndarray:
        return dj_get_displacements(self.h, self.n_nodes)

    def set_displacements(self, U0):
        dj_set_displacements(self.h, U0)

    def internal_forces(self, U) -> np.ndarray:
        return dj_internal_forces(self.h, U)

    def relax(self, tol, max_steps, stream=None, raise_on_fail=True):
        return dj_relax_to_tol(self.h, tol, max_steps, stream, raise_on_fail)

    def relax_adaptive(self, tol, max_steps, alpha_min=0.0, alpha_max=0.0, disp_tol=0.0, stream=None,
                       raise_on_fail=True):
        return dj_relax_adaptive(self.h, tol, max_steps, alpha_min, alpha_max, disp_tol, stream,
                                 raise_on_fail)

    def info(self) -> dj_info:
        return dj_get_info(self.h)

    def close(self):
        if self.h:
            dj_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Owning wrapper of a dj_batch built from workloads.Problem instances."""

    def __init__(self, problems, precompute=True, **param_kw):
        self.problems = list(problems)
        handles = []
        try:
            for p in self.problems:
                h = dj_mesh_create(p.elem_type, p.X, p.conn)
                handles.append(h)
                dj_mesh_set_materials(h, p.model, p.mu, p.kappa, p.rho, p.eta_a, p.eta_b, p.c01,
                                      p.a_dir, p.b_dir)
                dj_mesh_set_bcs(h, p.bc_dof, p.bc_target)
            self.b = dj_batch_create(handles)
        finally:
            for h in handles:
                dj_mesh_destroy(h)
        p0 = self.problems[0]
        kw = dict(dt=p0.dt, dt_scale=p0.dt_scale, alpha=p0.alpha, hg_coeff=p0.hg_coeff,
                  ramp_steps=p0.ramp_steps, ramp_kind=p0.ramp_kind)
        kw.update(param_kw)
        self.params = default_params(**kw)
        if precompute:
            dj_batch_precompute(self.b, self.params)

    def run(self, n, stream=None):
        dj_batch_run_n(self.b, n, stream)

    def sync(self, stream=None):
        dj_batch_sync(self.b, stream)

    def relax(self, tol, max_steps, stream=None, raise_on_fail=True):
        return dj_batch_relax_to_tol(self.b, tol, max_steps, stream, raise_on_fail)

    def displacements(self, i):
        return dj_batch_get_displacements(self.b, i, self.problems[i].n_nodes)

    def set_displacements(self, i, U0):
        dj_batch_set_displacements(self.b, i, U0)

    def instance_info(self, i):
        return dj_batch_instance_info(self.b, i)

    def info(self):
        return dj_batch_get_info(self.b)

    def close(self):
        if getattr(self, "b", None):
            dj_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dj_symmetric_eigen(A):
    """Eigenvalues (descending) and eigenvectors (columns) of a symmetric matrix."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    _check(lib().dj_symmetric_eigen(_dptr(A), n, _dptr(w), _dptr(V)), "dj_symmetric_eigen")
    return w, V


def dj_mlp_set_precision(m, precision):
    _mcheck(lib().dj_mlp_set_precision(m, int(precision)), "dj_mlp_set_precision", m)


# ------------------------------------------------------------ warm start --
def ws_params(**kw) -> dj_ws_params:
    p = dj_ws_params()
    lib().dj_ws_params_default(C.byref(p))
    for k, v in kw.items():
        if k == "hidden":
            v = list(v) + [0] * (4 - len(v))
            p.hidden = (C.c_int * 4)(*v)
            continue
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _wcheck(st, where, ws=None):
    if st != DJ_OK:
        msg = lib().dj_ws_last_error(ws) if ws else b""
        raise DJError(st, where, msg.decode() if msg else "")


def dj_ws_train(mesh_h, targets, tol, max_steps, params=None, stream=None):
    T = np.ascontiguousarray(targets, dtype=np.float64)
    w = _P()
    st = lib().dj_ws_train(mesh_h, _dptr(T), int(T.shape[0]), float(tol), int(max_steps),
                           C.byref(params) if params is not None else None, C.byref(w), _stream(stream))
    if st != DJ_OK:
        raise DJError(st, "dj_ws_train", dj_last_error(mesh_h))
    return w


def dj_ws_fit(bc_dof, n_nodes, d_targets, d_fields, n_loads, params=None, stream=None):
    dof = np.ascontiguousarray(bc_dof, dtype=np.int64)
    w = _P()
    _wcheck(lib().dj_ws_fit(dof.ctypes.data_as(_LL), int(dof.size), int(n_nodes), d_targets, d_fields,
                            int(n_loads), C.byref(params) if params is not None else None, C.byref(w),
                            _stream(stream)), "dj_ws_fit")
    return w


def dj_ws_predict(ws, targets, d_field, parts=DJ_WS_PARTS_FITTED, stream=None):
    t = _f64(targets)
    _wcheck(lib().dj_ws_predict(ws, _dptr(t), int(parts), d_field, _stream(stream)), "dj_ws_predict", ws)


def dj_ws_relax_to_tol(mesh_h, ws, targets, arm, tol, max_steps, stream=None, raise_on_fail=True):
    """Returns (status, result dict)."""
    t = _f64(targets)
    res = dj_ws_result()
    st = lib().dj_ws_relax_to_tol(mesh_h, ws, _dptr(t), int(arm), float(tol), int(max_steps), C.byref(res),
                                  _stream(stream))
    if raise_on_fail:
        _wcheck(st, "dj_ws_relax_to_tol", ws)
    return st, _struct_dict(res)


def dj_ws_save(ws) -> bytes:
    n = C.c_size_t(0)
    _wcheck(lib().dj_ws_save(ws, None, 0, C.byref(n)), "dj_ws_save", ws)
    buf = C.create_string_buffer(n.value)
    _wcheck(lib().dj_ws_save(ws, C.cast(buf, _P), n.value, C.byref(n)), "dj_ws_save", ws)
    return buf.raw[:n.value]


def dj_ws_load(blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    w = _P()
    _wcheck(lib().dj_ws_load(C.cast(buf, _P), len(blob), C.byref(w)), "dj_ws_load")
    return w


def dj_ws_get_info(ws) -> dict:
    info = dj_ws_info()
    _wcheck(lib().dj_ws_get_info(ws, C.byref(info)), "dj_ws_get_info", ws)
    return _struct_dict(info)


def dj_ws_destroy(ws):
    lib().dj_ws_destroy(ws)


def _addr(a: np.ndarray) -> int:
    """Address of an array's first element (the cheap route for writable
    buffers; the array interface otherwise)."""
    try:
        return C.addressof(C.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):
        return a.__array_interface__["data"][0]


_F64, _F32 = np.dtype(np.float64), np.dtype(np.float32)
_HOST_ADDR = {}  # id(array) -> (weak reference, address) of recent host buffers


def _host_addr(a: np.ndarray) -> int:
    """_addr with a small cache for buffers passed again and again (a host
    loop's targets and output); a weak reference tells a live entry from a
    reused id."""
    e = _HOST_ADDR.get(id(a))
    if e is not None and e[0]() is a:
        return e[1]
    addr = _addr(a)
    if len(_HOST_ADDR) >= 16:
        _HOST_ADDR.clear()
    _HOST_ADDR[id(a)] = (weakref.ref(a), addr)
    return addr


def dj_step_host(h, targets, U_out, stream=None):
    """One step with host input and output (include/dj_tled.h): targets (n_bc
    float64 or None), U_out a C-contiguous float64 or float32 array of
    n_nodes x 3 (or None).  Called once per step by a host-driven loop, so
    the marshalling takes the cheap routes (no ctypes pointer objects, cached
    addresses).  HostStep binds the buffers once and validates their sizes."""
    ta = None
    if targets is not None:
        if not (type(targets) is np.ndarray and targets.dtype is _F64 and targets.flags.c_contiguous):
            targets = _f64(targets)
        ta = _host_addr(targets) if targets.size else None
    ua, out_f64 = None, 1
    if U_out is not None:
        dt = U_out.dtype
        if not U_out.flags.c_contiguous or (dt is not _F32 and dt is not _F64 and dt not in (_F32, _F64)):
            raise ValueError("U_out must be a C-contiguous float64 or float32 array")
        out_f64 = 0 if dt == _F32 else 1
        ua = _host_addr(U_out) if U_out.size else None
    st = lib().dj_step_host(h, ta, ua, out_f64, _stream(stream))
    if st != DJ_OK:
        _check(st, "dj_step_host", h)
    return U_out


class HostStep:
    """dj_step_host bound to a mesh, a target array and an output array (the
    form for a loop that drives the solver from the host every step: the
    caller refills `targets` in place, calls the object, reads `U_out`).
    Types, layout and sizes are checked once, here; each call only passes
    the addresses.  Page-locked arrays (e.g. numpy views of pinned torch
    tensors) take the library's mapped paths."""

    def __init__(self, mesh, targets: Optional[np.ndarray], U_out: Optional[np.ndarray], stream=None):
        info = mesh.info()
        if targets is not None:
            if not (isinstance(targets, np.ndarray) and targets.dtype == _F64 and targets.flags.c_contiguous):
                raise ValueError("targets must be a C-contiguous float64 array (it is refilled in place)")
            if targets.size != info.n_bc_dofs:
                raise ValueError(f"targets has {targets.size} values, the mesh {info.n_bc_dofs} prescribed DOFs")
        if U_out is not None:
            if not (isinstance(U_out, np.ndarray) and U_out.flags.c_contiguous and U_out.dtype in (_F32, _F64)):
                raise ValueError("U_out must be a C-contiguous float64 or float32 array")
            if U_out.size != 3 * info.n_nodes:
                raise ValueError(f"U_out has {U_out.size} values, the mesh 3 x {info.n_nodes}")
        self.mesh, self.targets, self.U_out = mesh, targets, U_out  # held: the addresses stay valid
        self._args = (mesh.h, _addr(targets) if targets is not None and targets.size else None,
                      _addr(U_out) if U_out is not None and U_out.size else None,
                      0 if U_out is not None and U_out.dtype == _F32 else 1, _stream(stream))
        self._f = lib().dj_step_host

    def __call__(self) -> Optional[np.ndarray]:
        st = self._f(*self._args)
        if st != DJ_OK:
            _check(st, "dj_step_host", self.mesh.h)
        return self.U_out
