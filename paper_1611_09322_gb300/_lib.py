"""ctypes binding of libpse (include/pse.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
arrays are torch CUDA tensors passed as raw pointers with the current torch
stream; there is no CPU fallback: if the library cannot be loaded every call
raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libpse.so")

PSE_FP32, PSE_FP64 = 0, 1
PSE_PRECOND_NPARAM = 450
STAGES = ["cells", "sort", "real_noise", "neighbours", "matvec", "lanczos_update", "eigen", "final",
          "wave_noise", "fft", "interp", "grid_copy"]
STATUS = {0: "PSE_OK", 1: "PSE_EINVAL", 2: "PSE_ENOMEM", 3: "PSE_ECUDA", 4: "PSE_ECUFFT",
          5: "PSE_ENOTCONVERGED", 6: "PSE_ENOTSUPPORTED", 7: "PSE_ENOTREADY"}


class PseError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class pse_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("xi", ctypes.c_double), ("precision", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("fixed_iter", ctypes.c_int), ("grid_M", ctypes.c_int),
                ("support_P", ctypes.c_int), ("use_precond", ctypes.c_int), ("lanczos_tol", ctypes.c_double),
                ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int), ("system", ctypes.c_int),
                ("wave_noise", ctypes.c_int), ("spread_tile", ctypes.c_int),
                ("matvec_shape", ctypes.c_int), ("interp_form", ctypes.c_int), ("wave_fft", ctypes.c_int)]


class pse_plan_info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("a", ctypes.c_double), ("xi", ctypes.c_double), ("tol", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("k_cut", ctypes.c_double), ("m", ctypes.c_double),
                ("eta", ctypes.c_double), ("h", ctypes.c_double), ("self_mobility", ctypes.c_double),
                ("P", ctypes.c_int), ("M", ctypes.c_int), ("ncell", ctypes.c_int), ("precision", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class pse_stats(ctypes.Structure):
    _fields_ = [("lanczos_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("lanczos_rel_change", ctypes.c_double), ("n_pairs", ctypes.c_int64),
                ("overflow", ctypes.c_int), ("matvec_shape", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


PSE_XI_TRIALS = 8


class pse_xi_tuning(ctypes.Structure):
    _fields_ = [("xi_start", ctypes.c_double), ("t_real", ctypes.c_double), ("t_wave", ctypes.c_double),
                ("xi_model", ctypes.c_double), ("xi_best", ctypes.c_double), ("ms_start", ctypes.c_double),
                ("ms_best", ctypes.c_double), ("M_best", ctypes.c_int), ("n_grids", ctypes.c_int),
                ("n_tried", ctypes.c_int),
                ("xi_tried", ctypes.c_double * PSE_XI_TRIALS), ("ms_tried", ctypes.c_double * PSE_XI_TRIALS),
                ("ms_pred", ctypes.c_double * PSE_XI_TRIALS),
                ("iters_tried", ctypes.c_int * PSE_XI_TRIALS), ("M_tried", ctypes.c_int * PSE_XI_TRIALS)]

    def as_dict(self):
        n = self.n_tried
        out = {name: getattr(self, name) for name, _ in self._fields_[:10]}
        out["trials"] = [{"xi": self.xi_tried[i], "ms": self.ms_tried[i], "ms_pred": self.ms_pred[i],
                          "lanczos_iters": self.iters_tried[i], "M": self.M_tried[i]} for i in range(n)]
        return out


# name -> (restype, argtypes); the exported surface of include/pse.h
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_ST = ctypes.c_int
SIGNATURES = {
    "pse_plan": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.POINTER(pse_params), ctypes.POINTER(pse_plan_info)]),
    "pse_create": (_ST, [ctypes.POINTER(_VP), ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "pse_create_ex": (_ST, [ctypes.POINTER(_VP), ctypes.c_double, ctypes.c_double, ctypes.POINTER(pse_params)]),
    "pse_destroy": (None, [_VP]),
    "pse_get_plan": (_ST, [_VP, ctypes.POINTER(pse_plan_info)]),
    "pse_sample": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP]),
    "pse_sample_parts": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP, _VP, _VP]),
    "pse_sample_host": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP]),
    "pse_sample_host_async": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP]),
    "pse_host_sync": (_ST, [_VP]),
    "pse_sample_f64": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP, _VP, _VP]),
    "pse_real_matvec": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP]),
    "pse_sample_with_forces": (_ST, [_VP, _I64, _VP, _VP, _U64, _U64, ctypes.c_double, ctypes.c_double, _VP, _VP]),
    "pse_sample_with_forces_f64": (_ST, [_VP, _I64, _VP, _VP, _U64, _U64, ctypes.c_double, ctypes.c_double, _VP,
                                         _VP]),
    "pse_mobility_apply": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP]),
    "pse_sample_full_lanczos": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP]),
    "pse_sample_full_lanczos_f64": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP]),
    "pse_bd_step": (_ST, [_VP, _I64, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _U64, _U64, _VP]),
    "pse_bd_step_f64": (_ST, [_VP, _I64, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _U64, _U64,
                              _VP]),
    "pse_get_stats": (_ST, [_VP, ctypes.POINTER(pse_stats)]),
    "pse_strerror": (ctypes.c_char_p, [_ST]),
    "pse_profile_stages": (_ST, [_VP, _I64, _VP, _U64, _U64, _VP, _VP, _VP, _VP]),
    "pse_real_matvec_noalloc": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I64,
                                      _VP, _VP, _VP, _VP]),
    "pse_precond_features": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP]),
    "pse_precond_targets": (_ST, [_VP, _I64, _VP, _VP, _VP]),
    "pse_precond_loss_grad": (_ST, [_I64, _VP, _VP, _VP, _VP, ctypes.c_float, _VP, _VP, _VP]),
    "pse_precond_train": (_ST, [_I64, _VP, _VP, _VP, _VP, ctypes.c_float, ctypes.c_int, ctypes.c_float, _VP, _VP,
                                _VP]),
    "pse_precond_set_weights": (_ST, [_VP, _VP, ctypes.c_int]),
    "pse_precond_blocks": (_ST, [_VP, _I64, _VP, _VP, _VP]),
    "pse_create_poly": (_ST, [ctypes.POINTER(_VP), ctypes.c_double, ctypes.c_int, _VP, ctypes.POINTER(pse_params)]),
    "pse_get_species": (_ST, [_VP, ctypes.POINTER(ctypes.c_int), _VP]),
    "pse_sample_poly": (_ST, [_VP, _I64, _VP, _VP, _U64, _U64, _VP, _VP, _VP, _VP]),
    "pse_real_matvec_poly": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    "pse_batch_create": (_ST, [ctypes.POINTER(_VP), ctypes.c_int, _VP, _VP, _VP]),
    "pse_batch_grid": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.POINTER(pse_params), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)]),
    "pse_batch_sample": (_ST, [_VP, _VP, _VP, _U64, _U64, _VP, _VP]),
    "pse_batch_get_stats": (_ST, [_VP, ctypes.c_int, ctypes.POINTER(pse_stats)]),
    "pse_batch_get_plan": (_ST, [_VP, ctypes.c_int, ctypes.POINTER(pse_plan_info)]),
    "pse_batch_destroy": (None, [_VP]),
    "pse_batch_set_precond": (_ST, [_VP, ctypes.c_int, _VP, ctypes.c_int]),
    "pse_real_scalars": (_ST, [ctypes.c_double, ctypes.c_double, _I64, _VP, _VP, _VP]),
    "pse_real_scalars_poly": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _I64, _VP, _VP, _VP]),
    "pse_xi_model": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.POINTER(ctypes.c_double)]),
    "pse_tune_xi": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.POINTER(pse_params), _I64, _VP, ctypes.c_double,
                          ctypes.c_int, ctypes.POINTER(pse_xi_tuning), _VP]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libpse.so (built by paper_1611_09322_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libpse.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, where):
    if status != 0:
        raise PseError(status, where)
    return status
