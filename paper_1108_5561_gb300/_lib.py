"""ctypes binding of the C ABI in include/rlb.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RLB_OK, RLB_ERR_ARG, RLB_ERR_CUDA, RLB_ERR_NUMERIC, RLB_ERR_TIMEOUT, RLB_ERR_STATE, RLB_ERR_NOMEM = \
    0, -1, -2, -3, -4, -5, -6
RLB_F64, RLB_F32, RLB_BF16 = 0, 1, 2
RLB_EOS_CROSSOVER, RLB_EOS_CONST_MASS, RLB_EOS_CONFORMAL = 0, 1, 2
RLB_RADIAL_PAPER, RLB_RADIAL_LAGUERRE = 0, 1
RLB_MINKOWSKI, RLB_MILNE = 0, 1

EXPORTS = ["rlb_create", "rlb_destroy", "rlb_last_error", "rlb_init_eos", "rlb_workspace_size",
           "rlb_configure", "rlb_bind_buffers", "rlb_init_grid", "rlb_step", "rlb_get_tau",
           "rlb_moments", "rlb_check", "rlb_state_offsets", "rlb_lattice", "rlb_operators",
           "rlb_set_timing", "rlb_get_timing", "rlb_step_static_scratch", "rlb_observables",
           "rlb_state_blob_size", "rlb_save_state", "rlb_load_state", "rlb_configure_batch",
           "rlb_init_batch", "rlb_autotune", "rlb_set_stage_variant", "rlb_set_graphs", "rlb_adjoint_set_arithmetic", "rlb_adjoint_workspace_size",
           "rlb_adjoint_bind", "rlb_adjoint_seed_v2", "rlb_adjoint_seed", "rlb_adjoint_step", "rlb_adjoint_ic", "rlb_alu_peaks",
           "rlb_wait_selftest", "rlb_load_state_async", "rlb_adjoint_step_from", "rlb_moments_async",
           "rlb_moments_wait"]


class EosParamsC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("table_points", ctypes.c_int),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("Tc", ctypes.c_double),
                ("w", ctypes.c_double), ("m0", ctypes.c_double), ("Z", ctypes.c_double),
                ("T_min", ctypes.c_double), ("T_max", ctypes.c_double)]


class GridParamsC(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("metric", ctypes.c_int),
                ("n_xi", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_phi_half", ctypes.c_int),
                ("family", ctypes.c_int), ("prec", ctypes.c_int),
                ("dx", ctypes.c_double), ("z0", ctypes.c_double), ("T0", ctypes.c_double),
                ("eta_over_s", ctypes.c_double), ("tau0", ctypes.c_double),
                ("dtau", ctypes.c_double)]


class EventDescC(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("eta_over_s", ctypes.c_double)]


class RLBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librlb.so (librlb_checked.so, the build with device-side range
    checks, when the environment sets RLB_CHECKED=1); raises if it cannot be
    built or loaded (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("RLB_CHECKED", "") == "1"
    path = _build.LIB_CHECKED if checked else _build.LIB
    if build_if_missing:
        path = _build.build(checked=checked)
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing; run paper_1108_5561_gb300.build" % path)
    lib = ctypes.CDLL(path)
    P, vp, sz = ctypes.POINTER, ctypes.c_void_p, ctypes.c_size_t
    dp = P(ctypes.c_double)
    lib.rlb_create.argtypes = [P(vp), ctypes.c_int]
    lib.rlb_destroy.argtypes = [vp]
    lib.rlb_destroy.restype = None
    lib.rlb_last_error.argtypes = [vp]
    lib.rlb_last_error.restype = ctypes.c_char_p
    lib.rlb_init_eos.argtypes = [vp, P(EosParamsC)]
    lib.rlb_workspace_size.argtypes = [vp, P(GridParamsC), P(sz), P(sz)]
    lib.rlb_configure.argtypes = [vp, P(GridParamsC)]
    lib.rlb_bind_buffers.argtypes = [vp, vp, vp, vp]
    lib.rlb_init_grid.argtypes = [vp, dp, ctypes.c_int, vp]
    lib.rlb_step.argtypes = [vp, ctypes.c_int, vp]
    lib.rlb_get_tau.argtypes = [vp, dp]
    lib.rlb_moments.argtypes = [vp, dp, ctypes.c_int, vp]
    lib.rlb_check.argtypes = [vp, vp]
    lib.rlb_state_offsets.argtypes = [vp, P(sz), P(sz), P(sz)]
    lib.rlb_lattice.argtypes = [vp] + [dp] * 7
    lib.rlb_operators.argtypes = [vp, dp, dp]
    lib.rlb_set_timing.argtypes = [vp, ctypes.c_int]
    lib.rlb_alu_peaks.argtypes = [ctypes.c_int, dp]
    lib.rlb_load_state_async.argtypes = [vp, vp, sz, ctypes.c_double, vp]
    lib.rlb_moments_async.argtypes = [vp, vp, vp]
    lib.rlb_moments_wait.argtypes = [vp]
    lib.rlb_adjoint_step_from.argtypes = [vp, vp, sz, ctypes.c_double, vp]
    lib.rlb_wait_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, P(ctypes.c_int),
                                      P(ctypes.c_float)]
    lib.rlb_step_static_scratch.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.rlb_get_timing.argtypes = [vp, dp, P(ctypes.c_long), dp, P(ctypes.c_long)]
    lib.rlb_observables.argtypes = [vp, dp, dp, vp]
    lib.rlb_state_blob_size.argtypes = [vp, P(sz)]
    lib.rlb_save_state.argtypes = [vp, vp, sz, vp]
    lib.rlb_load_state.argtypes = [vp, vp, sz, vp]
    lib.rlb_configure_batch.argtypes = [vp, P(GridParamsC), ctypes.c_int, P(EventDescC)]
    lib.rlb_init_batch.argtypes = [vp, dp, ctypes.c_int, vp]
    lib.rlb_autotune.argtypes = [vp, vp, P(ctypes.c_int), dp, P(ctypes.c_int)]
    lib.rlb_set_graphs.argtypes = [vp, ctypes.c_int]
    lib.rlb_set_stage_variant.argtypes = [vp, ctypes.c_int, P(ctypes.c_int)]
    lib.rlb_adjoint_set_arithmetic.argtypes = [vp, ctypes.c_int]
    lib.rlb_adjoint_workspace_size.argtypes = [vp, P(sz)]
    lib.rlb_adjoint_bind.argtypes = [vp, vp]
    lib.rlb_adjoint_seed_v2.argtypes = [vp, dp, vp]
    lib.rlb_adjoint_seed.argtypes = [vp, vp, vp, vp]
    lib.rlb_adjoint_step.argtypes = [vp, vp]
    lib.rlb_adjoint_ic.argtypes = [vp, dp, dp, ctypes.c_int, dp, vp]
    for name in EXPORTS:
        if name not in ("rlb_destroy", "rlb_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib
