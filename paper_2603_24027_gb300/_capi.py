"""ctypes binding of include/fdtd.h (argument marshalling only).

Every function of the C ABI is exposed under its C name.  The shared library
is built in-tree by `paper_2603_24027_gb300.build`; if it is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# FDTD_BOUNDS_CHECKED=1 loads the bounds-checked test build instead.
LIB_PATH = os.path.join(HERE, "libfdtd_gb300_checked.so" if os.environ.get("FDTD_BOUNDS_CHECKED")
                        else "libfdtd_gb300.so")

FDTD_OK, FDTD_EINVAL, FDTD_ENOMEM, FDTD_ECUDA, FDTD_ESTATE, FDTD_ETIMEOUT, FDTD_ENONFINITE = (
    0, -1, -2, -3, -4, -5, -6)
STATUS_NAMES = {0: "FDTD_OK", -1: "FDTD_EINVAL", -2: "FDTD_ENOMEM", -3: "FDTD_ECUDA",
                -4: "FDTD_ESTATE", -5: "FDTD_ETIMEOUT", -6: "FDTD_ENONFINITE"}
# Tape element types: "e4m3" (alias "e4m3fn") is the hardware OCP float8; the
# other 8-bit names are the formats of Sec. 4, "e4m3ieee" the IEEE-style e4m3;
# "bdct" is the 8 x 8 block-transform codec ("bdct<K>" keeps K coefficients per
# block, plain "bdct" 10).
TAPE = {"f32": 0, "bf16": 1, "f16": 2, "e4m3": 3, "e4m3fn": 3, "e4m3b11fnuz": 4, "e5m2fnuz": 5,
        "e4m3fnuz": 6, "e4m3ieee": 7, "e3m4": 8, "bdct": 9}
BDCT_DEFAULT_COEFFS = 10
INTERP = {"linear": 0, "cubic": 1}
OPT_USE_GRAPHS, OPT_KERNEL, OPT_TILE_Y, OPT_ZCHUNK, OPT_SAMPLE_EVERY = range(5)
OPT_STAGES, OPT_PDL, OPT_PREFETCH, OPT_TILE_X, OPT_COMPACT_AUX, OPT_EXACT_REVERSAL, \
    OPT_ZCHUNK_FWD, OPT_ZGROUPS, OPT_INJECT_WAIT_TIMEOUT, OPT_REVERSE, OPT_FORWARD, \
    OPT_ZCHUNK_FWD2 = range(6, 18)
K_FWD_H, K_FWD_E, K_RECORD, K_RESTORE, K_REV_E, K_REV_H, K_REV_PRIMAL, K_REV_ADJOINT, K_MONITOR, \
    K_REV_ADJOINT_CPML, K_FWD_FUSED, K_FWD_2STEP = range(12)
KERNEL_NAMES = ["fwd_h", "fwd_e", "record", "restore_seed", "rev_e", "rev_h", "rev_primal",
                "rev_adjoint", "monitor", "rev_adjoint_cpml", "fwd_fused", "fwd_2step"]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class Pml(C.Structure):
    _fields_ = [("thickness", C.c_int), ("order", C.c_int), ("sigma_factor", C.c_double),
                ("kappa_max", C.c_double), ("alpha_factor", C.c_double)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("component", C.c_int), ("pos", C.c_int * 3),
                ("axis", C.c_int), ("sigma_uv", C.c_double * 2), ("lambda0", C.c_double),
                ("rel_bandwidth", C.c_double), ("t0_over_tau", C.c_double),
                ("amplitude", C.c_double)]


class Detector(C.Structure):
    _fields_ = [("kind", C.c_int), ("axis", C.c_int), ("index", C.c_int),
                ("lo", C.c_int * 2), ("hi", C.c_int * 2)]


class RecordCfg(C.Structure):
    _fields_ = [("dtype", C.c_int), ("k", C.c_int), ("interp", C.c_int), ("scaled", C.c_int),
                ("coeffs", C.c_int)]


class FdtdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_PROTOS = {
    "fdtd_create": (C.c_int, [C.POINTER(Grid), C.c_double, C.c_double, C.POINTER(Pml),
                              C.POINTER(Source), C.POINTER(Detector), C.c_int,
                              C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p,
                              C.POINTER(C.c_void_p)]),
    "fdtd_workspace_bytes": (C.c_int, [C.c_void_p, C.POINTER(RecordCfg), C.POINTER(C.c_size_t)]),
    "fdtd_bind_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fdtd_tape_bytes": (C.c_int, [C.c_void_p, C.POINTER(RecordCfg), C.POINTER(C.c_size_t)]),
    "fdtd_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RecordCfg),
                               C.POINTER(C.c_double)]),
    "fdtd_backward": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "fdtd_backward2": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_void_p]),
    "fdtd_set_detector2": (C.c_int, [C.c_void_p, C.POINTER(Detector)]),
    "fdtd_objectives": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "fdtd_value_and_grad_host": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RecordCfg),
                                           C.c_double, C.POINTER(C.c_double), C.c_void_p]),
    "fdtd_group_forward": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                     C.POINTER(RecordCfg), C.POINTER(C.c_double)]),
    "fdtd_group_backward": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_void_p)]),
    "fdtd_batch_forward": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                     C.POINTER(RecordCfg), C.POINTER(C.c_double)]),
    "fdtd_batch_backward": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_void_p)]),
    "fdtd_last_error": (C.c_char_p, [C.c_void_p]),
    "fdtd_destroy": (C.c_int, [C.c_void_p]),
    "fdtd_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "fdtd_get_option": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "fdtd_last_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fdtd_last_host_call_ms": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "fdtd_kernel_timing": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float),
                                     C.POINTER(C.c_int)]),
    "fdtd_pml_profile": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fdtd_source_waveform": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_interp_weights": (C.c_int, [C.c_void_p, C.POINTER(RecordCfg), C.c_int, C.c_int,
                                      C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "fdtd_read_fields": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_objective_history": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_encode": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "fdtd_decode": (C.c_int, [C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "fdtd_bdct_encode": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "fdtd_bdct_decode": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                   C.c_void_p]),
    "fdtd_bdct_basis": (C.c_int, [C.c_void_p]),
    "fdtd_state_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "fdtd_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fdtd_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "fdtd_zgroup_ranges": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fdtd_selftest_wait": (C.c_int, [C.c_void_p, C.c_longlong, C.c_void_p]),
    "fdtd_status_of_error_word": (C.c_int, [C.c_uint]),
    "fdtd_reverse_units": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.POINTER(C.c_int), C.c_void_p, C.c_int]),
    "fdtd_deep_units": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_int)]),
    "fdtd_value_and_grad_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(RecordCfg),
                                              C.c_double, C.POINTER(C.c_double), C.c_void_p]),
}


def lib():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2603_24027_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, handle=None) -> None:
    if status != FDTD_OK:
        msg = lib().fdtd_last_error(handle)
        raise FdtdError(status, msg.decode() if msg else "")


def record_cfg(dtype: str = "f32", k: int = 1, interp: str = "linear", scaled=None) -> RecordCfg:
    """Tape configuration; scaled defaults to per-face scales for f16 and the
    hardware e4m3 (the paper's 8-bit formats default to unscaled, as in Sec. 4).
    "bdct<K>" selects the block-transform codec with K coefficients per block."""
    coeffs = 0
    if dtype.startswith("bdct"):
        coeffs = int(dtype[4:]) if len(dtype) > 4 else BDCT_DEFAULT_COEFFS
        dtype = "bdct"
    if scaled is None:
        scaled = dtype in ("f16", "e4m3", "e4m3fn")
    return RecordCfg(TAPE[dtype], int(k), INTERP[interp], int(bool(scaled)), coeffs)
