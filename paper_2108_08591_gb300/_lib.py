"""ctypes binding of libmdf.so (include/mdf.h).  Argument marshalling only.

The shared library must have been built (``__graft_entry__.build()`` or
``python -m paper_2108_08591_gb300._build``); there is no fallback: loading
fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdf.so")

# mdf_status codes
OK, EINVAL, ENOMEM, ECUDA, EDIVERGED, ETIMEOUT, ENOTCONVERGED, EUNSUPPORTED, EIO = range(9)
STATUS_NAMES = ["MDF_OK", "MDF_EINVAL", "MDF_ENOMEM", "MDF_ECUDA", "MDF_EDIVERGED",
                "MDF_ETIMEOUT", "MDF_ENOTCONVERGED", "MDF_EUNSUPPORTED", "MDF_EIO"]
STORAGE = {"f32": 0, "f16": 1, "bf16": 2, "f64": 3, "f16eq": 4, "bf16eq": 5}
HOST, DEVICE = 0, 1


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class Rates(ctypes.Structure):
    _fields_ = [("s0", ctypes.c_double), ("s1", ctypes.c_double), ("s2", ctypes.c_double)]


class BC(ctypes.Structure):
    _fields_ = [("wall", ctypes.c_int * 3), ("lid", ctypes.c_int), ("lid_u", ctypes.c_double * 3)]


class Opts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("with_rho", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("vx", ctypes.c_int), ("block", ctypes.c_int), ("q", ctypes.c_int),
                ("inplace", ctypes.c_int)]


class Fields(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("P", "u", "rho", "G", "div", "S", "sigma", "omega")] + [
        ("where", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("q", ctypes.c_int), ("nsets", ctypes.c_int),
                ("storage", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("pitch", ctypes.c_int), ("nodes", ctypes.c_longlong),
                ("step", ctypes.c_longlong), ("bytes_per_update", ctypes.c_double),
                ("s0", ctypes.c_double), ("s1", ctypes.c_double), ("s2", ctypes.c_double),
                ("vx", ctypes.c_int), ("block", ctypes.c_int)]


H = ctypes.c_void_p
DP = ctypes.c_void_p  # double* (host or device address)

# name -> (restype, argtypes); every function declared in include/mdf.h
SIGNATURES = {
    "mdf_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.POINTER(Grid), ctypes.c_int,
                                  ctypes.POINTER(Rates), ctypes.POINTER(BC), ctypes.POINTER(Opts)]),
    "mdf_destroy": (None, [H]),
    "mdf_init": (ctypes.c_int, [H, DP, DP, ctypes.c_int]),
    "mdf_init_neq": (ctypes.c_int, [H, DP, DP, DP, ctypes.c_int]),
    "mdf_set_force": (ctypes.c_int, [H, DP, ctypes.c_int]),
    "mdf_set_forcing": (ctypes.c_int, [H, ctypes.c_int]),
    "mdf_slabs_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "mdf_slabs_init": (ctypes.c_int, [H, DP, DP]),
    "mdf_slabs_step": (ctypes.c_int, [H, ctypes.c_longlong]),
    "mdf_slabs_fields": (ctypes.c_int, [H, ctypes.c_void_p]),
    "mdf_slabs_destroy": (None, [H]),
    "mdf_slabs_last_error": (ctypes.c_char_p, [H]),
    "mdf_get_forcing": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_int)]),
    "mdf_step": (ctypes.c_int, [H, ctypes.c_longlong]),
    "mdf_step_fields": (ctypes.c_int, [H, ctypes.c_longlong, ctypes.POINTER(Fields)]),
    "mdf_fields": (ctypes.c_int, [H, ctypes.POINTER(Fields)]),
    "mdf_fields_host_noalloc": (ctypes.c_int, [H, ctypes.POINTER(Fields)]),
    "mdf_moments": (ctypes.c_int, [H, DP, DP, DP]),
    "mdf_gradients": (ctypes.c_int, [H, DP, DP, DP, DP, DP]),
    "mdf_sums": (ctypes.c_int, [H, DP]),
    "mdf_residual": (ctypes.c_int, [H, DP]),
    "mdf_mask": (ctypes.c_int, [H, DP]),
    "mdf_save": (ctypes.c_int, [H, ctypes.c_char_p]),
    "mdf_load": (ctypes.c_int, [H, ctypes.c_char_p]),
    "mdf_info": (ctypes.c_int, [H, ctypes.POINTER(Info)]),
    "mdf_autotune": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
    "mdf_sync": (ctypes.c_int, [H]),
    "mdf_last_error": (ctypes.c_char_p, [H]),
    "mdf_batch_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int, ctypes.c_int, DP, DP,
                                        ctypes.c_double, ctypes.POINTER(Opts)]),
    "mdf_batch_destroy": (None, [H]),
    "mdf_batch_init": (ctypes.c_int, [H, ctypes.c_int, DP, DP, ctypes.c_int]),
    "mdf_batch_seed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_int]),
    "mdf_batch_run": (ctypes.c_int, [H, ctypes.c_double, ctypes.c_longlong, ctypes.c_int, DP, DP, DP]),
    "mdf_batch_step": (ctypes.c_int, [H, ctypes.c_longlong]),
    "mdf_batch_fields": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(Fields)]),
    "mdf_batch_info": (ctypes.c_int, [H, DP, DP, DP]),
    "mdf_batch_set_timeout": (ctypes.c_int, [H, ctypes.c_longlong]),
    "mdf_batch_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mdf_batch_get_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mdf_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "mdf_batch_last_error": (ctypes.c_char_p, [H]),
    "mdf_ws_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int, ctypes.c_int, ctypes.c_int, DP,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_ulonglong, ctypes.c_void_p]),
    "mdf_ws_destroy": (None, [H]),
    "mdf_ws_param_count": (ctypes.c_longlong, [H]),
    "mdf_ws_get_params": (ctypes.c_int, [H, DP, DP]),
    "mdf_ws_set_params": (ctypes.c_int, [H, DP]),
    "mdf_ws_forward": (ctypes.c_int, [H, DP, ctypes.c_int, DP]),
    "mdf_ws_train_step": (ctypes.c_int, [H, DP, DP, ctypes.c_int, ctypes.c_float, DP]),
    "mdf_ws_last_error": (ctypes.c_char_p, [H]),
    "mdf_nn_conv_fwd": (ctypes.c_int, [DP, DP, DP, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "mdf_nn_wgrad_scratch": (ctypes.c_longlong, [ctypes.c_int] * 5),
    "mdf_nn_conv_wgrad": (ctypes.c_int, [DP, DP, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "mdf_nn_conv_dgrad": (ctypes.c_int, [DP, DP, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "mdf_nn_set_conv_kernel": (ctypes.c_int, [ctypes.c_int]),
    "mdf_nn_set_tc_tile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "mdf_nn_set_halo_tile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "mdf_nn_set_wgrad_kernel": (ctypes.c_int, [ctypes.c_int]),
    "mdf_nn_set_wgrad_tile": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mdf_nn_conv_error": (ctypes.c_int, [DP]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libmdf.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libmdf.so not found at {LIB_PATH}: build it first with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MdfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


def check(status: int, handle=None):
    if status != OK:
        msg = load().mdf_last_error(handle)
        raise MdfError(status, msg.decode() if msg else "")


def check_ws(status: int, handle=None):
    if status != OK:
        msg = load().mdf_ws_last_error(handle)
        raise MdfError(status, msg.decode() if msg else "")


def check_slabs(status: int, handle=None):
    if status != OK:
        msg = load().mdf_slabs_last_error(handle)
        raise MdfError(status, msg.decode() if msg else "")


def check_batch(status: int, handle=None):
    if status != OK:
        msg = load().mdf_batch_last_error(handle)
        raise MdfError(status, msg.decode() if msg else "")
