"""ctypes declarations of the C ABI in include/beamtrack.h (argument
marshalling only; every computation runs in libbeamtrack.so)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbeamtrack.so")

BX_OK, BX_BAD_ARG, BX_NONFINITE, BX_OUT_OF_MEMORY, BX_DEVICE_TIMEOUT, BX_CUDA, BX_COLLECTIVE = \
    range(7)
BX_OP_SUM, BX_OP_MIN, BX_OP_MAX = 0, 1, 2
BX_DRIFT, BX_QUAD, BX_SBEND, BX_DIPEDGE, BX_CONSTF, BX_MULTIPOLE = 0, 1, 2, 3, 4, 5
BX_MULTIPOLE_MAX_ORDER = 12
BX_NOALLOC_OUTSIDE, BX_NOALLOC_NONFINITE = 1, 2


class bx_options(ctypes.Structure):
    _fields_ = [("n_grid", c_int32), ("shape_order", c_int32), ("rebin_interval", c_int32),
                ("bin_edge", c_int32), ("cell_order", c_int32), ("reserved", c_int32 * 3)]


class bx_beam(ctypes.Structure):
    _fields_ = [("coord", c_void_p * 6), ("id", c_void_p), ("n", c_int64),
                ("charge_sign", c_double), ("bunch_charge_C", c_double),
                ("mass_MeV", c_double), ("kinetic_MeV", c_double)]


class bx_element(ctypes.Structure):
    _fields_ = [("type", c_int32), ("nslice", c_int32), ("length", c_double),
                ("k", c_double), ("angle", c_double), ("k2", c_double),
                ("order", c_int32), ("reserved", c_int32)]


class bx_lattice(ctypes.Structure):
    _fields_ = [("elements", POINTER(bx_element)), ("count", c_int32),
                ("space_charge", c_int32)]


class bx_grid(ctypes.Structure):
    _fields_ = [("n", c_int32), ("use_box", c_int32), ("lo", c_double * 3),
                ("hi", c_double * 3), ("h", c_double * 3), ("rho", c_void_p),
                ("phi", c_void_p)]


# int32_t (*)(int64_t *buf, int64_t count, int32_t op, void *stream, void *user)
bx_allreduce_fn = ctypes.CFUNCTYPE(c_int32, c_void_p, c_int64, c_int32, c_void_p, c_void_p)


class bx_shard(ctypes.Structure):
    _fields_ = [("allreduce", bx_allreduce_fn), ("user", c_void_p), ("n_total", c_int64)]


# name -> (restype, argtypes), one entry per declaration in include/beamtrack.h
SIGNATURES = {
    "bx_create": (c_int32, [POINTER(c_void_p), POINTER(bx_options)]),
    "bx_destroy": (c_int32, [c_void_p]),
    "bx_reset": (c_int32, [c_void_p]),
    "bx_track": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(bx_lattice), c_int64, c_int64,
                           c_void_p]),
    "bx_deposit": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(bx_grid), c_void_p]),
    "bx_solve": (c_int32, [c_void_p, POINTER(bx_grid), c_void_p]),
    "bx_gather_kick": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(bx_grid), c_double,
                                 c_void_p]),
    "bx_moments": (c_int32, [c_void_p, POINTER(bx_beam), c_void_p, c_void_p]),
    "bx_selftest_wait_timeout": (c_int32, [c_void_p, c_double, c_void_p]),
    "bx_green_table": (c_int32, [c_void_p, POINTER(c_double), c_void_p, c_void_p]),
    "bx_regrid_log": (c_int32, [c_void_p, POINTER(c_int64), c_int64, POINTER(c_int64)]),
    "bx_get_box": (c_int32, [c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    "bx_sync": (c_int32, [c_void_p, c_void_p]),
    "bx_profile": (c_int32, [c_void_p, c_int32]),
    "bx_profile_read": (c_int32, [c_void_p, POINTER(c_double), POINTER(c_int64), c_int32,
                                  POINTER(c_int32)]),
    "bx_kernel_name": (c_char_p, [c_int32]),
    "bx_deposit_noalloc": (c_int32, [POINTER(bx_beam), POINTER(c_double), POINTER(c_double),
                                     c_int32, c_void_p, c_void_p, c_void_p]),
    "bx_twiss_beam": (c_int32, [POINTER(c_double), POINTER(c_void_p), c_int64, POINTER(c_void_p),
                                c_void_p]),
    "bx_twiss_grad": (c_int32, [POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    "bx_grad_forward": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(bx_lattice), c_int32,
                                  POINTER(c_double), c_void_p]),
    "bx_grad_backward": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(c_double),
                                   POINTER(c_double), POINTER(c_double), POINTER(c_void_p),
                                   c_void_p]),
    "bx_grad_boxes": (c_int32, [c_void_p, POINTER(c_double), c_int64, POINTER(c_int64)]),
    "bx_batch_create": (c_int32, [POINTER(c_void_p), c_int32, POINTER(c_void_p),
                                  POINTER(POINTER(bx_beam)), POINTER(POINTER(bx_lattice)),
                                  c_void_p]),
    "bx_batch_launch": (c_int32, [c_void_p, c_void_p]),
    "bx_batch_destroy": (c_int32, [c_void_p]),
    "bx_batch_last_error": (c_char_p, [c_void_p]),
    "bx_set_binning": (c_int32, [c_void_p, c_int32, c_int32, c_int32]),
    "bx_autotune_binning": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(bx_lattice), c_int32,
                                      POINTER(c_int32), POINTER(c_double), c_int32,
                                      POINTER(c_int32), c_void_p]),
    "bx_track_diagnostics": (c_int32, [c_void_p, POINTER(bx_beam), POINTER(bx_lattice), c_int64,
                                       c_int64, c_void_p, c_void_p]),
    "bx_distribution_beam": (c_int32, [c_int32, POINTER(c_double), POINTER(c_void_p), c_void_p,
                                       c_int64, POINTER(c_void_p), c_void_p]),
    "bx_set_shard": (c_int32, [c_void_p, POINTER(bx_shard)]),
    "bx_objectives": (c_int32, [POINTER(c_double), POINTER(c_double)]),
    "bx_family_grad": (c_int32, [POINTER(c_double), POINTER(c_int32), c_int32, c_int32,
                                 POINTER(c_double)]),
    "bx_last_error": (c_char_p, [c_void_p]),
}

_LIB = None


class BeamtrackError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"beamtrack error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libbeamtrack.so; raise (never fall back) if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"libbeamtrack.so not built ({path}); run "
                          "`python -m paper_2208_02382_b300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib
