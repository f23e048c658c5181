"""ctypes declarations of the C ABI in include/fc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfc.so")

FC_OK = 0
STATUS = {0: "FC_OK", 1: "FC_ERR_INVALID_ARG", 2: "FC_ERR_PRECONDITION", 3: "FC_ERR_OOM",
          4: "FC_ERR_CUDA", 5: "FC_ERR_TIMEOUT", 6: "FC_ERR_STATE"}
F32, F64 = 0, 1
WALLS, PERIODIC, SPHERE, BRICK = 0, 1, 2, 3
VEL_CONST, VEL_SWIRL, VEL_ROTATION, VEL_DEFORM = 0, 1, 2, 3

INFO_LEVELS = 21

# allocator callbacks of fc_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)


class Info(ctypes.Structure):
    """Mirror of fc_info."""
    _fields_ = [(n, ctypes.c_int) for n in ("nleaves", "nforests", "mx", "mbc", "lmin", "lmax",
                                            "dtype", "domain")] + [
        ("leaves_per_level", ctypes.c_int * INFO_LEVELS), ("device_bytes", ctypes.c_int64),
        ("graphs", ctypes.c_int), ("tuned_buckets", ctypes.c_int),
        ("coarse_entries", ctypes.c_int), ("coarse_unlisted", ctypes.c_int)]


# every function that include/fc.h declares, with (restype, argtypes)
_vp, _ip, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)


class Desc(ctypes.Structure):
    """Mirror of fc_forest_desc."""
    _fields_ = [
        ("domain", ctypes.c_int), ("nforests", ctypes.c_int),
        ("mx", ctypes.c_int), ("mbc", ctypes.c_int),
        ("lmin", ctypes.c_int), ("lmax", ctypes.c_int),
        ("dtype", ctypes.c_int), ("vel_kind", ctypes.c_int),
        ("vel", ctypes.c_double * 4),
        ("order", ctypes.c_int), ("limiter", ctypes.c_int),
        ("transverse", ctypes.c_int),
        ("indicator", ctypes.c_int), ("smooth", ctypes.c_int),
        ("reflux", ctypes.c_int),
        ("brick_nx", ctypes.c_int), ("brick_ny", ctypes.c_int),
    ]


_DP = ctypes.POINTER(Desc)
SIGNATURES = {
    "fc_forest_create": (ctypes.c_int, [_DP, ctypes.c_int, _ip, ctypes.POINTER(_vp)]),
    "fc_forest_destroy": (ctypes.c_int, [_vp]),
    "fc_forest_num_leaves": (ctypes.c_int, [_vp, _ip]),
    "fc_forest_leaves": (ctypes.c_int, [_vp, _ip]),
    "fc_forest_set_q": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "fc_forest_get_q": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "fc_forest_get_q_full": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "fc_fill_ghosts": (ctypes.c_int, [_vp, _vp]),
    "fc_advance_level": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp]),
    "fc_step_global": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _vp]),
    "fc_step_multirate": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _vp]),
    "fc_tag_regrid": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _ip, _ip, _vp]),
    "fc_tag": (ctypes.c_int, [_vp, _dp, _vp]),
    "fc_forest_mass": (ctypes.c_int, [_vp, _dp, _vp]),
    "fc_layout_check": (ctypes.c_int, [_DP, ctypes.c_int, _ip]),
    "fc_layout_neighbours": (ctypes.c_int, [_DP, ctypes.c_int, _ip, _ip]),
    "fc_layout_reflux": (ctypes.c_int, [_DP, ctypes.c_int, _ip, _ip]),
    "fc_layout_regrid": (ctypes.c_int, [_DP, ctypes.c_int, _ip, _dp, ctypes.c_double,
                                        ctypes.c_double, _ip, ctypes.c_int, _ip, _ip]),
    "fc_timers_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fc_forest_poison": (ctypes.c_int, [_vp, ctypes.c_double, _vp]),
    "fc_set_graphs": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fc_autotune": (ctypes.c_int, [_vp, _ip, _vp]),
    "fc_set_fused_fill": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fc_set_velocity_scale": (ctypes.c_int, [_vp, ctypes.c_double]),
    "fc_adjoint_step_global": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _vp, _vp,
                                              _vp]),
    "fc_adjoint_step_multirate": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _vp,
                                                 _vp, _vp]),
    "fc_step_multirate_record": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_int, _vp]),
    "fc_adjoint_step_multirate_taped": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double,
                                                       ctypes.c_int, _vp, _vp, _vp]),
    "fc_tape_release": (ctypes.c_int, [_vp]),
    "fc_adjoint_advance": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          _vp, _vp, _vp, _vp]),
    "fc_forest_info": (ctypes.c_int, [_vp, _vp]),
    "fc_layout_partition": (ctypes.c_int, [_DP, ctypes.c_int, _ip, ctypes.c_int, _ip]),
    "fc_layout_halo": (ctypes.c_int, [_DP, ctypes.c_int, _ip, _ip, ctypes.c_int, _ip, _ip]),
    "fc_forest_create_part": (ctypes.c_int, [_DP, ctypes.c_int, _ip, _ip, ctypes.c_int,
                                             ctypes.POINTER(_vp)]),
    "fc_halo_count": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _ip, _ip]),
    "fc_halo_pack": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "fc_halo_unpack": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "fc_set_allocator": (ctypes.c_int, [_vp, _vp, _vp]),
    "fc_mass_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                       _vp, ctypes.c_int, _vp, _vp]),
    "fc_forest_get_capacity": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "fc_set_advance_variant": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "fc_set_limits": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "fc_timers_read": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64),
                                      _dp, ctypes.c_int]),
    "fc_last_error": (ctypes.c_char_p, []),
    "fc_launch_count": (ctypes.c_uint64, [ctypes.c_int]),
}

_lib = None


class FcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load libfc.so; raise if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
            "g.build()'` (nvcc, sm_103a).  There is no CPU fallback.")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int):
    if status != FC_OK:
        raise FcError(status, load().fc_last_error().decode())
