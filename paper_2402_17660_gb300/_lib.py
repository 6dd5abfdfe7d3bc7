"""ctypes binding of libtnet's C ABI (include/tnet.h): same names, argument
marshalling only.  Importing this module loads the CUDA library and fails
loudly when it is missing; there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build


class ModelDesc(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int), ("K", ctypes.c_int), ("L", ctypes.c_int), ("max_z", ctypes.c_int),
                ("cutoff_upper", ctypes.c_float), ("cutoff_lower", ctypes.c_float),
                ("precision", ctypes.c_int), ("recompute_edges", ctypes.c_int), ("radial_table", ctypes.c_int)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_f32 = ctypes.c_float

SIGNATURES = {
    "tnet_status_string": (ctypes.c_char_p, [_i32]),
    "tnet_weights_count": (_i64, [ctypes.POINTER(ModelDesc)]),
    "tnet_workspace_bytes": (_i64, [ctypes.POINTER(ModelDesc), _i32, _i32, _i64]),
    "tnet_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(ModelDesc), _i32, _i32, _i64, _vp,
                           ctypes.c_size_t]),
    "tnet_destroy": (_i32, [_vp]),
    "tnet_neighbors": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp, _f32, _vp, _vp, _i64, _vp, _vp, _vp]),
    "tnet_energy_forces": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp]),
    "tnet_radial_tables": (_i32, [_vp, _vp, _vp]),
    "tnet_md_step": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _f32, _f32, _i32, _i32, _vp, _vp,
                            _vp, _vp]),
    "tnet_md_rebuilds": (_i32, [_vp, _vp]),
    "tnet_md_neighbor_list": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, _vp]),
    "tnet_neighbors_noalloc": (_i32, [_i32, _i32, _vp, _vp, _vp, _f32, _vp, _vp, _i64, _vp, _vp, _vp]),
    "tnet_debug_tc_gemm": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "tnet_debug_tc_gemm_cluster": (_i32, [_i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tnet_debug_tc_gemm_f32": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tnet_debug_tc_gemm_timeout": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, ctypes.c_uint32, _vp, _vp]),
    "tnet_tuning_knobs": (_i32, []),
    "tnet_tuning_name": (ctypes.c_char_p, [_i32]),
    "tnet_tuning_candidates": (_i32, [_i32, ctypes.POINTER(_i32), _i32]),
    "tnet_get_tuning": (_i32, [_vp, ctypes.POINTER(_i32), _i32]),
    "tnet_set_tuning": (_i32, [_vp, ctypes.POINTER(_i32), _i32]),
    "tnet_launch_count": (_i64, []),
    "tnet_profile": (_i32, [_vp, _i32]),
    "tnet_profile_read": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_i64)]),
    "tnet_profile_tag": (ctypes.c_char_p, [_i32]),
}

STATUS = {0: "OK", 1: "ARG", 2: "CAPACITY", 3: "BOX", 4: "NAN", 5: "CUDA", 6: "TIMEOUT",
          7: "WORKSPACE", 8: "Z", 9: "UNSUPPORTED", 10: "SKIN"}


class TnetError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({status_string(code)})")


_LIB = None


def header_functions() -> list[str]:
    """Names of the functions include/tnet.h declares."""
    with open(os.path.join(_build.INCLUDE, "tnet.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tnet_[a-z_0-9]+)\s*\(", text)))


def load(path: str | None = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libtnet.so (building it first if needed) and bind every entry point."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    if path is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libtnet is not built ({path}); run paper_2402_17660_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == _build.LIB:
        _LIB = lib
    return lib


def status_string(code: int) -> str:
    return load().tnet_status_string(int(code)).decode()


def check(code: int, where: str) -> None:
    if code != 0:
        raise TnetError(code, where)
