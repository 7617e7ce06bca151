"""ctypes declarations of the C ABI in include/ds.h (libds.so).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libds.so")
# the range-checking variant (build.build(bounds=True)), selected with DS_LIBRARY=bounds
BOUNDS_LIB_PATH = os.path.join(PKG, "libds_bounds.so")

DS_OK = 0
DS_E_ARG = 1
DS_E_NOT_INCREASING = 2
DS_E_INDISTINGUISHABLE = 3
DS_E_OVERFLOW = 4
DS_E_TABLE_TOO_LARGE = 5
DS_E_NOMEM = 6
DS_E_CUDA = 7
DS_E_TIMEOUT = 8
DS_E_UNIMPLEMENTED = 9
DS_E_NO_CONVERGENCE = 10
DS_E_DEVICE = 11

DS_DEVERR_TIMEOUT = 1
DS_DEVERR_BOUNDS = 2
(DS_BS_K, DS_BS_K16, DS_BS_X, DS_BS_RANK, DS_BS_FPRINT, DS_BS_CMAP, DS_BS_CBLOCK, DS_BS_CESC, DS_BS_Y,
 DS_BS_LAYOUT) = range(1, 11)

DS_F32 = 0
DS_F64 = 1

DS_FMA = 1
DS_CACHE_LAYOUT = 2
DS_CHECKED = 4
DS_NO_SMEM = 8
DS_STRICT = 16
DS_GAP2 = 32
DS_NO_FINGERPRINT = 64
DS_REFINE_H = 128
DS_LS_CLASSIC, DS_LS_CLASSICMOD, DS_LS_LEADBIT, DS_LS_LEADBIT_NOPAD, DS_LS_OFFSET, DS_LS_EYTZINGER = range(6)
DS_LS_NAMES = ("classic", "classicmod", "leadbit", "leadbit_nopad", "offset", "eytzinger")

DS_LEARNED_FORCE = 1
DS_LEARNED_LINEAR = 2

DS_STATIC_MAX_KNOTS = 262144

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
F32 = ctypes.c_float
F64 = ctypes.c_double
ST = ctypes.c_int


class ds_info_t(ctypes.Structure):
    _fields_ = [
        ("kind", I32), ("dtype", I32), ("flags", U32), ("n_arrays", I32),
        ("n_knots", I64), ("H", F64), ("W", F64), ("X0", F64), ("XN", F64),
        ("R", U64), ("table_bytes", I64), ("h_updates", I64), ("hr_passes", I64),
        ("build_ms", F64), ("smem_resident", I32), ("n_direct", I32), ("n_learned", I32),
        ("n_fallback", I32), ("max_window", I64), ("train_steps", I64), ("train_ms", F64),
        ("final_loss", F64), ("fallback_queries", U64), ("device_error", I32), ("gap_q", I32),
        ("search_launches", I32), ("reserved_", I32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if not name.startswith("reserved")}


class ds_tune_t(ctypes.Structure):
    _fields_ = [("block", I32), ("items", I32), ("smem_limit", I32), ("blocks_per_sm", I32), ("ms", F32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ds_learned_cfg(ctypes.Structure):
    _fields_ = [("steps", I32), ("batch", I32), ("n_queries", I32), ("lr", F32), ("seed", U64),
                ("flags", U32), ("max_cells_per_knot", I32), ("cells_per_knot", F32), ("reserved", I32 * 3)]


_SIGS = {
    "ds_build": (ST, [P, I64, ST, U32, P, ctypes.POINTER(P)]),
    "ds_build_q": (ST, [P, I64, ST, U32, ctypes.c_int32, ctypes.c_int32, I64, P, ctypes.POINTER(P)]),
    "ds_search_sorted": (ST, [P, I64, ST, P, I64, P, P]),
    "ds_histogram": (ST, [P, P, I64, P, P]),
    "ds_learned_autotune": (ST, [P, P, P, I64, P, P, P, P, ctypes.POINTER(ds_tune_t)]),
    "ds_learned_build_xy": (ST, [P, P, P, I32, I64, ST, ctypes.POINTER(ds_learned_cfg), P, ctypes.POINTER(P)]),
    "ds_learned_cells": (ST, [P, I32, ctypes.POINTER(U64), ctypes.POINTER(I32), ctypes.POINTER(I64),
                              ctypes.POINTER(I64), ctypes.POINTER(F64), ctypes.POINTER(I32)]),
    "ds_learned_export_cells": (ST, [P, I32, P, P]),
    "ds_learned_search_host": (ST, [P, P, P, I64, P, P, P]),
    "ds_learned_set_tune": (ST, [P, ctypes.POINTER(ds_tune_t)]),
    "ds_learned_get_tune": (ST, [P, ctypes.POINTER(ds_tune_t)]),
    "ds_lsearch_constants": (ST, [ctypes.c_int32, I64, P, ctypes.POINTER(I64)]),
    "ds_lsearch_build": (ST, [P, I64, ST, ctypes.c_int32, U32, P, ctypes.POINTER(P)]),
    "ds_lsearch_search": (ST, [P, P, I64, P, P]),
    "ds_search": (ST, [P, P, I64, P, P]),
    "ds_search_host": (ST, [P, P, I64, P, P]),
    "ds_index_tables": (ST, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]),
    "ds_index_export": (ST, [P, P, P, P, P]),
    "ds_batch_build": (ST, [P, P, I32, ST, U32, P, ctypes.POINTER(P)]),
    "ds_batch_search": (ST, [P, P, P, P, P]),
    "ds_batch_autotune": (ST, [P, P, P, P, P, ctypes.POINTER(ds_tune_t)]),
    "ds_batch_set_tune": (ST, [P, ctypes.POINTER(ds_tune_t)]),
    "ds_batch_get_tune": (ST, [P, ctypes.POINTER(ds_tune_t)]),
    "ds_batch_array": (ST, [P, I32, ctypes.POINTER(F64), ctypes.POINTER(F64), ctypes.POINTER(U64),
                            ctypes.POINTER(I32)]),
    "ds_learned_cfg_default": (None, [ctypes.POINTER(ds_learned_cfg)]),
    "ds_learned_build": (ST, [P, P, I32, I64, ST, ctypes.POINTER(ds_learned_cfg), P, ctypes.POINTER(P)]),
    "ds_learned_search": (ST, [P, P, P, I64, P, P, P, P]),
    "ds_learned_array": (ST, [P, I32, P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
    "ds_mlp_forward": (ST, [P, P, I64, P, P]),
    "ds_mlp_loss_grad": (ST, [P, P, P, I64, P, P, P]),
    "ds_adam_step": (ST, [P, P, P, P, I32, F32, P]),
    "ds_build_table_static": (ST, [P, I64, ST, U32, P, I64, ctypes.POINTER(F64), ctypes.POINTER(F64),
                                   ctypes.POINTER(U64), P]),
    "ds_info": (ST, [P, ctypes.POINTER(ds_info_t)]),
    "ds_free": (None, [P]),
    "ds_status_str": (ctypes.c_char_p, [ST]),
    "ds_last_error": (ctypes.c_char_p, []),
    "ds_abi_version": (I32, []),
    "ds_debug_fail_alloc": (ST, [I64]),
    "ds_debug_alloc_stats": (ST, [ctypes.POINTER(I64), ctypes.POINTER(I64)]),
}

EXPORTED = sorted(_SIGS)

_lib = None


class DsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        L = lib()
        msg = L.ds_last_error().decode(errors="replace")
        super().__init__("%s: %s: %s" % (where, L.ds_status_str(status).decode(), msg))


def lib(path=None):
    """Load libds.so (built in-tree by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or (BOUNDS_LIB_PATH if os.environ.get("DS_LIBRARY") == "bounds" else LIB_PATH)
    if not os.path.exists(path):
        raise ImportError("libds.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'` "
                          "or `python -m paper_1506_08620_gb300.build`" % path)
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status, where):
    if status != DS_OK:
        raise DsError(status, where)
