"""ctypes view of libvdwdf (include/vdwdf.h): structs, prototypes, loader.

Argument marshalling only.  The library is built in-tree by
``paper_0810_2273_gb300.build`` (``__graft_entry__.build()``); if it is
missing, every entry point raises instead of falling back to anything else.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvdwdf.so")

VDWDF_FP32 = 0
VDWDF_FP64 = 1

_c_d = ctypes.c_double
_c_i = ctypes.c_int
_c_i32 = ctypes.c_int32
_c_i64 = ctypes.c_int64
_c_p = ctypes.c_void_p


class vdwdf_grid(ctypes.Structure):
    _fields_ = [("cell", (_c_d * 3) * 3), ("n", _c_i32 * 3), ("periodic", _c_i32 * 3), ("gradient", _c_i32)]


class vdwdf_result(ctypes.Structure):
    _fields_ = [("E", _c_d), ("E_diag", _c_d), ("n_active", _c_i64), ("pairs", _c_i64),
                ("pairs_evaluated", _c_i64), ("n_clamped", _c_i64), ("q0_min", _c_d),
                ("q0_max", _c_d), ("ms_prep", ctypes.c_float), ("ms_pairs", ctypes.c_float),
                ("ms_post", ctypes.c_float), ("launches", _c_i32), ("smem_row0", _c_i32),
                ("pair_threads", _c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vdwdf_semilocal_result(ctypes.Structure):
    _fields_ = [("Ex_lda", _c_d), ("Ec_lda", _c_d), ("Ex_pbe", _c_d), ("Ec_pbe", _c_d),
                ("Ex_revpbe", _c_d), ("n_points", _c_i64), ("ms", ctypes.c_float), ("launches", _c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vdwdf_diag_result(ctypes.Structure):
    _fields_ = [("E_diag_voxel", _c_d), ("E_diag_table", _c_d), ("q0_min", _c_d), ("q0_max", _c_d),
                ("n_active", _c_i64), ("nphi0", _c_i32), ("ms", ctypes.c_float), ("launches", _c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vdwdf_tail_result(ctypes.Structure):
    _fields_ = [("T", _c_d), ("n_active", _c_i64), ("nodes", _c_i32), ("planes", _c_i32),
                ("ms", ctypes.c_float), ("launches", _c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vdwdf_tuning(ctypes.Structure):
    _fields_ = [("threads", _c_i32), ("items_per_sm", _c_i32), ("smem_rows", _c_i32),
                ("smem_row0", _c_i32)]


# name -> (restype, argtypes); every function declared in include/vdwdf.h
PROTOTYPES = {
    "vdwdf_table_build": (_c_i, [_c_i, _c_d, _c_i, _c_i, _c_p, ctypes.POINTER(_c_p)]),
    "vdwdf_table_from_nodes": (_c_i, [_c_i, _c_d, _c_i, _c_p, ctypes.POINTER(_c_p)]),
    "vdwdf_table_nodes": (_c_i, [_c_p, _c_p]),
    "vdwdf_table_info": (_c_i, [_c_p, ctypes.POINTER(_c_i), ctypes.POINTER(_c_d), ctypes.POINTER(_c_i)]),
    "vdwdf_table_free": (None, [_c_p]),
    "vdwdf_kernel_eval": (_c_i, [_c_p, _c_i, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "vdwdf_q0": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, _c_d, _c_p, _c_p, _c_p, _c_p]),
    "vdwdf_gradient": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, _c_p]),
    "vdwdf_energy": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, _c_d, _c_d, _c_p, _c_i,
                            ctypes.POINTER(vdwdf_tuning), ctypes.POINTER(vdwdf_result), _c_p]),
    "vdwdf_potential": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_d, _c_d, _c_p, _c_i,
                               ctypes.POINTER(vdwdf_tuning), _c_p, _c_p, _c_p,
                               ctypes.POINTER(vdwdf_result), _c_p]),
    "vdwdf_energy_batched": (_c_i, [_c_i, ctypes.POINTER(vdwdf_grid), ctypes.POINTER(_c_p), _c_d, _c_d,
                                    _c_p, _c_i, ctypes.POINTER(vdwdf_tuning), _c_p,
                                    ctypes.POINTER(vdwdf_result), _c_p]),
    "vdwdf_semilocal": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, ctypes.POINTER(vdwdf_semilocal_result),
                               _c_p]),
    "vdwdf_phi0_eval": (_c_i, [_c_p, _c_p, _c_i64, _c_p, _c_p, _c_p]),
    "vdwdf_diag_voxel": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, _c_d, _c_p, _c_i,
                                ctypes.POINTER(vdwdf_diag_result), _c_p]),
    "vdwdf_diag_voxel_potential": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_d, _c_p, _c_i, _c_p,
                                          ctypes.POINTER(vdwdf_diag_result), _c_p]),
    "vdwdf_energy_noalloc": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, _c_d, _c_d, _c_p, _c_i,
                                    ctypes.POINTER(vdwdf_result), _c_p]),
    "vdwdf_autotune": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_d, _c_d, _c_p, _c_i,
                              ctypes.POINTER(vdwdf_tuning), _c_p]),
    "vdwdf_total_energy_nl": (_c_i, [_c_d, ctypes.POINTER(vdwdf_semilocal_result), _c_d, _c_i, _c_p]),
    "vdwdf_far_tail": (_c_i, [ctypes.POINTER(vdwdf_grid), _c_p, _c_p, _c_d, _c_d, _c_p,
                              ctypes.POINTER(vdwdf_tail_result), _c_p]),
    "vdwdf_strerror": (ctypes.c_char_p, [_c_i]),
    "vdwdf_version": (_c_i, []),
    "vdwdf_launch_count": (_c_i64, []),
    "vdwdf_lane_rate": (_c_i, [_c_i, _c_d, _c_p, _c_p, _c_p]),
}

_LIB = None


class VdwdfError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "unknown status"
        if _LIB is not None:
            msg = _LIB.vdwdf_strerror(status).decode()
        super().__init__("%s failed: %s (status %d)" % (where, msg, status))


def load():
    """The loaded libvdwdf (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libvdwdf.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_0810_2273_gb300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def check(status, where):
    if status != 0:
        raise VdwdfError(status, where)
