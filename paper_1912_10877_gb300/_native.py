"""ctypes view of libqsim.so (include/qsim.h).  Argument marshalling only.

Loading fails loudly when the CUDA library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsim.so")

QS_OK, QS_EINVAL, QS_ENOMEM, QS_EDEVICE, QS_ETIMEDOUT, QS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
QS_C64, QS_C128 = 0, 1
QS_MAXK = 5
QS_BATCH_RESET, QS_BATCH_GRAD = 1, 2
QS_BATCH_PRECISE = 1
QS_APPLY_PER_REGISTER, QS_APPLY_UNFUSED, QS_APPLY_TILES, QS_APPLY_BLOCKS = 1, 2, 4, 8
QS_APPLY_PRECISE = 32
QS_OPT_TENSOR_CORES = 1

GATE_KIND = {"I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8,
             "RX": 9, "RY": 10, "RZ": 11, "SHIFT": 12, "PHASE": 13, "SWAP": 14, "ROT": 15,
             "MATRIX": 16}
PAULI_CODE = {"X": 1, "Y": 2, "Z": 3}


class QsimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qsim status {code}: {msg}")
        self.code = code


class GateDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nlocs", ctypes.c_int32),
                ("locs", ctypes.c_int32 * QS_MAXK), ("paulis", ctypes.c_int32 * QS_MAXK),
                ("param", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ctrl_mask", ctypes.c_uint64), ("ctrl_vals", ctypes.c_uint64),
                ("mat_offset", ctypes.c_int64), ("theta", ctypes.c_double)]


class PauliTerm(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("x_mask", ctypes.c_uint64), ("z_mask", ctypes.c_uint64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PU64 = ctypes.POINTER(ctypes.c_uint64)
_PP = ctypes.POINTER(ctypes.c_void_p)
_PSZ = ctypes.POINTER(ctypes.c_size_t)

SIGNATURES = {
    "qs_last_error": ([], ctypes.c_char_p),
    "qs_state_bytes": ([_I, _PI32, _I, _PSZ], _I),
    "qs_state_create": ([_I, _I, _I, _P, _P, _PP], _I),
    "qs_batch_create": ([_I, _PI32, _I, _P, _P, _PP], _I),
    "qs_state_destroy": ([_P], _I),
    "qs_state_set_stream": ([_P, _P], _I),
    "qs_state_data": ([_P, _PP, _PSZ, _PI64], _I),
    "qs_state_reset": ([_P, _PU64], _I),
    "qs_state_upload": ([_P, _P], _I),
    "qs_state_download": ([_P, _P], _I),
    "qs_state_sync": ([_P], _I),
    "qs_state_copy": ([_P, _P], _I),
    "qs_state_inner": ([_P, _P, _PD], _I),
    "qs_state_axpy": ([_P, _D, _D, _P], _I),
    "qs_set_option": ([_I, _I], _I),
    "qs_get_option": ([_I, ctypes.POINTER(_I)], _I),
    "qs_selftest_bounded_wait": ([_D, ctypes.POINTER(_I)], _I),
    "qs_observable_groups": ([_P, ctypes.POINTER(_I)], _I),
    "qs_shot_expect": ([_P, _P, _PD, _I, _P, _PD], _I),
    "qs_faithful_gradient": ([_P, _PD, _P, _I, _I, _PD, _P, _P, _P, _PD], _I),
    "qs_mmd_gradient": ([_P, _PD, _PD, _D, _I, _I, _PD, _P, _P, _PD, _PD], _I),
    "qs_observable_csr_rows": ([_P, _I, _P, _P, _PI64, _P], _I),
    "qs_observable_csr_fill": ([_P, _I, _P, _P, _P, _P], _I),
    "qs_apply_gate": ([_P, _PD, _I, _PI32, _I, _PI32, _PI32], _I),
    "qs_apply_named": ([_P, _I, _I, _PI32, _PI32, _I, _PI32, _PI32, _D], _I),
    "qs_circuit_create": ([_I, ctypes.POINTER(GateDesc), _I, _PD, ctypes.c_int64, _I, _PP], _I),
    "qs_circuit_destroy": ([_P], _I),
    "qs_circuit_info": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "qs_circuit_gate_matrices": ([_P, _I, _PD, ctypes.POINTER(GateDesc), _PD, _PD, _PD], _I),
    "qs_circuit_schedule_info": ([_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "qs_circuit_tile_order": ([_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], _I),
    "qs_apply_circuit": ([_P, _P, _PD, _I], _I),
    "qs_circuit_blocks": ([_P, _PD, _I, ctypes.POINTER(_I), _PI32, _PI32, _PD], _I),
    "qs_autotune_circuit": ([_P, _P, _PD, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _PI32, _PD], _I),
    "qs_checkpoint_count": ([_P, _I, ctypes.POINTER(_I)], _I),
    "qs_apply_circuit_ckpt": ([_P, _P, _PD, _I, _P], _I),
    "qs_observable_create": ([ctypes.POINTER(PauliTerm), _I, _PP], _I),
    "qs_observable_destroy": ([_P], _I),
    "qs_expect": ([_P, _P, _PD], _I),
    "qs_expect_static": ([_P, _I, _I, _I, ctypes.POINTER(PauliTerm), _I, _P, _P], _I),
    "qs_backward_work_bytes": ([_I, _PSZ], _I),
    "qs_backward": ([_P, _P, _PD, _P, _I, _P, _P, _PD, _PD], _I),
    "qs_backward_tiled_work_bytes": ([_I, _PSZ], _I),
    "qs_backward_blocks_work_bytes": ([_I, _I, _PSZ], _I),
    "qs_backward_blocks": ([_P, _P, _PD, _P, _I, _P, _PD, _PD], _I),
    "qs_backward_tiled": ([_P, _P, _PD, _P, _I, _P, _PD, _PD], _I),
    "qs_measure": ([_P, _PD, _I, _PI64, _I], _I),
    "qs_measure_seeded": ([_P, ctypes.c_uint64, _I, _PI64, _I], _I),
    "qs_adjoint_step": ([_P, _P, _P, _PD, _PD, _P], _I),
    "qs_run_circuit_one_launch": ([_P, _P, _PD, _I, _P, _I, _P], _I),
    "qs_gate_desc_matrices": ([_P, _PD, _PD, _I, _PD, _PD, _PD], _I),
    "qs_sample_shards": ([_I, _PD, _I, _PD, _PI32, _PD], _I),
    "qs_batch_program_create": ([_I, _PP, _PP, _I, _PP], _I),
    "qs_batch_program_create_ex": ([_I, _PP, _PP, _I, _I, _I, _PP], _I),
    "qs_batch_program_shape": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "qs_batch_autotune_ex": ([_I, _PP, _PP, _I, _P, _P, _P, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(_I), _PI32, _PI32, _PD], _I),
    "qs_batch_program_destroy": ([_P], _I),
    "qs_batch_program_info": ([_P, ctypes.POINTER(_I), _PI64, _PI64, _PI64], _I),
    "qs_batch_run": ([_P, _P, _P, _P, _P, _I], _I),
    "qs_batch_autotune": ([_I, _PP, _PP, _P, _P, _P, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _PI32, _PD], _I),
}

_lib = None


def lib():
    """The loaded library; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def check(rc: int):
    if rc != QS_OK:
        raise QsimError(rc, lib().qs_last_error().decode(errors="replace"))
    return rc


def i32(vals):
    vals = list(vals)
    return (ctypes.c_int32 * max(1, len(vals)))(*vals)


def dptr(arr):
    return arr.ctypes.data_as(_PD)
