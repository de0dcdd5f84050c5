"""ctypes declarations of libanqs (include/anqs.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libanqs.so")

ANQS_OK = 0
ANQS_MODEL_MLP, ANQS_MODEL_TF, ANQS_MODEL_TABLE, ANQS_MODEL_NADE = 0, 1, 2, 3
ANQS_FORM_FP32, ANQS_FORM_BF16 = 0, 1
ANQS_BATCH_STREAMS, ANQS_BATCH_STATIC, ANQS_BATCH_DYNAMIC = 0, 1, 2
ERRORS = {-1: "ANQS_ERR_ARG", -2: "ANQS_ERR_CAPACITY", -3: "ANQS_ERR_SECTOR", -4: "ANQS_ERR_CUDA",
          -5: "ANQS_ERR_UNSUPPORTED"}


class ModelDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("form", C.c_int32), ("n_orb", C.c_int32), ("width", C.c_int32),
                ("n_hidden", C.c_int32), ("d_model", C.c_int32), ("n_heads", C.c_int32),
                ("n_layers", C.c_int32)]


class ElocProblem(C.Structure):
    """anqs_eloc_problem: the arguments of one anqs_local_energy call."""
    _fields_ = [("model", C.c_void_p), ("ham", C.c_void_p), ("x_dev", C.c_void_p), ("counts_dev", C.c_void_p),
                ("n_x", C.c_uint64), ("n_x_dev", C.c_void_p), ("eloc_re_dev", C.c_void_p),
                ("eloc_im_dev", C.c_void_p), ("stats_dev", C.c_void_p), ("workspace_dev", C.c_void_p),
                ("workspace_bytes", C.c_size_t)]


class AnqsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_VP = C.c_void_p
_U64 = C.c_uint64
_SZ = C.c_size_t

SIGNATURES = {
    "anqs_version": (C.c_char_p, []),
    "anqs_last_error": (C.c_int, [C.c_char_p, _SZ]),
    "anqs_hamiltonian_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, C.c_int, _VP, _VP, C.c_double]),
    "anqs_hamiltonian_destroy": (C.c_int, [_VP]),
    "anqs_hamiltonian_info": (C.c_int, [_VP, C.POINTER(_U64), C.POINTER(_U64)]),
    "anqs_hamiltonian_slot_masks": (C.c_int, [_VP, _VP, _SZ]),
    "anqs_connected": (C.c_int, [_VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP]),
    "anqs_model_param_count": (C.c_int, [C.POINTER(ModelDesc), C.POINTER(_U64)]),
    "anqs_model_create": (C.c_int, [C.POINTER(_VP), C.POINTER(ModelDesc), _VP]),
    "anqs_model_destroy": (C.c_int, [_VP]),
    "anqs_model_sync": (C.c_int, [_VP, _VP]),
    "anqs_logpsi": (C.c_int, [_VP, _VP, _VP, _U64, _VP, _VP, _VP]),
    "anqs_logpsi_vjp": (C.c_int, [_VP, _VP, _VP, _U64, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "anqs_logpsi_vjp_workspace_size": (C.c_int, [_VP, _VP, _U64, C.POINTER(_SZ)]),
    "anqs_sample_workspace_size": (C.c_int, [_VP, _VP, _U64, C.POINTER(_SZ)]),
    "anqs_sample": (C.c_int, [_VP, _VP, _U64, _U64, _U64, _VP, _VP, _VP, _U64, _VP, _VP, _SZ, _VP]),
    "anqs_sample_binomial": (C.c_int, [_VP, _VP, _U64, _U64, _U64, _VP, _VP, _VP, _U64, _VP, _VP, _SZ, _VP]),
    "anqs_sample_shard": (C.c_int, [_VP, _VP, _U64, _U64, _U64, _VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _U64, _VP,
                                     _VP, _SZ, _VP]),
    "anqs_hamiltonian_set_pruning": (C.c_int, [_VP, C.c_int]),
    "anqs_hamiltonian_status": (C.c_int, [_VP, C.POINTER(C.c_int), C.c_int]),
    "anqs_hamiltonian_set_z2": (C.c_int, [_VP, C.c_int, _VP]),
    "anqs_model_status": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "anqs_test_sampler_barrier": (C.c_int, [C.c_uint, _U64]),
    "anqs_stats_combine": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "anqs_local_energy_workspace_size": (C.c_int, [_VP, _VP, _U64, C.POINTER(_SZ)]),
    "anqs_local_energy": (C.c_int, [_VP, _VP, _VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "anqs_grad_workspace_size": (C.c_int, [_VP, _VP, _U64, C.POINTER(_SZ)]),
    "anqs_grad_workspace_size_min": (C.c_int, [_VP, _VP, _U64, C.POINTER(_SZ)]),
    "anqs_grad": (C.c_int, [_VP, _VP, _VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "anqs_local_energy_static": (C.c_int, [_VP, _VP, _VP, _VP, _U64, _VP, _VP, _VP, _VP]),
    "anqs_batch_create": (C.c_int, [C.POINTER(_VP), C.c_int]),
    "anqs_batch_destroy": (C.c_int, [_VP]),
    "anqs_batched_local_energy": (C.c_int, [_VP, _VP, C.c_int, _VP]),
    "anqs_batch_set_schedule": (C.c_int, [_VP, C.c_int, C.c_int]),
    "anqs_batch_get_schedule": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "anqs_batch_autotune": (C.c_int, [_VP, _VP, C.c_int, _VP, C.POINTER(C.c_float)]),
    "anqs_launch_count": (C.c_int, [C.POINTER(_U64)]),
    "anqs_profile_enable": (C.c_int, [C.c_int]),
    "anqs_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_char_p), C.POINTER(_U64), C.POINTER(C.c_double)]),
}

_lib = None


def load(path: str | None = None):
    """Load libanqs.so; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libanqs is not built ({p} missing); run __graft_entry__.build() "
                           "or python paper_2310_04166_gb300/build.py")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(code: int):
    if code != ANQS_OK:
        buf = C.create_string_buffer(512)
        load().anqs_last_error(buf, 512)
        raise AnqsError(code, buf.value.decode(errors="replace"))
