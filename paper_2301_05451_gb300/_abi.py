"""ctypes binding of the C ABI in include/tdq.h (argument marshalling only).

The library must be built (``paper_2301_05451_gb300.build.build()``); loading
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdq.so")

TDQ_OK, TDQ_ERR_ARG, TDQ_ERR_OOM, TDQ_ERR_CUDA, TDQ_ERR_TIMEOUT, TDQ_ERR_NONFINITE, \
    TDQ_ERR_UNSUPPORTED, TDQ_ERR_STATE = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_OOM", "ERR_CUDA", "ERR_TIMEOUT", "ERR_NONFINITE",
                "ERR_UNSUPPORTED", "ERR_STATE"]
GATES = {"H": 0, "X": 1, "Y": 2, "Z": 3, "RX": 4, "RY": 5, "RZ": 6, "U3": 7, "CNOT": 8, "CZ": 9,
         "RZZ": 10}
TDQ_FIXED = -1


def TDQ_INPUT(j):
    return -2 - j


TDQ_OUT_EXPVAL, TDQ_OUT_AMPLITUDE, TDQ_OUT_STATE, TDQ_OUT_PROBS = 0, 1, 2, 3
TDQ_GRAD_NONE, TDQ_GRAD_ADJOINT, TDQ_GRAD_PARAM_SHIFT = 0, 1, 2


class TdqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


class CompileOpts(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("output", ctypes.c_int), ("grad", ctypes.c_int),
                ("device", ctypes.c_int), ("max_smem_qubits", ctypes.c_int),
                ("tile_qubits", ctypes.c_int), ("plain", ctypes.c_int),
                ("workspace_bytes", ctypes.c_int64), ("record_timings", ctypes.c_int),
                ("interpret", ctypes.c_int), ("fwd_reg_bits", ctypes.c_int), ("rev_reg_bits", ctypes.c_int),
                ("subtree_log2", ctypes.c_int), ("autotune", ctypes.c_int), ("tc_min_log2", ctypes.c_int)]


class NetOpts(ctypes.Structure):
    _fields_ = [("output", ctypes.c_int), ("index", ctypes.c_int), ("lightcone", ctypes.c_int),
                ("split_2q", ctypes.c_int), ("hyper", ctypes.c_int)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("seed", ctypes.c_uint64), ("temperature", ctypes.c_double),
                ("target_log2", ctypes.c_int), ("repeats", ctypes.c_int), ("slice_trials", ctypes.c_int),
                ("slice_final", ctypes.c_int), ("rank_simplify", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("log2_flops_per_slice", ctypes.c_double), ("flops", ctypes.c_double),
                ("max_log2_width", ctypes.c_int), ("n_sliced", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("log2_bytes_per_slice", ctypes.c_double)]


TDQ_PATH_GREEDY, TDQ_PATH_RANDOM_GREEDY, TDQ_PATH_PARTITION = 0, 1, 2

# name -> (restype, argtypes); every symbol declared in include/tdq.h
_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)
_i = ctypes.c_int
SIGNATURES = {
    "tdq_last_error": (ctypes.c_char_p, []),
    "tdq_version": (_i, []),
    "tdq_circuit_create": (_i, [_i, ctypes.POINTER(_vp)]),
    "tdq_circuit_gate": (_i, [_vp, _i, _ip, _i, _ip, _dp]),
    "tdq_circuit_observable": (_i, [_vp, _ip, _i, ctypes.c_double, _i]),
    "tdq_circuit_amplitude": (_i, [_vp, ctypes.POINTER(ctypes.c_uint8)]),
    "tdq_circuit_info": (_i, [_vp, _ip, _ip, _ip, _ip, _ip, _ip]),
    "tdq_circuit_destroy": (_i, [_vp]),
    "tdq_network_build": (_i, [_vp, ctypes.POINTER(NetOpts), ctypes.POINTER(_vp)]),
    "tdq_network_info": (_i, [_vp, _ip, _ip, _ip, _ip]),
    "tdq_network_tensor": (_i, [_vp, _i, _ip, _ip, _ip, _ip, _ip, _ip]),
    "tdq_network_tensor_flips": (_i, [_vp, _i, _ip]),
    "tdq_network_destroy": (_i, [_vp]),
    "tdq_plan_find": (_i, [_vp, ctypes.POINTER(PlanOpts), ctypes.POINTER(_vp)]),
    "tdq_plan_from_path": (_i, [_vp, _ip, _i, _ip, _i, ctypes.POINTER(_vp)]),
    "tdq_plan_stats": (_i, [_vp, ctypes.POINTER(Stats)]),
    "tdq_plan_path": (_i, [_vp, _ip, _ip]),
    "tdq_plan_destroy": (_i, [_vp]),
    "tdq_compile_sweep": (_i, [_vp, ctypes.POINTER(CompileOpts), ctypes.POINTER(_vp)]),
    "tdq_compile_multi": (_i, [ctypes.POINTER(_vp), _ip, _i, ctypes.POINTER(CompileOpts), ctypes.POINTER(_vp)]),
    "tdq_multi_source": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i, ctypes.c_char_p, ctypes.c_size_t,
                              ctypes.POINTER(ctypes.c_size_t)]),
    "tdq_exec_config": (_i, [_vp, _ip]),
    "tdq_multi_layout": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int64), _ip]),
    "tdq_sweep_source": (_i, [_vp, _i, _i, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "tdq_plan_compile": (_i, [_vp, ctypes.POINTER(CompileOpts), ctypes.POINTER(_vp)]),
    "tdq_execute": (_i, [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]),
    "tdq_exec_status": (_i, [_vp]),
    "tdq_exec_set_initial_state": (_i, [_vp, _vp, ctypes.c_int64]),
    "tdq_cgemm_nt": (_i, [_i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]),
    "tdq_cgemm_nt_bounded": (_i, [_i, _i, _i, _i, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp]),
    "tdq_costmodel_create": (_i, [_i, _i, ctypes.c_uint64, _i, ctypes.POINTER(_vp)]),
    "tdq_costmodel_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), _ip, _i]),
    "tdq_costmodel_loss_grad": (_i, [_vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "tdq_costmodel_adam_step": (_i, [_vp, ctypes.c_float, _vp]),
    "tdq_costmodel_train": (_i, [_vp, _vp, _vp, _i, _i, ctypes.c_float, _vp, _vp]),
    "tdq_costmodel_predict": (_i, [_vp, _vp, _i, _vp, _vp]),
    "tdq_costmodel_destroy": (_i, [_vp]),
    "tdq_execute_param_shift_noalloc": (_i, [_vp, _i, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]),
    "tdq_exec_launches": (_i, [_vp]),
    "tdq_exec_timings": (_i, [_vp, ctypes.POINTER(ctypes.c_float), _i, _ip]),
    "tdq_exec_set_slice_range": (_i, [_vp, ctypes.c_int64, ctypes.c_int64]),
    "tdq_exec_launch_work": (_i, [_vp, _dp, _dp, _ip, _i, _ip]),
    "tdq_plan_features": (_i, [_vp, _i, ctypes.c_int64, ctypes.POINTER(ctypes.c_float), _i, _ip, _ip]),
    "tdq_exec_work": (_i, [_vp, _dp, _dp, _ip]),
    "tdq_exec_destroy": (_i, [_vp]),
}

_lib = None


def lib():
    """Load libtdq.so (raises if it is missing: the library has no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libtdq.so is not built; run paper_2301_05451_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != TDQ_OK:
        msg = lib().tdq_last_error()
        raise TdqError(status, msg.decode() if msg else "")


def call(name, *args):
    check(getattr(lib(), name)(*args))


def int_array(vals):
    vals = list(vals)
    return (ctypes.c_int * max(len(vals), 1))(*vals)


def double_array(vals):
    vals = list(vals)
    return (ctypes.c_double * max(len(vals), 1))(*vals)
