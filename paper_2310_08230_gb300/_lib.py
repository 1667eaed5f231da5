"""ctypes binding of the C ABI in ``include/disco.h`` (argument marshalling only).

Every function keeps its C name. The library must have been built by
``paper_2310_08230_gb300.build.build()``; loading fails loudly otherwise — there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

DISCO_OK = 0
ERRORS = {
    -1: "DISCO_ERR_INVALID_ARG", -2: "DISCO_ERR_NONMANIFOLD", -3: "DISCO_ERR_GENUS_MISMATCH",
    -4: "DISCO_ERR_INFEASIBLE", -5: "DISCO_ERR_PRIMAL_FAILED", -6: "DISCO_ERR_TIMEOUT", -7: "DISCO_ERR_CUDA",
    -8: "DISCO_ERR_OOM", -9: "DISCO_ERR_NOT_READY", -10: "DISCO_ERR_RANGE", -11: "DISCO_ERR_INTERNAL",
}
globals().update({v: k for k, v in ERRORS.items()})

c_float_p = ctypes.POINTER(ctypes.c_float)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_uint8_p = ctypes.POINTER(ctypes.c_uint8)
c_double_p = ctypes.POINTER(ctypes.c_double)


class disco_mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32), ("V", ctypes.c_void_p), ("T", ctypes.c_void_p)]


class disco_opts(ctypes.Structure):
    _fields_ = [
        ("omega", ctypes.c_float), ("split_chunk", ctypes.c_int32), ("lb_every", ctypes.c_int32),
        ("conv_rel_tol", ctypes.c_double), ("primal_rounds", ctypes.c_int32), ("primal_inner_iters", ctypes.c_int32),
        ("perturb_delta0", ctypes.c_float), ("perturb_growth", ctypes.c_float), ("tie_tau", ctypes.c_float),
        ("propagate_limit", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
        ("host_threads", ctypes.c_int32), ("split_max_segments", ctypes.c_int32),
        ("graph_iters", ctypes.c_int32), ("autotune", ctypes.c_int32), ("normalize_costs", ctypes.c_int32),
        ("qn_memory", ctypes.c_int32), ("cost_model", ctypes.c_int32), ("tile_order", ctypes.c_int32),
    ]


class disco_info_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "nvars", "nrows", "nvars_free", "nvars_aux", "nbdds", "nslots", "nnodes", "max_layers", "max_width",
        "ntiles", "device_bytes", "iterations")] + [("constant", ctypes.c_double), ("build_ms", ctypes.c_double),
                                                   ("bytes_per_iter", ctypes.c_int64),
                                                   ("upload_ms", ctypes.c_double),
                                                   ("launch_geometry", ctypes.c_int64),
                                                   ("reserved", ctypes.c_int64 * 3)]


V, P, I32, I64, D, F = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_float
SIGNATURES = {
    "disco_default_opts": (ctypes.c_int, [ctypes.POINTER(disco_opts)]),
    "disco_pair_costs": (ctypes.c_int, [P, P, I32, I32, I32, P, P]),
    "disco_pair_distances": (ctypes.c_int, [P, P, I32, I32, I32, P, P]),
    "disco_candidates": (ctypes.c_int, [P, I32, I32, I32, ctypes.POINTER(disco_mesh), ctypes.POINTER(disco_mesh), P, P]),
    "disco_candidates_noalloc": (ctypes.c_int, [P, I32, I32, I32, ctypes.POINTER(disco_mesh),
                                                ctypes.POINTER(disco_mesh), P, P]),
    "disco_build": (ctypes.c_int, [ctypes.POINTER(disco_mesh), ctypes.POINTER(disco_mesh), P, P,
                                   ctypes.POINTER(disco_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "disco_build_batch": (ctypes.c_int, [I32, ctypes.POINTER(disco_mesh), ctypes.POINTER(disco_mesh), P, P,
                                         ctypes.POINTER(disco_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "disco_batch_size": (ctypes.c_int, [P, c_int32_p]),
    "disco_lower_bounds": (ctypes.c_int, [P, c_double_p, I32]),
    "disco_instance_info": (ctypes.c_int, [P, I32, ctypes.POINTER(disco_info_t)]),
    "disco_primal_batch": (ctypes.c_int, [P, P, I64, c_double_p, c_int32_p, I32]),
    "disco_compile_host": (ctypes.c_int, [ctypes.POINTER(disco_mesh), ctypes.POINTER(disco_mesh), P, P, I32, I32,
                                          ctypes.POINTER(disco_info_t), P, P, I64, P, I64]),
    "disco_dual": (ctypes.c_int, [P, I32]),
    "disco_lower_bound": (ctypes.c_int, [P, c_double_p]),
    "disco_converge": (ctypes.c_int, [P, I32, c_int32_p, c_double_p]),
    "disco_min_marginals": (ctypes.c_int, [P, P, I64]),
    "disco_primal": (ctypes.c_int, [P, P, I64, c_double_p]),
    "disco_get_state": (ctypes.c_int, [P, P, I64, P, I64]),
    "disco_set_state": (ctypes.c_int, [P, P, I64, P, I64]),
    "disco_info": (ctypes.c_int, [P, ctypes.POINTER(disco_info_t)]),
    "disco_free": (None, [P]),
    "disco_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "disco_last_error": (ctypes.c_char_p, []),
    "disco_kernel_launches": (ctypes.c_int64, []),
    "disco_record": (ctypes.c_int, [P, I32, I32]),
    "disco_grad": (ctypes.c_int, [P, P, I64]),
    "disco_dual_qn": (ctypes.c_int, [P, I32, I32]),
    "disco_point_map": (ctypes.c_int, [P, P, I64, P, I64, ctypes.POINTER(ctypes.c_int64)]),
    "disco_candidates_coarse_to_fine": (ctypes.c_int, [P, I64, P, I32, P, I32, I32, ctypes.POINTER(disco_mesh),
                                                       ctypes.POINTER(disco_mesh), P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library {LIB} is missing: run __graft_entry__.build() "
                               "(paper_2310_08230_gb300.build.build()) first")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class DiscoError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().disco_last_error().decode(errors="replace")
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != DISCO_OK:
        raise DiscoError(code, where)
    return code


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
