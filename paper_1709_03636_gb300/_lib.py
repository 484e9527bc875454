"""ctypes binding of libqtc.so (argument marshalling only).

The shared library is built in-tree by ``paper_1709_03636_gb300.build``.
There is no fallback: if it is missing, importing the binding raises.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqtc.so")

c_int, c_int32, c_double, c_void_p, c_size_t, c_uint64 = (
    ctypes.c_int, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t,
    ctypes.c_uint64)
P = ctypes.POINTER


class qtc_observable(ctypes.Structure):
    _fields_ = [("kind", c_int), ("u", c_int), ("v", c_int),
                ("pauli", ctypes.c_char_p), ("bits", P(ctypes.c_uint8))]


class qtc_plan_opts(ctypes.Structure):
    _fields_ = [("kind", c_int), ("seed", c_uint64), ("max_rejections", c_int),
                ("restarts", c_int), ("budget_ms", c_double)]


class qtc_plan_info(ctypes.Structure):
    _fields_ = [("n_tensors", c_int), ("n_labels", c_int), ("n_steps", c_int),
                ("max_rank", c_int), ("cmacs", c_double), ("bytes_c64", c_double),
                ("lg_width", c_double)]


class qtc_batch_info(ctypes.Structure):
    _fields_ = [("n_networks", c_int), ("n_params", c_int), ("max_rank", c_int),
                ("n_steps_total", c_int), ("cmacs", c_double), ("bytes_c64", c_double),
                ("n_smem_networks", c_int), ("n_global_networks", c_int),
                ("grad_cmacs", c_double), ("grad_bytes_c64", c_double)]


class qtc_program_info(ctypes.Structure):
    _fields_ = [("graph", c_int), ("n_waves", c_int), ("n_tasks", c_int),
                ("n_global_steps", c_int), ("n_smem_tasks", c_int), ("smem_bytes", c_int),
                ("work_bytes", c_double), ("table_bytes", c_double), ("n_gemm_steps", c_int),
                ("warp_teams", c_int), ("n_ops", c_int), ("n_warp_steps", c_int),
                ("max_warp_steps", c_int), ("n_solo_steps", c_int), ("stage_ops", c_int),
                ("net_global_bytes", c_double), ("net_global_bytes_unshared", c_double),
                ("checkpoint_segments", c_int)]


# name -> (restype, argtypes)
SIGNATURES = {
    "qtc_last_error": (ctypes.c_char_p, []),
    "qtc_engine_create": (c_int, [c_int, c_void_p, c_size_t, P(c_void_p)]),
    "qtc_engine_destroy": (None, [c_void_p]),
    "qtc_engine_reset": (c_int, [c_void_p]),
    "qtc_engine_last_launches": (c_int, [c_void_p]),
    "qtc_circuit_create": (c_int, [c_int, c_int, P(c_void_p)]),
    "qtc_circuit_add_gate": (c_int, [c_void_p, c_int, P(c_int32), c_int, c_double, c_double]),
    "qtc_circuit_qaoa": (c_int, [c_int, P(c_int32), c_int, c_int, P(c_void_p)]),
    "qtc_plan_reuse": (c_int, [c_void_p, c_void_p, P(c_void_p)]),
    "qtc_circuit_qaoa_noisy": (c_int, [c_int, P(c_int32), c_int, c_int, c_int, c_double,
                                       P(c_void_p)]),
    "qtc_circuit_destroy": (None, [c_void_p]),
    "qtc_network_build": (c_int, [c_void_p, P(qtc_observable), c_int, c_int, P(c_void_p)]),
    "qtc_network_leaves": (c_int, [c_void_p, P(c_int32), P(c_int32), P(c_int32), P(c_int32),
                                   P(c_double), P(c_double), P(c_int32)]),
    "qtc_network_leaf_values": (c_int, [c_void_p, c_int, P(c_double), P(c_double), P(c_double)]),
    "qtc_network_destroy": (None, [c_void_p]),
    "qtc_plan_create": (c_int, [c_void_p, P(qtc_plan_opts), P(c_void_p)]),
    "qtc_plan_stats": (c_int, [c_void_p, P(qtc_plan_info)]),
    "qtc_plan_steps": (c_int, [c_void_p, P(c_int32), P(c_int32)]),
    "qtc_plan_step_shapes": (c_int, [c_void_p, P(c_int32)]),
    "qtc_plan_destroy": (None, [c_void_p]),
    "qtc_contract": (c_int, [c_void_p, c_void_p, P(c_double), c_int, c_void_p, P(c_double),
                             P(c_double)]),
    "qtc_batch_create": (c_int, [c_void_p, P(c_int32), c_int, c_int, c_int, P(qtc_plan_opts),
                                 P(c_void_p)]),
    "qtc_batch_stats": (c_int, [c_void_p, P(qtc_batch_info)]),
    "qtc_batch_destroy": (None, [c_void_p]),
    "qtc_batch_partition": (c_int, [c_void_p, c_int, c_int, P(c_int32), P(c_double)]),
    "qtc_batch_subset": (c_int, [c_void_p, P(c_int32), c_int, P(c_void_p)]),
    "qtc_batch_prepare": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "qtc_qaoa_expectation": (c_int, [c_void_p, c_void_p, P(c_double), P(c_double), c_int, c_int,
                                     c_void_p, P(c_double), P(c_double), P(c_double)]),
    "qtc_qaoa_expectation_device": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int,
                                            c_void_p, c_void_p]),
    "qtc_qaoa_expectation_static": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p,
                                            c_void_p]),
    "qtc_engine_set_limits": (c_int, [c_void_p, c_size_t, c_double]),
    "qtc_selftest_wait_timeout": (c_int, [c_void_p, c_void_p]),
    "qtc_engine_set_tile_mode": (c_int, [c_void_p, c_int]),
    "qtc_selftest_tile_steps": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int,
                                        P(c_double), P(c_int32)]),
    "qtc_engine_set_graph_options": (c_int, [c_void_p, c_int, c_int]),
    "qtc_engine_set_task_options": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
    "qtc_batch_launch_info": (c_int, [c_void_p, c_void_p, c_int, c_int, P(c_int32)]),
    "qtc_statevector_qaoa": (c_int, [c_void_p, c_void_p, P(c_double), P(c_double), c_int, c_int,
                                     c_void_p, P(c_double), P(c_double)]),
    "qtc_statevector_qaoa_device": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p,
                                            c_void_p]),
    "qtc_answer_string": (c_int, [c_void_p, c_void_p, P(c_double), c_int, P(qtc_plan_opts),
                                  c_uint64, c_void_p, P(ctypes.c_uint8), P(c_double)]),
    "qtc_batch_program_info": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_size_t, c_size_t,
                                       P(qtc_program_info)]),
}


def load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is not built; run paper_1709_03636_gb300.build.build() first "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()

STATUS = {0: "QTC_OK", 1: "QTC_ERR_INVALID", 2: "QTC_ERR_ARENA", 3: "QTC_ERR_TIMEOUT",
          4: "QTC_ERR_CUDA", 5: "QTC_ERR_UNSUPPORTED"}


class QtcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def check(status):
    if status != 0:
        raise QtcError(status, lib.qtc_last_error().decode())
