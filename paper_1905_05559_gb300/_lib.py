"""ctypes declarations of the C ABI in include/hessmlp.h."""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhessmlp.so")

HESS_OK = 0
HESS_ERR_INVALID_ARG = 1
HESS_ERR_OOM = 2
HESS_ERR_CUDA = 3
HESS_ERR_RANK_DEFICIENT = 4
HESS_ERR_NOT_CONVERGED = 5
HESS_ERR_TIMEOUT = 6
HESS_ERR_ADMISSION = 7
HESS_ERR_UNSUPPORTED = 8

STATUS_NAMES = {
    0: "HESS_OK", 1: "HESS_ERR_INVALID_ARG", 2: "HESS_ERR_OOM", 3: "HESS_ERR_CUDA",
    4: "HESS_ERR_RANK_DEFICIENT", 5: "HESS_ERR_NOT_CONVERGED", 6: "HESS_ERR_TIMEOUT",
    7: "HESS_ERR_ADMISSION", 8: "HESS_ERR_UNSUPPORTED",
}

ACT = {"sigmoid": 0, "tanh": 1, "relu": 2}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16x3": 3}

# every symbol the header declares
EXPORTS = (
    "hess_mlp_create", "hess_mlp_destroy", "hess_mlp_num_params", "hess_mlp_set_params",
    "hess_mlp_set_stream", "per_example_grads", "opg", "exact_hessian", "opg_topk_eig",
    "hess_param_permutation", "hess_last_error", "hess_timing_enable", "hess_timing_read",
    "hess_launch_count", "per_example_grads_noalloc", "hess_server_create",
    "hess_server_add_network", "hess_server_submit", "hess_server_wait", "hess_server_destroy",
    "hess_mlp_set_operand_limit", "hess_batch_create", "hess_batch_run", "hess_batch_destroy",
    "hess_autotune", "hess_autotune_entries", "hess_autotune_save", "hess_autotune_load",
    "hess_batch_set_graphs", "hess_curvature", "hessian_vector_products", "hessian_topk_eig",
    "hess_approx_form", "hess_approx_apply", "hessian_minibatches", "opg_topk_eig_streaming",
    "hess_check_devmath", "hess_debug_set_barrier_limit", "hess_probe_fp64", "hess_mlp_set_eig_blocks",
    "hess_server_wait_timed", "opg_topk_eig_lowmem",
)

REQUEST_KIND = {"hessian": 0, "opg": 1, "eig": 2}


class HessRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("net", ctypes.c_int), ("X", ctypes.c_void_p),
                ("Y", ctypes.c_void_p), ("N", ctypes.c_int64), ("prec", ctypes.c_int),
                ("k", ctypes.c_int), ("out", ctypes.c_void_p),
                ("evals", ctypes.POINTER(ctypes.c_double))]

class BatchItem(ctypes.Structure):
    _fields_ = [("net", ctypes.c_void_p), ("X", ctypes.c_void_p), ("Y", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("opg", ctypes.c_void_p), ("hessian", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("waves", ctypes.c_int), ("items_chunked", ctypes.c_int),
                ("tiles", ctypes.c_int64), ("flops", ctypes.c_double),
                ("launch_ms", ctypes.c_double), ("graph_replayed", ctypes.c_int)]


KERNEL_CLASS = {"syrk": 0, "hcontract": 1, "grads": 2, "rop": 3, "eig": 4, "hrest": 5, "hvp": 6,
                "hlanczos": 7, "approx": 8, "gram": 9, "digits": 10, "lanczos": 11, "tridiag": 12,
                "backproj": 13, "lowmem": 14}


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("sm_ms", ctypes.c_double)]


class HessDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("widths", ctypes.POINTER(ctypes.c_int)),
                ("act", ctypes.POINTER(ctypes.c_int))]


class HessError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the in-tree library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run paper_1905_05559_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    st = ctypes.c_int
    lib.hess_mlp_create.argtypes = [ctypes.POINTER(HessDesc), vp, vp, ctypes.POINTER(vp)]
    lib.hess_mlp_create.restype = st
    lib.hess_mlp_destroy.argtypes = [vp]
    lib.hess_mlp_destroy.restype = st
    lib.hess_mlp_num_params.argtypes = [vp]
    lib.hess_mlp_num_params.restype = i64
    lib.hess_mlp_set_params.argtypes = [vp, vp]
    lib.hess_mlp_set_params.restype = st
    lib.hess_mlp_set_stream.argtypes = [vp, vp]
    lib.hess_mlp_set_stream.restype = st
    for name in ("per_example_grads", "opg", "exact_hessian"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp]
        f.restype = st
    lib.opg_topk_eig.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.opg_topk_eig.restype = st
    lib.hess_curvature.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp]
    lib.hess_curvature.restype = st
    lib.hessian_vector_products.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, ctypes.c_int, vp]
    lib.hessian_vector_products.restype = st
    lib.hessian_topk_eig.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, vp,
                                     ctypes.POINTER(ctypes.c_int)]
    lib.hessian_topk_eig.restype = st
    lib.opg_topk_eig_streaming.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, i64, vp, vp]
    lib.opg_topk_eig_streaming.restype = st
    lib.opg_topk_eig_lowmem.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, vp, vp,
                                        ctypes.POINTER(ctypes.c_int)]
    lib.opg_topk_eig_lowmem.restype = st
    lib.hessian_minibatches.argtypes = [vp, vp, vp, i64, i64, ctypes.c_int, vp]
    lib.hessian_minibatches.restype = st
    lib.hess_approx_form.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, vp]
    lib.hess_approx_form.restype = st
    lib.hess_approx_apply.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_double, vp,
                                      ctypes.c_int, vp, vp]
    lib.hess_approx_apply.restype = st
    lib.hess_param_permutation.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int64)]
    lib.hess_param_permutation.restype = st
    lib.hess_timing_enable.argtypes = [vp, ctypes.c_int]
    lib.hess_timing_enable.restype = st
    lib.hess_timing_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(KernelStats)]
    lib.hess_timing_read.restype = st
    lib.per_example_grads_noalloc.argtypes = [ctypes.POINTER(HessDesc), vp, vp, vp, i64, vp, vp]
    lib.per_example_grads_noalloc.restype = st
    lib.hess_server_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(vp)]
    lib.hess_server_create.restype = st
    lib.hess_server_add_network.argtypes = [vp, ctypes.POINTER(HessDesc), vp, ctypes.POINTER(ctypes.c_int)]
    lib.hess_server_add_network.restype = st
    lib.hess_server_submit.argtypes = [vp, ctypes.POINTER(HessRequest), ctypes.POINTER(ctypes.c_int64)]
    lib.hess_server_submit.restype = st
    lib.hess_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    lib.hess_server_wait.restype = st
    lib.hess_server_wait_timed.argtypes = [vp, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.hess_server_wait_timed.restype = st
    lib.hess_server_destroy.argtypes = [vp]
    lib.hess_server_destroy.restype = st
    lib.hess_mlp_set_operand_limit.argtypes = [vp, i64]
    lib.hess_mlp_set_operand_limit.restype = st
    lib.hess_mlp_set_eig_blocks.argtypes = [vp, ctypes.c_int]
    lib.hess_mlp_set_eig_blocks.restype = st
    lib.hess_batch_create.argtypes = [i64, vp, ctypes.POINTER(vp)]
    lib.hess_batch_create.restype = st
    lib.hess_batch_run.argtypes = [vp, ctypes.POINTER(BatchItem), ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(BatchInfo)]
    lib.hess_batch_run.restype = st
    lib.hess_batch_set_graphs.argtypes = [vp, ctypes.c_int]
    lib.hess_batch_set_graphs.restype = st
    lib.hess_batch_destroy.argtypes = [vp]
    lib.hess_batch_destroy.restype = st
    lib.hess_autotune.argtypes = [ctypes.c_int]
    lib.hess_autotune.restype = st
    lib.hess_autotune_entries.argtypes = []
    lib.hess_autotune_entries.restype = ctypes.c_int
    lib.hess_autotune_save.argtypes = [ctypes.c_char_p]
    lib.hess_autotune_save.restype = st
    lib.hess_autotune_load.argtypes = [ctypes.c_char_p]
    lib.hess_autotune_load.restype = st
    lib.hess_check_devmath.argtypes = [vp, i64, vp, vp]
    lib.hess_check_devmath.restype = st
    lib.hess_debug_set_barrier_limit.argtypes = [i64]
    lib.hess_debug_set_barrier_limit.restype = st
    lib.hess_probe_fp64.argtypes = [i64, ctypes.POINTER(ctypes.c_double), vp, vp]
    lib.hess_probe_fp64.restype = st
    lib.hess_launch_count.argtypes = []
    lib.hess_launch_count.restype = ctypes.c_int64
    lib.hess_last_error.argtypes = []
    lib.hess_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def last_error() -> str:
    return load().hess_last_error().decode(errors="replace")


def check(status: int, allow=()) -> int:
    if status != HESS_OK and status not in allow:
        raise HessError(status, last_error())
    return status
