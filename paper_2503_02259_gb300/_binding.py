"""ctypes binding of libgp.so (include/gp.h).

Argument marshalling only: every arithmetic step runs in the library's CUDA
kernels.  Device memory comes from PyTorch tensors (outputs and workspaces are
allocated with torch on the tensors' device); streams are torch's current
stream.  If libgp.so is missing the first call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_size_t, c_uint64, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgp.so")

GP_OK = 0
GP_ERR_ARG = 1
GP_ERR_CUDA = 2
GP_ERR_OOM = 3
GP_ERR_NOT_CONVERGED = 4
GP_ERR_BREAKDOWN = 5
GP_ERR_TIMEOUT = 6
GP_ERR_UNIMPLEMENTED = 7
GP_ERR_NUMERIC = 8

GAUSSIAN = 0
MATERN32 = 1

PREC_FP32 = 0
PREC_TF32 = 1
PREC_BF16 = 2
PREC_TF32X3 = 3
PREC_BF16X3 = 4
PREC_SAME = -1   # slq_prec: the same arithmetic as prec

OP_MATMUL = 0
OP_GRAD_MATMUL = 1
OP_PCG = 2
OP_SLQ = 3
OP_LOSS_GRAD = 4
OP_PREDICT = 5
OP_RESIDUAL = 6
OP_PREDICT_VAR = 7
OP_LOSS_GRAD_BATCH = 8
OP_NYSTROM = 9
MAX_PRECOND_RANK = 4096

RESIDUAL_PAIR = 0   # compensated FP32-pair sums (the refinement default)
RESIDUAL_FP64 = 1   # FP64 entries and sums (the checker)

MAX_DIM = 16
MAX_COLS = 128
MAX_LANCZOS = 64


class gp_theta(ctypes.Structure):
    _fields_ = [("s", c_double), ("f", c_double), ("l", c_double)]


class gp_problem(ctypes.Structure):
    _fields_ = [("X", c_void_p), ("n", c_int64), ("d", c_int32), ("kernel", c_int32),
                ("theta", gp_theta), ("ls", c_void_p)]


class gp_solve_opts(ctypes.Structure):
    _fields_ = [("nprobe", c_int32), ("nlanczos", c_int32), ("cg_maxit", c_int32),
                ("prec", c_int32), ("cg_rtol", c_double), ("refine_rtol", c_double),
                ("seed", c_uint64), ("probes", c_void_p), ("refine_maxit", c_int32),
                ("slq_prec", c_int32), ("refine_residual", c_int32),
                ("precond_rank", c_int32), ("precond_tol", c_double)]


class gp_loss_info(ctypes.Structure):
    _fields_ = [("yalpha", c_double), ("logdet", c_double), ("logdet_stderr", c_double),
                ("quad", c_double * 3), ("trace", c_double * 3), ("trace_stderr", c_double * 3),
                ("cg_iters", c_int32), ("refine_steps", c_int32), ("relres_y", c_double),
                ("relres_max", c_double), ("logdet_m", c_double), ("trace_m", c_double * 3)]

    def as_dict(self) -> dict:
        return {"yalpha": self.yalpha, "logdet": self.logdet, "logdet_stderr": self.logdet_stderr,
                "quad": list(self.quad), "trace": list(self.trace),
                "trace_stderr": list(self.trace_stderr), "cg_iters": self.cg_iters,
                "refine_steps": self.refine_steps, "relres_y": self.relres_y,
                "relres_max": self.relres_max, "logdet_m": self.logdet_m,
                "trace_m": list(self.trace_m)}


class gp_request(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("d", c_int32), ("n", c_int64), ("kernel", c_int32),
                ("nprobe", c_int32), ("theta", gp_theta), ("X", c_void_p), ("y", c_void_p),
                ("Xstar", c_void_p), ("m", c_int64), ("cg_maxit", c_int32), ("nlanczos", c_int32),
                ("cg_rtol", c_double), ("seed", c_uint64), ("prec", c_int32), ("slq_prec", c_int32)]


class gp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("refused", c_int64),
                ("peak_active", c_int64), ("peak_bytes", c_size_t), ("budget_bytes", c_size_t),
                ("batches", c_int64), ("batched_requests", c_int64), ("largest_batch", c_int64)]


class gp_result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("cg_iters", c_int32), ("loss", c_double),
                ("grad", c_double * 3), ("relres", c_double), ("t_submit_s", c_double),
                ("t_start_s", c_double), ("t_done_s", c_double), ("mu", c_void_p)]


# Every exported symbol of include/gp.h with its ctypes prototype.
PROTOTYPES = {
    "gp_version": (c_char_p, []),
    "gp_last_error": (c_char_p, []),
    "gp_status_string": (c_char_p, [c_int32]),
    "gp_workspace_bytes": (c_size_t, [c_int32, POINTER(gp_problem), c_int32, POINTER(gp_solve_opts)]),
    "gp_kernel_matmul": (c_int32, [POINTER(gp_problem), c_void_p, c_int32, c_void_p, c_int32,
                                   c_void_p, c_size_t, c_void_p]),
    "gp_kernel_matmul_noalloc": (c_int32, [POINTER(gp_problem), c_void_p, c_int32, c_void_p,
                                           c_void_p]),
    "gp_kernel_grad_matmul": (c_int32, [POINTER(gp_problem), c_void_p, c_int32, c_void_p, c_void_p,
                                        c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "gp_pcg_solve": (c_int32, [POINTER(gp_problem), c_void_p, c_int32, c_void_p,
                               POINTER(gp_solve_opts), POINTER(c_int32), POINTER(c_double),
                               c_void_p, c_size_t, c_void_p]),
    "gp_pcg_solve_refined": (c_int32, [POINTER(gp_problem), c_void_p, c_int32, c_void_p,
                                       POINTER(gp_solve_opts), POINTER(c_int32), POINTER(c_double),
                                       c_void_p, c_size_t, c_void_p]),
    "gp_nystrom_apply": (c_int32, [POINTER(gp_problem), c_int32, c_double, c_void_p, c_int32,
                                   c_void_p, c_void_p, POINTER(c_int64), POINTER(c_int32),
                                   c_void_p, c_size_t, c_void_p]),
    "gp_true_residual": (c_int32, [POINTER(gp_problem), c_void_p, c_void_p, c_int32,
                                   POINTER(c_double), c_void_p, c_size_t, c_void_p]),
    "gp_residual_rows": (c_int32, [POINTER(gp_problem), c_void_p, c_void_p, c_int32, c_void_p,
                                   c_int64, c_int32, c_void_p, POINTER(c_double), c_void_p,
                                   c_size_t, c_void_p]),
    "gp_slq_logdet": (c_int32, [POINTER(gp_problem), POINTER(gp_solve_opts), POINTER(c_double),
                                POINTER(c_double), c_void_p, c_size_t, c_void_p]),
    "gp_loss_and_grad": (c_int32, [POINTER(gp_problem), c_void_p, POINTER(gp_solve_opts),
                                   POINTER(c_double), POINTER(c_double), POINTER(gp_loss_info),
                                   c_void_p, c_size_t, c_void_p]),
    "gp_loss_and_grad_batch": (c_int32, [c_int32, POINTER(gp_problem), POINTER(c_void_p),
                                         POINTER(gp_solve_opts), POINTER(c_double),
                                         POINTER(c_double), POINTER(gp_loss_info),
                                         POINTER(c_int32), POINTER(c_void_p), POINTER(c_size_t),
                                         c_void_p]),
    "gp_nll_forward": (c_int32, [POINTER(gp_problem), c_void_p, POINTER(gp_solve_opts), c_void_p,
                                 POINTER(c_double), POINTER(gp_loss_info), c_void_p, c_size_t,
                                 c_void_p]),
    "gp_nll_backward": (c_int32, [POINTER(gp_problem), POINTER(gp_solve_opts), c_void_p,
                                  POINTER(c_double), POINTER(gp_loss_info), c_void_p, c_size_t,
                                  c_void_p]),
    "gp_predict_mean": (c_int32, [POINTER(gp_problem), c_void_p, c_void_p, c_int64, c_void_p,
                                  c_int32, c_void_p, c_size_t, c_void_p]),
    "gp_predict_var": (c_int32, [POINTER(gp_problem), c_void_p, c_int64, c_void_p,
                                 POINTER(gp_solve_opts), POINTER(c_int32), POINTER(c_double),
                                 c_void_p, c_size_t, c_void_p]),
    "gp_generate_probes": (c_int32, [c_int64, c_int32, c_uint64, c_void_p, c_int64, c_void_p]),
    "gp_profile_begin": (c_int32, []),
    "gp_profile_end": (c_int32, [POINTER(c_double), POINTER(c_int64), POINTER(c_int64)]),
    "gp_measure_pipe_rates": (c_int32, [POINTER(c_double), POINTER(c_double), c_void_p]),
    "gp_server_create": (c_int32, [c_size_t, c_int32, POINTER(c_void_p)]),
    "gp_server_create_batched": (c_int32, [c_size_t, c_int32, c_int32, POINTER(c_void_p)]),
    "gp_server_submit": (c_int32, [c_void_p, POINTER(gp_request), POINTER(c_uint64)]),
    "gp_server_poll": (c_int32, [c_void_p, c_uint64, POINTER(gp_result)]),
    "gp_server_drain": (c_int32, [c_void_p, c_double]),
    "gp_server_get_stats": (c_int32, [c_void_p, POINTER(gp_server_stats)]),
    "gp_server_footprint": (c_size_t, [POINTER(gp_request)]),
    "gp_server_destroy": (c_int32, [c_void_p]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libgp.so (once) and declare the prototypes; raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libgp.so is not built ({LIB_PATH}); run `python -m paper_2503_02259_gb300.build`. "
                "There is no CPU fallback.")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GPError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        self.status = status
        msg = L.gp_last_error().decode()
        name = L.gp_status_string(status).decode()
        super().__init__(f"{where}: {name}: {msg}")


def check(status: int, where: str) -> None:
    if status != GP_OK:
        raise GPError(status, where)
