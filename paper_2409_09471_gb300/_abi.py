"""ctypes view of the C ABI in ``include/ttsg.h`` (structures, prototypes,
status codes) and the loader of the in-tree ``libttsg.so``."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttsg.so")

MODE_FP64, MODE_FP32, MODE_TF32, MODE_BF16 = 0, 1, 2, 3
STATUS = {0: "TT_OK", 1: "TT_ERR_ARG", 2: "TT_ERR_WORKSPACE", 3: "TT_ERR_CUDA",
          4: "TT_ERR_TIMEOUT", 5: "TT_ERR_NOT_CONVERGED", 6: "TT_ERR_UNSUPPORTED",
          7: "TT_ERR_BREAKDOWN"}

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_vpp = ctypes.POINTER(ctypes.c_void_p)


class TTVec(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", c_i64p), ("rank", c_i64p), ("core", c_vpp)]


class TTVecOut(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", c_i64p), ("cap", c_i64p), ("rank", c_i64p),
                ("core", c_vpp)]


class TTOp(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", c_i64p), ("rank", c_i64p), ("core", c_vpp)]


class TTPrecond(ctypes.Structure):
    _fields_ = [("zeta", ctypes.c_int), ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("beta", ctypes.POINTER(ctypes.c_double)), ("A1d", c_vpp)]


class SolverParams(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int), ("s", ctypes.c_int), ("tol", ctypes.c_double),
                ("round_tol", ctypes.c_double), ("eta", ctypes.c_double),
                ("stop_safety", ctypes.c_double), ("rmax", ctypes.c_int64),
                ("r_sol", ctypes.c_int64), ("oversample", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("max_restarts", ctypes.c_int), ("mode", ctypes.c_int),
                ("final_stta", ctypes.c_int), ("ell", ctypes.c_int)]


class SolverInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int),
                ("sketched_res", ctypes.c_double), ("true_res", ctypes.c_double),
                ("max_rank", ctypes.c_int64), ("status", ctypes.c_int),
                ("seconds", ctypes.c_double), ("res_hist", ctypes.POINTER(ctypes.c_double)),
                ("rank_hist", ctypes.POINTER(ctypes.c_int64)), ("hist_cap", ctypes.c_int),
                ("svd_nonconverged", ctypes.c_int), ("svd_max_sweeps", ctypes.c_int),
                ("svd_mean_sweeps", ctypes.c_double), ("breakdowns", ctypes.c_int)]


class TTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2409_09471_gb300/build.py` "
            "(there is no fallback implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    V, P = ctypes.c_void_p, ctypes.POINTER
    sz, i64, u64, dbl, cint = ctypes.c_size_t, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    protos = {
        "tt_version": (ctypes.c_char_p, []),
        "tt_last_error": (ctypes.c_char_p, []),
        "tt_matvec": (cint, [cint, P(TTOp), P(TTVec), P(TTVec), V, sz, V]),
        "tt_matvec_workspace": (sz, [cint, P(TTOp), P(TTVec)]),
        "tt_sketch": (cint, [cint, P(TTVec), i64, c_vpp, V, V, sz, V]),
        "tt_sketch_workspace": (sz, [cint, P(TTVec), i64]),
        "tt_dot": (cint, [cint, P(TTVec), P(TTVec), V, V, sz, V]),
        "tt_sketch_factors": (cint, [cint, cint, c_i64p, i64, u64, c_vpp, V]),
        "tt_dot_workspace": (sz, [cint, P(TTVec), P(TTVec)]),
        "tt_dot_noalloc": (cint, [cint, P(TTVec), P(TTVec), V, V]),
        "tt_round_rand": (cint, [cint, cint, P(TTVec), P(dbl), dbl, i64, i64, u64, c_vpp, c_i64p,
                                 P(TTVecOut), V, sz, V]),
        "tt_round_rand_workspace": (sz, [cint, cint, P(TTVec), i64, i64]),
        "tt_gaussian": (cint, [cint, V, i64, u64, u64, dbl, V]),
        "tt_qr_f64": (cint, [cint, V, i64, i64, i64, i64, V, V, V, sz, V]),
        "tt_qr_f64_workspace": (sz, [i64, i64]),
        "tt_lstsq_f64": (cint, [V, i64, i64, V, V, V, V, sz, V]),
        "tt_lstsq_f64_workspace": (sz, [i64, i64]),
        "tt_sgmres_solve": (cint, [P(TTOp), P(TTVec), P(SolverParams), P(TTVecOut),
                                   P(SolverInfo), V, sz, V]),
        "tt_sgmres_solve_workspace": (sz, [P(TTOp), P(TTVec), P(SolverParams)]),
        "tt_sgmres_solve_batched": (cint, [P(TTOp), cint, P(TTVec), P(SolverParams), P(TTVecOut),
                                           P(SolverInfo), cint, V, sz]),
        "tt_sgmres_solve_batched_workspace": (sz, [P(TTOp), cint, P(TTVec), P(SolverParams), cint]),
        "tt_qr_f64_batched": (cint, [cint, cint, c_vpp, c_i64p, c_i64p, c_vpp, c_vpp, V, sz, V]),
        "tt_qr_f64_batched_workspace": (sz, [cint, c_i64p, c_i64p]),
        "tt_dot_grad": (cint, [cint, P(TTVec), P(TTVec), c_vpp, V, sz, V]),
        "tt_dot_grad_workspace": (sz, [cint, P(TTVec), P(TTVec)]),
        "tt_local_dots": (cint, [cint, P(TTVec), P(TTVec), c_vpp, V, V, sz, V]),
        "tt_local_dots_workspace": (sz, [cint, P(TTVec), P(TTVec)]),
        "tt_kron_sum_op": (cint, [cint, cint, c_i64p, c_vpp, P(dbl), c_vpp, V]),
        "tt_op_transpose": (cint, [cint, P(TTOp), c_vpp, V]),
        "tt_stta_sketch": (cint, [cint, P(TTVec), dbl, cint, P(TTVec), P(TTVec), c_vpp, c_vpp,
                                  V, sz, V]),
        "tt_stta_sketch_workspace": (sz, [cint, P(TTVec), P(TTVec), P(TTVec)]),
        "tt_stta_recover": (cint, [cint, c_i64p, c_i64p, c_i64p, c_vpp, c_vpp, dbl, c_vpp, V, sz,
                                   V]),
        "tt_stta_recover_workspace": (sz, [cint, c_i64p, c_i64p, c_i64p]),
        "tt_exp_sum_coefficients": (cint, [dbl, dbl, dbl, cint, P(dbl), P(dbl)]),
        "tt_precond_apply": (cint, [cint, P(TTPrecond), P(TTVec), dbl, i64, i64, u64,
                                    P(TTVecOut), V, sz, V]),
        "tt_precond_apply_workspace": (sz, [cint, P(TTPrecond), P(TTVec), i64, i64]),
        "tt_spgmres_solve": (cint, [P(TTOp), P(TTPrecond), P(TTVec), P(SolverParams),
                                    P(TTVecOut), P(SolverInfo), V, sz, V]),
        "tt_spgmres_solve_workspace": (sz, [P(TTOp), P(TTPrecond), P(TTVec), P(SolverParams)]),
        "tt_profile": (cint, [cint]),
        "tt_profile_read": (cint, [cint, P(dbl), c_i64p, P(dbl), P(dbl)]),
        "tt_launch_count": (i64, []),
    }
    for name, (res, args) in protos.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def check(rc: int):
    if rc != 0:
        raise TTError(rc, lib.tt_last_error().decode())
