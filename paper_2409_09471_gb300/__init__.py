"""Python binding of the GB300 randomized sketched TT-GMRES library (libttsg.so).

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI declared in ``include/ttsg.h``.  PyTorch provides
device memory and the current CUDA stream.  The functions keep the C names:

``tt_matvec``, ``tt_sketch``, ``tt_dot``, ``tt_round_rand``, ``tt_gaussian``,
``tt_qr_f64``, ``tt_lstsq_f64``, ``tt_sgmres_solve``, and the adjoint helpers
``tt_dot_grad``, ``tt_local_dots``, ``tt_kron_sum_op``, ``tt_op_transpose``.
:func:`solve_loss` is a ``torch.autograd.Function`` over the solve whose
backward pass is the adjoint solve plus those backward contractions.

TT vectors are :class:`TT` objects (a list of contiguous CUDA tensors with
shapes ``[r_{k-1}, n_k, r_k]``); TT operators are lists of contiguous CUDA
tensors ``[R_{k-1}, n, n, R_k]``.  Importing this module fails loudly when the
compiled library is missing; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Sequence

import numpy as np
import torch

from ._abi import (lib, TTVec, TTVecOut, TTOp, TTPrecond, SolverParams, SolverInfo, MODE_FP64,
                   MODE_FP32, MODE_TF32, MODE_BF16, TTError, check, LIB_PATH)

__all__ = ["TT", "tt_matvec", "tt_sketch", "tt_sketch_factors", "tt_dot", "tt_round_rand", "tt_gaussian", "tt_qr_f64",
           "tt_lstsq_f64", "tt_sgmres_solve", "MODE_FP64", "MODE_FP32", "MODE_TF32", "MODE_BF16",
           "TTError",
           "LIB_PATH", "mode_dtype", "op_to_device", "tt_dot_grad", "tt_local_dots",
           "tt_kron_sum_op", "tt_op_transpose", "solve_loss", "tt_qr_f64_batched",
           "tt_sgmres_solve_batched", "tt_stta_sketch", "tt_stta_recover", "Precond",
           "exp_sum_coefficients", "tt_precond_apply", "tt_spgmres_solve"]


def mode_dtype(mode: int) -> torch.dtype:
    """Core dtype used by ``mode``."""
    return torch.float64 if mode == MODE_FP64 else torch.float32


class TT:
    """A TT vector on the device: ``cores[k]`` has shape ``[r_{k-1}, n_k, r_k]``."""

    def __init__(self, cores: Sequence[torch.Tensor]):
        self.cores = [c.contiguous() for c in cores]

    @property
    def d(self) -> int:
        return len(self.cores)

    @property
    def ns(self) -> List[int]:
        return [c.shape[1] for c in self.cores]

    @property
    def ranks(self) -> List[int]:
        return [c.shape[0] for c in self.cores] + [self.cores[-1].shape[2]]

    @classmethod
    def from_numpy(cls, cores, dtype=torch.float64, device="cuda"):
        return cls([torch.as_tensor(c, dtype=dtype, device=device) for c in cores])

    def numpy(self):
        return [c.detach().double().cpu().numpy() for c in self.cores]

    def to(self, dtype):
        return TT([c.to(dtype) for c in self.cores])

    def _desc(self):
        d = self.d
        n = (ctypes.c_int64 * d)(*self.ns)
        r = (ctypes.c_int64 * (d + 1))(*self.ranks)
        p = (ctypes.c_void_p * d)(*[c.data_ptr() for c in self.cores])
        keep = (n, r, p)
        return TTVec(d, n, r, p), keep


def op_to_device(op, dtype=torch.float64, device="cuda"):
    """TT operator cores (``[R_{k-1}, n_out, n_in, R_k]`` arrays or tensors) as
    contiguous device tensors of ``dtype`` (float64 for the solvers, the mode's
    dtype for :func:`tt_matvec`)."""
    return [torch.as_tensor(c, dtype=dtype, device=device).contiguous() for c in op]


def _op_desc(op):
    d = len(op)
    n = (ctypes.c_int64 * d)(*[c.shape[1] for c in op])
    r = (ctypes.c_int64 * (d + 1))(*([c.shape[0] for c in op] + [op[-1].shape[3]]))
    p = (ctypes.c_void_p * d)(*[c.data_ptr() for c in op])
    return TTOp(d, n, r, p), (n, r, p)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def _check_dtype(tensors, mode):
    want = mode_dtype(mode)
    for t in tensors:
        if t.dtype != want or not t.is_cuda or not t.is_contiguous():
            raise TTError(1, f"expected contiguous CUDA {want} tensors for mode {mode}")


def tt_matvec(op, x: TT, mode: int = MODE_FP64, stream=None) -> TT:
    """``A x`` without truncation; output ranks ``R_k r_k``."""
    _check_dtype(list(op) + x.cores, mode)
    R = [c.shape[0] for c in op] + [1]
    yr = [a * b for a, b in zip(R, x.ranks)]
    y = TT([torch.empty((yr[k], x.ns[k], yr[k + 1]), dtype=x.cores[0].dtype,
                        device=x.cores[0].device) for k in range(x.d)])
    od, k1 = _op_desc(op)
    xd, k2 = x._desc()
    yd, k3 = y._desc()
    ws = _workspace(lib.tt_matvec_workspace(mode, ctypes.byref(od), ctypes.byref(xd)),
                    x.cores[0].device)
    check(lib.tt_matvec(mode, ctypes.byref(od), ctypes.byref(xd), ctypes.byref(yd),
                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return y


def tt_sketch(x: TT, S: Sequence[torch.Tensor], mode: int = MODE_FP64, stream=None) -> torch.Tensor:
    """Khatri-Rao sketch ``S_odot x`` (float64 vector of length s)."""
    _check_dtype(list(S) + x.cores, mode)
    s = S[0].shape[0]
    out = torch.empty(s, dtype=torch.float64, device=x.cores[0].device)
    xd, k1 = x._desc()
    Sp = (ctypes.c_void_p * x.d)(*[t.data_ptr() for t in S])
    ws = _workspace(lib.tt_sketch_workspace(mode, ctypes.byref(xd), s), out.device)
    check(lib.tt_sketch(mode, ctypes.byref(xd), s, Sp, ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def tt_sketch_factors(ns: Sequence[int], s: int, seed: int = 0, mode: int = MODE_FP64,
                      device="cuda", stream=None) -> List[torch.Tensor]:
    """The Khatri-Rao factors ``S_k`` (``[s, n_k]``, entries N(0, s^(-1/d)))
    that :func:`tt_sgmres_solve` draws from ``seed``."""
    d = len(ns)
    S = [torch.empty((s, n), dtype=mode_dtype(mode), device=device) for n in ns]
    n_arr = (ctypes.c_int64 * d)(*ns)
    sp = (ctypes.c_void_p * d)(*[t.data_ptr() for t in S])
    check(lib.tt_sketch_factors(mode, d, n_arr, int(s), ctypes.c_uint64(seed), sp,
                                _stream(stream)))
    return S


def tt_dot(x: TT, y: TT, mode: int = MODE_FP64, stream=None) -> torch.Tensor:
    """``<x, y>`` as a one-element float64 device tensor."""
    _check_dtype(x.cores + y.cores, mode)
    out = torch.empty(1, dtype=torch.float64, device=x.cores[0].device)
    xd, k1 = x._desc()
    yd, k2 = y._desc()
    ws = _workspace(lib.tt_dot_workspace(mode, ctypes.byref(xd), ctypes.byref(yd)), out.device)
    check(lib.tt_dot(mode, ctypes.byref(xd), ctypes.byref(yd), ctypes.c_void_p(out.data_ptr()),
                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return out


def tt_round_rand(terms: Sequence[TT], coefs: Sequence[float], eps: float, rmax: int,
                  oversample: int = 10, seed: int = 0, drm=None, mode: int = MODE_FP64,
                  stream=None) -> TT:
    """Randomize-then-orthogonalize rounding of ``sum_b coefs[b] * terms[b]``.

    ``drm``: ``None`` (Philox TT-DRM from ``seed``) or a list of DRM cores
    ``[L_{k-1}, n_k, L_k]`` whose ranks cover the sketch ranks."""
    allc = [c for t in terms for c in t.cores] + (list(drm) if drm is not None else [])
    _check_dtype(allc, mode)
    nt = len(terms)
    descs, keep = [], []
    for t in terms:
        dsc, k = t._desc()
        descs.append(dsc)
        keep.append(k)
    arr = (TTVec * nt)(*descs)
    coef = (ctypes.c_double * nt)(*[float(c) for c in coefs])
    d = terms[0].d
    ns = terms[0].ns
    dev = terms[0].cores[0].device
    dt = terms[0].cores[0].dtype
    # output capacities: min(rmax, summed rank) per bond is always enough
    tsum = [sum(t.ranks[k] for t in terms) for k in range(d + 1)]
    cap = [1] + [min(int(rmax), tsum[k]) if True else 0 for k in range(1, d)] + [1]
    # the randomized sketch rank can exceed rmax before truncation only when eps == 0 and rmax
    # >= sketch rank, in which case cap = min(rmax, t) still covers it
    ycores = [torch.empty(cap[k] * ns[k] * cap[k + 1], dtype=dt, device=dev) for k in range(d)]
    n_arr = (ctypes.c_int64 * d)(*ns)
    cap_arr = (ctypes.c_int64 * (d + 1))(*cap)
    rank_arr = (ctypes.c_int64 * (d + 1))()
    yptr = (ctypes.c_void_p * d)(*[c.data_ptr() for c in ycores])
    yd = TTVecOut(d, n_arr, cap_arr, rank_arr, yptr)
    if drm is not None:
        drm_p = (ctypes.c_void_p * d)(*[c.data_ptr() for c in drm])
        drm_r = (ctypes.c_int64 * (d + 1))(*([c.shape[0] for c in drm] + [1]))
    else:
        drm_p, drm_r = None, None
    ws = _workspace(lib.tt_round_rand_workspace(mode, nt, arr, int(rmax), int(oversample)), dev)
    check(lib.tt_round_rand(mode, nt, arr, coef, float(eps), int(rmax), int(oversample),
                            ctypes.c_uint64(seed), drm_p, drm_r, ctypes.byref(yd),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    r = list(rank_arr)
    return TT([ycores[k][: r[k] * ns[k] * r[k + 1]].view(r[k], ns[k], r[k + 1]) for k in range(d)])


def tt_gaussian(count: int, seed: int, stream_id: int, std: float = 1.0,
                mode: int = MODE_FP64, device="cuda", stream=None) -> torch.Tensor:
    """Philox4x32-10 Gaussian stream elements ``0..count-1`` times ``std``."""
    out = torch.empty(count, dtype=mode_dtype(mode), device=device)
    check(lib.tt_gaussian(mode, ctypes.c_void_p(out.data_ptr()), count, ctypes.c_uint64(seed),
                          ctypes.c_uint64(stream_id), float(std), _stream(stream)))
    return out


def tt_qr_f64(Y: torch.Tensor, want_q: bool = True, stream=None):
    """FP64 Householder QR of a tall matrix (``m x l``, float64 or float32):
    returns ``(Q, R)`` with Q in Y's dtype and R float64."""
    mode = MODE_FP64 if Y.dtype == torch.float64 else MODE_FP32
    m, l = Y.shape
    Q = torch.empty((m, l), dtype=Y.dtype, device=Y.device) if want_q else None
    R = torch.empty((l, l), dtype=torch.float64, device=Y.device)
    ws = _workspace(lib.tt_qr_f64_workspace(m, l), Y.device)
    check(lib.tt_qr_f64(mode, ctypes.c_void_p(Y.data_ptr()), m, l, Y.stride(0), Y.stride(1),
                        ctypes.c_void_p(Q.data_ptr() if Q is not None else 0),
                        ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                        _stream(stream)))
    return Q, R


def tt_lstsq_f64(W: torch.Tensor, c: torch.Tensor, stream=None):
    """``y = argmin ||W y - c||`` (W: s x k float64) and ``||W y - c||``."""
    s, k = W.shape
    Wc = W.t().contiguous()  # column-major storage
    y = torch.empty(k, dtype=torch.float64, device=W.device)
    res = torch.empty(1, dtype=torch.float64, device=W.device)
    ws = _workspace(lib.tt_lstsq_f64_workspace(s, k), W.device)
    check(lib.tt_lstsq_f64(ctypes.c_void_p(Wc.data_ptr()), s, k,
                           ctypes.c_void_p(c.contiguous().data_ptr()), ctypes.c_void_p(y.data_ptr()),
                           ctypes.c_void_p(res.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                           ws.numel(), _stream(stream)))
    return y, res


def tt_sgmres_solve(op, b: TT, maxit: int, tol: float, rmax: int, mode: int = MODE_FP64,
                    s: int = 0, round_tol: float = 0.0, eta: float = 0.1,
                    stop_safety: float = 0.1, r_sol: int = 0, oversample: int = 10, seed: int = 0,
                    max_restarts: int = 5, hist_cap: int = 1024, workspace=None, stream=None,
                    raise_on_nonconvergence: bool = False, final_stta: bool = False,
                    ell: int = 1, precond=None):
    """Restarted TT-sGMRES.  ``op`` and ``b`` in float64 on the device.
    Returns ``(x, info)``; ``x`` is a float64 :class:`TT`.  ``final_stta``
    forms each cycle's correction by STTA from one-pass sketches of the basis
    vectors instead of rounding the stored basis; ``ell`` orthogonalises each
    new vector against the last ``ell`` basis vectors; ``precond`` (a
    :class:`Precond`) selects right preconditioning (TT-sPGMRES)."""
    _check_dtype(list(op) + b.cores, MODE_FP64)
    p = SolverParams(maxit, s, tol, round_tol, eta, stop_safety, rmax, r_sol, oversample, seed,
                     max_restarts, mode, int(bool(final_stta)), int(ell))
    od, k1 = _op_desc(op)
    bd, k2 = b._desc()
    dev = b.cores[0].device
    if precond is not None:
        precond.check_modes(b.ns)
        pdesc, k3 = precond._desc()
        need = lib.tt_spgmres_solve_workspace(ctypes.byref(od), ctypes.byref(pdesc),
                                              ctypes.byref(bd), ctypes.byref(p))
    else:
        need = lib.tt_sgmres_solve_workspace(ctypes.byref(od), ctypes.byref(bd), ctypes.byref(p))
    if need == 0:
        raise TTError(1, lib.tt_last_error().decode())
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    d = b.d
    rs = r_sol if r_sol > 0 else rmax
    cap = [1] + [rs] * (d - 1) + [1]
    xc = [torch.empty(cap[k] * b.ns[k] * cap[k + 1], dtype=torch.float64, device=dev)
          for k in range(d)]
    n_arr = (ctypes.c_int64 * d)(*b.ns)
    cap_arr = (ctypes.c_int64 * (d + 1))(*cap)
    rank_arr = (ctypes.c_int64 * (d + 1))()
    xp = (ctypes.c_void_p * d)(*[c.data_ptr() for c in xc])
    xd = TTVecOut(d, n_arr, cap_arr, rank_arr, xp)
    rh = (ctypes.c_double * hist_cap)()
    kh = (ctypes.c_int64 * hist_cap)()
    info = SolverInfo()
    info.res_hist = ctypes.cast(rh, ctypes.POINTER(ctypes.c_double))
    info.rank_hist = ctypes.cast(kh, ctypes.POINTER(ctypes.c_int64))
    info.hist_cap = hist_cap
    if precond is not None:
        rc = lib.tt_spgmres_solve(ctypes.byref(od), ctypes.byref(pdesc), ctypes.byref(bd),
                                  ctypes.byref(p), ctypes.byref(xd), ctypes.byref(info),
                                  ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                  _stream(stream))
    else:
        rc = lib.tt_sgmres_solve(ctypes.byref(od), ctypes.byref(bd), ctypes.byref(p),
                                 ctypes.byref(xd), ctypes.byref(info),
                                 ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                 _stream(stream))
    if rc not in (0, 5, 7) or (rc in (5, 7) and raise_on_nonconvergence):
        check(rc)
    r = list(rank_arr)
    x = TT([xc[k][: r[k] * b.ns[k] * r[k + 1]].view(r[k], b.ns[k], r[k + 1]) for k in range(d)])
    n = min(info.iters, hist_cap)
    out = dict(iters=info.iters, cycles=info.cycles, sketched_res=info.sketched_res,
               true_res=info.true_res, max_rank=info.max_rank, status=info.status,
               seconds=info.seconds, res_hist=list(rh[:n]), rank_hist=list(kh[:n]),
               svd_nonconverged=info.svd_nonconverged, svd_max_sweeps=info.svd_max_sweeps,
               svd_mean_sweeps=info.svd_mean_sweeps, breakdowns=info.breakdowns,
               workspace_bytes=int(need))
    return x, out


# ------------------------------------------------------------------ adjoint
def tt_dot_grad(x: TT, y: TT, mode: int = MODE_FP64, stream=None) -> List[torch.Tensor]:
    """Derivative of ``<x, y>`` with respect to every core of ``y`` (cores
    shaped like y's)."""
    _check_dtype(x.cores + y.cores, mode)
    g = [torch.empty_like(c) for c in y.cores]
    xd, k1 = x._desc()
    yd, k2 = y._desc()
    gp = (ctypes.c_void_p * y.d)(*[t.data_ptr() for t in g])
    ws = _workspace(lib.tt_dot_grad_workspace(mode, ctypes.byref(xd), ctypes.byref(yd)),
                    y.cores[0].device)
    check(lib.tt_dot_grad(mode, ctypes.byref(xd), ctypes.byref(yd), gp,
                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return g


class Precond:
    """Exponential-sum right preconditioner ``sum_i alpha_i (exp(-beta_i A_1) x
    .. x exp(-beta_i A_d))`` of a Kronecker-sum operator: host coefficients and
    the 1-D matrices ``A_k`` as float64 device tensors."""

    def __init__(self, alpha, beta, mats: Sequence[torch.Tensor]):
        self.alpha = np.ascontiguousarray(alpha, dtype=np.float64)
        self.beta = np.ascontiguousarray(beta, dtype=np.float64)
        if self.alpha.shape != self.beta.shape or self.alpha.ndim != 1:
            raise ValueError("alpha and beta: equal-length vectors")
        # device float64 copies (a host tensor or array is moved to the GPU)
        self.mats = [torch.as_tensor(m, dtype=torch.float64, device="cuda").contiguous()
                     for m in mats]
        for m in self.mats:
            if m.dim() != 2 or m.shape[0] != m.shape[1]:
                raise ValueError("preconditioner matrices must be square")

    @classmethod
    def for_interval(cls, a: float, b: float, tol: float, mats):
        """Coefficients for the spectral interval [a, b] at accuracy tol."""
        alpha, beta = exp_sum_coefficients(a, b, tol)
        return cls(alpha, beta, mats)

    def check_modes(self, ns):
        """The C descriptor carries no sizes: matrix k must be n_k x n_k."""
        if len(self.mats) != len(ns) or any(m.shape[0] != n for m, n in zip(self.mats, ns)):
            raise ValueError("preconditioner matrices must be n_k x n_k for every mode k")

    def _desc(self):
        ap = self.alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        bp = self.beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        mp = (ctypes.c_void_p * len(self.mats))(*[m.data_ptr() for m in self.mats])
        return TTPrecond(len(self.alpha), ap, bp, mp), (ap, bp, mp)


def exp_sum_coefficients(a: float, b: float, tol: float):
    """``(alpha, beta)`` of the exponential sum ``E(z) ~ 1/z`` on ``[a, b]``
    (trapezoidal rule on the Laplace integral; host computation)."""
    count = lib.tt_exp_sum_coefficients(float(a), float(b), float(tol), 0, None, None)
    if count < 0:
        raise TTError(1, "exp_sum_coefficients: need 0 < a < b and 0 < tol < 1")
    alpha = np.zeros(count)
    beta = np.zeros(count)
    lib.tt_exp_sum_coefficients(float(a), float(b), float(tol), count,
                                alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return alpha, beta


def tt_precond_apply(P: Precond, x: TT, eps: float, rmax: int, oversample: int = 10,
                     seed: int = 0, mode: int = MODE_FP64, stream=None) -> TT:
    """``Round(P^{-1} x)`` to ``eps`` and ranks ``<= rmax``."""
    _check_dtype(x.cores, mode)
    P.check_modes(x.ns)
    d, ns, dev, dt = x.d, x.ns, x.cores[0].device, x.cores[0].dtype
    cap = [1] + [int(rmax)] * (d - 1) + [1]
    ycores = [torch.empty(cap[k] * ns[k] * cap[k + 1], dtype=dt, device=dev) for k in range(d)]
    n_arr = (ctypes.c_int64 * d)(*ns)
    cap_arr = (ctypes.c_int64 * (d + 1))(*cap)
    rank_arr = (ctypes.c_int64 * (d + 1))()
    yptr = (ctypes.c_void_p * d)(*[c.data_ptr() for c in ycores])
    yd = TTVecOut(d, n_arr, cap_arr, rank_arr, yptr)
    xd, k1 = x._desc()
    pd, k2 = P._desc()
    need = lib.tt_precond_apply_workspace(mode, ctypes.byref(pd), ctypes.byref(xd), int(rmax),
                                          int(oversample))
    if need == 0:
        raise TTError(1, lib.tt_last_error().decode())
    ws = _workspace(need, dev)
    check(lib.tt_precond_apply(mode, ctypes.byref(pd), ctypes.byref(xd), float(eps), int(rmax),
                               int(oversample), ctypes.c_uint64(seed), ctypes.byref(yd),
                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    r = list(rank_arr)
    return TT([ycores[k][: r[k] * ns[k] * r[k + 1]].view(r[k], ns[k], r[k + 1]) for k in range(d)])


def tt_spgmres_solve(op, P: Precond, b: TT, maxit: int, tol: float, rmax: int, **kw):
    """Right-preconditioned TT-sGMRES (Algorithm 5); arguments as
    :func:`tt_sgmres_solve`."""
    return tt_sgmres_solve(op, b, maxit, tol, rmax, precond=P, **kw)


def tt_stta_sketch(x: TT, X: TT, Y: TT, mode: int = MODE_FP64, coef: float = 1.0,
                   out=None, stream=None):
    """Two-sided STTA sketches of ``x`` with right DRM ``X`` (target ranks) and
    left DRM ``Y``: ``(psi, omega)``, float64 device tensors ``psi[k]``
    ``[l_k, n_k, r_{k+1}]`` and ``omega[k]`` ``[l_{k+1}, r_{k+1}]``.  With
    ``out = (psi, omega)`` the sketches are accumulated into those tensors
    (``out += coef * sketch(x)``) and returned."""
    _check_dtype(x.cores + X.cores + Y.cores, mode)
    dev = x.cores[0].device
    r, l = X.ranks, Y.ranks
    if out is None:
        psi = [torch.empty((l[k], x.ns[k], r[k + 1]), dtype=torch.float64, device=dev)
               for k in range(x.d)]
        omega = [torch.empty((l[k + 1], r[k + 1]), dtype=torch.float64, device=dev)
                 for k in range(x.d - 1)]
        acc = 0
    else:
        psi, omega = out
        acc = 1
        want_p = [(l[k], x.ns[k], r[k + 1]) for k in range(x.d)]
        want_o = [(l[k + 1], r[k + 1]) for k in range(x.d - 1)]
        if ([tuple(t.shape) for t in psi] != want_p or [tuple(t.shape) for t in omega] != want_o
                or any(t.dtype != torch.float64 or t.device.type != "cuda" or
                       not t.is_contiguous() for t in list(psi) + list(omega))):
            raise ValueError("stta_sketch: out must hold contiguous float64 CUDA sketches of "
                             "the shapes this x, X, Y give")
    xd, k1 = x._desc()
    Xd, k2 = X._desc()
    Yd, k3 = Y._desc()
    pp = (ctypes.c_void_p * x.d)(*[t.data_ptr() for t in psi])
    op = (ctypes.c_void_p * max(1, x.d - 1))(*[t.data_ptr() for t in omega])
    ws = _workspace(lib.tt_stta_sketch_workspace(mode, ctypes.byref(xd), ctypes.byref(Xd),
                                                 ctypes.byref(Yd)), dev)
    check(lib.tt_stta_sketch(mode, ctypes.byref(xd), float(coef), acc, ctypes.byref(Xd),
                             ctypes.byref(Yd), pp, op, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                             _stream(stream)))
    return psi, omega


def tt_stta_recover(psi: Sequence[torch.Tensor], omega: Sequence[torch.Tensor],
                    rcond: float = 0.0, stream=None) -> TT:
    """FP64 cores of the STTA approximant from the sketches: core 1 = psi[0]
    and core k = pinv(omega[k-2]) psi[k-1] (right unfoldings), the
    pseudo-inverse with relative cutoff ``rcond`` (0: 1e-12)."""
    d = len(psi)
    dev = psi[0].device
    if len(omega) != d - 1:
        raise ValueError("stta_recover: d - 1 omega matrices expected")
    for t in list(psi) + list(omega):
        if t.dtype != torch.float64 or t.device.type != "cuda":
            raise ValueError("stta_recover: float64 CUDA tensors expected")
    if psi[0].shape[0] != 1 or psi[-1].shape[2] != 1:
        raise ValueError("stta_recover: boundary ranks must be 1")
    for k in range(d - 1):
        if tuple(omega[k].shape) != (psi[k + 1].shape[0], psi[k].shape[2]):
            raise ValueError("stta_recover: omega[k] must be l_{k+1} x r_{k+1}")
    n = [p.shape[1] for p in psi]
    l = [1] + [p.shape[0] for p in psi[1:]] + [1]
    r = [1] + [p.shape[2] for p in psi[:-1]] + [1]
    cores = [torch.empty((r[k], n[k], r[k + 1]), dtype=torch.float64, device=dev)
             for k in range(d)]
    n_a = (ctypes.c_int64 * d)(*n)
    r_a = (ctypes.c_int64 * (d + 1))(*r)
    l_a = (ctypes.c_int64 * (d + 1))(*l)
    psi = [p.contiguous() for p in psi]
    omega = [o.contiguous() for o in omega]
    pp = (ctypes.c_void_p * d)(*[p.data_ptr() for p in psi])
    op = (ctypes.c_void_p * max(1, d - 1))(*[o.data_ptr() for o in omega])
    cp = (ctypes.c_void_p * d)(*[c.data_ptr() for c in cores])
    need = lib.tt_stta_recover_workspace(d, n_a, r_a, l_a)
    if need == 0:
        raise TTError(1, lib.tt_last_error().decode())
    ws = _workspace(need, dev)
    check(lib.tt_stta_recover(d, n_a, r_a, l_a, pp, op, float(rcond), cp,
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)))
    return TT(cores)


def tt_local_dots(x: TT, y: TT, mats: Sequence[torch.Tensor], mode: int = MODE_FP64,
                  stream=None) -> torch.Tensor:
    """``out[k] = <x, (I x .. x mats[k] x .. x I) y>`` (float64 device tensor)."""
    _check_dtype(x.cores + y.cores + list(mats), mode)
    out = torch.empty(x.d, dtype=torch.float64, device=x.cores[0].device)
    xd, k1 = x._desc()
    yd, k2 = y._desc()
    mp = (ctypes.c_void_p * x.d)(*[m.data_ptr() for m in mats])
    ws = _workspace(lib.tt_local_dots_workspace(mode, ctypes.byref(xd), ctypes.byref(yd)),
                    out.device)
    check(lib.tt_local_dots(mode, ctypes.byref(xd), ctypes.byref(yd), mp,
                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                            ws.numel(), _stream(stream)))
    return out


def tt_kron_sum_op(mats: Sequence[torch.Tensor], theta=None, mode: int = MODE_FP64,
                   stream=None) -> List[torch.Tensor]:
    """Cores of ``sum_k theta_k (I x .. x mats[k] x .. x I)`` (rank 2)."""
    _check_dtype(list(mats), mode)
    d = len(mats)
    ns = [m.shape[0] for m in mats]
    R = [1] + [2] * (d - 1) + [1]
    cores = [torch.empty((R[k], ns[k], ns[k], R[k + 1]), dtype=mats[0].dtype,
                         device=mats[0].device) for k in range(d)]
    n_arr = (ctypes.c_int64 * d)(*ns)
    mp = (ctypes.c_void_p * d)(*[m.data_ptr() for m in mats])
    cp = (ctypes.c_void_p * d)(*[c.data_ptr() for c in cores])
    th = None
    if theta is not None:
        vals = [float(t) for t in (theta.detach().cpu().tolist() if torch.is_tensor(theta)
                                   else theta)]
        th = (ctypes.c_double * d)(*vals)
    check(lib.tt_kron_sum_op(mode, d, n_arr, mp, th, cp, _stream(stream)))
    return cores


def tt_op_transpose(op: Sequence[torch.Tensor], mode: int = MODE_FP64,
                    stream=None) -> List[torch.Tensor]:
    """Cores of ``A^T``."""
    _check_dtype(list(op), mode)
    out = [torch.empty_like(c) for c in op]
    od, k1 = _op_desc(op)
    cp = (ctypes.c_void_p * len(op))(*[c.data_ptr() for c in out])
    check(lib.tt_op_transpose(mode, ctypes.byref(od), cp, _stream(stream)))
    return out


class _SolveLoss(torch.autograd.Function):
    """``loss(theta, b) = ||x - x_t||^2`` with ``A(theta) x = b`` and
    ``A(theta) = sum_k theta_k (I x .. x M x .. x I)``.

    The difference ``x - x_t`` is formed as a TT by the FP64 randomized rounding
    at full rank (sum of the two rank caps, tolerance far below the solver's),
    which leaves it left-orthogonal, so the loss is its squared norm without
    the cancellation of ``<x, x> - 2 <x, x_t> + <x_t, x_t>`` when x is close to
    x_t.

    Backward: ``lambda = A^{-T} 2 (x - x_t)`` by a second TT-sGMRES solve on the
    transposed operator, then ``dL/dtheta_k = -<lambda, (I x .. M .. x I) x>``
    (tt_local_dots), ``dL/db_k = d<lambda, b>/db_k`` and ``dL/dxt_k =
    -d<2(x - x_t), x_t>/dxt_k`` (tt_dot_grad)."""

    @staticmethod
    def forward(ctx, theta, M, cfg, *cores):
        d = cfg["d"]
        b = TT(cores[:d])
        xt = TT(cores[d:])
        mats = [M] * d
        op = tt_kron_sum_op(mats, theta)
        sv = cfg["solver"]
        x, info = tt_sgmres_solve(op, b, **sv)
        rmax_r = max(x.ranks) + max(xt.ranks)
        diff = tt_round_rand([x, xt], [1.0, -1.0], 1e-12, rmax_r,
                             oversample=sv.get("oversample", 10), seed=sv.get("seed", 0) + 1)
        loss = tt_dot(diff, diff).reshape(())
        ctx.cfg = cfg
        ctx.info = info
        ctx.save_for_backward(theta, M, *x.cores, *cores, *diff.cores)
        ctx.xd = x.d
        cfg["last_info"] = info
        return loss

    @staticmethod
    def backward(ctx, gout):
        cfg = ctx.cfg
        d = cfg["d"]
        saved = ctx.saved_tensors
        theta, M = saved[0], saved[1]
        x = TT(saved[2:2 + d])
        b = TT(saved[2 + d:2 + 2 * d])
        xt = TT(saved[2 + 2 * d:2 + 3 * d])
        diff = saved[2 + 3 * d:2 + 4 * d]
        sv = cfg["solver"]
        # right-hand side of the adjoint system: 2 (x - x_t), the forward's
        # FP64 rounding of the difference scaled by 2
        r = TT([2.0 * diff[0], *diff[1:]])
        opT = tt_op_transpose(tt_kron_sum_op([M] * d, theta))
        lam, info = tt_sgmres_solve(opT, r, **sv)
        cfg["last_adjoint_info"] = info
        g = gout.to(torch.float64)
        dtheta = -tt_local_dots(lam, x, [M] * d) * g
        db = [t * g for t in tt_dot_grad(lam, b)]
        dxt = [-t * g for t in tt_dot_grad(r, xt)]
        dtheta = dtheta.to(device=theta.device, dtype=theta.dtype)
        return (dtheta, None, None, *db, *dxt)


def solve_loss(theta: torch.Tensor, M: torch.Tensor, b_cores: Sequence[torch.Tensor],
               xt_cores: Sequence[torch.Tensor], **solver) -> torch.Tensor:
    """Differentiable ``||x(theta, b) - x_t||^2`` (float64 scalar on the device).

    ``theta``: d coefficients; ``M``: the n x n 1-D operator (float64, CUDA);
    ``b_cores``, ``xt_cores``: float64 CUDA cores.  ``solver``: keyword
    arguments of :func:`tt_sgmres_solve` (``maxit``, ``tol``, ``rmax``,
    ``mode``, ...), used for both the forward and the adjoint solve.  After a
    call, ``solve_loss.last`` holds the forward and adjoint solver info."""
    d = len(b_cores)
    cfg = {"d": d, "solver": dict(solver)}
    loss = _SolveLoss.apply(theta, M, cfg, *b_cores, *xt_cores)
    solve_loss.last = cfg
    return loss


# ------------------------------------------------------------------ batched
def tt_qr_f64_batched(Ys: Sequence[torch.Tensor], want_q: bool = True, stream=None):
    """FP64 Householder QR of several tall matrices in one launch (one CTA per
    matrix); returns lists ``Q`` (each in its Y's dtype) and ``R`` (float64)."""
    mode = MODE_FP64 if Ys[0].dtype == torch.float64 else MODE_FP32
    _check_dtype(list(Ys), mode)
    cnt = len(Ys)
    ms = [y.shape[0] for y in Ys]
    ls = [y.shape[1] for y in Ys]
    Qs = [torch.empty_like(y) for y in Ys] if want_q else None
    Rs = [torch.zeros((l, l), dtype=torch.float64, device=y.device) for y, l in zip(Ys, ls)]
    m_arr = (ctypes.c_int64 * cnt)(*ms)
    l_arr = (ctypes.c_int64 * cnt)(*ls)
    yp = (ctypes.c_void_p * cnt)(*[y.data_ptr() for y in Ys])
    qp = (ctypes.c_void_p * cnt)(*[q.data_ptr() for q in Qs]) if want_q else None
    rp = (ctypes.c_void_p * cnt)(*[r.data_ptr() for r in Rs])
    ws = _workspace(lib.tt_qr_f64_batched_workspace(cnt, m_arr, l_arr), Ys[0].device)
    check(lib.tt_qr_f64_batched(mode, cnt, yp, m_arr, l_arr, qp, rp, ctypes.c_void_p(ws.data_ptr()),
                                ws.numel(), _stream(stream)))
    return Qs, Rs


def tt_sgmres_solve_batched(op, bs: Sequence[TT], maxit: int, tol: float, rmax: int,
                            mode: int = MODE_FP64, s: int = 0, round_tol: float = 0.0,
                            eta: float = 0.1, stop_safety: float = 0.1, r_sol: int = 0,
                            oversample: int = 10, seed: int = 0, max_restarts: int = 5,
                            nworkers: int = 16, workspace=None, final_stta: bool = False,
                            ell: int = 1):
    """Independent solves ``A x_i = b_i`` for all right-hand sides (uneven ranks
    allowed) on ``nworkers`` library threads and streams.  Returns a list of
    ``(x_i, info_i)`` like :func:`tt_sgmres_solve`; synchronises."""
    _check_dtype(list(op) + [c for b in bs for c in b.cores], MODE_FP64)
    p = SolverParams(maxit, s, tol, round_tol, eta, stop_safety, rmax, r_sol, oversample, seed,
                     max_restarts, mode, int(bool(final_stta)), int(ell))
    nrhs = len(bs)
    od, k1 = _op_desc(op)
    descs, keep = [], []
    for b in bs:
        dsc, k = b._desc()
        descs.append(dsc)
        keep.append(k)
    barr = (TTVec * nrhs)(*descs)
    dev = bs[0].cores[0].device
    need = lib.tt_sgmres_solve_batched_workspace(ctypes.byref(od), nrhs, barr, ctypes.byref(p),
                                                 nworkers)
    if need == 0:
        raise TTError(1, lib.tt_last_error().decode())
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    rs = r_sol if r_sol > 0 else rmax
    outs, odescs = [], []
    infos = (SolverInfo * nrhs)()
    for i, b in enumerate(bs):
        d = b.d
        cap = [1] + [rs] * (d - 1) + [1]
        xc = [torch.empty(cap[k] * b.ns[k] * cap[k + 1], dtype=torch.float64, device=dev)
              for k in range(d)]
        n_arr = (ctypes.c_int64 * d)(*b.ns)
        cap_arr = (ctypes.c_int64 * (d + 1))(*cap)
        rank_arr = (ctypes.c_int64 * (d + 1))()
        xp = (ctypes.c_void_p * d)(*[c.data_ptr() for c in xc])
        odescs.append(TTVecOut(d, n_arr, cap_arr, rank_arr, xp))
        outs.append((xc, rank_arr, n_arr, cap_arr, xp))
        infos[i].hist_cap = 0
    xarr = (TTVecOut * nrhs)(*odescs)
    torch.cuda.synchronize(dev)
    rc = lib.tt_sgmres_solve_batched(ctypes.byref(od), nrhs, barr, ctypes.byref(p), xarr, infos,
                                     int(nworkers), ctypes.c_void_p(workspace.data_ptr()),
                                     workspace.numel())
    if rc not in (0, 5, 7):
        check(rc)
    res = []
    for i, b in enumerate(bs):
        xc = outs[i][0]
        r = list(xarr[i].rank[k] for k in range(b.d + 1))
        x = TT([xc[k][: r[k] * b.ns[k] * r[k + 1]].view(r[k], b.ns[k], r[k + 1]) for k in range(b.d)])
        inf = infos[i]
        res.append((x, dict(iters=inf.iters, cycles=inf.cycles, sketched_res=inf.sketched_res,
                            true_res=inf.true_res, max_rank=inf.max_rank, status=inf.status,
                            seconds=inf.seconds, svd_nonconverged=inf.svd_nonconverged,
                            breakdowns=inf.breakdowns, workspace_bytes=int(need))))
    return res
