"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every function ``include/ttsg.h`` declares, and the binding's ctypes
prototypes name exactly those functions.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(tt_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for required in ("tt_matvec", "tt_sketch", "tt_round_rand", "tt_sgmres_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_prototypes_match_header(built_lib):
    from paper_2409_09471_gb300 import _abi
    src = open(_abi.__file__).read()
    bound = set(re.findall(r'"(tt_\w+)"\s*:', src))
    assert bound == declared_functions()


def test_version_and_error_strings(built_lib):
    built_lib.tt_version.restype = ctypes.c_char_p
    built_lib.tt_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in built_lib.tt_version()
    assert built_lib.tt_last_error() == b""


def test_argument_errors_are_caught_on_the_host(built_lib):
    # a null descriptor is rejected before any CUDA call, so this runs without a GPU
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    rc = lib.tt_dot(0, None, None, None, None, 0, None)
    assert rc == 1 and b"null descriptor" in lib.tt_last_error()
    rc = lib.tt_matvec(7, None, None, None, None, 0, None)
    assert rc == 1 and b"unknown mode" in lib.tt_last_error()


def test_workspace_queries_run_without_a_gpu(built_lib):
    # every *_workspace entry point is a dry run on the host (no CUDA call):
    # descriptors with placeholder device pointers must give a positive size
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    d, ns = 4, [7, 5, 8, 6]

    def desc(ranks):
        n = (ctypes.c_int64 * d)(*ns)
        r = (ctypes.c_int64 * (d + 1))(*ranks)
        p = (ctypes.c_void_p * d)(*([0x1000] * d))
        return _abi.TTVec(d, n, r, p), (n, r, p)

    x, kx = desc([1, 4, 9, 3, 1])
    y, ky = desc([1, 2, 6, 5, 1])
    for mode in (0, 1, 2):
        assert lib.tt_dot_workspace(mode, ctypes.byref(x), ctypes.byref(y)) > 0
        assert lib.tt_dot_grad_workspace(mode, ctypes.byref(x), ctypes.byref(y)) > 0
        assert lib.tt_local_dots_workspace(mode, ctypes.byref(x), ctypes.byref(y)) > 0
        assert lib.tt_sketch_workspace(mode, ctypes.byref(x), 40) > 0
        arr = (_abi.TTVec * 2)(x, y)
        assert lib.tt_round_rand_workspace(mode, 2, arr, 8, 4) > 0


def test_new_entry_points_reject_bad_arguments_on_the_host(built_lib):
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    assert lib.tt_sgmres_solve_batched(None, 0, None, None, None, None, 4, None, 0) == 1
    assert b"nrhs" in lib.tt_last_error()
    assert lib.tt_qr_f64_batched(0, 0, None, None, None, None, None, None, 0, None) == 1
    assert lib.tt_qr_f64_batched_workspace(0, None, None) == 0
    assert lib.tt_dot_grad(0, None, None, None, None, 0, None) == 1
    assert lib.tt_local_dots(0, None, None, None, None, None, 0, None) == 1
    assert lib.tt_kron_sum_op(0, 0, None, None, None, None, None) == 1
    assert lib.tt_op_transpose(0, None, None, None) == 1
    assert lib.tt_kron_sum_op(7, 1, None, None, None, None, None) == 1  # unknown mode
    assert b"mode" in lib.tt_last_error()


def test_solver_workspace_queries_are_dry_runs(built_lib):
    # the solver's workspace query runs the whole solve on the host with
    # placeholder pointers and no CUDA work; the batched query is at least the
    # per-worker slice times the workers
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    d, ns = 4, [8, 8, 8, 8]
    n = (ctypes.c_int64 * d)(*ns)
    R = (ctypes.c_int64 * (d + 1))(1, 2, 2, 2, 1)
    opc = (ctypes.c_void_p * d)(*([0x1000] * d))
    op = _abi.TTOp(d, n, R, opc)
    r = (ctypes.c_int64 * (d + 1))(1, 3, 4, 2, 1)
    bc = (ctypes.c_void_p * d)(*([0x2000] * d))
    b = _abi.TTVec(d, n, r, bc)
    for mode in (0, 1, 2):
        p = _abi.SolverParams(20, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode)
        one = lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b), ctypes.byref(p))
        assert one > 0, lib.tt_last_error()
        bs = (_abi.TTVec * 3)(b, b, b)
        many = lib.tt_sgmres_solve_batched_workspace(ctypes.byref(op), 3, bs, ctypes.byref(p), 2)
        assert many >= 2 * 256 and many > 0
        # the STTA form of the correction (its DRMs and stored sketches, and a
        # basis window of ell + 1 vectors instead of the whole basis)
        ps = _abi.SolverParams(20, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode, 1)
        st = lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b), ctypes.byref(ps))
        assert st > 0, lib.tt_last_error()
        # orthogonalising against 4 vectors rounds 5-term sums
        pl = _abi.SolverParams(20, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode, 0, 4)
        four = lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b), ctypes.byref(pl))
        assert four >= one, lib.tt_last_error()
        # invalid parameters are rejected by the query itself
        bad = _abi.SolverParams(0, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode)
        assert lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b), ctypes.byref(bad)) == 0
        bad2 = _abi.SolverParams(20, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode, 3)
        assert lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b),
                                             ctypes.byref(bad2)) == 0


def test_stta_entry_points_validate_and_size_on_the_host(built_lib):
    # workspace queries of the STTA entry points are host dry runs; the
    # recovery rejects left ranks below the target ranks
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    d, ns = 4, [7, 5, 8, 6]

    def desc(ranks):
        n = (ctypes.c_int64 * d)(*ns)
        r = (ctypes.c_int64 * (d + 1))(*ranks)
        p = (ctypes.c_void_p * d)(*([0x1000] * d))
        return _abi.TTVec(d, n, r, p), (n, r, p)

    x, kx = desc([1, 4, 9, 3, 1])
    X, kX = desc([1, 3, 5, 2, 1])
    Y, kY = desc([1, 6, 8, 4, 1])
    for mode in (0, 1, 2):
        assert lib.tt_stta_sketch_workspace(mode, ctypes.byref(x), ctypes.byref(X),
                                            ctypes.byref(Y)) > 0, lib.tt_last_error()
    Z, kZ = desc([1, 3, 5, 2, 1])
    Z.n[1] = 6                       # mode sizes differ from x
    assert lib.tt_stta_sketch_workspace(0, ctypes.byref(x), ctypes.byref(X), ctypes.byref(Z)) == 0
    assert b"mode sizes" in lib.tt_last_error()
    n = (ctypes.c_int64 * d)(*ns)
    r = (ctypes.c_int64 * (d + 1))(1, 3, 5, 2, 1)
    ok = (ctypes.c_int64 * (d + 1))(1, 6, 8, 4, 1)
    short = (ctypes.c_int64 * (d + 1))(1, 6, 4, 4, 1)
    assert lib.tt_stta_recover_workspace(d, n, r, ok) > 0, lib.tt_last_error()
    assert lib.tt_stta_recover_workspace(d, n, r, short) == 0
    assert b"l_k >= r_k" in lib.tt_last_error()
    assert lib.tt_stta_recover(d, n, r, ok, None, None, 0.0, None, None, 0, None) == 1
    assert lib.tt_stta_sketch(0, None, 1.0, 0, None, None, None, None, None, 0, None) == 1


def test_exp_sum_coefficients_match_the_oracle(built_lib):
    # the library's host coefficients and the oracle's are independent codes
    # of the same rule (trapezoidal rule on the Laplace integral of 1/z)
    import numpy as np
    import paper_2409_09471_gb300 as g
    from oracle import precond as opc
    for a, b, tol in [(1.0, 100.0, 1e-2), (39.4, 1.1e4, 1e-4), (2.0, 3e6, 1e-8)]:
        al, be = g.exp_sum_coefficients(a, b, tol)
        ao, bo = opc.exp_sum_coefficients(a, b, tol)
        assert al.shape == ao.shape
        assert np.allclose(al, ao, rtol=1e-13, atol=0) and np.allclose(be, bo, rtol=1e-13, atol=0)
    from paper_2409_09471_gb300 import _abi
    assert _abi.lib.tt_exp_sum_coefficients(2.0, 1.0, 1e-2, 0, None, None) == -1
    assert _abi.lib.tt_exp_sum_coefficients(1.0, 2.0, 1.5, 0, None, None) == -1


def test_precond_entry_points_validate_and_size_on_the_host(built_lib):
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    d, ns = 3, [8, 8, 8]
    n = (ctypes.c_int64 * d)(*ns)
    r = (ctypes.c_int64 * (d + 1))(1, 3, 4, 1)
    xc = (ctypes.c_void_p * d)(*([0x1000] * d))
    x = _abi.TTVec(d, n, r, xc)
    alpha = (ctypes.c_double * 5)(1.0, 0.5, 0.25, 0.1, 0.05)
    beta = (ctypes.c_double * 5)(0.01, 0.02, 0.04, 0.08, 0.16)
    mats = (ctypes.c_void_p * d)(*([0x3000] * d))
    P = _abi.TTPrecond(5, alpha, beta, mats)
    for mode in (0, 1, 2):
        assert lib.tt_precond_apply_workspace(mode, ctypes.byref(P), ctypes.byref(x), 6, 2) > 0, \
            lib.tt_last_error()
    bad = _abi.TTPrecond(0, alpha, beta, mats)
    assert lib.tt_precond_apply_workspace(0, ctypes.byref(bad), ctypes.byref(x), 6, 2) == 0
    assert b"zeta" in lib.tt_last_error()
    negb = (ctypes.c_double * 5)(0.01, -0.02, 0.04, 0.08, 0.16)
    bad2 = _abi.TTPrecond(5, alpha, negb, mats)
    assert lib.tt_precond_apply_workspace(0, ctypes.byref(bad2), ctypes.byref(x), 6, 2) == 0
    # the preconditioned solve's workspace query is a host dry run too
    R = (ctypes.c_int64 * (d + 1))(1, 2, 2, 1)
    opc = (ctypes.c_void_p * d)(*([0x2000] * d))
    op = _abi.TTOp(d, n, R, opc)
    for mode in (0, 2):
        p = _abi.SolverParams(20, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode)
        plain = lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(x), ctypes.byref(p))
        pre = lib.tt_spgmres_solve_workspace(ctypes.byref(op), ctypes.byref(P), ctypes.byref(x),
                                             ctypes.byref(p))
        assert pre > plain > 0, lib.tt_last_error()
        ps = _abi.SolverParams(20, 40, 1e-6, 0.0, 0.1, 0.1, 16, 16, 4, 0, 2, mode, 1)
        assert lib.tt_spgmres_solve_workspace(ctypes.byref(op), ctypes.byref(P), ctypes.byref(x),
                                              ctypes.byref(ps)) == 0
        assert b"final_stta" in lib.tt_last_error()


def test_stta_correction_drops_the_basis_storage(built_lib):
    # With the STTA correction only the ell + 1 basis vectors of the
    # Gram-Schmidt window are stored; each basis vector leaves its sketches
    # (target ranks r_sol, left ranks r_sol + 20) instead.  In the regime the
    # paper's streaming form is for, basis ranks (here 128) above the
    # solution's (here 24), the workspace is 0.4 of the rounding form's,
    # which keeps all maxit + 1 basis vectors (d = 10, n = 64, maxit = 80).
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    d, nn = 10, 64
    n = (ctypes.c_int64 * d)(*([nn] * d))
    R = (ctypes.c_int64 * (d + 1))(*([1] + [2] * (d - 1) + [1]))
    op = _abi.TTOp(d, n, R, (ctypes.c_void_p * d)(*([0x1000] * d)))
    r = (ctypes.c_int64 * (d + 1))(*([1] + [4] * (d - 1) + [1]))
    b = _abi.TTVec(d, n, r, (ctypes.c_void_p * d)(*([0x2000] * d)))
    for mode in (0, 1):
        rnd = _abi.SolverParams(80, 160, 1e-6, 0.0, 0.1, 0.1, 128, 24, 10, 0, 4, mode, 0, 1)
        sta = _abi.SolverParams(80, 160, 1e-6, 0.0, 0.1, 0.1, 128, 24, 10, 0, 4, mode, 1, 1)
        w_rnd = lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b), ctypes.byref(rnd))
        w_sta = lib.tt_sgmres_solve_workspace(ctypes.byref(op), ctypes.byref(b), ctypes.byref(sta))
        assert w_rnd > 0 and w_sta > 0, lib.tt_last_error()
        vec = (2 * nn * 128 + (d - 2) * 128 * nn * 128) * (8 if mode == 0 else 4)
        assert w_rnd >= 81 * vec
        # the 79 basis vectors beyond the window of two are gone; their
        # sketches (80 x 10 cores of 44 x 64 x 24 doubles) cost far less
        sketches = 80 * (d * 44 * nn * 24) * 8
        assert w_rnd - w_sta >= 79 * vec - sketches - (64 << 20)
        assert w_sta < 0.5 * w_rnd, (w_sta, w_rnd)
