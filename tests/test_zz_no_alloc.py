"""The allocation-free inner product ``tt_dot_noalloc`` (for callers that cannot
allocate device memory) against the workspace-based ``tt_dot``, called through
the C ABI twice in a row on the same inputs (the shared scratch array keeps the
previous call's contents, so the second call checks that nothing stale leaks
in).  This file runs last; it must also pass alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as ott

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_09471_gb300 as g
    return g


def _noalloc(g, x, y, mode):
    from paper_2409_09471_gb300._abi import lib
    xd, k1 = x._desc()
    yd, k2 = y._desc()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.tt_dot_noalloc(mode, ctypes.byref(xd), ctypes.byref(yd),
                            ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, out.item()


@pytest.mark.parametrize("mode,tol", [(0, 1e-12), (1, 2e-5), (2, 2e-5)])
def test_noalloc_dot_matches_tt_dot_twice(g, mode, tol):
    ns = [13, 64, 7, 30, 64]
    dt = g.mode_dtype(mode)
    pairs = [(ti.random_tt(ns, [1, 5, 70, 3, 64, 1], seed=1), ti.random_tt(ns, [1, 2, 9, 65, 8, 1], seed=2)),
             (ti.random_tt(ns, [1, 3, 4, 5, 6, 1], seed=3), ti.random_tt(ns, [1, 7, 1, 2, 3, 1], seed=4))]
    for xc, yc in pairs:
        x, y = g.TT.from_numpy(xc, dt), g.TT.from_numpy(yc, dt)
        ref = g.tt_dot(x, y, mode=mode).item()
        scale = np.sqrt(g.tt_dot(x, x, mode=mode).item() * g.tt_dot(y, y, mode=mode).item())
        exact = ott.dot(x.numpy(), y.numpy())  # the oracle, on the stored values
        for _ in range(2):
            rc, val = _noalloc(g, x, y, mode)
            assert rc == 0
            assert abs(val - ref) <= tol * scale
            assert abs(val - exact) <= tol * scale


def test_noalloc_rejects_inputs_beyond_the_fixed_scratch(g):
    from paper_2409_09471_gb300._abi import lib
    # ranks 300 at n = 64: the Gram sweep needs far more than the fixed scratch;
    # the check happens on the host before any device work
    ns = [64, 64, 64]
    x = g.TT([torch.zeros((1, 64, 300), device="cuda"), torch.zeros((300, 64, 300), device="cuda"),
              torch.zeros((300, 64, 1), device="cuda")])
    rc, _ = _noalloc(g, x, x, 1)
    assert rc == 1
    assert b"fixed" in lib.tt_last_error()
