"""The Markov-chain workload on the GPU (Section 5.1.2; the steady state of
d = 5 coupled random walks of n = 32 states, read as the rank-one-normalised
system ``(-G_c + 1 1^T / N) rho = 1`` whose solution is ``rho = N pi``), solved
by the right-preconditioned TT-sPGMRES (Algorithm 5, exponential sum of the
shifted independent part) in FP64 and TF32 modes.  Each solution is checked
with the oracle's exact FP64 residual, and as a probability distribution: its
entries sum to N (``<rho, 1> = N``, by the oracle's inner product)."""
import numpy as np
import pytest
import torch

import ttinputs as ti
from oracle import tt as ott, solvers as osol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_09471_gb300 as g
    return g


@pytest.mark.parametrize("mode", [0, 2])
def test_markov_preconditioned_solve(g, mode):
    w = ti.workload("markov")
    p = w.params
    blocks, a, b = ti.markov_precond_blocks(w.extra["Q"])
    P = g.Precond.for_interval(a, b, 1e-2, [torch.as_tensor(B, device="cuda") for B in blocks])
    x, info = g.tt_spgmres_solve(g.op_to_device(w.op), P, g.TT.from_numpy(w.b), maxit=p["maxit"],
                                 tol=p["tol"], rmax=p["rmax"], mode=mode, s=p["s"], eta=p["eta"],
                                 r_sol=p["r_sol"], oversample=p["oversample"], max_restarts=10)
    assert info["status"] == 0, info
    xc = x.numpy()
    res = osol.true_residual_norm(w.op, xc, w.b) / ott.norm(w.b)
    assert res <= 1e-6
    assert abs(res - info["true_res"]) <= 1e-2 * res + 1e-14
    N = float(np.prod(w.ns))
    # <rho, 1> = N exactly for the exact solution; a residual r changes it by at
    # most |<1, A^{-T} r>|, and 1^T A = 1^T (columns of G_c sum to zero), so
    # <1, A^{-1} r> = <1, r>: the sum is within ||1|| ||r|| = sqrt(N) ||r||
    total = ott.dot(xc, w.b)
    assert abs(total - N) <= np.sqrt(N) * res * ott.norm(w.b) * 1.01 + 1e-9 * N
