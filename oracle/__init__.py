"""FP64 CPU oracle for randomized sketched TT-GMRES (arXiv 2409.09471).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the CUDA library and its Python binding never do, and this package never
imports them.  The two share no code; the only common dependency is the seeded
input generator module ``ttinputs``, which holds none of the method's arithmetic.

Every routine is written in float64 with NumPy, following the paper's
definitions in the paper's order.  Library primitives (matrix products,
LAPACK QR/SVD/lstsq) serve as single steps; there is no blocking, fusion or
reordering beyond what the definitions state.

Modules
-------
``tt``          TT containers, dense reconstruction, matvec, inner products,
                Khatri-Rao sketch (sweep and explicit dense form).
``rounding``    TT-SVD rounding and randomize-then-orthogonalize rounding of
                (implicit) sums of TT vectors.
``solvers``     sketched least squares, TT-sGMRES (Algorithm 4 with l = 1),
                restarted driver, full-orthogonalisation TT-GMRES (Algorithm 2).
``philox``      Philox4x32-10 counter-based generator + Box-Muller Gaussians.
``closed_forms`` closed-form eigenpairs of the 1-D model matrices and the
                fast-diagonalisation dense solve of Kronecker sums.
``adjoint``     dense gradient of ``||x(theta, b) - x_t||^2`` on tiny grids.
``stta``        streaming TT approximation: two-sided sketches with Gaussian
                TT-DRMs (dense definition and partial contractions) and the
                recovery of the approximant from them.
``precond``     exponential-sum right preconditioning of Kronecker-sum
                operators and TT-sPGMRES (Algorithm 5).

Parity status: every function has at least one pin in ``tests/test_oracle_*``
except where a docstring says "parity unpinned".
"""
from . import tt, rounding, solvers, philox, closed_forms, adjoint, stta, precond  # noqa: F401
