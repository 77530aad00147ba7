// Restarted TT-sGMRES driver (solver.cu).
#pragma once
#include "tt_ops.cuh"

namespace ttsg {

struct SolveParams {
  int maxit = 50;
  int64_t s = 0;
  double tol = 1e-6;
  double round_tol = 0.0;
  double eta = 0.1;
  double stop_safety = 0.1;
  int64_t rmax = 40;
  int64_t r_sol = 0;
  int64_t oversample = 10;
  uint64_t seed = 0;
  int max_restarts = 5;
  int final_stta = 0;
  int ell = 1;
  const PrecondArgs* pre = nullptr;  // right preconditioner (Algorithm 5), or none
};

struct SolveResult {
  int iters = 0, cycles = 0, status = TT_OK, svd_nonconverged = 0, svd_max_sweeps = 0;
  int breakdowns = 0;  // cycles that ended on h_{k+1,k} = 0 (Krylov space invariant)
  double svd_mean_sweeps = 0.0;
  double sketched_res = 0, true_res = 0, seconds = 0;
  int64_t max_rank = 0;
  std::vector<double> res_hist;
  std::vector<int64_t> rank_hist;
};

// Solves A x = b (A, b in FP64, A in the caller's [a][i][j][a'] layout) in the
// precision of c.mode; x (FP64 cores with capacity r_sol) receives the result.
template <typename T>
SolveResult sgmres_solve(const Ctx& c, const TTop<double>& A, const TTv<double>& b,
                         const SolveParams& p, TTv<double>& x);

}  // namespace ttsg
