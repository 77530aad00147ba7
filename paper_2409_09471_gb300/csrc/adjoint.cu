// Backward contractions of the differentiable solve.
//
// For the loss L(theta, b) = ||x - x_t||^2 with A(theta) x = b the adjoint
// vector lambda solves A^T lambda = 2 (x - x_t) (one more TT-sGMRES solve), and
//   dL/dtheta_k = - <lambda, (dA/dtheta_k) x>,   dL/db = lambda.
// Both reduce to the inner-product sweep of Section 2.2 differentiated with
// respect to one core: with the left and right interface matrices of x
// against y,
//   P_0 = 1,  P_{k+1} = sum_i X_k[:, i, :]^T P_k Y_k[:, i, :]      (x.r[k] x y.r[k])
//   Q_d = 1,  Q_k     = sum_i X_k[:, i, :] Q_{k+1} Y_k[:, i, :]^T
// the derivative of <x, y> with respect to Y_k is
//   G_k[b, i, c] = sum_{a, a'} P_k[a, b] X_k[a, i, a'] Q_{k+1}[a', c],
// and <x, (I x .. x M x .. x I) y> (M acting on mode k) = <G_k, M x_2 Y_k>.
// Every step is a grouped GEMM; the per-core inner products accumulate in
// FP64.
#include "tt_ops.cuh"

namespace ttsg {

namespace {

// Rank-2 Kronecker-sum operator core k of sum_k theta_k (I x .. x M_k x .. x I):
// first [theta M, I], middle [[I, 0], [theta M, I]], last [I; theta M]; d == 1
// gives [[theta M]].
template <typename T>
__global__ void kron_core_kernel(T* core, const T* M, int64_t n, int R0, int R1, int first,
                                 int last, double theta) {
  const int64_t total = (int64_t)R0 * n * n * R1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a1 = (int)(e % R1);
    const int64_t j = (e / R1) % n, i = (e / (R1 * n)) % n;
    const int a0 = (int)(e / (R1 * n * n));
    const double mij = theta * (double)M[i * n + j];
    const double id = i == j ? 1.0 : 0.0;
    double v;
    if (first && last) v = mij;
    else if (first) v = a1 == 0 ? mij : id;
    else if (last) v = a0 == 0 ? id : mij;
    else v = (a0 == 0 && a1 == 0) ? id : (a0 == 1 && a1 == 0) ? mij : (a0 == 1 && a1 == 1) ? id : 0.0;
    core[e] = (T)v;
  }
}

}  // namespace

template <typename T>
void tt_dot_grad_dev(const Ctx& c, const TTv<T>& x, const TTv<T>& y, T* const* g,
                     const T* const* M, double* dots) {
  const int d = x.d;
  const size_t mk = c.ar->mark();
  const int f64 = sizeof(T) == 8;
  int64_t nmax = 1, umax = 1;
  std::vector<T*> P(d + 1, nullptr), Q(d + 1, nullptr);
  for (int k = 0; k < d; ++k) {
    nmax = std::max(nmax, x.n[k]);
    umax = std::max(umax, std::max(x.r[k], y.r[k]) * x.n[k] * std::max(x.r[k + 1], y.r[k + 1]));
  }
  for (int k = 1; k < d; ++k) {
    P[k] = c.ar->take<T>(x.r[k] * y.r[k]);
    Q[k] = c.ar->take<T>(x.r[k] * y.r[k]);
  }
  T* U = c.ar->take<T>(umax);
  // G_k goes to a scratch buffer unless only the gradient is wanted (the dry
  // run's arena returns null pointers, so ownership is a flag, not a test)
  const bool own_g = !(g && !M);
  T* Gs = own_g ? c.ar->take<T>(umax) : nullptr;
  T* MY = M ? c.ar->take<T>(umax) : nullptr;

  // left interfaces: U = P_k Y_k ((x.r[k]) x (n y.r[k+1])), P_{k+1} = X_k^T U
  for (int k = 0; k + 1 < d; ++k) {
    const int64_t t0 = x.r[k], t1 = x.r[k + 1], q0 = y.r[k], q1 = y.r[k + 1], n = x.n[k];
    const T* Uk = y.core[k];
    if (k > 0) {
      gemm(c.mode, {gemm_rm((int)t0, (int)(n * q1), (int)q0, P[k], q0, y.core[k], n * q1, U, n * q1)},
           c.st);
      Uk = U;
    }
    GemmProblem gp;
    gp.M = (int)t1; gp.N = (int)q1; gp.K = (int)(t0 * n);
    gp.A = x.core[k]; gp.sAm = 1; gp.sAk = t1;
    gp.B = Uk; gp.sBk = q1; gp.sBn = 1;
    gp.C = P[k + 1]; gp.sCm = q1; gp.sCn = 1;
    gemm(c.mode, {gp}, c.st);
  }
  // right interfaces: V = X_k Q_{k+1} ((x.r[k] n) x y.r[k+1]), Q_k = V Y_k^T
  for (int k = d - 1; k >= 1; --k) {
    const int64_t t0 = x.r[k], t1 = x.r[k + 1], q0 = y.r[k], q1 = y.r[k + 1], n = x.n[k];
    const T* Vk = x.core[k];
    if (k < d - 1) {
      gemm(c.mode, {gemm_rm((int)(t0 * n), (int)q1, (int)t1, x.core[k], t1, Q[k + 1], q1, U, q1)},
           c.st);
      Vk = U;
    }
    GemmProblem gp;
    gp.M = (int)t0; gp.N = (int)q0; gp.K = (int)(n * q1);
    gp.A = Vk; gp.sAm = n * q1; gp.sAk = 1;
    gp.B = y.core[k]; gp.sBk = 1; gp.sBn = n * q1;
    gp.C = Q[k]; gp.sCm = q0; gp.sCn = 1;
    gemm(c.mode, {gp}, c.st);
  }
  // per core: W = X_k Q_{k+1}, G_k = P_k^T W
  for (int k = 0; k < d; ++k) {
    const int64_t t0 = x.r[k], t1 = x.r[k + 1], q0 = y.r[k], q1 = y.r[k + 1], n = x.n[k];
    T* Gk = own_g ? Gs : g[k];
    const T* Wk = x.core[k];
    if (k < d - 1) {
      T* W = (k == 0) ? Gk : U;  // P_0 = 1: G_0 = W directly
      gemm(c.mode, {gemm_rm((int)(t0 * n), (int)q1, (int)t1, x.core[k], t1, Q[k + 1], q1, W, q1)},
           c.st);
      Wk = W;
    } else if (k == 0) {
      CopySeg cs;
      cs.src = x.core[0]; cs.dst = Gk; cs.A = n; cs.sa = 1; cs.src_f64 = cs.dst_f64 = f64;
      copy3d({cs}, c.st);
    }
    if (k > 0) {
      GemmProblem gp;
      gp.M = (int)q0; gp.N = (int)(n * q1); gp.K = (int)t0;
      gp.A = P[k]; gp.sAm = 1; gp.sAk = q0;
      gp.B = Wk; gp.sBk = n * q1; gp.sBn = 1;
      gp.C = Gk; gp.sCm = n * q1; gp.sCn = 1;
      gemm(c.mode, {gp}, c.st);
    }
    if (M) {
      // MY[b][i][c] = sum_j M[i][j] Y_k[b][j][c], then <G_k, MY> in FP64
      GemmProblem gp;
      gp.M = (int)n; gp.N = (int)q1; gp.K = (int)n; gp.nb1 = (int)q0;
      gp.A = M[k]; gp.sAm = n; gp.sAk = 1; gp.sAb1 = 0;
      gp.B = y.core[k]; gp.sBk = q1; gp.sBn = 1; gp.sBb1 = n * q1;
      gp.C = MY; gp.sCm = q1; gp.sCn = 1; gp.sCb1 = n * q1;
      gemm(c.mode, {gp}, c.st);
      dot_acc(Gk, MY, f64, q0 * n * q1, dots + k, c.scratch + 16, c.st);
      if (g && g[k] != Gk) {
        CopySeg cs;
        cs.src = Gk; cs.dst = g[k]; cs.A = q0 * n * q1; cs.sa = 1; cs.src_f64 = cs.dst_f64 = f64;
        copy3d({cs}, c.st);
      }
    }
  }
  c.ar->release(mk);
}

template <typename T>
void tt_kron_sum_op_dev(cudaStream_t st, int d, const int64_t* n, const T* const* M,
                        const double* theta, T* const* cores) {
  if (g_dry_run) return;
  for (int k = 0; k < d; ++k) {
    const int R0 = k == 0 ? 1 : 2, R1 = k == d - 1 ? 1 : 2;
    const int64_t total = (int64_t)R0 * n[k] * n[k] * R1;
    const int blocks = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(total, (int64_t)256), 1), 4096);
    kron_core_kernel<T><<<blocks, 256, 0, st>>>(cores[k], M[k], n[k], R0, R1, k == 0, k == d - 1,
                                                theta ? theta[k] : 1.0);
    check_launch("kron_core_kernel");
  }
}

template <typename T>
void tt_op_transpose_dev(cudaStream_t st, const TTop<T>& A, T* const* cores) {
  std::vector<CopySeg> segs;
  const int f64 = sizeof(T) == 8;
  for (int k = 0; k < A.d; ++k) {
    const int64_t R0 = A.R[k], R1 = A.R[k + 1], n = A.n[k];
    for (int64_t a = 0; a < R0; ++a) {
      // dst[a][j][i][a'] = src[a][i][j][a']: A index j, B index i, C index a'
      CopySeg s;
      s.src = A.core[k] + a * n * n * R1;
      s.dst = cores[k] + a * n * n * R1;
      s.A = n; s.B = n; s.C = R1;
      s.sa = R1; s.sb = n * R1; s.sc = 1;
      s.da = n * R1; s.db = R1; s.dc = 1;
      s.src_f64 = s.dst_f64 = f64;
      segs.push_back(s);
    }
  }
  copy3d(segs, st);
}

template void tt_dot_grad_dev<float>(const Ctx&, const TTv<float>&, const TTv<float>&, float* const*,
                                     const float* const*, double*);
template void tt_dot_grad_dev<double>(const Ctx&, const TTv<double>&, const TTv<double>&,
                                      double* const*, const double* const*, double*);
template void tt_kron_sum_op_dev<float>(cudaStream_t, int, const int64_t*, const float* const*,
                                        const double*, float* const*);
template void tt_kron_sum_op_dev<double>(cudaStream_t, int, const int64_t*, const double* const*,
                                         const double*, double* const*);
template void tt_op_transpose_dev<float>(cudaStream_t, const TTop<float>&, float* const*);
template void tt_op_transpose_dev<double>(cudaStream_t, const TTop<double>&, double* const*);

}  // namespace ttsg
