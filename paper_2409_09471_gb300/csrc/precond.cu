// Exponential-sum right preconditioning of a Kronecker-sum operator (Section
// 4, Algorithm 5):
//   P^{-1} = sum_i alpha_i (exp(-beta_i A_1) x .. x exp(-beta_i A_d)),
// an exponential sum E(z) = sum_i alpha_i exp(-beta_i z) ~ 1/z evaluated at the
// Kronecker sum (its terms commute, so exp(-beta sum_j A_j) is the Kronecker
// product of the exp(-beta A_j)).  Applying it to a TT vector multiplies every
// core by exp(-beta_i A_k) along its mode index (ranks unchanged) and rounds the
// zeta-term sum to a rank cap (the bounded-rank rounding of Section 4.2).
//
// The coefficients come from the trapezoidal rule on 1/z = int_R exp(t - e^t z) dt
// (Trefethen and Weideman, "The exponentially convergent trapezoidal rule",
// SIAM Review 2014).  For z = a u, u in [1, b/a], with nodes t_k = k h:
// alpha_k = h e^{t_k} / a, beta_k = e^{t_k} / a; lower cutoff log(tol a / b)
// (tail below u e^t), upper cutoff log(log(1/tol)) (tail exp(-e^t u) / u), and
// step h = pi^2 / (2 log(1/tol)) from a strip of half-width pi/4 about the
// real axis, where the integrand keeps decaying.
//
// The matrix exponentials are FP64: Taylor polynomial of degree 18 on
// X = -beta A / 2^s with ||X||_1 <= 1/2 (Horner steps P <- I + X P / k), then s
// squarings (Moler and Van Loan, "Nineteen dubious ways to compute the
// exponential of a matrix, twenty-five years later", SIAM Review 2003).
#include "tt_ops.cuh"

#include <cmath>

namespace ttsg {

namespace {

__global__ void set_identity_kernel(double* __restrict__ C, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x)
    C[e] = (e / n == e % n) ? 1.0 : 0.0;
}

void set_identity(double* C, int64_t n, cudaStream_t st) {
  if (g_dry_run) return;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>(ceil_div(n * n, threads), 152 * 4);
  set_identity_kernel<<<blocks, threads, 0, st>>>(C, n);
  check_launch("set_identity_kernel");
}

constexpr int EXPM_DEGREE = 18;

// E = exp(-beta A), A n x n row-major FP64 with ||A||_1 = anorm1; W0, W1 are
// n x n scratch; E may not alias them.
void expm_neg_f64(const double* A, int64_t n, double beta, double anorm1, double* E, double* W0,
                  double* W1, cudaStream_t st) {
  const double xn = beta * anorm1;
  int s = 0;
  if (xn > 0.5) s = (int)std::ceil(std::log2(xn / 0.5));
  const double scale = -beta / std::ldexp(1.0, s);
  set_identity(W0, n, st);
  for (int k = EXPM_DEGREE; k >= 1; --k) {
    // W1 = I + (X / k) W0, X = scale * A
    set_identity(W1, n, st);
    gemm(TT_MODE_FP64,
         {gemm_rm((int)n, (int)n, (int)n, A, n, W0, n, W1, n, scale / (double)k, 1.0)}, st);
    std::swap(W0, W1);
  }
  for (int i = 0; i < s; ++i) {
    gemm(TT_MODE_FP64, {gemm_rm((int)n, (int)n, (int)n, W0, n, W0, n, W1, n)}, st);
    std::swap(W0, W1);
  }
  CopySeg cs;
  cs.src = W0; cs.dst = E; cs.A = n * n; cs.sa = 1; cs.src_f64 = cs.dst_f64 = 1;
  copy3d({cs}, st);
}

}  // namespace

int exp_sum_coefficients(double a, double b, double tol, int cap, double* alpha, double* beta) {
  if (!(a > 0.0) || !(b > a) || !(tol > 0.0) || !(tol < 1.0)) return -1;
  const double kappa = b / a;
  const double t_lo = std::log(tol / kappa);
  const double t_hi = std::log(std::log(1.0 / tol));
  const double h = M_PI * M_PI / (2.0 * std::log(1.0 / tol));
  const int64_t k0 = (int64_t)std::floor(t_lo / h);
  const int64_t k1 = (int64_t)std::ceil(t_hi / h);
  const int64_t count = k1 - k0 + 1;
  if (alpha && beta && count <= cap) {
    for (int64_t k = k0; k <= k1; ++k) {
      const double t = h * (double)k;
      alpha[k - k0] = h * std::exp(t) / a;
      beta[k - k0] = std::exp(t) / a;
    }
  }
  return (int)count;
}

template <typename T>
void precond_setup(const Ctx& c, const PrecondArgs& P, int d, const int64_t* n,
                   PrecondDev<T>& out) {
  TT_CHECK_ARG(P.zeta >= 1 && P.zeta <= TT_MAX_PRECOND_TERMS,
               "precond: 1 <= zeta <= " + std::to_string(TT_MAX_PRECOND_TERMS));
  Arena& ar = *c.ar;
  out.zeta = P.zeta;
  out.d = d;
  out.alpha.assign(P.alpha, P.alpha + P.zeta);
  int64_t nmax = 1;
  for (int k = 0; k < d; ++k) nmax = std::max(nmax, n[k]);
  // ||A_k||_1 from host copies (setup only; the dry run uses placeholders)
  std::vector<double> norm1(d, 1.0);
  if (!g_dry_run) {
    std::vector<double> h(nmax * nmax);
    for (int k = 0; k < d; ++k) {
      TT_CUDA(cudaMemcpyAsync(h.data(), P.A1d[k], sizeof(double) * n[k] * n[k],
                              cudaMemcpyDeviceToHost, c.st));
      TT_CUDA(cudaStreamSynchronize(c.st));
      double m = 0.0;
      for (int64_t col = 0; col < n[k]; ++col) {
        double acc = 0.0;
        for (int64_t row = 0; row < n[k]; ++row) acc += std::fabs(h[row * n[k] + col]);
        m = std::max(m, acc);
      }
      norm1[k] = m;
    }
  }
  out.E.assign((size_t)P.zeta * d, nullptr);
  for (int i = 0; i < P.zeta; ++i)
    for (int k = 0; k < d; ++k) out.E[(size_t)i * d + k] = ar.take<T>(n[k] * n[k]);
  const size_t mk = ar.mark();
  double* W0 = ar.take<double>(nmax * nmax);
  double* W1 = ar.take<double>(nmax * nmax);
  double* E64 = sizeof(T) == 8 ? nullptr : ar.take<double>(nmax * nmax);
  for (int i = 0; i < P.zeta; ++i) {
    for (int k = 0; k < d; ++k) {
      T* dst = out.E[(size_t)i * d + k];
      double* e = sizeof(T) == 8 ? (double*)dst : E64;
      expm_neg_f64(P.A1d[k], n[k], P.beta[i], norm1[k], e, W0, W1, c.st);
      if (sizeof(T) != 8) {
        CopySeg cs;
        cs.src = E64; cs.dst = dst; cs.A = n[k] * n[k]; cs.sa = 1; cs.src_f64 = 1;
        cs.dst_f64 = 0;
        copy3d({cs}, c.st);
      }
    }
  }
  ar.release(mk);
}

template <typename T>
void precond_apply_dev(const Ctx& c, const PrecondDev<T>& P, const TTv<T>& x, double eps,
                       int64_t rmax, int64_t oversample, const DRMSource<T>& drm,
                       std::vector<TTv<T>>& bufs, TTv<T>& y) {
  const int d = x.d;
  TT_CHECK_ARG((int)bufs.size() >= P.zeta, "precond: too few term buffers");
  // term i, core k: exp(-beta_i A_k) applied along the mode index of x's core,
  // a GEMM batched over the left rank
  std::vector<GemmProblem> probs;
  for (int i = 0; i < P.zeta; ++i) {
    TTv<T>& b = bufs[i];
    b.d = d;
    for (int k = 0; k <= d; ++k) b.r[k] = x.r[k];
    for (int k = 0; k < d; ++k) {
      b.n[k] = x.n[k];
      const int64_t nn = x.n[k], r0 = x.r[k], r1 = x.r[k + 1];
      GemmProblem g;
      g.M = (int)nn; g.N = (int)r1; g.K = (int)nn;
      g.nb1 = (int)r0;
      g.A = P.E[(size_t)i * d + k]; g.sAm = nn; g.sAk = 1; g.sAb1 = 0;
      g.B = x.core[k]; g.sBk = r1; g.sBn = 1; g.sBb1 = nn * r1;
      g.C = b.core[k]; g.sCm = r1; g.sCn = 1; g.sCb1 = nn * r1;
      probs.push_back(g);
    }
  }
  gemm(c.mode, probs, c.st);
  std::vector<Term<T>> terms(P.zeta);
  for (int i = 0; i < P.zeta; ++i) {
    terms[i].X = bufs[i];
    terms[i].coef = P.alpha[i];
  }
  tt_round_rand_dev<T>(c, terms, eps, rmax, oversample, drm, y);
}

template void precond_setup<float>(const Ctx&, const PrecondArgs&, int, const int64_t*,
                                   PrecondDev<float>&);
template void precond_setup<double>(const Ctx&, const PrecondArgs&, int, const int64_t*,
                                    PrecondDev<double>&);
template void precond_apply_dev<float>(const Ctx&, const PrecondDev<float>&, const TTv<float>&,
                                       double, int64_t, int64_t, const DRMSource<float>&,
                                       std::vector<TTv<float>>&, TTv<float>&);
template void precond_apply_dev<double>(const Ctx&, const PrecondDev<double>&, const TTv<double>&,
                                        double, int64_t, int64_t, const DRMSource<double>&,
                                        std::vector<TTv<double>>&, TTv<double>&);

}  // namespace ttsg
