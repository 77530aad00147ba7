// TT operations of the solver iteration, expressed as grouped GEMMs plus the
// FP64 QR / Jacobi kernels.  All functions enqueue work on ctx.st; functions
// that must learn data-dependent ranks synchronise that stream.
#pragma once
#include "kernels.cuh"

namespace ttsg {

struct Ctx {
  int mode = TT_MODE_FP32;
  cudaStream_t st = nullptr;
  Arena* ar = nullptr;
  int* err = nullptr;        // device flags: err[0] bit 0 = QR barrier timeout,
                             // err[1] = Jacobi sweep-cap count
  double* scratch = nullptr; // device scratch for reductions (>= 256 doubles)
  // randomized rounding only: an event the left-to-right sweep waits for (the
  // term coefficients on the device are read from that sweep on; the
  // right-to-left partial contractions before it do not need them)
  cudaEvent_t left_wait = nullptr;
  bool f64() const { return mode == TT_MODE_FP64; }
};

// One term of an implicit sum: coef * (*coef_dev if set) * X.
template <typename T>
struct Term {
  TTv<T> X;
  double coef = 1.0;
  const double* coef_dev = nullptr;
};

// Source of the Gaussian TT-DRM of a randomized rounding: explicit cores with
// capacity ranks L, or the Philox stream (seed, 2048 + k) read as a virtual
// array of capacity ranks L.
template <typename T>
struct DRMSource {
  const T* const* core = nullptr;  // nullptr => Philox
  int64_t L[MAXD + 1] = {};
  uint64_t seed = 0;
};

template <typename T>
void tt_matvec_dev(const Ctx& c, const TTop<T>& A, const TTv<T>& x, const TTv<T>& y);

template <typename T>
void tt_sketch_dev(const Ctx& c, const TTv<T>& x, int64_t s, const T* const* S, double* out);

template <typename T>
void tt_dot_dev(const Ctx& c, const TTv<T>& x, const TTv<T>& y, double* out);
// Derivative of <x, y> with respect to every core of y (g[k] shaped like
// y's core k; nullptr skips it) and, when M is given, dots[k] = <x, (I x .. x
// M[k] x .. x I) y> in FP64 (adjoint.cu).
template <typename T>
void tt_dot_grad_dev(const Ctx& c, const TTv<T>& x, const TTv<T>& y, T* const* g,
                     const T* const* M, double* dots);
// Cores of the rank-2 operator sum_k theta_k (I x .. x M[k] x .. x I).
template <typename T>
void tt_kron_sum_op_dev(cudaStream_t st, int d, const int64_t* n, const T* const* M,
                        const double* theta, T* const* cores);
// Cores of A^T (input and output mode indices swapped in every core).
template <typename T>
void tt_op_transpose_dev(cudaStream_t st, const TTop<T>& A, T* const* cores);

// Randomize-then-orthogonalize rounding of sum_b terms[b] into y (cores with
// capacity; y.r[] is filled in).  Returns after a stream synchronisation.
template <typename T>
void tt_round_rand_dev(const Ctx& c, const std::vector<Term<T>>& terms, double eps, int64_t rmax,
                       int64_t oversample, const DRMSource<T>& drm, TTv<T>& y);

// STTA sketches of x with right DRM X and left DRM Y, accumulated into FP64
// psi[0..d-1] and omega[0..d-2] (see tt_stta_sketch), and the recovery of the
// approximant's FP64 cores from them (see tt_stta_recover).
template <typename T>
void tt_stta_sketch_dev(const Ctx& c, const TTv<T>& x, double coef, int accumulate,
                        const TTv<T>& X, const TTv<T>& Y, double* const* psi,
                        double* const* omega);
void tt_stta_recover_dev(const Ctx& c, int d, const int64_t* n, const int64_t* r,
                         const int64_t* l, const double* const* psi, const double* const* omega,
                         double rcond, double* const* cores);
// out = sum_{i < k} y[i] S_i for k sketches stored ssz doubles apart (y on the device).
void stta_combine(const double* S, int64_t ssz, int k, const double* y, double* out,
                  cudaStream_t st);

// Exponential-sum preconditioner (see tt_precond_apply): host description
// (coefficients, device pointers to the 1-D FP64 matrices A_k) and its device
// form (the matrices exp(-beta_i A_k) in the working precision).
constexpr int TT_MAX_PRECOND_TERMS = 256;
struct PrecondArgs {
  int zeta = 0;
  const double* alpha = nullptr;      // host [zeta]
  const double* beta = nullptr;       // host [zeta]
  const double* const* A1d = nullptr; // host array of d device pointers
};
template <typename T>
struct PrecondDev {
  int zeta = 0, d = 0;
  std::vector<double> alpha;
  std::vector<T*> E;  // E[i * d + k] = exp(-beta_i A_k), n_k x n_k row-major
};
// Coefficients of the exponential sum for 1/z on [a, b] at relative accuracy
// tol; returns the number of terms (written only when it is <= cap), or -1.
int exp_sum_coefficients(double a, double b, double tol, int cap, double* alpha, double* beta);
template <typename T>
void precond_setup(const Ctx& c, const PrecondArgs& P, int d, const int64_t* n,
                   PrecondDev<T>& out);
// y = Round(P^{-1} x) to eps and rmax; bufs: zeta TT buffers with capacity >= x's ranks.
template <typename T>
void precond_apply_dev(const Ctx& c, const PrecondDev<T>& P, const TTv<T>& x, double eps,
                       int64_t rmax, int64_t oversample, const DRMSource<T>& drm,
                       std::vector<TTv<T>>& bufs, TTv<T>& y);

// Sketch ranks l_mu of the randomized rounding (see tt_round_rand).
void rto_ranks(const std::vector<const int64_t*>& term_ranks, const int64_t* n, int d,
               int64_t rmax, int64_t oversample, int64_t* ells);

// Exact ||b - A x|| in FP64 (QR sweep of the explicit sum; A x is formed in
// FP64).  x in the working precision, A and b in FP64 (A permuted layout).
template <typename T>
double true_residual_norm(const Ctx& c, const TTop<double>& A, const TTv<double>& b,
                          const TTv<T>& x);

// Raise TT_ERR_TIMEOUT if a device wait expired (synchronises).
void check_device_flags(const Ctx& c);

}  // namespace ttsg
