// Declarations of the element-wise / data-movement kernels (kernels.cu), the
// FP64 Householder QR (qr.cu), the small Jacobi SVD (svd.cu) and the sketched
// least-squares kernel (lstsq.cu).
#pragma once
#include "common.cuh"

namespace ttsg {

// Batched strided copy with conversion (element types: 0 = float, 1 = double).
// dst[a*da + b*db + c*dc] = scale * src[a*sa + b*sb + c*sc]; with da = db = dc = 0
// the destination is compact [A][B][C].
struct CopySeg {
  const void* src = nullptr;
  void* dst = nullptr;
  int64_t A = 0, B = 1, C = 1;
  int64_t sa = 0, sb = 0, sc = 0;
  int64_t da = 0, db = 0, dc = 0;
  double scale = 1.0;
  const double* scale_dev = nullptr;  // multiplies scale when set
  int scale_dev_inv = 0;              // use 1 / *scale_dev instead
  int src_f64 = 0, dst_f64 = 0;
};
void copy3d(const std::vector<CopySeg>& segs, cudaStream_t st);

// out[e] = std * g(seed, stream, e) for e < count (Philox4x32-10 + Box-Muller).
void gaussian_fill(void* out, int out_f64, int64_t count, uint64_t seed, uint64_t stream,
                   double std_, cudaStream_t st);
// Sub-block [rows][n][cols] of a virtual [*][n][ldc] Gaussian array (element
// (q,i,c) is stream element q*n*ldc + i*ldc + c).
void gaussian_subblock(void* out, int out_f64, int64_t rows, int64_t n, int64_t cols,
                       int64_t ldc, uint64_t seed, uint64_t stream, double std_, cudaStream_t st);

// out[0] = sum of squares of x[0..count) (FP64 accumulation); x float or double.
void sumsq(const void* x, int x_f64, int64_t count, double* out, double* scratch,
           cudaStream_t st);
// out[0] = sum_e a[e] b[e] (FP64 accumulation); a, b both float or both double.
void dot_acc(const void* a, const void* b, int f64, int64_t count, double* out, double* scratch,
             cudaStream_t st);
// x <- 2^-e x with e the binary exponent of ||x||_2 (so 1 <= ||x|| < 2 after
// it): an exact rescaling that keeps long products of small or large factors
// inside the float range.  scratch: 256 doubles.
void pow2_normalize(void* x, int x_f64, int64_t count, double* scratch, cudaStream_t st);
// y[0] = sqrt(x[0]).
void sqrt_scalar(const double* x, double* y, cudaStream_t st);

// ------------------------------------------------------------- QR (qr.cu)
// FP64 Householder QR of Y (m x l, element (i,j) at Y[i*sr + j*sc], float or
// double) on a cooperative grid.  Writes Q (m x l, row-major, ldq, float or
// double) when Q != nullptr and R (l x l row-major double) when R != nullptr.
size_t qr_workspace(int64_t m, int64_t l);
// One matrix of a batched QR (Y element (i,j) at Y[i*sr + j*sc]).
struct QRProblem {
  const void* Y;
  int y_f64;
  int64_t m, l, sr, sc;
  void* Q;
  int q_f64;
  int64_t ldq;
  double* R;
};
// Batched form: one CTA per matrix, rows in global memory, one launch.
size_t qr_batch_workspace(int count, const int64_t* m, const int64_t* l);
void qr_f64_batched(int count, const QRProblem* probs, void* ws, size_t ws_bytes, int* err_flag,
                    cudaStream_t st);
// When set on the calling thread, qr_f64 uses the narrow cooperative form: the
// fewest CTAs whose row blocks fit in shared memory (many independent solves
// running side by side on their own streams).
extern thread_local bool g_qr_narrow;
void qr_f64(const void* Y, int y_f64, int64_t m, int64_t l, int64_t sr, int64_t sc, void* Q,
            int q_f64, int64_t ldq, double* R, void* ws, size_t ws_bytes, int* err_flag,
            cudaStream_t st);

// ----------------------------------------------------- Gram / Cholesky (chol.cu)
// G (l x l, double, full symmetric) = Y^T Y in FP64 for Y (m x l, element
// (i,j) at Y[i*sr + j*sc], float or double).
size_t gram_workspace(int64_t m, int64_t l);
void gram_f64(const void* Y, int y_f64, int64_t m, int64_t l, int64_t sr, int64_t sc, double* G,
              void* ws, size_t ws_bytes, cudaStream_t st);
// G + rel_shift * trace(G) * I = R^T R with R upper triangular (row-major,
// double); clamped non-positive pivots increment *err_flag.
void chol_f64(const double* G, int64_t l, double rel_shift, double* R, int* err_flag,
              cudaStream_t st);
// Batched form: problem i factors G[i] (l[i] x l[i]) into R[i], one CTA each.
void chol_f64_batched(int count, const double* const* G, const int64_t* l, double rel_shift,
                      double* const* R, int* err_flag, cudaStream_t st);

// ------------------------------------------------------------ SVD (svd.cu)
// One-sided Jacobi on the columns of G (l x l, row-major double input, or its
// transpose when ``trans``):
// finds an orthogonal V with G V = U Sigma (orthogonal columns), sorted by
// decreasing column norm.  Outputs (double): GV (l x l, columns scaled by the
// singular values), V (l x l), sigma (l).  ``f32`` selects FP32 arithmetic.
// Then picks the truncation rank r (smallest with tail <= delta, <= rmax, >= 1)
// where delta = eps * nrm / sqrt(dm1) and nrm = *norm_in if norm_in, else
// sqrt(sum sigma^2) (written to *norm_out if set).  r written to *rank_out.
// A sweep cap reached without convergence increments *err_flag.
void jacobi_svd(const double* G, int64_t l, int trans, int f32, double* GV, double* V, double* sigma,
                double eps, int64_t dm1, int64_t rmax, const double* norm_in, double* norm_out,
                int* rank_out, int* err_flag, cudaStream_t st, double* vtmp = nullptr,
                double* pre = nullptr);
// (pre: 4 l x l doubles of scratch; with f32 == 0 the FP64 result is then
// reached by an FP32 pass, an FP64 re-orthogonalisation of its rotations and
// FP64 sweeps from them)

// Batched form: one CTA per problem; every problem uses the same rank rule
// parameters.  With norm_in == nullptr each problem takes its own sqrt(sum
// sigma^2) as ||T||; norm_out (if set) receives problem 0's norm.
struct JacobiBatchArgs {
  int count = 0, trans = 0, f32 = 1;
  double eps = 0.0;
  int64_t dm1 = 1, rmax = 1;
  const double* norm_in = nullptr;
  double* norm_out = nullptr;
  int* err = nullptr;
  const double* G[TT_MAX_D] = {};
  int64_t l[TT_MAX_D] = {};
  double* GV[TT_MAX_D] = {};
  double* V[TT_MAX_D] = {};
  double* sigma[TT_MAX_D] = {};
  int* rank_out[TT_MAX_D] = {};
  double* vtmp[TT_MAX_D] = {};  // l x l scratch each, used when l is too large for shared memory
  const double* v0[TT_MAX_D] = {};  // initial rotations (row-major l x l), null = identity
};
void jacobi_svd_batched(const JacobiBatchArgs& a, cudaStream_t st);

// ---------------------------------------------------------- LS (lstsq.cu)
size_t lstsq_workspace(int64_t s, int64_t kmax);
// Incremental FP64 Householder least squares: state lives in ws and persists
// across calls.  lstsq_reset(c) starts a new problem with right-hand side c;
// lstsq_add_column appends column k of W (column-major, leading dimension s),
// then solves and writes y[0..k] and res[0] = ||W y - c||.
void lstsq_reset(const double* c, int64_t s, int64_t kmax, void* ws, cudaStream_t st);
void lstsq_add_column(const double* W, const double* c, int64_t s, int64_t k, int64_t kmax,
                      void* ws, double* y, double* res, cudaStream_t st);

}  // namespace ttsg
