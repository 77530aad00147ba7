/*
 * ttsg.h - C ABI of the GB300 randomized sketched TT-GMRES library.
 *
 * Solves A x = b where A is a tensor-train (TT) operator and x, b are TT
 * vectors, with the sketched TT-GMRES of Bucci, Palitta and Robol,
 * "Randomized sketched TT-GMRES for linear systems with tensor structure"
 * (arXiv 2409.09471), Algorithm 4 with incomplete orthogonalisation l = 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.  All arrays are row-major (C order).
 *   TT vector core k  : [r_{k-1}][n_k][r_k], r_0 = r_d = 1           (Sec. 2.2, eq. tt-format)
 *   TT operator core k: [R_{k-1}][n_k (out)][n_k (in)][R_k], R_0=R_d=1 (Sec. 2.2, eq. operator tt-format)
 *   Khatri-Rao factor k: [s][n_k]                                       (Sec. 3.1)
 *   The merged rank index of a matvec output is a * r + l (operator rank a
 *   slowest), so output core k has ranks R_{k-1} r_{k-1} and R_k r_k.
 * Memory.  Core pointers, factor pointers, workspaces and outputs marked
 *   "device" are CUDA device pointers on the current device; arrays of
 *   pointers and of sizes (n, rank, ...) are HOST arrays.  The caller owns all
 *   memory; the library allocates nothing except where stated.
 * Precision.  ``mode`` selects the arithmetic:
 *   TT_MODE_FP64  cores are double; every step in FP64.
 *   TT_MODE_FP32  cores are float; contractions in FP32 (CUDA cores),
 *                 Householder QR, least squares and residual checks in FP64.
 *   TT_MODE_TF32  cores are float; the matvec core contractions (mode sizes a
 *                 multiple of 4) on tcgen05 tensor cores in split TF32 (each
 *                 operand as hi + lo TF32 parts, three products, FP32
 *                 accumulation, about 2^-20 relative error per product);
 *                 the other contractions as in TT_MODE_FP32; QR, least
 *                 squares and residual checks in FP64.
 *   TT_MODE_BF16  as TT_MODE_TF32 with the matvec's tensor-core products in
 *                 split BF16 (each FP32 operand as bf16 hi + bf16 lo, three
 *                 kind::f16 products, FP32 accumulation, about 2^-17 relative
 *                 per product; plain BF16, 2^-9, could not contract the
 *                 refinement of these operators).
 * Streams.  ``stream`` is a cudaStream_t (NULL = default stream).  Calls that
 *   return host values or data-dependent ranks synchronise that stream.
 * Workspace.  Entry points that need scratch take ``ws`` (device) and
 *   ``ws_bytes``; the matching *_workspace function returns the bytes needed.
 *   A workspace may be reused by consecutive calls on the same stream.
 * Errors.  Every function returns TT_OK (0) or a TT_ERR_* code; tt_last_error()
 *   returns a message for the calling thread's last failure.  Argument errors
 *   are detected on the host before any launch.
 * Devices.  Kernel attributes and the SM count are set up once per process, on
 *   the device of the first call; use one device per process.
 * Memory model.  The library never allocates device memory for its outputs or
 *   scratch: every call takes caller-owned buffers, sized by the *_workspace
 *   queries and by the capacities of tt_vec_out.  There is therefore no
 *   library context, allocator callback or free function, and no out-of-memory
 *   status (a workspace below the query's answer gives TT_ERR_WORKSPACE); the
 *   element type of every buffer follows from ``mode``.
 */
#ifndef TTSG_H
#define TTSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_OK 0
#define TT_ERR_ARG 1           /* bad shape, rank, pointer or parameter */
#define TT_ERR_WORKSPACE 2     /* ws_bytes smaller than the *_workspace answer */
#define TT_ERR_CUDA 3          /* a CUDA runtime call or kernel failed */
#define TT_ERR_TIMEOUT 4       /* a bounded device-side wait expired */
#define TT_ERR_NOT_CONVERGED 5 /* solver stopped at maxit / restarts; x is returned */
#define TT_ERR_UNSUPPORTED 6   /* mode or size the library does not support */
#define TT_ERR_BREAKDOWN 7     /* solver: h_{k+1,k} = 0 (the Krylov space became invariant
                                  under A) in a cycle and the true residual stayed above tol;
                                  x is returned (exact in that space) */

#define TT_MODE_FP64 0
#define TT_MODE_FP32 1
#define TT_MODE_TF32 2
#define TT_MODE_BF16 3

#define TT_MAX_D 64

/* TT vector (input).  n[d], rank[d+1]: host arrays; core[d]: host array of
 * device pointers. */
typedef struct {
  int d;
  const int64_t* n;
  const int64_t* rank;
  void* const* core;
} tt_vec;

/* TT vector (output with data-dependent ranks).  core[k] must hold at least
 * cap[k] * n[k] * cap[k+1] elements; the result is written compactly as
 * [rank[k]][n[k]][rank[k+1]] and rank[] (host, d+1 entries) is filled in. */
typedef struct {
  int d;
  const int64_t* n;
  const int64_t* cap;
  int64_t* rank;
  void* const* core;
} tt_vec_out;

/* TT operator (square modes).  n[d], rank[d+1]: host; core[d]: device. */
typedef struct {
  int d;
  const int64_t* n;
  const int64_t* rank;
  void* const* core;
} tt_op;

/* Library version string. */
const char* tt_version(void);
/* Message of the calling thread's last error ("" if none). */
const char* tt_last_error(void);

/*
 * tt_matvec - y = A x without truncation (Sec. 2.2, matvec formula):
 *   G_k[(a,l), i, (a',l')] = sum_j D_k[a, i, j, a'] C_k[l, j, l'].
 * y->core[k] (device) must hold (R_{k-1} r_{k-1}) * n_k * (R_k r_k) elements;
 * y's ranks are R_k r_k exactly and y->n/rank must say so (checked).
 * Operator and vector cores use the precision of ``mode``.
 */
int tt_matvec(int mode, const tt_op* A, const tt_vec* x, const tt_vec* y,
              void* ws, size_t ws_bytes, void* stream);
size_t tt_matvec_workspace(int mode, const tt_op* A, const tt_vec* x);

/*
 * tt_sketch - Khatri-Rao sketch of a TT vector (Sec. 3.1):
 *   out[j] = prod_k ( sum_i S_k[j, i] C_k[:, i, :] ),  j = 0..s-1,
 * computed as one left-to-right sweep over the cores for all s rows.
 * S[k] (device): factor k, [s][n_k], same precision as the cores.
 * out (device, double[s]).
 */
int tt_sketch(int mode, const tt_vec* x, int64_t s, void* const* S, double* out,
              void* ws, size_t ws_bytes, void* stream);
size_t tt_sketch_workspace(int mode, const tt_vec* x, int64_t s);

/*
 * tt_sketch_factors - the Khatri-Rao factors S_k of the solver's sketch
 * (Sec. 3.1; Alg. 4's input S): S[k] (device, [s][n_k], double for
 * TT_MODE_FP64, float otherwise) receives i.i.d. N(0, s^(-1/d)) entries, factor k
 * being element 0..s*n_k-1 of the Gaussian stream (seed, 1024 + k) of
 * tt_gaussian.  The variance s^(-1/d) makes E ||S_odot x||^2 = ||x||^2.
 * tt_sgmres_solve draws exactly these factors from its ``seed``.
 * n: host array [d].  Errors: TT_ERR_ARG for d outside 1..TT_MAX_D, s < 1,
 * n[k] < 1 or null pointers.
 */
int tt_sketch_factors(int mode, int d, const int64_t* n, int64_t s, uint64_t seed, void* const* S,
                      void* stream);

/*
 * tt_dot - <x, y> by the left-to-right Gram sweep (used for h_{k,k} = w^T v_k
 * and the norms of Alg. 4).  out (device, double[1]).
 */
int tt_dot(int mode, const tt_vec* x, const tt_vec* y, double* out,
           void* ws, size_t ws_bytes, void* stream);
size_t tt_dot_workspace(int mode, const tt_vec* x, const tt_vec* y);

/*
 * tt_dot_noalloc - the inner product of tt_dot for callers that cannot
 * allocate device memory: for example code that runs while a memory manager
 * owns all device memory, or inside a host program that must not call
 * cudaMalloc once it is running.  The paper has no counterpart; this is an
 * interface convenience.  No workspace is passed: the Gram sweep uses a fixed
 * TT_NOALLOC_SCRATCH_BYTES device array inside the library, which every GPU
 * that loads the library keeps until the process exits.  Inputs that would
 * need more scratch than that are rejected with TT_ERR_ARG before any device
 * work.  The first call on a device looks up the array's device address; make
 * that first call before any stream capture, and at start-up, before a memory
 * manager takes the device's memory: with lazy module loading the array itself
 * is created at that first look-up.  The looked-up address is cached per device
 * index for the life of the process; after a cudaDeviceReset the cache is
 * stale, so do not call this function after resetting a device.  All calls
 * share the one array, so calls that overlap on the GPU (different streams, or
 * threads, at the same time) race; serialise them.  The function calls no
 * cudaMalloc or cudaFree.  Errors: the status of the size query for bad
 * arguments (TT_ERR_ARG, TT_ERR_UNSUPPORTED), TT_ERR_ARG for inputs beyond the
 * fixed array, TT_ERR_CUDA if the look-up fails.
 * out (device, double[1]); x, y as for tt_dot.
 */
#define TT_NOALLOC_SCRATCH_BYTES (16u << 20)
#define TT_MAX_DEVICES 64
int tt_dot_noalloc(int mode, const tt_vec* x, const tt_vec* y, double* out, void* stream);

/*
 * tt_round_rand - randomize-then-orthogonalize rounding (Sec. 3.3) of the
 * implicit sum  sum_b coef[b] * X_b  (nterms >= 1 TT vectors with equal mode
 * sizes), without forming the block cores:
 *   1. sketch ranks l_mu = min(rmax + oversample, t_mu, l_{mu-1} n_mu,
 *      prod_{k>mu} n_k) with t_mu the summed representation ranks;
 *   2. right partial contractions of every term with a Gaussian TT-DRM;
 *   3. left-to-right sweep: Y = Z W, FP64 Householder QR of Y, core <- Q,
 *      M = Q^T Z carried into the next core;
 *   4. truncation to the tolerance eps ||T|| and ranks <= rmax.  TT_MODE_FP64:
 *      right-to-left TT-SVD sweep (FP64 Householder QR of each core unfolding
 *      and a small Jacobi SVD, per-bond threshold eps ||T|| / sqrt(d-1)); cores
 *      2..d of the result are right-orthogonal.  Float modes: every bond is cut
 *      from the same left-orthogonal tensor (eigenvectors of its right Gram
 *      matrices, FP64 Cholesky + Jacobi, all bonds in one launch, threshold
 *      eps ||T|| / (d-1)); the result is not orthogonalised.
 * coef: host array [nterms].  drm: NULL to draw the TT-DRM from the Philox
 * stream (seed, streams 2048 + k) with capacity ranks rmax + oversample, or a
 * host array of d device pointers to DRM cores [L_{k-1}][n_k][L_k] with ranks
 * drm_rank[d+1] (host) at least the sketch ranks (leading sub-blocks are used).
 * y: output with capacities; ranks written to y->rank.  Synchronises.
 */
int tt_round_rand(int mode, int nterms, const tt_vec* terms, const double* coef,
                  double eps, int64_t rmax, int64_t oversample, uint64_t seed,
                  void* const* drm, const int64_t* drm_rank, const tt_vec_out* y,
                  void* ws, size_t ws_bytes, void* stream);
size_t tt_round_rand_workspace(int mode, int nterms, const tt_vec* terms, int64_t rmax,
                               int64_t oversample);

/*
 * Backward contractions of the adjoint gradient.  The paper solves A x = b
 * only; these differentiate its inner-product sweep (Sec. 2.2) so that the
 * loss ||x - x_t||^2 can be differentiated through an adjoint solve
 * A^T lambda = 2 (x - x_t) (Alg. 4 applied to A^T):
 *   dL/dtheta_k = -<lambda, (dA/dtheta_k) x>,  dL/db = lambda.
 *
 * tt_dot_grad - derivative of <x, y> with respect to every core of y:
 *   g_k[b, i, c] = sum_{a, a'} P_k[a, b] X_k[a, i, a'] Q_{k+1}[a', c],
 * where P_k (x.rank[k] x y.rank[k]) and Q_{k+1} are the left and right
 * interface matrices of x against y (P_0 = Q_d = 1).
 * g (host array of d device pointers): output core k has y's core-k shape
 * [y.rank[k]][n_k][y.rank[k+1]], in the mode's precision; the caller owns it.
 * Errors: TT_ERR_ARG for mismatched d or mode sizes, null pointers.
 */
int tt_dot_grad(int mode, const tt_vec* x, const tt_vec* y, void* const* g, void* ws,
                size_t ws_bytes, void* stream);
size_t tt_dot_grad_workspace(int mode, const tt_vec* x, const tt_vec* y);

/*
 * tt_local_dots - out[k] = <x, (I x .. x M_k x .. x I) y> for k = 0..d-1
 * (M_k acting on mode k), i.e. <g_k, M_k x_2 Y_k> with g_k as in tt_dot_grad.
 * With M_k the 1-D operator of term k this is the theta-gradient of the loss
 * up to sign.  M (host array of d device pointers): n_k x n_k row-major
 * matrices in the mode's precision (entries may repeat).  out (device,
 * double[d]), accumulated in FP64.
 */
int tt_local_dots(int mode, const tt_vec* x, const tt_vec* y, void* const* M, double* out,
                  void* ws, size_t ws_bytes, void* stream);
size_t tt_local_dots_workspace(int mode, const tt_vec* x, const tt_vec* y);

/*
 * tt_kron_sum_op - cores of the rank-2 TT operator
 *   A(theta) = sum_k theta_k (I x .. x M_k x .. x I)
 * (first core [theta_1 M_1, I], middle [[I, 0], [theta_k M_k, I]], last
 * [I; theta_d M_d]; d == 1 gives theta_1 M_1).  n (host, d), M (host array of
 * d device pointers to n_k x n_k row-major matrices), theta (host, d; NULL =
 * all ones), cores (host array of d device pointers; core k holds
 * R_{k-1} n_k n_k R_k elements with R = 1, 2, .., 2, 1).
 */
int tt_kron_sum_op(int mode, int d, const int64_t* n, void* const* M, const double* theta,
                   void* const* cores, void* stream);

/*
 * tt_op_transpose - cores of A^T: out core k [R_{k-1}][n][n][R_k] with the
 * output and input mode indices of A's core k swapped.  cores: host array of d
 * device pointers, each sized like A's core k; must not alias A's cores.
 */
int tt_op_transpose(int mode, const tt_op* A, void* const* cores, void* stream);

/*
 * tt_gaussian - fill out (device, ``count`` elements: double for TT_MODE_FP64,
 * float otherwise) with std times element e of the Gaussian stream (seed,
 * stream_id): Philox4x32-10 (Salmon et al., SC'11) with counter (lo(e/2),
 * hi(e/2), lo(stream_id), hi(stream_id)) and key (lo(seed), hi(seed)); the
 * output words w0..w3 give u1 = ((w0<<32|w1)>>11 + 0.5) 2^-53 and u2 likewise
 * from (w2, w3); element e is sqrt(-2 ln u1) cos(2 pi u2) for even e and
 * sqrt(-2 ln u1) sin(2 pi u2) for odd e.  The solver draws Khatri-Rao factor k
 * from stream 1024 + k and TT-DRM core k from stream 2048 + k.
 */
int tt_gaussian(int mode, void* out, int64_t count, uint64_t seed, uint64_t stream_id,
                double std_, void* stream);

/*
 * tt_qr_f64 - FP64 Householder QR of a tall matrix Y (m x l, m >= l) read
 * with strides (row stride sr, column stride sc) in the mode's type.  Writes
 * the explicit Q (m x l, row-major, mode's type) if Q != NULL and R (l x l,
 * row-major, double) if R != NULL.  Used inside tt_round_rand; exposed for
 * testing.  All pointers device.
 */
int tt_qr_f64(int mode, const void* Y, int64_t m, int64_t l, int64_t sr, int64_t sc,
              void* Q, double* R, void* ws, size_t ws_bytes, void* stream);
size_t tt_qr_f64_workspace(int64_t m, int64_t l);

/*
 * tt_qr_f64_batched - FP64 Householder QR of count independent tall matrices
 * in one launch, one CTA per matrix with its rows in global memory (the form
 * batched solves use; Sec. 3.3's QR).  Y[i] (device): m[i] x l[i] row-major in
 * the mode's precision; Q[i] (device, may be NULL): m[i] x l[i] row-major, same
 * precision; R[i] (device double, may be NULL): l[i] x l[i] upper triangular.
 * m, l: host arrays.  Requires m[i] >= l[i] >= 1.
 */
int tt_qr_f64_batched(int mode, int count, void* const* Y, const int64_t* m, const int64_t* l,
                      void* const* Q, double* const* R, void* ws, size_t ws_bytes, void* stream);
size_t tt_qr_f64_batched_workspace(int count, const int64_t* m, const int64_t* l);

/*
 * tt_lstsq_f64 - sketched least squares of eq. pseudo_inv:
 *   y = argmin ||W y - c||_2 with W (s x k, column-major, device double) and
 * c (device double[s]); writes y (device double[k]) and res = ||W y - c||
 * (device double[1]).  Householder QR in FP64 on the device.
 */
int tt_lstsq_f64(const double* W, int64_t s, int64_t k, const double* c, double* y,
                 double* res, void* ws, size_t ws_bytes, void* stream);
size_t tt_lstsq_f64_workspace(int64_t s, int64_t k);

/* Solver parameters (Alg. 4 inputs plus the restart loop of Sec. 3.4). */
typedef struct {
  int maxit;          /* Krylov dimension cap per cycle (maxit) */
  int s;              /* sketch rows; 0 => 2 * maxit (Sec. 3.6) */
  double tol;         /* target true relative residual ||b - A x|| / ||b|| */
  double round_tol;   /* Gram-Schmidt rounding tolerance; 0 => eta * tol */
  double eta;         /* rounding threshold factor (Alg. 4 input eta) */
  double stop_safety; /* sketched stop at stop_safety * tol (relative) */
  int64_t rmax;       /* rank cap of the basis vectors (Sec. 4.2) */
  int64_t r_sol;      /* rank cap of the solution; 0 => rmax */
  int64_t oversample; /* randomized-rounding oversampling p */
  uint64_t seed;      /* Khatri-Rao factors: stream 1024+k; TT-DRM: 2048+k */
  int max_restarts;   /* restart cycles after the first */
  int mode;           /* TT_MODE_* */
  int final_stta;     /* 1: each cycle's correction sum_i y_i v_i by STTA (Sec. 3.3,
                         Alg. 4) from one-pass FP64 sketches of the basis vectors
                         (target ranks r_sol, left ranks r_sol + 20, DRM streams
                         4096 + k and 6144 + k), then rounded in FP64 with x (meant
                         for TT_MODE_FP64: in the float modes its refinement converged
                         far more slowly than the default); 0: randomized rounding of
                         the stored basis (default) */
  int ell;            /* incomplete orthogonalisation (Alg. 4, Sec. 3.4): v~ = Round(w -
                         sum of h_{i,k} v_i over the last ell basis vectors); 0 => 1 */
} tt_solver_params;

typedef struct {
  int iters;            /* total Krylov iterations over all cycles */
  int cycles;           /* restart cycles run */
  double sketched_res;  /* last sketched relative residual */
  double true_res;      /* final true relative residual (FP64, exact TT) */
  int64_t max_rank;     /* largest basis rank seen */
  int status;           /* TT_OK, TT_ERR_NOT_CONVERGED or TT_ERR_BREAKDOWN */
  double seconds;       /* host wall time of the call */
  double* res_hist;     /* optional host array [hist_cap]: sketched residuals */
  int64_t* rank_hist;   /* optional host array [hist_cap]: basis max ranks */
  int hist_cap;
  int svd_nonconverged; /* small SVDs that reached their sweep cap (diagnostic) */
  int svd_max_sweeps;   /* most Jacobi sweeps any small SVD took (diagnostic) */
  double svd_mean_sweeps; /* mean Jacobi sweeps per small SVD (diagnostic) */
  int breakdowns;       /* cycles that ended on h_{k+1,k} = 0 */
} tt_solver_info;

/*
 * tt_sgmres_solve - restarted TT-sGMRES (Alg. 4, l = 1, randomized rounding),
 * x0 = 0.  Each cycle stops when ||W y - S r0|| <= stop_safety * tol * ||b|| /
 * ||r|| * ||S r0||; the final x of a cycle is one randomized rounding of
 * sum_i y_i v_i (Sec. 3.5); the true residual is then computed exactly in FP64
 * and the loop restarts from it until ||b - A x|| <= tol ||b||.
 * A and b are given in FP64 (double cores, device); x (device, double cores,
 * capacities >= r_sol) receives the solution.  Synchronises.
 * Each iteration's inner products <A v_k, v_i> and sketch S A v_k run on a
 * second CUDA stream that the call creates (with three events) and releases
 * before it returns; ``stream`` waits on it where their results are used, so
 * the call is ordered on ``stream`` as a whole.  (Inside
 * tt_sgmres_solve_batched every solve stays on its worker's stream.)
 */
int tt_sgmres_solve(const tt_op* A, const tt_vec* b, const tt_solver_params* p,
                    const tt_vec_out* x, tt_solver_info* info, void* ws, size_t ws_bytes,
                    void* stream);
size_t tt_sgmres_solve_workspace(const tt_op* A, const tt_vec* b, const tt_solver_params* p);

/*
 * tt_sgmres_solve_batched - nrhs independent solves A x_i = b_i (same operator,
 * same parameters, uneven TT ranks allowed), each exactly as tt_sgmres_solve.
 * The library runs them on min(nworkers, nrhs) worker threads of its own, each
 * with its own CUDA stream and workspace slice; inside a batch every Householder
 * QR runs on the fewest CTAs whose row blocks fit in shared memory, so the
 * factorisations of different right-hand sides run side by side on different
 * SMs.
 * b, x, info: host arrays of nrhs descriptors (info may be NULL).  Returns
 * TT_ERR_NOT_CONVERGED if any right-hand side stopped above tol (its info says
 * which), another TT_ERR_* if a solve failed.  Synchronises.
 */
int tt_sgmres_solve_batched(const tt_op* A, int nrhs, const tt_vec* b, const tt_solver_params* p,
                            const tt_vec_out* x, tt_solver_info* info, int nworkers, void* ws,
                            size_t ws_bytes);
size_t tt_sgmres_solve_batched_workspace(const tt_op* A, int nrhs, const tt_vec* b,
                                         const tt_solver_params* p, int nworkers);

/*
 * Streaming tensor-train approximation (STTA, Sec. 3.3): two-sided sketches of
 * TT vectors with Gaussian TT-DRMs, linear in the tensor, from which an
 * approximant of fixed ranks is recovered without the tensor itself.  With x's
 * cores C_k [t_{k-1}][n_k][t_k] (paper's 1-based numbering), a right DRM X of
 * ranks r_k (the target ranks) and a left DRM Y of ranks l_k:
 *   Psi_k   = (Y_{<=k-1}^T kron I) x_{<=k} X_{>k}, shape [l_{k-1}][n_k][r_k],
 *             k = 1..d,
 *   Omega_k = Y_{<=k}^T x_{<=k} X_{>k}, l_k x r_k row-major, k = 1..d-1,
 * where x_{<=k} is the unfolding of x with rows (i_1..i_k), Y_{<=k} and X_{>k}
 * the left and right interface matrices of the DRMs,
 * computed through the left and right partial contractions of x.
 *
 * tt_stta_sketch - psi[k] = coef * Psi_{k+1} (+ psi[k] if accumulate) and
 * omega[k] = coef * Omega_{k+1} (+ omega[k] if accumulate), so the sketches of
 * a sum sum_i a_i x_i build up one term at a time.
 * x, X, Y: TT vectors with equal d and mode sizes, cores in the mode's
 * precision (TT_MODE_TF32 contracts in FP32 on CUDA cores); X->rank gives r,
 * Y->rank gives l.  psi: host array of d device pointers (double); omega: host
 * array of d-1 device pointers (double); the caller owns all of them.
 * Errors: TT_ERR_ARG for mismatched d or mode sizes, null pointers.
 */
int tt_stta_sketch(int mode, const tt_vec* x, double coef, int accumulate, const tt_vec* X,
                   const tt_vec* Y, double* const* psi, double* const* omega, void* ws,
                   size_t ws_bytes, void* stream);
size_t tt_stta_sketch_workspace(int mode, const tt_vec* x, const tt_vec* X, const tt_vec* Y);

/*
 * tt_stta_recover - cores of the STTA approximant from the sketches (FP64):
 * core 1 = Psi_1 and, for k = 2..d, the right unfolding of core k is
 * Omega_{k-1}^+ Psi_k (r_{k-1} x n_k r_k).  The pseudo-inverse is formed from
 * the FP64 Householder QR Omega = Q R and the FP64 Jacobi SVD R = U S V^T:
 * Omega^+ Psi = V S^-2 (R V)^T Q^T Psi, singular values at or below
 * rcond * s_max treated as zero (rcond <= 0 selects 1e-12).
 * n[d], r[d+1], l[d+1]: host arrays (r_0 = r_d = l_0 = l_d = 1, l_k >= r_k).
 * psi, omega: as written by tt_stta_sketch.  cores: host array of d device
 * pointers (double, [r_{k-1}][n_k][r_k]), owned by the caller.
 * Errors: TT_ERR_ARG for bad sizes (l_k < r_k) or null pointers.  A
 * rank-deficient Omega is handled by the cutoff, not reported.
 */
int tt_stta_recover(int d, const int64_t* n, const int64_t* r, const int64_t* l,
                    const double* const* psi, const double* const* omega, double rcond,
                    double* const* cores, void* ws, size_t ws_bytes, void* stream);
size_t tt_stta_recover_workspace(int d, const int64_t* n, const int64_t* r, const int64_t* l);

/*
 * Exponential-sum right preconditioning (Sec. 4.1, Alg. 5) of an operator whose
 * dominant part is a Kronecker sum A_0 = sum_k (I x .. x A_k x .. x I):
 *   P^{-1} = sum_i alpha_i (exp(-beta_i A_1) x .. x exp(-beta_i A_d)) ~ A_0^{-1}.
 * zeta: number of terms (1..256); alpha, beta: host arrays [zeta]; A1d: host
 * array of d device pointers to the n_k x n_k row-major FP64 matrices A_k.
 * The descriptor carries no sizes: matrix k must have n_k x n_k entries for the
 * n_k of the TT vectors it is applied to (the caller's responsibility).
 */
typedef struct {
  int zeta;
  const double* alpha;
  const double* beta;
  const double* const* A1d;
} tt_precond;

/*
 * tt_exp_sum_coefficients - alpha, beta with |z E(z) - 1| <~ tol on [a, b]
 * (0 < a < b, 0 < tol < 1): the trapezoidal rule on 1/z = int exp(t - e^t z) dt
 * (Trefethen-Weideman 2014) with step pi^2 / (2 log(1/tol)).  Returns the
 * number of terms; alpha, beta (host, cap entries) are written only when it is
 * <= cap.  Returns -1 for invalid arguments.  Host only.
 */
int tt_exp_sum_coefficients(double a, double b, double tol, int cap, double* alpha,
                            double* beta);

/*
 * tt_precond_apply - y = Round(P^{-1} x): every core of x multiplied along its
 * mode index by exp(-beta_i A_k) (FP64 Taylor of degree 18 with scaling and
 * squaring, then the mode's precision), and the zeta-term sum rounded by the
 * randomized rounding of tt_round_rand (DRM from the Philox stream seed,
 * streams 2048 + k) to tolerance eps and ranks <= rmax.  y: output with
 * capacities >= min(rmax, sketch ranks); ranks written to y->rank.
 * Synchronises (reads the A_k to size the scaling).
 */
int tt_precond_apply(int mode, const tt_precond* P, const tt_vec* x, double eps, int64_t rmax,
                     int64_t oversample, uint64_t seed, const tt_vec_out* y, void* ws,
                     size_t ws_bytes, void* stream);
size_t tt_precond_apply_workspace(int mode, const tt_precond* P, const tt_vec* x, int64_t rmax,
                                  int64_t oversample);

/*
 * tt_spgmres_solve - right-preconditioned TT-sGMRES (TT-sPGMRES, Alg. 5): as
 * tt_sgmres_solve, with w = A P^{-1} v_k (P^{-1} v_k rounded to rmax, the
 * bounded-rank rounding of Sec. 4.2) and each cycle's correction
 * P^{-1} Round(sum_i y_i v_i) rounded to r_sol.  The true residual is that of
 * A x = b.  p->final_stta must be 0.
 */
int tt_spgmres_solve(const tt_op* A, const tt_precond* P, const tt_vec* b,
                     const tt_solver_params* p, const tt_vec_out* x, tt_solver_info* info,
                     void* ws, size_t ws_bytes, void* stream);
size_t tt_spgmres_solve_workspace(const tt_op* A, const tt_precond* P, const tt_vec* b,
                                  const tt_solver_params* p);

/*
 * Measurement support (no counterpart in the method): tt_profile(mask) clears
 * the launch records and, for every class bit set in mask (1 CUDA-core GEMM,
 * 2 FP64 Householder QR, 4 Jacobi SVD, 8 least squares, 16 copies / generators,
 * 32 FP64 Gram, 64 FP64 Cholesky, 128 tensor-core matvec), brackets each later
 * launch of that class with CUDA events on its stream.
 * tt_profile_read synchronises those events and returns, for one class index
 * (0..7), the summed
 * event time in milliseconds, the number of launches and their algorithmic
 * FLOPs and bytes (host outputs, any may be NULL).  tt_profile(0) disables it.
 */
int tt_profile(int mask);
int tt_profile_read(int cls, double* ms_total, int64_t* launches, double* flops, double* bytes);
/* Number of kernel launches this library has enqueued since it was loaded
 * (all classes, counted on the host whether or not profiling is enabled). */
int64_t tt_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TTSG_H */
