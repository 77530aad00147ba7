// FP64 Gram matrix and shifted Cholesky factor of a tall-skinny matrix, used
// by the truncation sweep of the randomized rounding in the float modes: the
// singular values and left singular vectors of a core unfolding X (l x c) are
// those of the Cholesky factor L of X X^T + s I (s a tiny shift that keeps the
// factorisation defined when X is rank deficient), which a small Jacobi SVD
// then resolves.
#include "kernels.cuh"
#include "prof.cuh"

namespace ttsg {

namespace {

constexpr int GT = 256;

// part[c][p][q] (p <= q) = sum over the rows of block c of Y[i,p] Y[i,q].
__global__ void __launch_bounds__(GT)
gram_partial_kernel(const void* Y, int y_f64, int64_t m, int l, int64_t sr, int64_t sc, int rows,
                    double* part) {
  extern __shared__ double ys[];  // [rows][l]
  const int c = blockIdx.x;
  const int64_t r0 = (int64_t)c * rows;
  const int nloc = (int)(m - r0 < rows ? m - r0 : rows);
  for (int e = threadIdx.x; e < nloc * l; e += GT) {
    const int li = e / l, j = e % l;
    const int64_t src = (r0 + li) * sr + (int64_t)j * sc;
    ys[e] = y_f64 ? ((const double*)Y)[src] : (double)((const float*)Y)[src];
  }
  __syncthreads();
  double* out = part + (size_t)c * l * l;
  for (int e = threadIdx.x; e < l * l; e += GT) {
    const int p = e / l, q = e % l;
    if (q < p) continue;
    double s = 0.0;
    for (int li = 0; li < nloc; ++li) s += ys[li * l + p] * ys[li * l + q];
    out[e] = s;
  }
}

__global__ void gram_reduce_kernel(const double* part, int P, int l, double* G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int p = e / l, q = e % l;
    if (q < p) continue;
    double s = 0.0;
    for (int c = 0; c < P; ++c) s += part[(size_t)c * l * l + e];
    G[e] = s;
    G[(size_t)q * l + p] = s;
  }
}

// G + shift I = R^T R (R upper triangular, written row-major into R) with
// shift = rel_shift * trace(G); a non-positive pivot is clamped to the shift
// and counted in *err.
struct CholBatch {
  const double* G[TT_MAX_D];
  double* R[TT_MAX_D];
  int l[TT_MAX_D];
};

__global__ void __launch_bounds__(GT)
chol_kernel(const __grid_constant__ CholBatch cb, double rel_shift, int* err, int gm) {
  extern __shared__ double sA[];  // [l][l]
  const double* G = cb.G[blockIdx.x];
  double* R = cb.R[blockIdx.x];
  // gm: l x l does not fit in shared memory; the factorisation runs in place in
  // R (global memory, ordered within the CTA by the same block barriers)
  double* A = gm ? R : sA;
  const int l = cb.l[blockIdx.x];
  __shared__ double s_shift;
  for (int e = threadIdx.x; e < l * l; e += GT) A[e] = G[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < l; ++i) tr += A[i * l + i];
    s_shift = rel_shift * tr;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < l; i += GT) A[i * l + i] += s_shift;
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j * l + j];
      if (!(d > 0.0)) {
        atomicAdd(err, 1);
        d = s_shift > 0.0 ? s_shift : 1e-300;
      }
      A[j * l + j] = sqrt(d);
    }
    __syncthreads();
    const double rjj = A[j * l + j];
    for (int k = j + 1 + threadIdx.x; k < l; k += GT) A[j * l + k] /= rjj;
    __syncthreads();
    const int nt = l - j - 1;
    for (int e = threadIdx.x; e < nt * nt; e += GT) {
      const int i = j + 1 + e / nt, k = j + 1 + e % nt;
      if (k >= i) A[i * l + k] -= A[j * l + i] * A[j * l + k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < l * l; e += GT) {
    const int i = e / l, k = e % l;
    R[e] = k >= i ? A[e] : 0.0;
  }
}

int sm_count() {
  // thread-safe one-time query (batched solves call this from several threads)
  static const int sms = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

}  // namespace

size_t gram_workspace(int64_t m, int64_t l) {
  // at most one partial Gram per SM (256 bounds the SM count) plus slack
  const int64_t P = std::min<int64_t>(256, std::max<int64_t>(1, ceil_div(m, 8)));
  return sizeof(double) * (size_t)(P * l * l) + 1024;
}

void gram_f64(const void* Y, int y_f64, int64_t m, int64_t l, int64_t sr, int64_t sc, double* G,
              void* ws, size_t ws_bytes, cudaStream_t st) {
  if (g_dry_run) return;
  int64_t P = std::min<int64_t>(sm_count(), std::max<int64_t>(1, ceil_div(m, 8)));
  int rows = (int)ceil_div(m, P);
  while ((size_t)rows * l * sizeof(double) > 200 * 1024) { ++P; rows = (int)ceil_div(m, P); }
  P = ceil_div(m, rows);
  if ((size_t)P * l * l * sizeof(double) > ws_bytes)
    throw Error(TT_ERR_WORKSPACE, "gram_f64: workspace too small");
  static const bool attr = [] {
    TT_CUDA(cudaFuncSetAttribute(gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 210 * 1024));
    return true;
  }();
  (void)attr;
  const int tok = prof_begin(PROF_GRAM, st);
  gram_partial_kernel<<<(unsigned)P, GT, (size_t)rows * l * sizeof(double), st>>>(
      Y, y_f64, m, (int)l, sr, sc, rows, (double*)ws);
  check_launch("gram_partial_kernel");
  gram_reduce_kernel<<<(unsigned)std::min<int64_t>(ceil_div(l * l, 256), 64), 256, 0, st>>>(
      (const double*)ws, (int)P, (int)l, G);
  check_launch("gram_reduce_kernel");
  prof_end(tok, st, (double)m * l * (l + 1), (double)m * l * (y_f64 ? 8 : 4));
}

void chol_f64_batched(int count, const double* const* G, const int64_t* l, double rel_shift,
                      double* const* R, int* err_flag, cudaStream_t st) {
  if (g_dry_run || count == 0) return;
  if (count > TT_MAX_D) throw Error(TT_ERR_UNSUPPORTED, "chol_f64: batch too large");
  CholBatch cb;
  int64_t lmax = 1;
  for (int i = 0; i < count; ++i) {
    cb.G[i] = G[i]; cb.R[i] = R[i]; cb.l[i] = (int)l[i];
    lmax = std::max(lmax, l[i]);
  }
  size_t smem = (size_t)lmax * lmax * sizeof(double);
  const int gm = smem > 220 * 1024 ? 1 : 0;
  if (gm) smem = 0;
  static const bool attr = [] {
    TT_CUDA(cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 220 * 1024));
    return true;
  }();
  (void)attr;
  const int tok = prof_begin(PROF_CHOL, st);
  chol_kernel<<<count, GT, smem, st>>>(cb, rel_shift, err_flag, gm);
  check_launch("chol_kernel");
  prof_end(tok, st, (double)count * lmax * lmax * lmax / 3.0, 2.0 * count * lmax * lmax * 8.0);
}

void chol_f64(const double* G, int64_t l, double rel_shift, double* R, int* err_flag,
              cudaStream_t st) {
  chol_f64_batched(1, &G, &l, rel_shift, &R, err_flag, st);
}

}  // namespace ttsg
