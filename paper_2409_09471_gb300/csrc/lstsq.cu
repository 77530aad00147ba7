// Sketched least squares y_k = argmin ||W_k y - S r_0|| (eq. pseudo_inv) with
// an incrementally updated FP64 Householder QR of W_k (one column appended per
// Krylov iteration, Algorithm 4), one CTA.
//
// State in the workspace: Householder vectors (column j of Vh, unit leading
// entry implicit), their tau, the triangular factor R (column-major, kmax x
// kmax) and Q^T c.  A pivot |R_jj| <= 1e-14 max|R_ii| is treated as zero in the
// back substitution (that component of y is set to 0), and the reported
// residual is recomputed explicitly as ||W y - c||.
#include "kernels.cuh"

namespace ttsg {

namespace {

constexpr int LS_THREADS = 256;

struct LSState {
  double* Vh;    // [kmax][s]   (column j stored contiguously)
  double* tau;   // [kmax]
  double* R;     // [kmax][kmax] column-major
  double* qtc;   // [s]
};

LSState carve(void* ws, int64_t s, int64_t kmax) {
  Arena ar(ws, ~size_t(0) >> 1);
  LSState st;
  st.Vh = ar.take<double>(s * kmax);
  st.tau = ar.take<double>(kmax);
  st.R = ar.take<double>(kmax * kmax);
  st.qtc = ar.take<double>(s);
  return st;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < LS_THREADS / 32; ++w) t += red[w];
  return t;
}

__global__ void ls_reset_kernel(const double* c, int s, LSState S) {
  for (int i = threadIdx.x; i < s; i += blockDim.x) S.qtc[i] = c[i];
}

__global__ void __launch_bounds__(LS_THREADS)
ls_step_kernel(const double* W, const double* c, int s, int k, int kmax, LSState S, double* y,
               double* res) {
  extern __shared__ double sh[];
  double* x = sh;            // [s] new column
  double* ys = x + s;        // [kmax]
  double* r = ys + kmax;     // [s] residual
  __shared__ double red[LS_THREADS / 32];
  const int tid = threadIdx.x;
  for (int i = tid; i < s; i += LS_THREADS) x[i] = W[(size_t)k * s + i];
  __syncthreads();
  // apply the previous reflectors H_j = I - tau_j v_j v_j^T to the new column
  for (int j = 0; j < k && j < s; ++j) {
    const double* v = S.Vh + (size_t)j * s;
    double p = 0.0;
    for (int i = j + tid; i < s; i += LS_THREADS) p += (i == j ? 1.0 : v[i]) * x[i];
    p = block_sum(p, red) * S.tau[j];
    for (int i = j + tid; i < s; i += LS_THREADS) x[i] -= p * (i == j ? 1.0 : v[i]);
    __syncthreads();
  }
  // new reflector for x[k:]
  if (k < s) {
    double sg = 0.0;
    for (int i = k + 1 + tid; i < s; i += LS_THREADS) sg += x[i] * x[i];
    sg = block_sum(sg, red);
    const double alpha = x[k];
    double t = 0.0, beta = alpha, scale = 0.0;
    if (sg > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sg), alpha);
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    double* v = S.Vh + (size_t)k * s;
    for (int i = tid; i < s; i += LS_THREADS) v[i] = i > k ? x[i] * scale : (i == k ? 1.0 : 0.0);
    for (int i = tid; i < k; i += LS_THREADS) S.R[(size_t)k * kmax + i] = x[i];
    if (tid == 0) { S.R[(size_t)k * kmax + k] = beta; S.tau[k] = t; }
    __syncthreads();
    // Q^T c update with H_k
    double p = 0.0;
    for (int i = k + tid; i < s; i += LS_THREADS) p += v[i] * S.qtc[i];
    p = block_sum(p, red) * t;
    for (int i = k + tid; i < s; i += LS_THREADS) S.qtc[i] -= p * v[i];
    __syncthreads();
  }
  // back substitution R y = (Q^T c)[0..k]
  const int kk = min(k, s - 1);
  if (tid == 0) {
    double rmaxd = 0.0;
    for (int i = 0; i <= kk; ++i) rmaxd = fmax(rmaxd, fabs(S.R[(size_t)i * kmax + i]));
    for (int i = kk; i >= 0; --i) {
      double acc = S.qtc[i];
      for (int j = i + 1; j <= kk; ++j) acc -= S.R[(size_t)j * kmax + i] * ys[j];
      const double piv = S.R[(size_t)i * kmax + i];
      ys[i] = (fabs(piv) <= 1e-14 * rmaxd || piv == 0.0) ? 0.0 : acc / piv;
    }
    for (int i = kk + 1; i <= k; ++i) ys[i] = 0.0;
  }
  __syncthreads();
  for (int i = tid; i <= k; i += LS_THREADS) y[i] = ys[i];
  // explicit residual ||W y - c||
  double acc2 = 0.0;
  for (int i = tid; i < s; i += LS_THREADS) {
    double v = -c[i];
    for (int j = 0; j <= k; ++j) v += W[(size_t)j * s + i] * ys[j];
    r[i] = v;
    acc2 += v * v;
  }
  acc2 = block_sum(acc2, red);
  if (tid == 0) *res = sqrt(acc2);
}

}  // namespace

size_t lstsq_workspace(int64_t s, int64_t kmax) {
  return sizeof(double) * (s * kmax + kmax + kmax * kmax + s) + 4 * 256;
}

void lstsq_reset(const double* c, int64_t s, int64_t kmax, void* ws, cudaStream_t st) {
  if (g_dry_run) return;
  LSState S = carve(ws, s, kmax);
  ls_reset_kernel<<<1, 256, 0, st>>>(c, (int)s, S);
  check_launch("ls_reset_kernel");
}

void lstsq_add_column(const double* W, const double* c, int64_t s, int64_t k, int64_t kmax,
                      void* ws, double* y, double* res, cudaStream_t st) {
  if (g_dry_run) return;
  LSState S = carve(ws, s, kmax);
  const size_t smem = sizeof(double) * (2 * s + kmax);
  if (smem > 200 * 1024) throw Error(TT_ERR_UNSUPPORTED, "lstsq: sketch size too large");
  static const bool attr = [] {
    TT_CUDA(cudaFuncSetAttribute(ls_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    return true;
  }();
  (void)attr;
  ls_step_kernel<<<1, LS_THREADS, smem, st>>>(W, c, (int)s, (int)k, (int)kmax, S, y, res);
  check_launch("ls_step_kernel");
}

}  // namespace ttsg
