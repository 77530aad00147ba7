// One-sided Jacobi SVD of a small square matrix (one CTA) and the truncation
// rank rule of the TT-SVD rounding (Section 2.2: per-bond threshold
// eps ||T|| / sqrt(d - 1), smallest rank meeting it, capped at rmax).
//
// Columns of G are rotated pairwise (parallel round-robin ordering, one warp
// per pair) until they are mutually orthogonal: G V = U Sigma.  The rotation
// angle zeroes the pair's inner product gamma given the squared norms
// alpha, beta: zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t.
// A sweep without any rotation above the threshold l * eps ends the iteration.
#include "kernels.cuh"
#include "prof.cuh"

namespace ttsg {

namespace {

constexpr int SVD_THREADS = 1024;
constexpr int MAX_SWEEPS = 60;

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(SVD_THREADS)
jacobi_kernel(const double* G, int l, int trans, double* GV, double* V, double* sigma, double eps,
              long long dm1, long long rmax, const double* norm_in, double* norm_out,
              int* rank_out, int* err) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = (T*)sm_raw;            // column-major: column p at A + p*l
  T* Vm = A + (size_t)l * l;    // column-major
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = SVD_THREADS / 32;

  for (int e = tid; e < l * l; e += SVD_THREADS) {
    const int i = e / l, j = e % l;           // element (i, j) of G
    A[(size_t)j * l + i] = (T)(trans ? G[(size_t)j * l + i] : G[e]);
    Vm[(size_t)j * l + i] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  const T eps_t = sizeof(T) == 4 ? (T)1.1920929e-07 : (T)2.220446049250313e-16;
  const T tol = (T)l * eps_t;
  // columns whose squared norm is below eps^4 ||G||_F^2 are numerically zero
  __shared__ double s_tot;
  if (warp == 0) {
    double acc = 0.0;
    for (int e = lane; e < l * l; e += 32) { const double x = (double)A[e]; acc += x * x; }
    acc = warp_sum_t(acc);
    if (lane == 0) s_tot = acc;
  }
  __syncthreads();
  // thresholds in the kernel's own precision (FP64 math is slow on this part)
  const T tot_t = (T)s_tot;
  const T tiny = (T)(s_tot * (double)eps_t * (double)eps_t * (double)eps_t * (double)eps_t);
  const T abs_thr = tol * eps_t * tot_t;
  const int lp = l + (l & 1);   // even number of players (index l is a dummy when l is odd)
  int sweep = 0;
  for (; sweep < MAX_SWEEPS; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < lp - 1; ++step) {
      for (int k = warp; k < lp / 2; k += nwarps) {
        int p, q;
        if (k == 0) { p = lp - 1; q = step; }
        else { p = (step + k) % (lp - 1); q = (step - k + (lp - 1)) % (lp - 1); }
        if (p >= l || q >= l) continue;
        if (p > q) { const int t = p; p = q; q = t; }
        T* ap = A + (size_t)p * l;
        T* aq = A + (size_t)q * l;
        T al = 0, be = 0, ga = 0;
        for (int i = lane; i < l; i += 32) {
          const T x = ap[i], y = aq[i];
          al += x * x; be += y * y; ga += x * y;
        }
        al = warp_sum_t(al); be = warp_sum_t(be); ga = warp_sum_t(ga);
        // converged pair: relative test, or an inner product at the rounding
        // level of the whole matrix (columns at noise level cannot be made
        // relatively orthogonal in this precision)
        if (ga == T(0) || al <= tiny || be <= tiny || fabs(ga) <= tol * sqrt(al) * sqrt(be) ||
            fabs(ga) <= abs_thr)
          continue;
        const T zeta = (be - al) / (T(2) * ga);
        const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
        for (int i = lane; i < l; i += 32) {
          const T x = ap[i], y = aq[i];
          ap[i] = c * x - s * y;
          aq[i] = s * x + c * y;
        }
        T* vp = Vm + (size_t)p * l;
        T* vq = Vm + (size_t)q * l;
        for (int i = lane; i < l; i += 32) {
          const T x = vp[i], y = vq[i];
          vp[i] = c * x - s * y;
          vq[i] = s * x + c * y;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep == MAX_SWEEPS && tid == 0) atomicAdd(err, 1);  // non-convergence counter
  // column norms and descending order (ties by index)
  double* sg = (double*)(Vm + (size_t)l * l);
  for (int j = warp; j < l; j += nwarps) {
    double acc = 0.0;
    for (int i = lane; i < l; i += 32) { const double x = (double)A[(size_t)j * l + i]; acc += x * x; }
    acc = warp_sum_t(acc);
    if (lane == 0) sg[j] = sqrt(acc);
  }
  __syncthreads();
  for (int j = tid; j < l; j += SVD_THREADS) {
    int rank = 0;
    for (int i = 0; i < l; ++i)
      if (sg[i] > sg[j] || (sg[i] == sg[j] && i < j)) ++rank;
    sigma[rank] = sg[j];
    for (int i = 0; i < l; ++i) {
      GV[(size_t)i * l + rank] = (double)A[(size_t)j * l + i];
      V[(size_t)i * l + rank] = (double)Vm[(size_t)j * l + i];
    }
  }
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int i = 0; i < l; ++i) tot += sigma[i] * sigma[i];
    const double nrm = norm_in ? *norm_in : sqrt(tot);
    if (norm_out) *norm_out = nrm;
    const double delta = eps * nrm / sqrt((double)(dm1 > 0 ? dm1 : 1));
    // smallest r with ||sigma[r:]|| <= delta
    double tail = 0.0;
    int r = l;
    for (int i = l - 1; i >= 0; --i) {
      tail += sigma[i] * sigma[i];
      if (sqrt(tail) <= delta) r = i; else break;
    }
    if (r > rmax) r = (int)rmax;
    if (r < 1) r = 1;
    *rank_out = r;
  }
}

}  // namespace

void jacobi_svd(const double* G, int64_t l, int trans, int f32, double* GV, double* V, double* sigma,
                double eps, int64_t dm1, int64_t rmax, const double* norm_in, double* norm_out,
                int* rank_out, int* err_flag, cudaStream_t st) {
  if (g_dry_run) return;
  const size_t es = f32 ? 4 : 8;
  const size_t smem = 2 * (size_t)l * l * es + (size_t)l * sizeof(double) + 16;
  if (smem > 220 * 1024)
    throw Error(TT_ERR_UNSUPPORTED, "jacobi_svd: l = " + std::to_string(l) + " too large for " +
                                        (f32 ? "FP32" : "FP64"));
  static bool attr[2] = {false, false};
  const int tok = prof_begin(PROF_SVD, st);
  if (f32) {
    if (!attr[0]) {
      TT_CUDA(cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   220 * 1024));
      attr[0] = true;
    }
    jacobi_kernel<float><<<1, SVD_THREADS, smem, st>>>(G, (int)l, trans, GV, V, sigma, eps, dm1, rmax,
                                                       norm_in, norm_out, rank_out, err_flag);
  } else {
    if (!attr[1]) {
      TT_CUDA(cudaFuncSetAttribute(jacobi_kernel<double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      attr[1] = true;
    }
    jacobi_kernel<double><<<1, SVD_THREADS, smem, st>>>(G, (int)l, trans, GV, V, sigma, eps, dm1, rmax,
                                                        norm_in, norm_out, rank_out, err_flag);
  }
  check_launch("jacobi_kernel");
  prof_end(tok, st, 0.0, 3.0 * l * l * 8.0);
}

}  // namespace ttsg
