// Streaming tensor-train approximation (STTA, Section 3.3): the two-sided
// sketch of a TT vector with two Gaussian TT-DRMs, and the recovery of the
// approximant from the sketches alone.
//
// With x's cores C_k [t_k][n_k][t_{k+1}], a right DRM X of ranks r_k (the
// target ranks) and a left DRM Y of ranks l_k:
//   right partial contractions  W_k = C_{>k}^T X_{>k}    (t_k x r_k),
//   left partial contractions   L_k = Y_{<=k}^T C_{<=k}  (l_k x t_k),
//   Psi_k   = L_{k-1} x_1 C_k x_3 W_k^T        ([l_{k-1}][n_k][r_k]),
//   Omega_k = L_k W_k                          (l_k x r_k),
// (bond indices as in the paper, cores numbered from 1) and the recovered
// cores, right unfoldings C^_1 = Psi_1, C^_k = Omega_{k-1}^+ Psi_k.
//
// Every contraction is one grouped GEMM in the mode's precision; the sketches
// are accumulated into FP64 outputs (dst = coef * sketch + [dst]), so sums of
// TT vectors are sketched one term at a time.  The recovery is FP64: the
// Householder QR of Omega, the Jacobi SVD of its R factor, and
// Omega^+ Psi = V Sigma^-2 (R V)^T Q^T Psi with singular values below
// rcond * sigma_max dropped.
#include "tt_ops.cuh"

namespace ttsg {

namespace {

template <typename S>
__global__ void stta_axpy_kernel(const S* __restrict__ src, double* __restrict__ dst,
                                 int64_t count, double coef, int accumulate) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = coef * (double)src[e];
    dst[e] = accumulate ? dst[e] + v : v;
  }
}

template <typename S>
void stta_axpy(const S* src, double* dst, int64_t count, double coef, int accumulate,
               cudaStream_t st) {
  if (g_dry_run || count <= 0) return;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>(ceil_div(count, threads), 152 * 8);
  stta_axpy_kernel<S><<<blocks, threads, 0, st>>>(src, dst, count, coef, accumulate);
  check_launch("stta_axpy_kernel");
}

// B[i][:] *= 1 / sigma_i^2 when sigma_i > rcond * sigma_0, else 0 (sigma sorted
// in decreasing order).
__global__ void stta_pinv_scale_kernel(double* __restrict__ B, int64_t rows, int64_t cols,
                                       const double* __restrict__ sigma, double rcond) {
  const double cut = rcond * sigma[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double s = sigma[e / cols];
    B[e] = (s > cut && s > 0.0) ? B[e] / (s * s) : 0.0;
  }
}

// out[e] = sum_{i < k} y[i] * S[i * ssz + e]: the sketch of sum_i y_i v_i from
// the stored sketches of the v_i (coefficients on the device).
__global__ void stta_combine_kernel(const double* __restrict__ S, int64_t ssz, int k,
                                    const double* __restrict__ y, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ssz;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc = fma(y[i], S[(int64_t)i * ssz + e], acc);
    out[e] = acc;
  }
}

}  // namespace

void stta_combine(const double* S, int64_t ssz, int k, const double* y, double* out,
                  cudaStream_t st) {
  if (g_dry_run || ssz <= 0) return;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>(ceil_div(ssz, threads), 152 * 8);
  stta_combine_kernel<<<blocks, threads, 0, st>>>(S, ssz, k, y, out);
  check_launch("stta_combine_kernel");
}

template <typename T>
void tt_stta_sketch_dev(const Ctx& c, const TTv<T>& x, double coef, int accumulate,
                        const TTv<T>& X, const TTv<T>& Y, double* const* psi,
                        double* const* omega) {
  const int d = x.d;
  const int64_t* n = x.n;
  const int64_t* t = x.r;
  const int64_t* r = X.r;
  const int64_t* l = Y.r;
  Arena& ar = *c.ar;
  const size_t mk = ar.mark();

  // 1. right partial contractions W_k (t_k x r_k), k = d-1..1 (0-based bonds)
  std::vector<T*> W(d + 1, nullptr);
  for (int k = 1; k < d; ++k) W[k] = ar.take<T>(t[k] * r[k]);
  int64_t t1max = 1;
  for (int k = 1; k < d - 1; ++k) t1max = std::max(t1max, t[k] * n[k] * r[k + 1]);
  T* T1 = ar.take<T>(t1max);
  for (int k = d - 1; k >= 1; --k) {  // core k (0-based) gives W at bond k
    const int64_t nn = n[k];
    if (k == d - 1) {
      GemmProblem g;
      g.M = (int)t[k]; g.K = (int)nn; g.N = (int)r[k];
      g.A = x.core[k]; g.sAm = nn; g.sAk = 1;
      g.B = X.core[k]; g.sBk = 1; g.sBn = nn;
      g.C = W[k]; g.sCm = r[k]; g.sCn = 1;
      gemm(c.mode, {g}, c.st);
    } else {
      // T1 = C_k W_{k+1}: (t_k n) x r_{k+1}
      gemm(c.mode, {gemm_rm((int)(t[k] * nn), (int)r[k + 1], (int)t[k + 1], x.core[k], t[k + 1],
                            W[k + 1], r[k + 1], T1, r[k + 1])},
           c.st);
      // W_k = T1 (t_k x n r_{k+1}) times X_k^T (X_k viewed r_k x n r_{k+1})
      GemmProblem g;
      g.M = (int)t[k]; g.K = (int)(nn * r[k + 1]); g.N = (int)r[k];
      g.A = T1; g.sAm = nn * r[k + 1]; g.sAk = 1;
      g.B = X.core[k]; g.sBk = 1; g.sBn = nn * r[k + 1];
      g.C = W[k]; g.sCm = r[k]; g.sCn = 1;
      gemm(c.mode, {g}, c.st);
    }
  }

  // 2. left sweep: Z = L_{k} C_k, Psi = Z W_{k+1}, L_{k+1} = Y_k^T Z, Omega = L_{k+1} W_{k+1}
  int64_t zmax = 1, lmax = 1, pmax = 1, omax = 1;
  for (int k = 0; k < d; ++k) {
    zmax = std::max(zmax, l[k] * n[k] * t[k + 1]);
    pmax = std::max(pmax, l[k] * n[k] * r[k + 1]);
    if (k + 1 < d) {
      lmax = std::max(lmax, l[k + 1] * t[k + 1]);
      omax = std::max(omax, l[k + 1] * r[k + 1]);
    }
  }
  T* Z = ar.take<T>(zmax);
  T* L = ar.take<T>(lmax);
  T* P = ar.take<T>(pmax);
  T* O = ar.take<T>(omax);
  for (int k = 0; k < d; ++k) {
    const int64_t nn = n[k];
    const T* Zk = x.core[0];
    if (k > 0) {
      // Z = L_k (l_k x t_k) times C_k (t_k x n t_{k+1})
      gemm(c.mode, {gemm_rm((int)l[k], (int)(nn * t[k + 1]), (int)t[k], L, t[k], x.core[k],
                            nn * t[k + 1], Z, nn * t[k + 1])},
           c.st);
      Zk = Z;
    }
    if (k == d - 1) {
      // Psi_d = Z (r_d = 1, W_d = 1)
      stta_axpy<T>(Zk, psi[k], l[k] * nn, coef, accumulate, c.st);
      break;
    }
    // Psi = Z ((l_k n) x t_{k+1}) times W_{k+1} (t_{k+1} x r_{k+1})
    gemm(c.mode, {gemm_rm((int)(l[k] * nn), (int)r[k + 1], (int)t[k + 1], Zk, t[k + 1], W[k + 1],
                          r[k + 1], P, r[k + 1])},
         c.st);
    stta_axpy<T>(P, psi[k], l[k] * nn * r[k + 1], coef, accumulate, c.st);
    // L_{k+1} = Y_k^T Z: Y_k viewed (l_k n) x l_{k+1}
    GemmProblem g;
    g.M = (int)l[k + 1]; g.K = (int)(l[k] * nn); g.N = (int)t[k + 1];
    g.A = Y.core[k]; g.sAm = 1; g.sAk = l[k + 1];
    g.B = Zk; g.sBk = t[k + 1]; g.sBn = 1;
    g.C = L; g.sCm = t[k + 1]; g.sCn = 1;
    gemm(c.mode, {g}, c.st);
    // Omega_{k+1} = L_{k+1} W_{k+1}
    gemm(c.mode, {gemm_rm((int)l[k + 1], (int)r[k + 1], (int)t[k + 1], L, t[k + 1], W[k + 1],
                          r[k + 1], O, r[k + 1])},
         c.st);
    stta_axpy<T>(O, omega[k], l[k + 1] * r[k + 1], coef, accumulate, c.st);
  }
  ar.release(mk);
}

void tt_stta_recover_dev(const Ctx& c, int d, const int64_t* n, const int64_t* r,
                         const int64_t* l, const double* const* psi, const double* const* omega,
                         double rcond, double* const* cores) {
  Arena& ar = *c.ar;
  const size_t mk = ar.mark();
  // C^_1 = Psi_1
  stta_axpy<double>(psi[0], cores[0], n[0] * r[1], 1.0, 0, c.st);
  int64_t rm = 1, bmax = 1, qmax = 1;
  size_t qws = 0;
  for (int k = 1; k < d; ++k) {
    rm = std::max(rm, r[k]);
    bmax = std::max(bmax, r[k] * n[k] * r[k + 1]);
    qmax = std::max(qmax, l[k] * r[k]);
    qws = std::max(qws, qr_workspace(l[k], r[k]));
  }
  if (d > 1) {
    double* Q = ar.take<double>(qmax);
    double* R = ar.take<double>(rm * rm);
    double* GV = ar.take<double>(rm * rm);
    double* V = ar.take<double>(rm * rm);
    double* sig = ar.take<double>(rm);
    double* vtmp = ar.take<double>(rm * rm);
    double* pre = ar.take<double>(4 * rm * rm);
    int* rank = ar.take<int>(1);
    double* B1 = ar.take<double>(bmax);
    double* B2 = ar.take<double>(bmax);
    void* qw = ar.take<char>((int64_t)qws);
    for (int k = 1; k < d; ++k) {
      const int64_t lk = l[k], rk = r[k], cols = n[k] * r[k + 1];
      // Omega_k = Q R (FP64 Householder)
      qr_f64(omega[k - 1], 1, lk, rk, rk, 1, Q, 1, rk, R, qw, qws, c.err, c.st);
      // R = U Sigma V^T (FP64 one-sided Jacobi): GV = R V = U Sigma
      jacobi_svd(R, rk, 0, 0, GV, V, sig, 0.0, 1, rk, nullptr, nullptr, rank, c.err + 1, c.st,
                 vtmp, pre);
      // B1 = Q^T Psi_k  (Psi_k right unfolding: l_k x n r_{k+1})
      GemmProblem g1;
      g1.M = (int)rk; g1.K = (int)lk; g1.N = (int)cols;
      g1.A = Q; g1.sAm = 1; g1.sAk = rk;
      g1.B = psi[k]; g1.sBk = cols; g1.sBn = 1;
      g1.C = B1; g1.sCm = cols; g1.sCn = 1;
      gemm(TT_MODE_FP64, {g1}, c.st);
      // B2 = GV^T B1, then rows scaled by 1 / sigma^2 (cut below rcond)
      GemmProblem g2;
      g2.M = (int)rk; g2.K = (int)rk; g2.N = (int)cols;
      g2.A = GV; g2.sAm = 1; g2.sAk = rk;
      g2.B = B1; g2.sBk = cols; g2.sBn = 1;
      g2.C = B2; g2.sCm = cols; g2.sCn = 1;
      gemm(TT_MODE_FP64, {g2}, c.st);
      if (!g_dry_run) {
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>(ceil_div(rk * cols, threads), 152 * 8);
        stta_pinv_scale_kernel<<<blocks, threads, 0, c.st>>>(B2, rk, cols, sig, rcond);
        check_launch("stta_pinv_scale_kernel");
      }
      // C^_k = V B2
      gemm(TT_MODE_FP64, {gemm_rm((int)rk, (int)cols, (int)rk, V, rk, B2, cols, cores[k], cols)},
           c.st);
    }
  }
  ar.release(mk);
}

template void tt_stta_sketch_dev<float>(const Ctx&, const TTv<float>&, double, int,
                                        const TTv<float>&, const TTv<float>&, double* const*,
                                        double* const*);
template void tt_stta_sketch_dev<double>(const Ctx&, const TTv<double>&, double, int,
                                         const TTv<double>&, const TTv<double>&, double* const*,
                                         double* const*);

}  // namespace ttsg
