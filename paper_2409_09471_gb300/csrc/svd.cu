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
constexpr int MAX_SVD_BATCH = TT_MAX_D;
constexpr int MAX_SWEEPS = 60;

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct JacobiBatch {
  int count;
  int trans, f32;
  double eps;
  long long dm1, rmax;
  const double* norm_in;   // shared input norm (nullptr: each problem's own)
  double* norm_out;        // written by problem 0 when set
  const double* G[MAX_SVD_BATCH];
  int l[MAX_SVD_BATCH];
  double* GV[MAX_SVD_BATCH];
  double* V[MAX_SVD_BATCH];
  double* sigma[MAX_SVD_BATCH];
  int* rank_out[MAX_SVD_BATCH];
  double* vtmp[MAX_SVD_BATCH];  // V in global memory when it does not fit (else null)
  const double* v0[MAX_SVD_BATCH];  // initial rotations, row-major (else the identity)
};

constexpr int GL = 8;             // lanes per column pair
constexpr int PPW = 32 / GL;      // column pairs per warp

template <typename T>
__device__ __forceinline__ T group_sum(T v) {
  // sum over the GL lanes of a lane group
#pragma unroll
  for (int o = GL / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One pair of columns per group of GL = 8 lanes (4 pairs per warp).  Measured
// on GB300 at l = 74: a parallel step costs ~3K cycles, one dependent chain
// (dot product, reduction, rotation, update) plus the block barrier; 16 lanes
// per pair (twice the warps) was slower.
template <typename T>
__global__ void __launch_bounds__(SVD_THREADS)
jacobi_kernel(const __grid_constant__ JacobiBatch jb, int* err) {
  const int bi = blockIdx.x;
  const double* G = jb.G[bi];
  const int l = jb.l[bi], trans = jb.trans;
  double* GV = jb.GV[bi];
  double* V = jb.V[bi];
  double* sigma = jb.sigma[bi];
  int* rank_out = jb.rank_out[bi];
  const double eps = jb.eps;
  const long long dm1 = jb.dm1, rmax = jb.rmax;
  const double* norm_in = jb.norm_in;
  double* norm_out = bi == 0 ? jb.norm_out : nullptr;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = (T*)sm_raw;            // column-major: column p at A + p*l
  // V (column-major) in shared memory after A, or in global scratch for large l
  T* Vm = jb.vtmp[bi] ? (T*)jb.vtmp[bi] : A + (size_t)l * l;
  T* after = A + (size_t)l * l * (jb.vtmp[bi] ? 1 : 2);
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x, nwarps = nthreads / 32;
  const int grp = lane / GL, sub = lane % GL;

  for (int e = tid; e < l * l; e += nthreads) {
    const int i = e / l, j = e % l;           // element (i, j) of G
    A[(size_t)j * l + i] = (T)(trans ? G[(size_t)j * l + i] : G[e]);
    Vm[(size_t)j * l + i] = jb.v0[bi] ? (T)jb.v0[bi][e] : ((i == j) ? T(1) : T(0));
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
  const int npairs = lp / 2;
  T* nrm2 = after;               // squared column norms, updated with the rotations
  int sweep = 0;
  for (; sweep < MAX_SWEEPS; ++sweep) {
    // exact column norms at the start of every sweep
    for (int j = warp; j < l; j += nwarps) {
      T acc = 0;
      for (int i = lane; i < l; i += 32) { const T x = A[(size_t)j * l + i]; acc += x * x; }
      acc = warp_sum_t(acc);
      if (lane == 0) nrm2[j] = acc;
    }
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < lp - 1; ++step) {
      for (int k0 = warp * PPW; k0 < npairs; k0 += nwarps * PPW) {
        const int k = k0 + grp;
        int p = -1, q = -1;
        if (k < npairs) {
          // round-robin pairing: player lp-1 stays, the others rotate (no
          // integer division: 0 <= step < lp-1 and 0 < k < lp/2)
          if (k == 0) { p = lp - 1; q = step; }
          else {
            p = step + k;
            if (p >= lp - 1) p -= lp - 1;
            q = step - k;
            if (q < 0) q += lp - 1;
          }
          if (p >= l || q >= l) p = q = -1;
          else if (p > q) { const int t = p; p = q; q = t; }
        }
        T ga = 0;
        if (p >= 0) {
          // two independent chains per lane (the loop is latency-bound)
          const T* ap = A + (size_t)p * l;
          const T* aq = A + (size_t)q * l;
          T g0 = 0, g1 = 0;
          int i = sub;
          for (; i + GL < l; i += 2 * GL) {
            g0 = fma(ap[i], aq[i], g0);
            g1 = fma(ap[i + GL], aq[i + GL], g1);
          }
          if (i < l) g0 = fma(ap[i], aq[i], g0);
          ga = g0 + g1;
        }
        ga = group_sum(ga);
        if (p < 0) continue;
        const T al = nrm2[p], be = nrm2[q];
        // converged pair: relative test, or an inner product at the rounding
        // level of the whole matrix (columns at noise level cannot be made
        // relatively orthogonal in this precision)
        if (ga == T(0) || al <= tiny || be <= tiny || fabs(ga) <= tol * sqrt(al) * sqrt(be) ||
            fabs(ga) <= abs_thr)
          continue;
        T t, c, s;
        if (sizeof(T) == 4) {
          const float zeta = __fdividef((float)(be - al), 2.0f * (float)ga);
          t = (T)__fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          c = (T)rsqrtf(1.f + (float)(t * t));
        } else {
          const T zeta = (be - al) / (T(2) * ga);
          t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          c = T(1) / sqrt(T(1) + t * t);
        }
        s = c * t;
        T* ap = A + (size_t)p * l;
        T* aq = A + (size_t)q * l;
        T* vp = Vm + (size_t)p * l;
        T* vq = Vm + (size_t)q * l;
        int i = sub;
        for (; i + GL < l; i += 2 * GL) {
          // two rows per iteration, all loads before the stores
          const T x0 = ap[i], y0 = aq[i], u0 = vp[i], w0 = vq[i];
          const T x1 = ap[i + GL], y1 = aq[i + GL], u1 = vp[i + GL], w1 = vq[i + GL];
          ap[i] = c * x0 - s * y0;
          aq[i] = s * x0 + c * y0;
          vp[i] = c * u0 - s * w0;
          vq[i] = s * u0 + c * w0;
          ap[i + GL] = c * x1 - s * y1;
          aq[i + GL] = s * x1 + c * y1;
          vp[i + GL] = c * u1 - s * w1;
          vq[i + GL] = s * u1 + c * w1;
        }
        if (i < l) {
          const T x = ap[i], y = aq[i], u = vp[i], w = vq[i];
          ap[i] = c * x - s * y;
          aq[i] = s * x + c * y;
          vp[i] = c * u - s * w;
          vq[i] = s * u + c * w;
        }
        if (sub == 0) {
          nrm2[p] = al - t * ga;
          nrm2[q] = be + t * ga;
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (tid == 0) {
    if (sweep == MAX_SWEEPS) atomicAdd(err, 1);  // non-convergence counter
    // sweep statistics: err[2] maximum, err[3] total, err[4] problems
    atomicMax(err + 2, sweep);
    atomicAdd(err + 3, sweep);
    atomicAdd(err + 4, 1);
  }
  // column norms and descending order (ties by index)
  double* sg = (double*)(after + ((l + 1) & ~1));
  for (int j = warp; j < l; j += nwarps) {
    double acc = 0.0;
    for (int i = lane; i < l; i += 32) { const double x = (double)A[(size_t)j * l + i]; acc += x * x; }
    acc = warp_sum_t(acc);
    if (lane == 0) sg[j] = sqrt(acc);
  }
  __syncthreads();
  for (int j = tid; j < l; j += nthreads) {
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

void jacobi_svd_batched(const JacobiBatchArgs& a, cudaStream_t st) {
  if (g_dry_run || a.count == 0) return;
  if (a.count > MAX_SVD_BATCH) throw Error(TT_ERR_UNSUPPORTED, "jacobi_svd: batch too large");
  JacobiBatch jb;
  jb.count = a.count; jb.trans = a.trans; jb.f32 = a.f32; jb.eps = a.eps;
  jb.dm1 = a.dm1; jb.rmax = a.rmax; jb.norm_in = a.norm_in; jb.norm_out = a.norm_out;
  int64_t lmax = 1;
  for (int i = 0; i < a.count; ++i) {
    jb.G[i] = a.G[i]; jb.l[i] = (int)a.l[i]; jb.GV[i] = a.GV[i]; jb.V[i] = a.V[i];
    jb.sigma[i] = a.sigma[i]; jb.rank_out[i] = a.rank_out[i];
    jb.vtmp[i] = nullptr;
    jb.v0[i] = a.v0[i];
    lmax = std::max<int64_t>(lmax, a.l[i]);
  }
  const size_t es = a.f32 ? 4 : 8;
  const size_t tail = (size_t)(lmax + 2) * es + (size_t)lmax * sizeof(double) + 16;
  size_t smem = 2 * (size_t)lmax * lmax * es + tail;
  if (smem > 220 * 1024) {
    // V moves to the callers' global scratch; A stays in shared memory
    smem = (size_t)lmax * lmax * es + tail;
    for (int i = 0; i < a.count; ++i) {
      if (!a.vtmp[i])
        throw Error(TT_ERR_UNSUPPORTED, "jacobi_svd: l = " + std::to_string(lmax) +
                                            " needs a V scratch");
      jb.vtmp[i] = a.vtmp[i];
    }
  }
  if (smem > 220 * 1024)
    throw Error(TT_ERR_UNSUPPORTED, "jacobi_svd: l = " + std::to_string(lmax) + " too large for " +
                                        (a.f32 ? "FP32" : "FP64"));
  static bool attr[2] = {false, false};
  // PPW column pairs per warp
  const int pairs = (int)((lmax + 1) / 2);
  const int threads =
      (int)std::min<int64_t>(SVD_THREADS, std::max<int64_t>(64, ceil_div(pairs, PPW) * 32));
  const int tok = prof_begin(PROF_SVD, st);
  if (a.f32) {
    if (!attr[0]) {
      TT_CUDA(cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   220 * 1024));
      attr[0] = true;
    }
    jacobi_kernel<float><<<a.count, threads, smem, st>>>(jb, a.err);
  } else {
    if (!attr[1]) {
      TT_CUDA(cudaFuncSetAttribute(jacobi_kernel<double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      attr[1] = true;
    }
    jacobi_kernel<double><<<a.count, threads, smem, st>>>(jb, a.err);
  }
  check_launch("jacobi_kernel");
  prof_end(tok, st, 0.0, 3.0 * lmax * lmax * 8.0 * a.count);
}

void jacobi_svd(const double* G, int64_t l, int trans, int f32, double* GV, double* V,
                double* sigma, double eps, int64_t dm1, int64_t rmax, const double* norm_in,
                double* norm_out, int* rank_out, int* err_flag, cudaStream_t st, double* vtmp,
                double* pre) {
  JacobiBatchArgs a;
  a.vtmp[0] = vtmp;
  a.count = 1; a.trans = trans; a.f32 = f32; a.eps = eps; a.dm1 = dm1; a.rmax = rmax;
  a.norm_in = norm_in; a.norm_out = norm_out; a.err = err_flag;
  a.G[0] = G; a.l[0] = l; a.GV[0] = GV; a.V[0] = V; a.sigma[0] = sigma; a.rank_out[0] = rank_out;
  if (f32 || !pre) {
    jacobi_svd_batched(a, st);
    return;
  }
  // FP64 result in two passes: FP32 sweeps give rotations V32 (orthogonal to
  // about single precision); two Newton-Schulz steps X <- X (3 I - X^T X) / 2
  // in FP64 make them orthogonal to double rounding (each step squares the
  // error); FP64 sweeps on op(G) V32 starting from V32 then only have the
  // remaining rotations to do (the FP64 pipe is slow on this part)
  double* V32 = pre;
  double* A0 = pre + l * l;
  double* Tm = pre + 2 * l * l;
  double* Cn = pre + 3 * l * l;
  JacobiBatchArgs p1 = a;
  p1.f32 = 1;
  p1.norm_in = nullptr;
  p1.norm_out = nullptr;
  p1.V[0] = V32;
  jacobi_svd_batched(p1, st);
  for (int it = 0; it < 2; ++it) {
    GemmProblem t;  // Tm = X^T X
    t.M = (int)l; t.N = (int)l; t.K = (int)l;
    t.A = V32; t.sAm = 1; t.sAk = l;
    t.B = V32; t.sBk = l; t.sBn = 1;
    t.C = Tm; t.sCm = l; t.sCn = 1;
    gemm(TT_MODE_FP64, {t}, st);
    CopySeg cs;
    cs.src = V32; cs.dst = Cn; cs.A = l * l; cs.sa = 1; cs.src_f64 = cs.dst_f64 = 1;
    copy3d({cs}, st);
    GemmProblem u = gemm_rm((int)l, (int)l, (int)l, V32, l, Tm, l, Cn, l, -0.5, 1.5);
    gemm(TT_MODE_FP64, {u}, st);
    std::swap(V32, Cn);
  }
  GemmProblem g;
  g.M = (int)l; g.N = (int)l; g.K = (int)l;
  g.A = G; g.sAm = trans ? 1 : l; g.sAk = trans ? l : 1;  // op(G)
  g.B = V32; g.sBk = l; g.sBn = 1;
  g.C = A0; g.sCm = l; g.sCn = 1;
  gemm(TT_MODE_FP64, {g}, st);
  JacobiBatchArgs p2 = a;
  p2.trans = 0;
  p2.G[0] = A0;
  p2.v0[0] = V32;
  jacobi_svd_batched(p2, st);
}

}  // namespace ttsg
