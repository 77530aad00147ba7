// FP64 Householder QR of a tall matrix on a cooperative grid.
//
// The rounding of Section 3.3 orthogonalises the sketch Y = Z W (l columns, up
// to l_{mu-1} n_mu rows) once per bond, and the truncation sweep factorises the
// transposed core unfoldings the same way.  On GB300 the FP64 pipe delivers
// about 8 GFLOP/s per SM, so the factorisation is spread over up to one CTA
// per SM: CTA c keeps a contiguous block of rows in shared memory (FP64).
//
// Reflector convention (LAPACK dlarfg): for x = Y[j:, j] with alpha = x_0,
// sigma^2 = ||x_{1:}||^2: beta = -sign(alpha) sqrt(alpha^2 + sigma^2),
// tau = (beta - alpha) / beta, v = [1; x_{1:} / (alpha - beta)];
// sigma^2 == 0 gives tau = 0 (identity).  R's diagonal holds beta.
//
// Synchronisation.  Cross-CTA sums go through FP64 atomics into per-column
// slots that are zeroed before the launch, so every CTA reads one finished
// value after a grid barrier (all CTAs read the same memory, hence build the
// same reflector).  Factorisation step j needs one barrier: besides the
// products w = v^T Y[:, j+1:], each CTA contributes the three sums that give
// the next column's norm after the update, sigma^2_{j+1} = S1 - 2 tau w S2 +
// tau^2 w^2 S3 (S1 = sum Y^2, S2 = sum v Y, S3 = sum v^2 over rows > j+1).  When
// that downdate could lose accuracy (sigma^2 < S1 / 100) the norm is recomputed
// exactly with a second barrier; the decision is uniform across CTAs.
// The explicit Q = H_0 ... H_{l-1} [I; 0] is accumulated backwards in blocks
// of QB reflectors in the compact-WY form I - V T V^T (T from the block's
// V^T V), one barrier per block.
//
// Grid barriers spin a bounded number of times; on expiry the kernel sets bit 0
// of the error flag and every CTA returns (the host reports TT_ERR_TIMEOUT).
#include "kernels.cuh"
#include "prof.cuh"

namespace ttsg {

namespace {

constexpr int QR_THREADS = 256;
constexpr int QB = 8;                        // reflectors per Q-formation block
constexpr int NREP = 8;                      // replicas of every reduction slot
constexpr long long SPIN_LIMIT = 1ll << 24;  // bounded spin (well under a second)

struct QRArgs {
  const void* Y;
  int y_f64;
  int64_t m, l, sr, sc;
  void* Q;
  int q_f64;
  int64_t ldq;
  double* R;
  double* acc;     // [l][l + 4] factorisation slots (zeroed)
  double* nrm;     // [l] exact column norms (zeroed)
  double* pub;     // [2 (l + 1)] values published by the owner of a row
  double* vtv;     // [nblk][QB][QB] block-diagonal part of V^T V (zeroed)
  double* accq;    // [nblk][QB][l] Q-formation slots (zeroed)
  unsigned* bar;   // [0] arrivals, [1] generation
  int* err;
  int rows;        // rows per CTA
  int ldy;         // shared-memory row stride (l + 1)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier on a monotonic arrival counter (bar[0], zeroed before the
// launch): barrier number b completes when the counter reaches (b + 1) * P, so
// each CTA keeps a running target and needs one release fence, one atomic and
// a poll of the same word; no reset, no second word.  Returns false when the
// barrier timed out (bit 0 of the error flag is then set).
__device__ bool grid_barrier(unsigned* bar, unsigned& target, int* err) {
  __shared__ int fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    fail = 0;
    target += gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    volatile unsigned* vc = bar;
    long long spins = 0;
    while ((int)(*vc - target) < 0) {
      if (++spins > SPIN_LIMIT || (*(volatile int*)err & 1)) {
        atomicOr(err, 1);
        fail = 1;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
  }
  __syncthreads();
  return fail == 0;
}

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

// Block-wide sum; every thread gets the result.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < QR_THREADS / 32; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(QR_THREADS) qr_coop_kernel(const QRArgs a) {
  extern __shared__ double smem[];
  const int l = (int)a.l, ldy = a.ldy, L4 = l + 4;
  double* Yl = smem;                             // [rows][ldy]: R above, v below the diagonal
  double* Ql = Yl + (size_t)a.rows * ldy;        // [rows][ldy]: explicit Q rows
  double* wv = Ql + (a.Q ? (size_t)a.rows * ldy : 0);  // [l + 4]
  double* tau = wv + L4;                         // [l]
  double* Tb = tau + l;                          // [QB][QB]
  double* Wb = Tb + QB * QB;                     // [QB][l]
  double* Vb = Wb + QB * l;                      // [QB][rows]
  __shared__ double red[QR_THREADS / 32];
  __shared__ double sc[8];

  const int c = blockIdx.x;
  unsigned btarget = 0;  // running grid-barrier target (used by thread 0)
  const int64_t r0 = (int64_t)c * a.rows;
  const int64_t r1 = a.m < r0 + a.rows ? a.m : r0 + a.rows;
  const int nloc = r1 > r0 ? (int)(r1 - r0) : 0;
  const int tid = threadIdx.x;

  for (int e = tid; e < nloc * l; e += QR_THREADS) {
    const int li = e / l, j = e % l;
    const int64_t src = (r0 + li) * a.sr + (int64_t)j * a.sc;
    Yl[li * ldy + j] = a.y_f64 ? ((const double*)a.Y)[src] : (double)((const float*)a.Y)[src];
  }
  __syncthreads();
  // v_i of reflector j at local row li (1 on the diagonal, 0 above)
  auto vval = [&](int li, int j) -> double {
    const int64_t gi = r0 + li;
    return gi < j ? 0.0 : (gi == j ? 1.0 : Yl[li * ldy + j]);
  };

  // ------------------------------------------------ exact norm of column 0
  {
    double s = 0.0;
    for (int li = tid; li < nloc; li += QR_THREADS)
      if (r0 + li > 0) { const double v = Yl[li * ldy]; s += v * v; }
    s = block_sum(s, red);
    if (tid == 0) {
      if (s != 0.0) atomicAdd(a.nrm, s);
      if (r0 == 0 && nloc > 0) a.pub[0] = Yl[0];
    }
    if (!grid_barrier(a.bar, btarget, a.err)) return;
    if (tid == 0) { sc[0] = __ldcg(a.nrm); sc[1] = __ldcg(a.pub); }
    __syncthreads();
  }
  double sigma2 = sc[0], alpha = sc[1];

  // ------------------------------------------------------------ factorise
  for (int j = 0; j < l; ++j) {
    double t = 0.0, beta = alpha, scale = 0.0;
    if (sigma2 > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sigma2), alpha);
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    for (int li = tid; li < nloc; li += QR_THREADS) {
      const int64_t gi = r0 + li;
      if (gi > j) Yl[li * ldy + j] *= scale;
      else if (gi == j) Yl[li * ldy + j] = beta;
    }
    if (tid == 0) tau[j] = t;
    __syncthreads();
    if (j + 1 >= l) break;
    double* slot = a.acc + ((size_t)(c % NREP) * l + j) * L4;  // this CTA's replica
    // local rows holding v_j: the diagonal row (v = 1) and the rows below it
    const int64_t jl = (int64_t)j - r0;
    const int ldiag = (jl >= 0 && jl < nloc) ? (int)jl : -1;
    const int lbeg = jl + 1 > 0 ? (int)imin64(jl + 1, nloc) : 0;
    // partial products w[col] = sum_{i >= j} v_i Y[i, col], one thread per column
    for (int col = j + 1 + tid; col < l; col += QR_THREADS) {
      double p = ldiag >= 0 ? Yl[ldiag * ldy + col] : 0.0;
      for (int li = lbeg; li < nloc; ++li) p = fma(Yl[li * ldy + j], Yl[li * ldy + col], p);
      atomicAdd(slot + col, p);
    }
    // S1, S2, S3 of column j+1 over rows > j+1 (before the update)
    {
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      const int lb2 = jl + 2 > 0 ? (int)imin64(jl + 2, nloc) : 0;
      for (int li = lb2 + tid; li < nloc; li += QR_THREADS) {
        const double y = Yl[li * ldy + j + 1], v = Yl[li * ldy + j];
        s1 = fma(y, y, s1); s2 = fma(v, y, s2); s3 = fma(v, v, s3);
      }
      s1 = block_sum(s1, red);
      s2 = block_sum(s2, red);
      s3 = block_sum(s3, red);
      if (tid == 0) {
        atomicAdd(slot + l, s1);
        atomicAdd(slot + l + 1, s2);
        atomicAdd(slot + l + 2, s3);
        const int64_t o = j + 1 - r0;
        if (o >= 0 && o < nloc) {
          a.pub[2 * (j + 1)] = Yl[o * ldy + j + 1];
          a.pub[2 * (j + 1) + 1] = Yl[o * ldy + j];
        }
      }
    }
    if (!grid_barrier(a.bar, btarget, a.err)) return;
    for (int col = j + 1 + tid; col < L4; col += QR_THREADS) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < NREP; ++q) v += __ldcg(a.acc + ((size_t)q * l + j) * L4 + col);
      wv[col] = v;
    }
    if (tid == 0) { sc[2] = __ldcg(a.pub + 2 * (j + 1)); sc[3] = __ldcg(a.pub + 2 * (j + 1) + 1); }
    __syncthreads();
    // update rows >= j: Y[i, col] -= (tau v_i) w[col]
    for (int col = j + 1 + tid; col < l; col += QR_THREADS) wv[col] *= -t;
    __syncthreads();
    {
      const int ncols = l - j - 1;
      const int r_lo = ldiag >= 0 ? ldiag : lbeg;
      const int nr = nloc - r_lo;
      for (int e = tid; e < nr * ncols; e += QR_THREADS) {
        const int li = r_lo + e / ncols, col = j + 1 + e % ncols;
        const double v = li == ldiag ? 1.0 : Yl[li * ldy + j];
        Yl[li * ldy + col] = fma(v, wv[col], Yl[li * ldy + col]);
      }
    }
    // wv[j+1] now holds -tau w[j+1]
    const double mtw = wv[j + 1], S1 = wv[l], S2 = wv[l + 1], S3 = wv[l + 2];
    alpha = sc[2] + sc[3] * mtw;
    sigma2 = S1 + 2.0 * mtw * S2 + mtw * mtw * S3;
    __syncthreads();
    if (!(sigma2 >= 0.01 * S1)) {
      // possible cancellation: recompute the norm of the updated column exactly
      double s = 0.0;
      const int lb2 = jl + 2 > 0 ? (int)imin64(jl + 2, nloc) : 0;
      for (int li = lb2 + tid; li < nloc; li += QR_THREADS) {
        const double v = Yl[li * ldy + j + 1];
        s = fma(v, v, s);
      }
      s = block_sum(s, red);
      if (tid == 0) atomicAdd(a.nrm + j + 1, s);
      if (!grid_barrier(a.bar, btarget, a.err)) return;
      if (tid == 0) sc[4] = __ldcg(a.nrm + j + 1);
      __syncthreads();
      sigma2 = sc[4];
    }
  }

  // ------------------------------------------------------------ R factor
  if (a.R) {
    for (int e = tid; e < nloc * l; e += QR_THREADS) {
      const int li = e / l, col = e % l;
      const int64_t gi = r0 + li;
      if (gi < l) a.R[gi * l + col] = col >= gi ? Yl[li * ldy + col] : 0.0;
    }
  }
  if (!a.Q) return;

  // ------------------------------------------------------------ explicit Q
  const int nblk = (l + QB - 1) / QB;
  // block-diagonal part of V^T V, one thread per (block, p, q) with p <= q
  for (int e = tid; e < nblk * QB * QB; e += QR_THREADS) {
    const int bi = e / (QB * QB), p = (e / QB) % QB, q = e % QB;
    const int jp = bi * QB + p, jq = bi * QB + q;
    if (q < p || jq >= l) continue;
    double s = 0.0;
    for (int li = 0; li < nloc; ++li) s += vval(li, jp) * vval(li, jq);
    if (s != 0.0) atomicAdd(a.vtv + e, s);
  }
  for (int e = tid; e < nloc * l; e += QR_THREADS) {
    const int li = e / l, col = e % l;
    Ql[li * ldy + col] = (r0 + li == col) ? 1.0 : 0.0;
  }
  if (!grid_barrier(a.bar, btarget, a.err)) return;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int j0 = bi * QB, kb = min(QB, l - j0);
    if (tid == 0) {
      // forward recurrence: T[i][i] = tau_i, T[r][i] = -tau_i sum_{q=r}^{i-1} T[r][q] v_q^T v_i
      const double* G = a.vtv + (size_t)bi * QB * QB;
      for (int i = 0; i < kb; ++i) {
        const double ti = tau[j0 + i];
        for (int r = 0; r < i; ++r) {
          double s = 0.0;
          for (int q = r; q < i; ++q) s += Tb[r * QB + q] * __ldcg(G + q * QB + i);
          Tb[r * QB + i] = -ti * s;
        }
        Tb[i * QB + i] = ti;
        for (int r = i + 1; r < QB; ++r) Tb[r * QB + i] = 0.0;
      }
    }
    // stage v of the block's reflectors (unit diagonal, zeros above) in Vb
    for (int e = tid; e < QB * nloc; e += QR_THREADS) {
      const int r = e / nloc, li = e % nloc;
      Vb[e] = r < kb ? vval(li, j0 + r) : 0.0;
    }
    __syncthreads();
    // W = V_b^T Q over the local rows, columns j0..l-1
    const int nblk_all = (l + QB - 1) / QB;
    double* slot = a.accq + ((size_t)(c % NREP) * nblk_all + bi) * QB * l;
    const int ncols = l - j0;
    const int vlo = (int)imax64(0, imin64((int64_t)j0 - r0, nloc));
    for (int e = tid; e < kb * ncols; e += QR_THREADS) {
      const int r = e / ncols, col = j0 + e % ncols;
      double s = 0.0;
      for (int li = vlo; li < nloc; ++li) s = fma(Vb[r * nloc + li], Ql[li * ldy + col], s);
      atomicAdd(slot + (size_t)r * l + col, s);
    }
    if (!grid_barrier(a.bar, btarget, a.err)) return;
    for (int e = tid; e < QB * l; e += QR_THREADS) {
      double v = 0.0;
      if (e < kb * l) {
#pragma unroll
        for (int q = 0; q < NREP; ++q)
          v += __ldcg(a.accq + ((size_t)q * nblk_all + bi) * QB * l + e);
      }
      Wb[e] = v;
    }
    __syncthreads();
    // Wb <- T Wb
    for (int col = j0 + tid; col < l; col += QR_THREADS) {
      double w[QB];
#pragma unroll
      for (int r = 0; r < QB; ++r) w[r] = r < kb ? Wb[r * l + col] : 0.0;
#pragma unroll
      for (int r = 0; r < QB; ++r) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < QB; ++q) s += (q >= r && q < kb) ? Tb[r * QB + q] * w[q] : 0.0;
        if (r < kb) Wb[r * l + col] = s;
      }
    }
    __syncthreads();
    // Q -= V_b (T W)
    for (int e = tid; e < (nloc - vlo) * ncols; e += QR_THREADS) {
      const int li = vlo + e / ncols, col = j0 + e % ncols;
      double s = Ql[li * ldy + col];
#pragma unroll
      for (int r = 0; r < QB; ++r) s = fma(-Vb[r * nloc + li], Wb[r * l + col], s);
      Ql[li * ldy + col] = s;
    }
    __syncthreads();
  }
  for (int e = tid; e < nloc * l; e += QR_THREADS) {
    const int li = e / l, col = e % l;
    const double v = Ql[li * ldy + col];
    const int64_t dst = (r0 + li) * a.ldq + col;
    if (a.q_f64) ((double*)a.Q)[dst] = v;
    else ((float*)a.Q)[dst] = (float)v;
  }
}

struct QRPlan {
  int P, rows, ldy;
  size_t smem;
};

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

QRPlan plan(int64_t m, int64_t l, int sms, bool want_q) {
  QRPlan p;
  const int64_t min_rows = 16;
  int64_t P = std::min<int64_t>(sms, std::max<int64_t>(1, ceil_div(m, min_rows)));
  p.rows = (int)ceil_div(m, P);
  p.P = (int)ceil_div(m, p.rows);
  p.ldy = (int)l + 1;
  p.smem = ((size_t)p.rows * p.ldy * (want_q ? 2 : 1) + (l + 4) + l + QB * QB + QB * l +
            (size_t)QB * p.rows) * sizeof(double);
  return p;
}

size_t slots_doubles(int64_t l) {
  const int64_t nblk = (l + QB - 1) / QB;
  return (size_t)(NREP * l * (l + 4) + l + 2 * (l + 1) + nblk * QB * QB + NREP * nblk * QB * l);
}

}  // namespace

size_t qr_workspace(int64_t m, int64_t l) {
  (void)m;
  return 2048 + sizeof(double) * slots_doubles(l);
}

void qr_f64(const void* Y, int y_f64, int64_t m, int64_t l, int64_t sr, int64_t sc, void* Q,
            int q_f64, int64_t ldq, double* R, void* ws, size_t ws_bytes, int* err_flag,
            cudaStream_t st) {
  if (m < l || l <= 0) throw Error(TT_ERR_ARG, "qr_f64: need m >= l >= 1");
  if (g_dry_run) return;
  const int sms = num_sms();
  QRPlan p = plan(m, l, sms, Q != nullptr);
  if (p.smem > 220 * 1024)
    throw Error(TT_ERR_UNSUPPORTED, "qr_f64: block of " + std::to_string(p.rows) + " x " +
                                        std::to_string(l) + " does not fit in shared memory");
  Arena ar(ws, ws_bytes);
  unsigned* bar = ar.take<unsigned>(64);
  double* slots = ar.take<double>((int64_t)slots_doubles(l));
  QRArgs a;
  a.Y = Y; a.y_f64 = y_f64; a.m = m; a.l = l; a.sr = sr; a.sc = sc;
  a.Q = Q; a.q_f64 = q_f64; a.ldq = ldq; a.R = R;
  const int64_t nblk = (l + QB - 1) / QB;
  a.acc = slots;
  a.nrm = a.acc + NREP * l * (l + 4);
  a.pub = a.nrm + l;
  a.vtv = a.pub + 2 * (l + 1);
  a.accq = a.vtv + nblk * QB * QB;
  a.bar = bar; a.err = err_flag; a.rows = p.rows; a.ldy = p.ldy;
  TT_CUDA(cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned), st));
  TT_CUDA(cudaMemsetAsync(slots, 0, sizeof(double) * slots_doubles(l), st));
  static bool attr = false;
  if (!attr) {
    TT_CUDA(cudaFuncSetAttribute(qr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 220 * 1024));
    attr = true;
  }
  void* args[] = {(void*)&a};
  const int tok = prof_begin(PROF_QR, st);
  TT_CUDA(cudaLaunchCooperativeKernel((const void*)qr_coop_kernel, dim3(p.P), dim3(QR_THREADS),
                                      args, p.smem, st));
  count_launch();
  if (tok >= 0) {
    // Householder factorisation 2 m l^2 - 2 l^3 / 3, explicit Q the same again
    const double md = (double)m, ld = (double)l;
    const double f1 = 2.0 * md * ld * ld - 2.0 * ld * ld * ld / 3.0;
    prof_end(tok, st, Q ? 2.0 * f1 : f1,
             (double)m * l * (y_f64 ? 8 : 4) + (Q ? (double)m * l * (q_f64 ? 8 : 4) : 0.0));
  }
}

}  // namespace ttsg
