// FP64 Householder QR of a tall matrix on a cooperative grid.
//
// The rounding of Section 3.3 orthogonalises the sketch Y = Z W (l columns, up
// to l_{mu-1} n_mu rows) once per bond, and the truncation sweep factorises the
// transposed core unfoldings the same way.  On GB300 the FP64 pipe delivers
// about 2 FMA per clock per SM, so the factorisation is spread over up to one
// CTA per SM: CTA c keeps a contiguous block of rows in shared memory (FP64),
// and every FP64 instruction that is not an FMA of the factorisation itself
// counts.
//
// Reflector convention (LAPACK dlarfg): for x = Y[j:, j] with alpha = x_0,
// sigma^2 = ||x_{1:}||^2: beta = -sign(alpha) sqrt(alpha^2 + sigma^2),
// tau = (beta - alpha) / beta, v = [1; x_{1:} / (alpha - beta)]; sigma^2 == 0
// gives tau = 0 (identity).  R's diagonal holds beta.
//
// One grid-wide reduction per column.  At step j every CTA sums, over its rows
// r > j, t_c = Y[r][j] Y[r][c] for all columns c (FP64 atomics into replicated
// per-step slots), and the owner of row j publishes that row.  With scale =
// 1 / (alpha - beta) the same formula u_c = Y[j][c] + scale t_c gives
//   c > j:  v^T Y[:, c], the product the reflector update needs, and
//   c < j:  V[:, c]^T v, the column of the compact-WY factor T
//           (H_0 ... H_j = I - V T V^T, T[0:j, j] = -tau_j T[0:j, 0:j] V^T v_j),
// because column c < j already holds the normalised reflector below its
// diagonal.  t_j itself is sigma^2.  Rows of T are independent of each other,
// so CTA c keeps rows c, c + P, ... of T.
//
// Explicit Q = (I - V T V^T)[I; 0] = E - V K with K = T V_1^T (V_1 the top l x l
// block of V, unit lower triangular): two more barriers (publish T and V_1,
// then K), after which every CTA forms its own rows of Q.  When Q is stored in
// float, that product runs on the FP32 pipe (K and V rounded to float,
// accumulation in blocks of 8); in FP64 it stays in FP64.
//
// Forms of the same factorisation body (qr_body):
//  * cooperative (qr_coop_kernel): up to one CTA per SM, row blocks in shared
//    memory; the single-solve default;
//  * narrow: the fewest CTAs whose row blocks fit in shared memory, used when
//    many independent solves share the GPU (g_qr_narrow);
//  * global rows (qr_coop_gm_kernel): row blocks too large for shared memory
//    stay in global memory (L2), everything else unchanged;
//  * batched (qr_batch_kernel / qr_one_kernel): one CTA per matrix with its
//    rows in global memory, many matrices in one launch.
//
// Grid barriers spin a bounded number of times; on expiry the kernel sets bit 0
// of the error flag and every CTA returns (the host reports TT_ERR_TIMEOUT).
#include "kernels.cuh"
#include "prof.cuh"

namespace ttsg {

namespace {

constexpr int QR_THREADS = 256;
constexpr int NREP = 8;                      // replicas of every reduction slot
constexpr int QR_RPMAX = 4;                  // row phases of the partial sums
static_assert(NREP == 8, "the replica sums below are written out for 8 replicas");
constexpr long long SPIN_LIMIT = 1ll << 24;  // bounded spin (well under a second)

struct QRArgs {
  const void* Y;
  int y_f64;
  int64_t m, l, sr, sc;
  void* Q;
  int q_f64;
  int64_t ldq;
  double* R;
  double* acc;     // [l][NREP][l] per-step sums (zeroed)
  double* pub;     // [l][l] row j as published at step j
  double* Tg;      // [l][l] compact-WY factor T
  double* V1g;     // [l][l] V_1 (unit lower triangular)
  double* Kg;      // [l][l] K = T V_1^T
  unsigned* bar;   // [0] arrivals
  int* err;
  int rows;        // rows per CTA
  int ldy;         // shared-memory row stride (l + 1)
  int nown;        // rows of T per CTA
  int cw;          // Q-formation column chunk
  double* Yg;      // one-CTA mode: working copy of Y in global memory (else null)
  float* Vfg;      // one-CTA mode: float reflectors [m][l]
  float* yjfg;     // one-CTA mode: float column j [m]
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier on a monotonic arrival counter (bar[0], zeroed before the
// launch): barrier number b completes when the counter reaches (b + 1) * P, so
// each CTA keeps a running target; thread 0 arrives with a release reduction
// (ordering the CTA's earlier writes and atomics, which it has observed through
// the block barrier) and polls with acquire loads.  Returns false when the
// barrier timed out (bit 0 of the error flag is then set).
__device__ bool grid_barrier(unsigned* bar, unsigned& target, int* err) {
  __shared__ int fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    fail = 0;
    target += gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    long long spins = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if (++spins > SPIN_LIMIT || (*(volatile int*)err & 1)) {
        atomicOr(err, 1);
        fail = 1;
        break;
      }
    }
  }
  __syncthreads();
  return fail == 0;
}

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

// Rows of Q owned by this CTA: Q[g][x] = delta(g, x) - sum_q V[g][q] K[q][x],
// with V[g][q] = Vr[li][q] for q < g, 1 for q == g, 0 above.
template <typename E>
__device__ void form_q(const QRArgs& a, const E* Vr, int ldv, E* Kc, int nloc, int64_t r0) {
  const int l = (int)a.l, cw = a.cw, tid = threadIdx.x;
  const int G = QR_THREADS / cw;
  const int x = tid % cw, rg = tid / cw;
  for (int c0 = 0; c0 < l; c0 += cw) {
    const int w = imin(cw, l - c0);
    __syncthreads();
    for (int e = tid; e < l * w; e += QR_THREADS) {
      const int q = e / w, xx = e % w;
      Kc[q * cw + xx] = (E)__ldcg(a.Kg + (size_t)q * l + c0 + xx);
    }
    __syncthreads();
    if (x >= w) continue;
    const int col = c0 + x;
    for (int li = rg; li < nloc; li += G) {
      const int64_t gi = r0 + li;
      const int qn = gi < l ? (int)gi : l;
      const E* vr = Vr + (size_t)li * ldv;
      E s = 0;
      for (int q0 = 0; q0 < qn; q0 += 8) {
        E t = 0;
        const int q1 = imin(q0 + 8, qn);
        for (int q = q0; q < q1; ++q) t = fma(vr[q], Kc[q * cw + x], t);
        s += t;
      }
      if (gi < l) s += Kc[gi * cw + x];
      const E qv = (gi == col ? (E)1 : (E)0) - s;
      const int64_t dst = gi * a.ldq + col;
      if (a.q_f64) ((double*)a.Q)[dst] = (double)qv;
      else ((float*)a.Q)[dst] = (float)qv;
    }
  }
}

// Grid-wide synchronisation of one factorisation: the block barrier when one
// CTA owns the whole matrix, otherwise the bounded grid barrier.
__device__ __forceinline__ bool sync_all(const QRArgs& a, int P, unsigned& target) {
  if (P == 1) {
    __syncthreads();
    return true;
  }
  return grid_barrier(a.bar, target, a.err);
}

// The factorisation of one matrix by P CTAs (CTA c of P).  gm: the rows and the
// float copies live in global memory (one CTA per matrix, batched launches);
// otherwise CTA c keeps its row block in shared memory.
__device__ __forceinline__ void qr_body(const QRArgs& a, int P, int c, bool gm) {
  extern __shared__ double smem[];
  const int l = (int)a.l, ldy = a.ldy;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool want_q = a.Q != nullptr;
  // float Q: the compact-WY products (columns < j) run on the FP32 pipe from a
  // float copy of the normalised reflectors (also the V operand of form_q)
  const bool tf = want_q && !a.q_f64;
  const int64_t r0 = (int64_t)c * a.rows;                // first row of this CTA
  double* sp = smem;
  double* Yl = gm ? a.Yg + r0 * ldy : sp;                // [rows][ldy]: R above, v below
  if (!gm) sp += (size_t)a.rows * ldy;
  double* ts = sp;                                       // [l] reduced sums t_c
  double* rj = ts + l;                                   // [l] published row j
  double* uu = rj + l;                                   // [l] u_c (tau u_c for c > j)
  double* part = uu + l;                                 // [QR_RPMAX][l]
  double* Tl = part + (size_t)QR_RPMAX * l;              // [nown][l] owned rows of T
  float* partf = (float*)(Tl + (size_t)a.nown * l);      // [QR_RPMAX][l]
  float* fp = partf + (size_t)QR_RPMAX * l;
  float* yjf = gm ? a.yjfg + r0 : fp;                    // [rows] column j in float
  if (!gm) fp += a.rows;
  float* Vf = gm ? a.Vfg + r0 * l : fp;                  // [rows][l] reflectors in float
  if (!gm && tf) fp += (size_t)a.rows * l;
  unsigned char* qx =                                    // Q-formation chunk, 16-byte aligned
      (unsigned char*)(((uintptr_t)fp + 15) & ~(uintptr_t)15);
  __shared__ double hs[4];  // beta, tau, scale of the current reflector
  unsigned btarget = 0;  // running grid-barrier target (used by thread 0)
  if (gm && P == 1) {
    // one CTA: its own reduction slots are cleared here instead of by the host
    for (int e = tid; e < NREP * l * l; e += QR_THREADS) a.acc[e] = 0.0;
    __syncthreads();
  }
  const int64_t r1 = a.m < r0 + a.rows ? a.m : r0 + a.rows;
  const int nloc = r1 > r0 ? (int)(r1 - r0) : 0;

  for (int e = tid; e < nloc * l; e += QR_THREADS) {
    const int li = e / l, j = e % l;
    const int64_t src = (r0 + li) * a.sr + (int64_t)j * a.sc;
    Yl[li * ldy + j] = a.y_f64 ? ((const double*)a.Y)[src] : (double)((const float*)a.Y)[src];
  }
  for (int e = tid; e < a.nown * l; e += QR_THREADS) Tl[e] = 0.0;
  __syncthreads();
  if (tf)
    for (int li = tid; li < nloc; li += QR_THREADS) yjf[li] = (float)Yl[li * ldy];
  __syncthreads();

  // column jj of the owned rows of T: T[i][jj] = -tau_jj sum_{q=i}^{jj-1} T[i][q] p_q
  // with p_q = uu[q] and tau_jj = hs[1] of step jj
  auto t_column = [&](int jj) {
    const double tj = hs[1];
    for (int w = warp; w < a.nown; w += QR_THREADS / 32) {
      const int i = c + P * w;
      if (i > jj) continue;
      double* Ti = Tl + (size_t)w * l;
      if (i == jj) {
        if (lane == 0) Ti[jj] = tj;
        continue;
      }
      double s = 0.0;
      for (int q = i + lane; q < jj; q += 32) s = fma(Ti[q], uu[q], s);
      s = warp_sum(s);
      if (lane == 0) Ti[jj] = -tj * s;
    }
  };

  for (int j = 0; j < l; ++j) {
    const int64_t jl = (int64_t)j - r0;                     // local index of row j
    const int lb = (int)(jl + 1 < 0 ? 0 : (jl + 1 > nloc ? nloc : jl + 1));  // first row > j
    const int ncol = l - j;                                 // FP64 columns j .. l-1
    const int RPd = imin(QR_RPMAX, ncol >= QR_THREADS ? 1 : QR_THREADS / ncol);
    const int RPt = j == 0 ? 1 : imin(QR_RPMAX, j >= QR_THREADS ? 1 : QR_THREADS / j);
    // (a) partial sums over the local rows r > j
    if (lb < nloc) {
      for (int e = tid; e < RPd * ncol; e += QR_THREADS) {
        const int col = j + e % ncol, rp = e / ncol;
        // two independent chains: dependent FP64 FMAs are slow on this part
        double s0 = 0.0, s1 = 0.0;
        int li = lb + rp;
        for (; li + RPd < nloc; li += 2 * RPd) {
          s0 = fma(Yl[li * ldy + j], Yl[li * ldy + col], s0);
          s1 = fma(Yl[(li + RPd) * ldy + j], Yl[(li + RPd) * ldy + col], s1);
        }
        if (li < nloc) s0 = fma(Yl[li * ldy + j], Yl[li * ldy + col], s0);
        part[rp * l + col] = s0 + s1;
      }
      if (want_q && j > 0) {
        for (int e = tid; e < RPt * j; e += QR_THREADS) {
          const int col = e % j, rp = e / j;
          if (tf) {
            float s = 0.f;
            for (int li = lb + rp; li < nloc; li += RPt) s = fmaf(yjf[li], Vf[li * l + col], s);
            partf[rp * l + col] = s;
          } else {
            double s0 = 0.0, s1 = 0.0;
            int li = lb + rp;
            for (; li + RPt < nloc; li += 2 * RPt) {
              s0 = fma(Yl[li * ldy + j], Yl[li * ldy + col], s0);
              s1 = fma(Yl[(li + RPt) * ldy + j], Yl[(li + RPt) * ldy + col], s1);
            }
            if (li < nloc) s0 = fma(Yl[li * ldy + j], Yl[li * ldy + col], s0);
            part[rp * l + col] = s0 + s1;
          }
        }
      }
      __syncthreads();
      double* slot = a.acc + ((size_t)j * NREP + (c % NREP)) * l;
      for (int col = (want_q ? 0 : j) + tid; col < l; col += QR_THREADS) {
        double s;
        if (col >= j) {
          s = part[col];
          for (int rp = 1; rp < RPd; ++rp) s += part[rp * l + col];
        } else if (tf) {
          float f = partf[col];
          for (int rp = 1; rp < RPt; ++rp) f += partf[rp * l + col];
          s = (double)f;
        } else {
          s = part[col];
          for (int rp = 1; rp < RPt; ++rp) s += part[rp * l + col];
        }
        if (__double_as_longlong(s) != 0) atomicAdd(slot + col, s);
      }
    }
    // column j-1 of T while the other CTAs catch up (uu and tau still hold step j-1)
    if (want_q && j > 0) t_column(j - 1);
    if (jl >= 0 && jl < nloc)
      for (int col = tid; col < l; col += QR_THREADS) a.pub[(size_t)j * l + col] = Yl[jl * ldy + col];
    if (!sync_all(a, P, btarget)) return;
    // (b) the reduced sums and row j; lane 0 of warp 0 meanwhile forms the
    // reflector's scalars from x = alpha^2 + sigma^2 with one reciprocal square
    // root and one reciprocal: beta = -sign(alpha) sqrt(x), tau = (beta -
    // alpha) / beta = 1 + |alpha| / sqrt(x), scale = 1 / (alpha - beta)
    const int c_lo = want_q ? 0 : j;
    if (warp == 0) {
      if (lane == 0) {
        double v[NREP];
#pragma unroll
        for (int q = 0; q < NREP; ++q) v[q] = __ldcg(a.acc + ((size_t)j * NREP + q) * l + j);
        const double y0 = __ldcg(a.pub + (size_t)j * l + j);
        const double sig2 = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        double beta = y0, tau = 0.0, scale = 0.0;
        if (sig2 > 0.0) {
          const double x = fma(y0, y0, sig2);
          const double rs = rsqrt(x);
          beta = -copysign(x * rs, y0);
          tau = fma(fabs(y0), rs, 1.0);
          scale = 1.0 / (y0 - beta);
        }
        hs[0] = beta; hs[1] = tau; hs[2] = scale;
      }
    } else {
      for (int col = tid - 32; col < l; col += QR_THREADS - 32) {
        double s = 0.0;
        if (col >= c_lo) {
          double v[NREP];
#pragma unroll
          for (int q = 0; q < NREP; ++q) v[q] = __ldcg(a.acc + ((size_t)j * NREP + q) * l + col);
          s = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        }
        ts[col] = s;
        rj[col] = __ldcg(a.pub + (size_t)j * l + col);
      }
    }
    __syncthreads();
    const double beta = hs[0], tau = hs[1], scale = hs[2];
    for (int col = c_lo + tid; col < l; col += QR_THREADS) {
      const double u = fma(scale, ts[col], rj[col]);
      uu[col] = col > j ? tau * u : u;
    }
    for (int li = tid; li < nloc; li += QR_THREADS) {
      const int64_t gi = r0 + li;
      if (gi > j) {
        const double v = Yl[li * ldy + j] * scale;
        Yl[li * ldy + j] = v;
        if (tf) Vf[li * l + j] = (float)v;
      } else if (gi == j) {
        Yl[li * ldy + j] = beta;
      }
    }
    __syncthreads();
    // (c) update rows >= j, columns > j: Y[r][c] -= v_r tau u_c (column j+1
    // also refreshes its float copy for the next step)
    {
      const int ncols = l - j - 1;
      const int r_lo = (jl >= 0 && jl < nloc) ? (int)jl : lb;
      if (ncols > 0 && r_lo < nloc) {
        const int RPu = ncols >= QR_THREADS ? 1 : QR_THREADS / ncols;
        for (int e = tid; e < RPu * ncols; e += QR_THREADS) {
          const int col = j + 1 + e % ncols, rp = e / ncols;
          const double w = uu[col];
          const bool fj = tf && col == j + 1;
          int li = r_lo + rp;
          // four rows at a time, loads before the FMAs
          for (; li + 3 * RPu < nloc; li += 4 * RPu) {
            double v[4], y[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int lk = li + k * RPu;
              v[k] = (r0 + lk == j) ? 1.0 : Yl[lk * ldy + j];
              y[k] = Yl[lk * ldy + col];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int lk = li + k * RPu;
              y[k] = fma(-v[k], w, y[k]);
              Yl[lk * ldy + col] = y[k];
              if (fj) yjf[lk] = (float)y[k];
            }
          }
          for (; li < nloc; li += RPu) {
            const double v = (r0 + li == j) ? 1.0 : Yl[li * ldy + j];
            const double y = fma(-v, w, Yl[li * ldy + col]);
            Yl[li * ldy + col] = y;
            if (fj) yjf[li] = (float)y;
          }
        }
      }
    }
    __syncthreads();
  }
  if (want_q) t_column(l - 1);
  __syncthreads();

  if (a.R) {
    for (int e = tid; e < nloc * l; e += QR_THREADS) {
      const int li = e / l, col = e % l;
      const int64_t gi = r0 + li;
      if (gi < l) a.R[gi * l + col] = col >= gi ? Yl[li * ldy + col] : 0.0;
    }
  }
  if (!want_q) return;

  // ------------------------------------------------------------ explicit Q
  for (int w = 0; w < a.nown; ++w) {
    const int i = c + P * w;
    if (i >= l) break;
    for (int col = tid; col < l; col += QR_THREADS) a.Tg[(size_t)i * l + col] = Tl[w * l + col];
  }
  for (int e = tid; e < nloc * l; e += QR_THREADS) {
    const int li = e / l, col = e % l;
    const int64_t gi = r0 + li;
    if (gi < l) a.V1g[gi * l + col] = col < gi ? Yl[li * ldy + col] : (col == gi ? 1.0 : 0.0);
  }
  if (!sync_all(a, P, btarget)) return;
  // K[i][x] = sum_{q = i}^{x} T[i][q] V_1[x][q] for the owned rows i, one warp per (i, x)
  for (int task = warp; task < a.nown * l; task += QR_THREADS / 32) {
    const int w = task / l, x = task % l;
    const int i = c + P * w;
    if (i >= l) continue;
    const double* Ti = Tl + (size_t)w * l;
    double s = 0.0;
    for (int q = i + lane; q <= x; q += 32) s = fma(Ti[q], __ldcg(a.V1g + (size_t)x * l + q), s);
    s = warp_sum(s);
    if (lane == 0) a.Kg[(size_t)i * l + x] = s;
  }
  if (!sync_all(a, P, btarget)) return;
  if (a.q_f64) {
    form_q<double>(a, Yl, ldy, (double*)qx, nloc, r0);
  } else {
    form_q<float>(a, Vf, l, (float*)qx, nloc, r0);
  }
}

__global__ void __launch_bounds__(QR_THREADS) qr_coop_kernel(const QRArgs a) {
  qr_body(a, (int)gridDim.x, (int)blockIdx.x, false);
}
// The same with the row blocks in global memory (matrices whose row blocks do
// not fit in shared memory).
__global__ void __launch_bounds__(QR_THREADS) qr_coop_gm_kernel(const QRArgs a) {
  qr_body(a, (int)gridDim.x, (int)blockIdx.x, true);
}

// One CTA per matrix: problem blockIdx.x of a batch.
__global__ void __launch_bounds__(QR_THREADS) qr_batch_kernel(const QRArgs* probs) {
  const QRArgs a = probs[blockIdx.x];
  qr_body(a, 1, 0, true);
}
// The same for a single matrix, arguments by value (no host-to-device copy,
// which from pageable memory would synchronise the stream).
__global__ void __launch_bounds__(QR_THREADS) qr_one_kernel(const QRArgs a) {
  qr_body(a, 1, 0, true);
}

struct QRPlan {
  int P, rows, ldy, nown, cw;
  size_t smem;
};

int num_sms() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

constexpr size_t QR_SMEM_MAX = 220 * 1024;

// gm: the row blocks and their float copies live in global memory (the
// batched one-CTA form, and matrices whose row blocks exceed shared memory).
QRPlan plan(int64_t m, int64_t l, int sms, bool want_q, bool q_f64, bool gm) {
  QRPlan p;
  const int64_t min_rows = 16;
  int64_t P = std::min<int64_t>(sms, std::max<int64_t>(1, ceil_div(m, min_rows)));
  p.rows = (int)ceil_div(m, P);
  p.P = (int)ceil_div(m, p.rows);
  p.ldy = (int)l + 1;
  p.nown = (int)ceil_div(l, p.P);
  const bool tf = want_q && !q_f64;
  const size_t rows_sm = gm ? 0 : (size_t)p.rows;
  const size_t base = (rows_sm * p.ldy + 3 * l + (size_t)QR_RPMAX * l + (size_t)p.nown * l) *
                          sizeof(double) +
                      ((size_t)QR_RPMAX * l + rows_sm + (tf ? rows_sm * l : 0)) * sizeof(float) +
                      16;
  p.cw = 8;
  p.smem = base;
  if (want_q) {
    // widest column chunk (a divisor of the block size) that fits
    for (int cw : {64, 32, 16, 8}) {
      p.cw = cw;
      p.smem = base + (size_t)l * cw * (q_f64 ? sizeof(double) : sizeof(float));
      if (p.smem <= QR_SMEM_MAX) break;
    }
  }
  return p;
}

size_t slots_doubles(int64_t l) { return (size_t)(NREP * l * l + 4 * l * l); }

// Narrow form (concurrent solves): the fewest CTAs whose row blocks fit in
// shared memory, so that independent factorisations on other streams find
// free SMs.
QRPlan plan_narrow(int64_t m, int64_t l, int sms, bool want_q, bool q_f64) {
  for (int64_t P = 1; P <= sms; ++P) {
    QRPlan p = plan(m, l, (int)P, want_q, q_f64, false);
    if (p.P <= P && p.smem <= QR_SMEM_MAX) return p;
  }
  return plan(m, l, sms, want_q, q_f64, false);
}

// Global scratch of one problem in the batched form: slots, the FP64 working
// copy of Y and the float copies, each 256-byte aligned.
size_t batch_problem_bytes(int64_t m, int64_t l) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return al(sizeof(double) * slots_doubles(l)) + al(sizeof(double) * m * (l + 1)) +
         al(sizeof(float) * m * l) + al(sizeof(float) * m) + 256;
}

void fill_args(QRArgs& a, const QRProblem& pb, const QRPlan& p) {
  a.Y = pb.Y; a.y_f64 = pb.y_f64; a.m = pb.m; a.l = pb.l; a.sr = pb.sr; a.sc = pb.sc;
  a.Q = pb.Q; a.q_f64 = pb.q_f64; a.ldq = pb.ldq; a.R = pb.R;
  a.rows = p.rows; a.ldy = p.ldy; a.nown = p.nown; a.cw = p.cw;
  a.Yg = nullptr; a.Vfg = nullptr; a.yjfg = nullptr;
}

void prof_qr(int tok, cudaStream_t st, const QRProblem* pbs, int count) {
  if (tok < 0) return;
  // algorithmic work: the factorisation's leading term 2 m l^2 (for the
  // rounding's Y of l n rows this is 2 n l^3); the explicit Q is not counted
  double fl = 0.0, by = 0.0;
  for (int i = 0; i < count; ++i) {
    const QRProblem& pb = pbs[i];
    const double md = (double)pb.m, ld = (double)pb.l;
    fl += 2.0 * md * ld * ld;
    by += md * ld * (pb.y_f64 ? 8 : 4) + (pb.Q ? md * ld * (pb.q_f64 ? 8 : 4) : 0.0);
  }
  prof_end(tok, st, fl, by);
}

}  // namespace

thread_local bool g_qr_narrow = false;

size_t qr_batch_workspace(int count, const int64_t* m, const int64_t* l) {
  size_t b = 4096 + (size_t)count * sizeof(QRArgs);
  for (int i = 0; i < count; ++i) b += batch_problem_bytes(m[i], l[i]);
  return b;
}

void qr_f64_batched(int count, const QRProblem* pbs, void* ws, size_t ws_bytes, int* err_flag,
                    cudaStream_t st) {
  if (count <= 0) return;
  for (int i = 0; i < count; ++i)
    if (pbs[i].m < pbs[i].l || pbs[i].l <= 0) throw Error(TT_ERR_ARG, "qr_f64: need m >= l >= 1");
  if (g_dry_run) return;
  Arena ar(ws, ws_bytes);
  QRArgs* dargs = ar.take<QRArgs>(count);
  std::vector<QRArgs> hargs(count);
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    const QRProblem& pb = pbs[i];
    const int64_t m = pb.m, l = pb.l;
    QRPlan p = plan(m, l, 1, pb.Q != nullptr, pb.q_f64 != 0, true);
    if (p.smem > QR_SMEM_MAX)
      throw Error(TT_ERR_UNSUPPORTED, "qr_f64: " + std::to_string(l) +
                                          " columns do not fit the one-CTA form");
    smem = std::max(smem, p.smem);
    QRArgs& a = hargs[i];
    fill_args(a, pb, p);
    a.acc = ar.take<double>((int64_t)slots_doubles(l));
    a.pub = a.acc + NREP * l * l;
    a.Tg = a.pub + l * l;
    a.V1g = a.Tg + l * l;
    a.Kg = a.V1g + l * l;
    a.Yg = ar.take<double>(m * (l + 1));
    a.Vfg = ar.take<float>(m * l);
    a.yjfg = ar.take<float>(m);
    a.bar = nullptr;
    a.err = err_flag;
  }
  static const bool attr = [] {
    TT_CUDA(cudaFuncSetAttribute(qr_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)QR_SMEM_MAX));
    TT_CUDA(cudaFuncSetAttribute(qr_one_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)QR_SMEM_MAX));
    return true;
  }();
  (void)attr;
  const int tok = prof_begin(PROF_QR, st);
  if (count == 1) {
    qr_one_kernel<<<1, QR_THREADS, smem, st>>>(hargs[0]);
    check_launch("qr_one_kernel");
  } else {
    // from pageable memory this copy completes (staged) before it returns
    TT_CUDA(cudaMemcpyAsync(dargs, hargs.data(), sizeof(QRArgs) * count, cudaMemcpyHostToDevice,
                            st));
    qr_batch_kernel<<<count, QR_THREADS, smem, st>>>(dargs);
    check_launch("qr_batch_kernel");
  }
  prof_qr(tok, st, pbs, count);
}

// The shared-memory plan does not fit for some precision pair: the rows go to
// global memory (an FP64 copy of Y, float copies of the reflectors and of the
// current column).
static bool needs_global_rows(int64_t m, int64_t l) {
  const int sms = num_sms();
  for (int want_q = 0; want_q < 2; ++want_q)
    for (int q64 = 0; q64 < 2; ++q64) {
      const QRPlan p = g_qr_narrow ? plan_narrow(m, l, sms, want_q, q64)
                                   : plan(m, l, sms, want_q, q64, false);
      if (p.smem > QR_SMEM_MAX) return true;
    }
  return false;
}
static size_t global_rows_bytes(int64_t m, int64_t l) {
  return sizeof(double) * m * (l + 1) + sizeof(float) * m * l + sizeof(float) * m + 3 * 256;
}

size_t qr_workspace(int64_t m, int64_t l) {
  return 2048 + sizeof(double) * slots_doubles(l) +
         (needs_global_rows(m, l) ? global_rows_bytes(m, l) : 0);
}

void qr_f64(const void* Y, int y_f64, int64_t m, int64_t l, int64_t sr, int64_t sc, void* Q,
            int q_f64, int64_t ldq, double* R, void* ws, size_t ws_bytes, int* err_flag,
            cudaStream_t st) {
  if (m < l || l <= 0) throw Error(TT_ERR_ARG, "qr_f64: need m >= l >= 1");
  if (g_dry_run) return;
  const int sms = num_sms();
  QRPlan p = g_qr_narrow ? plan_narrow(m, l, sms, Q != nullptr, q_f64 != 0)
                          : plan(m, l, sms, Q != nullptr, q_f64 != 0, false);
  bool gm = false;
  if (p.smem > QR_SMEM_MAX) {
    // row blocks too large for shared memory: keep them in global memory
    p = plan(m, l, sms, Q != nullptr, q_f64 != 0, true);
    gm = true;
  }
  if (p.smem > QR_SMEM_MAX)
    throw Error(TT_ERR_UNSUPPORTED, "qr_f64: " + std::to_string(l) +
                                        " columns do not fit in shared memory");
  Arena ar(ws, ws_bytes);
  unsigned* bar = ar.take<unsigned>(64);
  double* slots = ar.take<double>((int64_t)slots_doubles(l));
  QRArgs a;
  QRProblem pb{Y, y_f64, m, l, sr, sc, Q, q_f64, ldq, R};
  fill_args(a, pb, p);
  if (gm) {
    a.Yg = ar.take<double>(m * (l + 1));
    a.Vfg = ar.take<float>(m * l);
    a.yjfg = ar.take<float>(m);
  }
  a.acc = slots;
  a.pub = a.acc + NREP * l * l;
  a.Tg = a.pub + l * l;
  a.V1g = a.Tg + l * l;
  a.Kg = a.V1g + l * l;
  a.bar = bar; a.err = err_flag;
  TT_CUDA(cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned), st));
  TT_CUDA(cudaMemsetAsync(a.acc, 0, sizeof(double) * NREP * l * l, st));
  static const bool attr = [] {
    TT_CUDA(cudaFuncSetAttribute(qr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)QR_SMEM_MAX));
    TT_CUDA(cudaFuncSetAttribute(qr_coop_gm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)QR_SMEM_MAX));
    return true;
  }();
  (void)attr;
  void* args[] = {(void*)&a};
  const int tok = prof_begin(PROF_QR, st);
  TT_CUDA(cudaLaunchCooperativeKernel(gm ? (const void*)qr_coop_gm_kernel
                                         : (const void*)qr_coop_kernel,
                                      dim3(p.P), dim3(QR_THREADS), args, p.smem, st));
  count_launch();
  prof_qr(tok, st, &pb, 1);
}

}  // namespace ttsg
