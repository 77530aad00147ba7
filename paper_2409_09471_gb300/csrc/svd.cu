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
// Double-precision problems run in a cluster form (jacobi_cluster_kernel): the
// pairs of a step are spread over up to 16 CTAs that pass the rotated columns
// to each other through distributed shared memory.
#include <cooperative_groups.h>

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

// Shared-memory column stride of the one-CTA kernel: the smallest ld >= l with
// ld = 8 or 24 (mod 32).  The PPW lane groups of a warp work on consecutive
// players p (and q), so their columns start ld apart; with ld = 8 (mod 32) the
// four groups' 8-lane slices cover four disjoint sets of banks.  (A stride of
// l itself puts all four groups on the same banks when 32 divides l.)
__host__ __device__ __forceinline__ int jacobi_ld(int l) {
  const int r = l & 31;
  return l + (r <= 8 ? 8 - r : (r <= 24 ? 24 - r : 40 - r));
}

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
  const int ld = jacobi_ld(l);
  T* A = (T*)sm_raw;            // column-major: column p at A + p*ld
  // V (column-major) in shared memory after A (stride ld), or in global
  // scratch of l x l doubles for large l (stride l)
  const int ldv = jb.vtmp[bi] ? l : ld;
  T* Vm = jb.vtmp[bi] ? (T*)jb.vtmp[bi] : A + (size_t)ld * l;
  T* after = A + (size_t)ld * l * (jb.vtmp[bi] ? 1 : 2);
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x, nwarps = nthreads / 32;
  const int grp = lane / GL, sub = lane % GL;

  for (int e = tid; e < l * l; e += nthreads) {
    const int i = e / l, j = e % l;           // element (i, j) of G
    A[(size_t)j * ld + i] = (T)(trans ? G[(size_t)j * l + i] : G[e]);
    Vm[(size_t)j * ldv + i] = jb.v0[bi] ? (T)jb.v0[bi][e] : ((i == j) ? T(1) : T(0));
  }
  __syncthreads();
  const T eps_t = sizeof(T) == 4 ? (T)1.1920929e-07 : (T)2.220446049250313e-16;
  const T tol = (T)l * eps_t;
  // columns whose squared norm is below eps^4 ||G||_F^2 are numerically zero
  __shared__ double s_tot;
  if (warp == 0) {
    double acc = 0.0;
    for (int e = lane; e < l * l; e += 32) {
      const double x = (double)A[(size_t)(e / l) * ld + e % l];
      acc += x * x;
    }
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
      for (int i = lane; i < l; i += 32) { const T x = A[(size_t)j * ld + i]; acc += x * x; }
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
          const T* ap = A + (size_t)p * ld;
          const T* aq = A + (size_t)q * ld;
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
          // t may be approximate, but c and s must satisfy c^2 + s^2 = 1 to
          // rounding: the approximate rsqrtf (up to 2 ulp, with a bias) drifts
          // the orthogonality of V linearly over the ~sweeps * l rotations a
          // column takes (1e-4 at l = 72); correctly rounded sqrt and division
          // keep the drift at the level of a random walk
          c = (T)(1.0f / sqrtf(1.f + (float)(t * t)));
        } else {
          const T zeta = (be - al) / (T(2) * ga);
          t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          c = T(1) / sqrt(T(1) + t * t);
        }
        s = c * t;
        T* ap = A + (size_t)p * ld;
        T* aq = A + (size_t)q * ld;
        T* vp = Vm + (size_t)p * ldv;
        T* vq = Vm + (size_t)q * ldv;
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
    for (int i = lane; i < l; i += 32) { const double x = (double)A[(size_t)j * ld + i]; acc += x * x; }
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
      GV[(size_t)i * l + rank] = (double)A[(size_t)j * ld + i];
      if (sizeof(T) == 8) V[(size_t)i * l + rank] = (double)Vm[(size_t)j * ldv + i];
    }
  }
  __syncthreads();
  if (sizeof(T) == 4) {
    // Single precision: the rounding errors of applying some sweeps * l
    // rotations to every column leave V orthogonal only to ~1e-5; one
    // Newton-Schulz step V <- V (3 I - V^T V) / 2 (quadratic, so 1e-5 -> 1e-10)
    // restores it to the level of FP32 rounding.  M = V^T V goes where A was
    // (GV is written out already), with compensated sums; one row of V at a
    // time goes through the norm buffer.
    T* M = A;
    for (int e = tid; e < l * l; e += nthreads) {
      const int p = e / l, q = e % l;
      if (q < p) continue;
      const T* vp = Vm + (size_t)p * ldv;
      const T* vq = Vm + (size_t)q * ldv;
      T sum = 0, comp = 0;
      for (int i = 0; i < l; ++i) {
        const T y = fma(vp[i], vq[i], -comp);
        const T t2 = sum + y;
        comp = (t2 - sum) - y;
        sum = t2;
      }
      M[(size_t)p * l + q] = sum;
      M[(size_t)q * l + p] = sum;
    }
    __syncthreads();
    T* row = nrm2;
    for (int i = 0; i < l; ++i) {
      for (int k = tid; k < l; k += nthreads) row[k] = Vm[(size_t)k * ldv + i];
      __syncthreads();
      for (int j = tid; j < l; j += nthreads) {
        T acc = 0;
        for (int k = 0; k < l; ++k) acc = fma(row[k], M[(size_t)k * l + j], acc);
        Vm[(size_t)j * ldv + i] = T(1.5) * row[j] - T(0.5) * acc;
      }
      __syncthreads();
    }
    for (int j = tid; j < l; j += nthreads) {
      int rank = 0;
      for (int i = 0; i < l; ++i)
        if (sg[i] > sg[j] || (sg[i] == sg[j] && i < j)) ++rank;
      for (int i = 0; i < l; ++i) V[(size_t)i * l + rank] = (double)Vm[(size_t)j * ldv + i];
    }
    __syncthreads();
  }
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

// ---------------------------------------------------------------- cluster form
// The same sweeps with one problem spread over a cluster of CS CTAs: in every
// parallel step, pair k is rotated by warp k / CS of CTA k % CS, which holds both
// columns (of G V and of V, with their tracked squared norms) in its own shared
// memory.  After the rotation each column is written straight into the shared
// memory of the CTA that rotates it in the next step (double-buffered by step
// parity), so one cluster barrier per step orders the whole exchange.  Every
// CTA then does CS times less arithmetic per step; the FP64 pipe of one SM is
// what bounds the one-CTA kernel in double precision.
constexpr int JC_MAX_CS = 16;
constexpr int JC_THREADS = 512;  // one warp per local pair

// player held by slot (k, role) in round-robin step `step` (lp players)
__device__ __forceinline__ int jc_col(int k, int role, int step, int lp) {
  const int m = lp - 1;
  if (k == 0) return role == 0 ? m : step;
  int x = role == 0 ? step + k : step - k;
  if (x >= m) x -= m;
  if (x < 0) x += m;
  return x;
}
// inverse: slot (k, role) of player x in step `step`
__device__ __forceinline__ void jc_slot(int x, int step, int lp, int& k, int& role) {
  const int m = lp - 1, npairs = lp >> 1;
  if (x == m) { k = 0; role = 0; return; }
  int d = x - step;
  if (d < 0) d += m;
  if (d == 0) { k = 0; role = 1; }
  else if (d <= npairs - 1) { k = d; role = 0; }
  else { k = m - d; role = 1; }
}

// Shared memory per CTA (ld = largest l of the launch, nplm = pairs per CTA):
// A and V slots [2 buffers][nplm][2 roles][ld], norms [2][nplm][2], then the
// gathered singular values (double[ld]) and the sweep flags (int[2][16]).
__host__ __device__ inline size_t jc_smem_bytes(int ld, int nplm, size_t es) {
  const size_t t = (8 * (size_t)nplm * ld + 4 * (size_t)nplm) * es;
  return ((t + 7) & ~(size_t)7) + (size_t)ld * sizeof(double) + 2 * JC_MAX_CS * sizeof(int);
}

template <typename T>
__global__ void __launch_bounds__(JC_THREADS)
jacobi_cluster_kernel(const __grid_constant__ JacobiBatch jb, int ld, int nplm, int* err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int cr = (int)cl.block_rank();
  const int bi = blockIdx.x / CS;
  const double* G = jb.G[bi];
  const int l = jb.l[bi], trans = jb.trans;
  double* GV = jb.GV[bi];
  double* V = jb.V[bi];
  double* sigma = jb.sigma[bi];
  const double* v0 = jb.v0[bi];
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* Ab = (T*)sm_raw;
  T* Vb = Ab + (size_t)4 * nplm * ld;
  T* Nb = Vb + (size_t)4 * nplm * ld;
  double* nall = (double*)(sm_raw + (((8 * (size_t)nplm * ld + 4 * (size_t)nplm) * sizeof(T) + 7) &
                                     ~(size_t)7));
  int* flags = (int*)(nall + ld);
  __shared__ int rotated;
  __shared__ double s_tot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x;
  const int lp = l + (l & 1), m = lp - 1, npairs = lp / 2;
  const int kk = warp;              // local pair of this warp
  const int k = kk * CS + cr;       // its pair index
  const bool has_pair = kk < nplm && k < npairs;
  auto slotA = [&](int b, int q, int role) { return Ab + ((size_t)(b * nplm + q) * 2 + role) * ld; };
  auto slotV = [&](int b, int q, int role) { return Vb + ((size_t)(b * nplm + q) * 2 + role) * ld; };
  auto slotN = [&](int b, int q, int role) { return Nb + (size_t)(b * nplm + q) * 2 + role; };

  // ||G||_F^2 read by every CTA in the same order (identical thresholds)
  if (warp == 0) {
    double acc = 0.0;
    for (int e = lane; e < l * l; e += 32) { const double x = (double)(T)G[e]; acc += x * x; }
    acc = warp_sum_t(acc);
    if (lane == 0) s_tot = acc;
  }
  // step-0 slots of this CTA's pairs
  if (has_pair) {
    for (int role = 0; role < 2; ++role) {
      const int x = jc_col(k, role, 0, lp);
      if (x >= l) continue;
      T* a = slotA(0, kk, role);
      T* v = slotV(0, kk, role);
      for (int i = lane; i < l; i += 32) {
        a[i] = (T)(trans ? G[(size_t)x * l + i] : G[(size_t)i * l + x]);
        v[i] = v0 ? (T)v0[(size_t)i * l + x] : ((i == x) ? T(1) : T(0));
      }
    }
  }
  __syncthreads();
  const T eps_t = sizeof(T) == 4 ? (T)1.1920929e-07 : (T)2.220446049250313e-16;
  const T tol = (T)l * eps_t;
  const T tot_t = (T)s_tot;
  const T tiny = (T)(s_tot * (double)eps_t * (double)eps_t * (double)eps_t * (double)eps_t);
  const T abs_thr = tol * eps_t * tot_t;
  const T tol2 = tol * tol;
  int buf = 0, sweep = 0;
  for (; sweep < MAX_SWEEPS; ++sweep) {
    // exact squared norms of the columns at the start of every sweep
    if (has_pair) {
      for (int role = 0; role < 2; ++role) {
        if (jc_col(k, role, 0, lp) >= l) continue;
        const T* a = slotA(buf, kk, role);
        T acc = 0;
        for (int i = lane; i < l; i += 32) acc = fma(a[i], a[i], acc);
        acc = warp_sum_t(acc);
        if (lane == 0) *slotN(buf, kk, role) = acc;
      }
    }
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < m; ++step) {
      const int nstep = step + 1 == m ? 0 : step + 1;
      if (has_pair) {
        const int xa = jc_col(k, 0, step, lp), xb = jc_col(k, 1, step, lp);
        const T* a0 = slotA(buf, kk, 0);
        const T* a1 = slotA(buf, kk, 1);
        const T* u0p = slotV(buf, kk, 0);
        const T* u1p = slotV(buf, kk, 1);
        T n0 = *slotN(buf, kk, 0), n1 = *slotN(buf, kk, 1);
        // where each column goes for the next step
        T *da0 = nullptr, *dv0 = nullptr, *dn0 = nullptr;
        T *da1 = nullptr, *dv1 = nullptr, *dn1 = nullptr;
        if (xa < l) {
          int k2, r2;
          jc_slot(xa, nstep, lp, k2, r2);
          const int dst = k2 % CS, q2 = k2 / CS;
          da0 = cl.map_shared_rank(slotA(buf ^ 1, q2, r2), dst);
          dv0 = cl.map_shared_rank(slotV(buf ^ 1, q2, r2), dst);
          dn0 = cl.map_shared_rank(slotN(buf ^ 1, q2, r2), dst);
        }
        if (xb < l) {
          int k2, r2;
          jc_slot(xb, nstep, lp, k2, r2);
          const int dst = k2 % CS, q2 = k2 / CS;
          da1 = cl.map_shared_rank(slotA(buf ^ 1, q2, r2), dst);
          dv1 = cl.map_shared_rank(slotV(buf ^ 1, q2, r2), dst);
          dn1 = cl.map_shared_rank(slotN(buf ^ 1, q2, r2), dst);
        }
        bool rot = false;
        T c = 1, sg = 0;
        if (xa < l && xb < l) {
          // rotation of (p, q) = (lower, higher index), as in the one-CTA kernel
          const bool sw = xa > xb;
          T g0 = 0, g1 = 0;
          int i = lane;
          for (; i + 32 < l; i += 64) {
            g0 = fma(a0[i], a1[i], g0);
            g1 = fma(a0[i + 32], a1[i + 32], g1);
          }
          if (i < l) g0 = fma(a0[i], a1[i], g0);
          const T ga = warp_sum_t(g0 + g1);
          const T al = sw ? n1 : n0, be = sw ? n0 : n1;
          // (double: the squared form of the relative test saves two dependent
          // square roots; float keeps the square roots against overflow)
          const bool rel_ok = sizeof(T) == 4 ? fabs(ga) <= tol * sqrt(al) * sqrt(be)
                                             : ga * ga <= tol2 * al * be;
          if (!(ga == T(0) || al <= tiny || be <= tiny || rel_ok || fabs(ga) <= abs_thr)) {
            T t;
            // for |zeta| > 1e4, t = 1 / (2 zeta) to a relative 1/(4 zeta^2),
            // below single rounding (and zeta^2 would overflow a float first)
            if (sizeof(T) == 4) {
              const float zeta = __fdividef((float)(be - al), 2.0f * (float)ga);
              t = fabsf(zeta) > 1e4f ? (T)__fdividef(0.5f, zeta)
                                     : (T)__fdividef(zeta >= 0.f ? 1.f : -1.f,
                                                     fabsf(zeta) + sqrtf(1.f + zeta * zeta));
              // correctly rounded: c^2 + s^2 = 1 to rounding (see jacobi_kernel)
              c = (T)(1.0f / sqrtf(1.f + (float)(t * t)));
            } else {
              // the angle only needs single precision (it sets how much of
              // gamma is removed); c = 1/sqrt(1+t^2), s = c t in double keep
              // the rotation orthogonal to double rounding
              const double zeta = (double)(be - al) / (2.0 * (double)ga);
              const float zf = (float)zeta;
              t = fabs(zeta) > 1e4 ? (T)(0.5 / zeta)
                                   : (T)__fdividef(zf >= 0.f ? 1.f : -1.f,
                                                   fabsf(zf) + sqrtf(1.f + zf * zf));
              c = (T)rsqrt(1.0 + (double)t * (double)t);
            }
            const T s = c * t;
            const T nal = al - t * ga, nbe = be + t * ga;
            if (sw) { n1 = nal; n0 = nbe; } else { n0 = nal; n1 = nbe; }
            // role form of p' = c p - s q, q' = s p + c q
            sg = sw ? -s : s;
            rot = true;
          }
        }
        for (int i = lane; i < l; i += 32) {
          const T x0 = a0[i], x1 = a1[i], w0 = u0p[i], w1 = u1p[i];
          if (da0) {
            da0[i] = rot ? c * x0 - sg * x1 : x0;
            dv0[i] = rot ? c * w0 - sg * w1 : w0;
          }
          if (da1) {
            da1[i] = rot ? sg * x0 + c * x1 : x1;
            dv1[i] = rot ? sg * w0 + c * w1 : w1;
          }
        }
        if (lane == 0) {
          if (dn0) *dn0 = n0;
          if (dn1) *dn1 = n1;
          if (rot) rotated = 1;
        }
      }
      if (step == m - 1) {
        __syncthreads();
        if (tid == 0) *cl.map_shared_rank(flags + (sweep & 1) * JC_MAX_CS + cr, 0) = rotated;
      }
      cl.sync();
      buf ^= 1;
    }
    // every CTA reads the same flags: the decision is uniform over the cluster
    int any = 0;
    for (int r = 0; r < CS; ++r) any |= *cl.map_shared_rank(flags + (sweep & 1) * JC_MAX_CS + r, 0);
    if (!any) break;
  }
  if (cr == 0 && tid == 0) {
    if (sweep == MAX_SWEEPS) atomicAdd(err, 1);  // non-convergence counter
    atomicMax(err + 2, sweep);
    atomicAdd(err + 3, sweep);
    atomicAdd(err + 4, 1);
  }
  // column norms gathered in CTA 0, then descending order (ties by index)
  if (has_pair) {
    for (int role = 0; role < 2; ++role) {
      const int x = jc_col(k, role, 0, lp);
      if (x >= l) continue;
      const T* a = slotA(buf, kk, role);
      double acc = 0.0;
      for (int i = lane; i < l; i += 32) { const double y = (double)a[i]; acc += y * y; }
      acc = warp_sum_t(acc);
      if (lane == 0) *cl.map_shared_rank(nall + x, 0) = sqrt(acc);
    }
  }
  cl.sync();
  if (cr != 0)
    for (int j = tid; j < l; j += nthreads) nall[j] = *cl.map_shared_rank(nall + j, 0);
  __syncthreads();
  if (has_pair) {
    for (int role = 0; role < 2; ++role) {
      const int x = jc_col(k, role, 0, lp);
      if (x >= l) continue;
      int rank = 0;
      for (int i = 0; i < l; ++i)
        if (nall[i] > nall[x] || (nall[i] == nall[x] && i < x)) ++rank;
      const T* a = slotA(buf, kk, role);
      const T* v = slotV(buf, kk, role);
      for (int i = lane; i < l; i += 32) {
        GV[(size_t)i * l + rank] = (double)a[i];
        V[(size_t)i * l + rank] = (double)v[i];
      }
    }
  }
  if (cr == 0) {
    for (int j = tid; j < l; j += nthreads) {
      int rank = 0;
      for (int i = 0; i < l; ++i)
        if (nall[i] > nall[j] || (nall[i] == nall[j] && i < j)) ++rank;
      sigma[rank] = nall[j];
    }
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int i = 0; i < l; ++i) tot += sigma[i] * sigma[i];
      const double nrm = jb.norm_in ? *jb.norm_in : sqrt(tot);
      if (bi == 0 && jb.norm_out) *jb.norm_out = nrm;
      const double delta = jb.eps * nrm / sqrt((double)(jb.dm1 > 0 ? jb.dm1 : 1));
      double tail = 0.0;
      int r = l;
      for (int i = l - 1; i >= 0; --i) {
        tail += sigma[i] * sigma[i];
        if (sqrt(tail) <= delta) r = i; else break;
      }
      if (r > jb.rmax) r = (int)jb.rmax;
      if (r < 1) r = 1;
      *jb.rank_out[bi] = r;
    }
  }
  // CTA 0's shared memory stays in place until every CTA has read the norms
  cl.sync();
}

}  // namespace

// Cluster launch of jacobi_cluster_kernel; false when the launch configuration
// is refused (the caller then uses the one-CTA kernel).
template <typename T>
static bool launch_jacobi_cluster(const JacobiBatch& jb, int count, int cs, int ld, int nplm,
                                  size_t smem, int* err, cudaStream_t st) {
  static const bool attr_set = [] {
    TT_CUDA(cudaFuncSetAttribute(jacobi_cluster_kernel<T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    TT_CUDA(cudaFuncSetAttribute(jacobi_cluster_kernel<T>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return true;
  }();
  (void)attr_set;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * cs));
  cfg.blockDim = dim3((unsigned)(nplm * 32));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<T>, jb, ld, nplm, err) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  check_launch("jacobi_cluster_kernel");
  return true;
}

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
  if (!a.f32) {
    // cluster form for double precision, where one SM's FP64 pipe bounds the
    // one-CTA kernel (GB300, l = 74: 4.4 ms -> 1.35 ms).  In single precision
    // a step is bound by its dependent chain and the barrier, not by the
    // arithmetic, and the cluster form measured slower (9 problems, l = 74:
    // 874 us against 786 us), so floats keep the one-CTA kernel.
    // 16 CTAs per problem for up to 4 problems, else 8; never more CTAs than
    // column pairs.
    const int npm = (int)((lmax + 1) / 2);
    int cs = a.count > 4 ? 8 : 16;
    while (cs > 1 && cs / 2 >= npm) cs /= 2;
    int nplm = (int)ceil_div(npm, cs);
    size_t jsm = jc_smem_bytes((int)lmax, nplm, es);
    if (jsm > 200 * 1024 && cs < JC_MAX_CS) {
      cs = JC_MAX_CS;
      nplm = (int)ceil_div(npm, cs);
      jsm = jc_smem_bytes((int)lmax, nplm, es);
    }
    if (jsm <= 200 * 1024 && nplm * 32 <= JC_THREADS) {
      const int tok = prof_begin(PROF_SVD, st);
      const bool ok = launch_jacobi_cluster<double>(jb, a.count, cs, (int)lmax, nplm, jsm, a.err, st);
      prof_end(tok, st, 0.0, 3.0 * lmax * lmax * 8.0 * a.count);
      if (ok) return;
    }
  }
  const size_t tail = (size_t)(lmax + 2) * es + (size_t)lmax * sizeof(double) + 16;
  const size_t ldm = (size_t)jacobi_ld((int)lmax);  // padded column stride (>= l of every problem)
  size_t smem = 2 * ldm * lmax * es + tail;
  if (smem > 220 * 1024) {
    // V moves to the callers' global scratch (l x l doubles, stride l); A
    // stays in shared memory
    smem = ldm * lmax * es + tail;
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
  // PPW column pairs per warp
  const int pairs = (int)((lmax + 1) / 2);
  const int threads =
      (int)std::min<int64_t>(SVD_THREADS, std::max<int64_t>(64, ceil_div(pairs, PPW) * 32));
  const int tok = prof_begin(PROF_SVD, st);
  if (a.f32) {
    static const bool attr_f = [] {
      TT_CUDA(cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   220 * 1024));
      return true;
    }();
    (void)attr_f;
    jacobi_kernel<float><<<a.count, threads, smem, st>>>(jb, a.err);
  } else {
    static const bool attr_d = [] {
      TT_CUDA(cudaFuncSetAttribute(jacobi_kernel<double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      return true;
    }();
    (void)attr_d;
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
