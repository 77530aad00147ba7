// Grouped strided batched GEMM on CUDA cores (FP64 and FP32).
//
// Every contraction of the TT-sGMRES iteration (matvec cores, Khatri-Rao sketch
// steps, Gram sweeps, partial contractions and projections of the randomized
// rounding) is expressed as one or a few of these problems; see tt_ops.cu for
// the mapping.  One launch covers up to MAXG problems of different shapes:
// blockIdx.z selects the problem, blockIdx.y the batch entry and blockIdx.x the
// 64x64 output tile.  Tiles beyond a problem's extent exit immediately.
#include "prof.cuh"

namespace ttsg {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// Split-K partials of problem z go to part[z] + ((split * nb + b) * M + m) * N + n.
struct SplitInfo {
  int splits[MAXG];
  int64_t part_off[MAXG];
};

template <typename T>
__global__ void __launch_bounds__(NT)
gemm_simt_kernel(const __grid_constant__ GemmGroup g, const __grid_constant__ SplitInfo si,
                 T* part) {
  const GemmProblem& p = g.p[blockIdx.z];
  const int M = p.M, N = p.N;
  const int tiles_n = (N + BN - 1) / BN;
  const int tiles_m = (M + BM - 1) / BM;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int nb = p.nb1 * p.nb2;
  const int splits = si.splits[blockIdx.z];
  if ((int)blockIdx.y >= nb * splits) return;
  const int split = blockIdx.y / nb, bidx = blockIdx.y % nb;
  const int kchunk = ((p.K + splits - 1) / splits + BK - 1) / BK * BK;
  const int kbeg = split * kchunk;
  const int K = min(p.K, kbeg + kchunk);
  const int b1 = bidx / p.nb2, b2 = bidx % p.nb2;
  const int m0 = (blockIdx.x / tiles_n) * BM, n0 = (blockIdx.x % tiles_n) * BN;

  const T* A = (const T*)p.A;
  const T* B = (const T*)p.B + b1 * p.sBb1 + b2 * p.sBb2;
  T* C = (T*)p.C + b1 * p.sCb1 + b2 * p.sCb2;
  if (A) A += b1 * p.sAb1 + b2 * p.sAb2;
  const T* S = (const T*)p.kr_S;

  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Bs[BK][BN + 4];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  const bool a_kfast = (p.a_mode == 1) || (p.sAk == 1);
  const bool b_nfast = (p.sBn == 1);

  // global -> registers for one K tile (A: BM x BK, B: BK x BN); the next
  // tile's loads are issued before the current tile's FMAs (register double
  // buffering), so their latency overlaps the arithmetic
  constexpr int RA = (BM * BK) / NT, RB = (BN * BK) / NT;
  T ra[RA], rb[RB];
  auto load_tile = [&](int k0) {
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      const int e = tid + r * NT;
      int mm, kk;
      if (a_kfast) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
      const int m = m0 + mm, k = k0 + kk;
      T v = T(0);
      if (m < M && k < K) {
        if (p.a_mode == 1) {
          const int pz = k / p.kr_n, iz = k - pz * p.kr_n;
          const T z = A ? A[(int64_t)m * p.sAm + (int64_t)pz * p.sAk] : T(1);
          v = z * S[(int64_t)m * p.kr_sS + iz];
        } else {
          v = A[(int64_t)m * p.sAm + (int64_t)k * p.sAk];
        }
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int e = tid + r * NT;
      int nn, kk;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
      const int n = n0 + nn, k = k0 + kk;
      rb[r] = (n < N && k < K) ? B[(int64_t)k * p.sBk + (int64_t)n * p.sBn] : T(0);
    }
  };
  auto store_tile = [&]() {
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      const int e = tid + r * NT;
      int mm, kk;
      if (a_kfast) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
      As[kk][mm] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int e = tid + r * NT;
      int nn, kk;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
      Bs[kk][nn] = rb[r];
    }
  };

  if (kbeg < K) load_tile(kbeg);
  for (int k0 = kbeg; k0 < K; k0 += BK) {
    store_tile();
    __syncthreads();
    if (k0 + BK < K) load_tile(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (splits > 1) {
    T* P = part + si.part_off[blockIdx.z] + ((int64_t)split * nb + bidx) * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty * 4 + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx * 4 + j;
        if (n < N) P[(int64_t)m * N + n] = acc[i][j];
      }
    }
    return;
  }
  T alpha = (T)p.alpha;
  if (p.alpha_dev) alpha *= (T)(*p.alpha_dev);
  const T beta = (T)p.beta;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      T* c = C + (int64_t)m * p.sCm + (int64_t)n * p.sCn;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v += beta * (*c);
      *c = v;
    }
  }
}

// C = alpha * sum_s part[s] + beta * C for every split problem of a launch.
template <typename T>
__global__ void splitk_reduce_kernel(const __grid_constant__ GemmGroup g,
                                     const __grid_constant__ SplitInfo si, const T* part) {
  const GemmProblem& p = g.p[blockIdx.y];
  const int splits = si.splits[blockIdx.y];
  if (splits <= 1) return;
  const int64_t nb = (int64_t)p.nb1 * p.nb2, MN = (int64_t)p.M * p.N, total = nb * MN;
  T alpha = (T)p.alpha;
  if (p.alpha_dev) alpha *= (T)(*p.alpha_dev);
  const T beta = (T)p.beta;
  const T* P = part + si.part_off[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int s = 0; s < splits; ++s) acc += P[(int64_t)s * total + e];
    const int64_t b = e / MN, mn = e % MN;
    const int m = (int)(mn / p.N), n = (int)(mn % p.N);
    const int b1 = (int)(b / p.nb2), b2 = (int)(b % p.nb2);
    T* c = (T*)p.C + b1 * p.sCb1 + b2 * p.sCb2 + (int64_t)m * p.sCm + (int64_t)n * p.sCn;
    T v = alpha * acc;
    if (beta != T(0)) v += beta * (*c);
    *c = v;
  }
}

int gemm_num_sms() {
  // thread-safe one-time query (batched solves call this from several threads)
  static const int sms = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

thread_local void* g_split_ws = nullptr;
thread_local size_t g_split_bytes = 0;

template <typename T>
void launch_simt(const std::vector<GemmProblem>& probs, cudaStream_t st) {
  const int target = 2 * gemm_num_sms();
  for (size_t s0 = 0; s0 < probs.size(); s0 += MAXG) {
    GemmGroup g;
    SplitInfo si;
    int64_t max_tiles = 0, max_yb = 0, part_used = 0, max_red = 0;
    bool any_split = false;
    for (size_t i = s0; i < probs.size() && g.count < MAXG; ++i) {
      const GemmProblem& p = probs[i];
      if (p.M <= 0 || p.N <= 0 || p.nb1 * p.nb2 <= 0) continue;
      const int64_t tiles = ceil_div(p.M, BM) * ceil_div(p.N, BN);
      const int64_t nb = (int64_t)p.nb1 * p.nb2;
      // split the reduction when the output tiles cannot fill the GPU
      int splits = 1;
      if (tiles * nb < target && p.K >= 4 * BK * 8) {
        splits = (int)std::min<int64_t>(ceil_div(target, tiles * nb), p.K / (BK * 8));
        splits = std::max(1, std::min(splits, 64));
        const int64_t need = (int64_t)splits * nb * p.M * p.N;
        if ((part_used + need) * (int64_t)sizeof(T) > (int64_t)g_split_bytes) splits = 1;
      }
      si.splits[g.count] = splits;
      si.part_off[g.count] = part_used;
      if (splits > 1) {
        part_used += (int64_t)splits * nb * p.M * p.N;
        any_split = true;
        max_red = std::max<int64_t>(max_red, nb * p.M * p.N);
      }
      g.p[g.count++] = p;
      max_tiles = std::max<int64_t>(max_tiles, tiles);
      max_yb = std::max<int64_t>(max_yb, nb * splits);
    }
    if (g.count == 0) continue;
    if (max_yb > 65535 || max_tiles > 0x7fffffff)
      throw Error(TT_ERR_UNSUPPORTED, "gemm: batch or tile count too large");
    dim3 grid((unsigned)max_tiles, (unsigned)max_yb, (unsigned)g.count);
    const int tok = prof_begin(PROF_GEMM, st);
    gemm_simt_kernel<T><<<grid, NT, 0, st>>>(g, si, (T*)g_split_ws);
    check_launch("gemm_simt_kernel");
    if (any_split) {
      const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(max_red, 256), 1024);
      splitk_reduce_kernel<T><<<dim3(blocks, g.count), 256, 0, st>>>(g, si, (const T*)g_split_ws);
      check_launch("splitk_reduce_kernel");
    }
    if (tok >= 0) {
      double fl = 0, by = 0;
      for (int i = 0; i < g.count; ++i) {
        const GemmProblem& p = g.p[i];
        const double nb = (double)p.nb1 * p.nb2;
        fl += 2.0 * p.M * p.N * p.K * nb;
        by += sizeof(T) * nb * ((double)p.M * p.K + (double)p.K * p.N + (double)p.M * p.N *
                                                                          (p.beta != 0 ? 2 : 1));
      }
      prof_end(tok, st, fl, by);
    }
  }
}

}  // namespace

void gemm_tf32(const std::vector<GemmProblem>& probs, cudaStream_t st);

void set_gemm_scratch(void* ws, size_t bytes) {
  g_split_ws = ws;
  g_split_bytes = ws ? bytes : 0;
}
void* gemm_split_ws() { return g_split_ws; }
size_t gemm_split_bytes() { return g_split_bytes; }

void gemm_fp32_simt(const std::vector<GemmProblem>& probs, cudaStream_t st) {
  if (g_dry_run) return;
  launch_simt<float>(probs, st);
}

void gemm(int mode, const std::vector<GemmProblem>& probs, cudaStream_t st) {
  if (g_dry_run) return;
  if (mode == TT_MODE_FP64) launch_simt<double>(probs, st);
  else if (mode == TT_MODE_FP32) launch_simt<float>(probs, st);
  else gemm_tf32(probs, st);
}

}  // namespace ttsg
