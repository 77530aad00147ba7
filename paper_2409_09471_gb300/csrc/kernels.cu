// Data movement and element-wise kernels: batched strided 3-D copies with type
// conversion (operator permutation, DRM sub-blocks, core stacking), the
// Philox4x32-10 Gaussian generator, and FP64 sum-of-squares reductions.
#include "kernels.cuh"

namespace ttsg {

namespace {

constexpr int MAXSEG = 64;
struct CopyBatch {
  int count;
  CopySeg s[MAXSEG];
};

__global__ void copy3d_kernel(const __grid_constant__ CopyBatch b) {
  const CopySeg& s = b.s[blockIdx.y];
  const int64_t total = s.A * s.B * s.C;
  double scale = s.scale;
  if (s.scale_dev) scale *= s.scale_dev_inv ? 1.0 / (*s.scale_dev) : (*s.scale_dev);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % s.C;
    const int64_t ab = e / s.C;
    const int64_t bb = ab % s.B, a = ab / s.B;
    const int64_t src = a * s.sa + bb * s.sb + c * s.sc;
    const int64_t dst = (s.da | s.db | s.dc) ? a * s.da + bb * s.db + c * s.dc : e;
    if (!s.src_f64 && !s.dst_f64) {
      // float to float in float arithmetic (FP64 throughput is low on this part)
      ((float*)s.dst)[dst] = ((const float*)s.src)[src] * (float)scale;
      continue;
    }
    double v = s.src_f64 ? ((const double*)s.src)[src] : (double)((const float*)s.src)[src];
    v *= scale;
    if (s.dst_f64) ((double*)s.dst)[dst] = v;
    else ((float*)s.dst)[dst] = (float)v;
  }
}

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11) and the Gaussian stream: element e uses
// counter (lo(e/2), hi(e/2), lo(stream), hi(stream)), key (lo(seed), hi(seed));
// two 53-bit uniforms from the output words, Box-Muller cos (even e) / sin (odd).
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
}

__device__ __forceinline__ double gauss_elem(uint64_t e, uint64_t seed, uint64_t stream) {
  const uint64_t c = e >> 1;
  uint32_t w0 = (uint32_t)c, w1 = (uint32_t)(c >> 32), w2 = (uint32_t)stream,
           w3 = (uint32_t)(stream >> 32);
  philox4x32_10(w0, w1, w2, w3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t a = ((((uint64_t)w0) << 32) | w1) >> 11;
  const uint64_t b = ((((uint64_t)w2) << 32) | w3) >> 11;
  const double u1 = ((double)a + 0.5) * 0x1p-53;
  const double u2 = ((double)b + 0.5) * 0x1p-53;
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586 * u2;
  return (e & 1) ? rad * sin(ang) : rad * cos(ang);
}

__global__ void gauss_kernel(void* out, int f64, int64_t rows, int64_t n, int64_t cols,
                             int64_t ldc, uint64_t seed, uint64_t stream, double std_) {
  const int64_t total = rows * n * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % cols, qi = e / cols;
    const int64_t src = qi * ldc + c;  // (q*n + i)*ldc + c
    const double g = gauss_elem((uint64_t)src, seed, stream) * std_;
    if (f64) ((double*)out)[e] = g;
    else ((float*)out)[e] = (float)g;
  }
}

// --------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void sumsq_partial(const void* x, int f64, int64_t count, double* part) {
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = f64 ? ((const double*)x)[e] : (double)((const float*)x)[e];
    acc += v * v;
  }
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void dot_partial(const void* a, const void* b, int f64, int64_t count, double* part) {
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double u = f64 ? ((const double*)a)[e] : (double)((const float*)a)[e];
    const double v = f64 ? ((const double*)b)[e] : (double)((const float*)b)[e];
    acc = fma(u, v, acc);
  }
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void sum_final(const double* part, int np, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}

__global__ void sqrt_kernel(const double* x, double* y) { *y = sqrt(fmax(*x, 0.0)); }

// x *= 2^-e with e the binary exponent of sqrt(sum of the np partial sums of
// squares): every CTA reduces the partials itself, then scales its share.  A
// power of two changes no significand bit, so the scaling itself is exact.
template <typename T>
__global__ void pow2_scale_kernel(T* x, int64_t count, const double* part, int np) {
  __shared__ double fac;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += 32) v += part[i];
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      const double s = sqrt(v);
      // the factor itself must be finite in T
      const int lim = sizeof(T) == 4 ? 120 : 1000;
      const int e = (s > 0.0 && isfinite(s)) ? max(-lim, min(lim, ilogb(s))) : 0;
      fac = ldexp(1.0, -e);
    }
  }
  __syncthreads();
  const T f = (T)fac;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] *= f;
}

}  // namespace

void copy3d(const std::vector<CopySeg>& segs, cudaStream_t st) {
  if (g_dry_run) return;
  for (size_t s0 = 0; s0 < segs.size(); s0 += MAXSEG) {
    CopyBatch b;
    b.count = 0;
    int64_t maxe = 0;
    for (size_t i = s0; i < segs.size() && b.count < MAXSEG; ++i) {
      b.s[b.count++] = segs[i];
      maxe = std::max<int64_t>(maxe, segs[i].A * segs[i].B * segs[i].C);
    }
    if (maxe == 0) continue;
    const int64_t blocks = std::min<int64_t>(ceil_div(maxe, 256), 4096);
    copy3d_kernel<<<dim3((unsigned)blocks, (unsigned)b.count), 256, 0, st>>>(b);
    check_launch("copy3d_kernel");
  }
}

void gaussian_fill(void* out, int out_f64, int64_t count, uint64_t seed, uint64_t stream,
                   double std_, cudaStream_t st) {
  gaussian_subblock(out, out_f64, 1, 1, count, count, seed, stream, std_, st);
}

void gaussian_subblock(void* out, int out_f64, int64_t rows, int64_t n, int64_t cols,
                       int64_t ldc, uint64_t seed, uint64_t stream, double std_, cudaStream_t st) {
  if (g_dry_run) return;
  const int64_t total = rows * n * cols;
  if (total <= 0) return;
  const int64_t blocks = std::min<int64_t>(ceil_div(total, 256), 8192);
  gauss_kernel<<<(unsigned)blocks, 256, 0, st>>>(out, out_f64, rows, n, cols, ldc, seed, stream,
                                                 std_);
  check_launch("gauss_kernel");
}

void sumsq(const void* x, int x_f64, int64_t count, double* out, double* scratch,
           cudaStream_t st) {
  if (g_dry_run) return;
  const int np = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(count, 1024), 1), 256);
  sumsq_partial<<<np, 256, 0, st>>>(x, x_f64, count, scratch);
  check_launch("sumsq_partial");
  sum_final<<<1, 256, 0, st>>>(scratch, np, out);
  check_launch("sum_final");
}

void dot_acc(const void* a, const void* b, int f64, int64_t count, double* out, double* scratch,
             cudaStream_t st) {
  if (g_dry_run) return;
  const int np = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(count, 1024), 1), 256);
  dot_partial<<<np, 256, 0, st>>>(a, b, f64, count, scratch);
  check_launch("dot_partial");
  sum_final<<<1, 256, 0, st>>>(scratch, np, out);
  check_launch("sum_final");
}

void pow2_normalize(void* x, int x_f64, int64_t count, double* scratch, cudaStream_t st) {
  if (g_dry_run || count <= 0) return;
  const int np = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(count, 1024), 1), 256);
  sumsq_partial<<<np, 256, 0, st>>>(x, x_f64, count, scratch);
  check_launch("sumsq_partial");
  if (x_f64) pow2_scale_kernel<double><<<np, 256, 0, st>>>((double*)x, count, scratch, np);
  else pow2_scale_kernel<float><<<np, 256, 0, st>>>((float*)x, count, scratch, np);
  check_launch("pow2_scale_kernel");
}

void sqrt_scalar(const double* x, double* y, cudaStream_t st) {
  if (g_dry_run) return;
  sqrt_kernel<<<1, 1, 0, st>>>(x, y);
  check_launch("sqrt_kernel");
}

}  // namespace ttsg
