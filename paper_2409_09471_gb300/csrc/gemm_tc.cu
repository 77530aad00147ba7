// Tensor-core contractions for TT_MODE_TF32 and TT_MODE_BF16: the TT matvec
// core contraction (Section 2.2, matvec formula) on tcgen05 in split TF32 or
// split BF16 with FP32 accumulation.
//
// Per core k the contraction is a batch over (a, l) of GEMMs
//   G[(a,l)][(i,a')][l'] = sum_j Dp[a][(i,a')][j] * Ct[l][l'][j],
// with both operands K-major (j innermost): the working operator layout
// [a][i][a'][j] already is, and the vector core C[l][j][l'] is first copied to
// Ct[l][l'][j].  One CTA computes a 128 x 64 output tile: thread 0 issues the
// TMA loads (128-byte swizzle, 32 FP32 values of K per row) and the tcgen05.mma
// instructions (M=128, N=64, K=8 each) into a TMEM accumulator, and the four
// warps read the accumulator back with tcgen05.ld for the epilogue.  Rows and
// columns outside the tile's batch entry are computed on zero-filled or
// neighbouring data and never stored.
//
// Split TF32 (the three-product error compensation of Ootomo and Yokota,
// "Recovering single precision accuracy from Tensor Cores while surpassing the
// FP32 theoretical peak performance", 2022): after each tile lands, the CTA
// splits every FP32 value x in shared memory into hi = x with the low 13
// mantissa bits cleared (exactly a TF32 value) and lo = x - hi (exact in FP32),
// and accumulates hi*hi + lo*hi + hi*lo.  The dropped lo*lo term and the TF32
// rounding of lo are below 2^-20 relative, against 2^-11 for plain TF32: the
// matvec defines the operator of the Krylov solve, and its relative error times
// the condition number is the contraction factor of each refinement cycle.
//
// Every mbarrier wait is bounded; on expiry the CTA sets bit 2 of the error
// word, waits (bounded) for its own copies, frees its TMEM and returns.
#include "common.cuh"
#include "prof.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

namespace ttsg {

namespace {

constexpr int TM = 128, TN = 64, TK = 32;       // tile: rows, columns, K per TMA box
constexpr int TC_THREADS = 128;
constexpr long long WAIT_LIMIT = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the given phase parity; returns false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start address,
// leading byte offset 16 (unused inside one swizzle row), stride byte offset
// 1024 (8 rows of 128 bytes), descriptor version 1, layout type 2 (SW128).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor for kind::tf32: D F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)             // D format F32
         | (2u << 7)           // A format TF32
         | (2u << 10)          // B format TF32
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One core of the matvec: the operator slices (A operand) and the transposed
// vector core (B operand) as tensor maps, with the core's GEMM sizes.
struct TcCore {
  CUtensorMap mA, mB;
  int M;        // n * R1 rows of one operator slice (i, a')
  int N;        // r1
  int K;        // n
  int r0, R0;   // batch: a in [0, R0), l in [0, r0)
  float* G;     // output core
};
// All cores of one matvec in one launch: blockIdx.z selects the core,
// blockIdx.y the batch entry (a, l), blockIdx.x the output tile; entries past a
// core's own extent exit before any setup.
constexpr int TC_MAXC = 16;
struct TcBatch {
  TcCore c[TC_MAXC];
  int count;
  int* err;
};

// hi/lo split of one staged tile, elementwise (so the swizzled layout is
// kept): hi keeps sign, exponent and the 10 leading mantissa bits.
__device__ __forceinline__ void split_tf32(float* hi, float* lo, int count) {
  for (int e = threadIdx.x * 4; e < count; e += TC_THREADS * 4) {
    float4 v = *reinterpret_cast<float4*>(hi + e);
    float4 h, r;
    h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
    h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
    h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
    h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
    r.x = v.x - h.x; r.y = v.y - h.y; r.z = v.z - h.z; r.w = v.w - h.w;
    *reinterpret_cast<float4*>(hi + e) = h;
    *reinterpret_cast<float4*>(lo + e) = r;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
matvec_tc_kernel(const __grid_constant__ TcBatch b) {
  if ((int)blockIdx.z >= b.count) return;
  const TcCore& p = b.c[blockIdx.z];
  const CUtensorMap& mapA = p.mA;
  const CUtensorMap& mapB = p.mB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tiles for the 128-byte swizzle: [A hi | B hi | A lo | B lo]
  unsigned char* base =
      (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int TILE = (TM + TN) * TK;        // floats of one A+B stage (24 KB)
  float* sA = (float*)base;                    // [TM][TK] swizzled, 16 KB
  float* sB = sA + TM * TK;                    // [TN][TK] swizzled, 8 KB
  float* sAl = sA + TILE;
  float* sBl = sAl + TM * TK;
  __shared__ __align__(8) uint64_t bar_full, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;

  const int tiles_m = (p.M + TM - 1) / TM, tiles_n = (p.N + TN - 1) / TN;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  if (tn >= tiles_n || (int)blockIdx.y >= p.R0 * p.r0) return;
  const int a = blockIdx.y / p.r0, l = blockIdx.y % p.r0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    fail = 0;
    mbar_init(&bar_full, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  const int ktiles = (p.K + TK - 1) / TK;
  const int rowA = a * p.M + tm * TM;      // operator rows of slice a
  const int rowB = l * p.N + tn * TN;      // rows (l, l') of Ct
  uint32_t phase = 0;
  int stage = 0;                           // 1: copies issued, 2: MMAs issued
  for (int kt = 0; kt < ktiles; ++kt) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bar_full, TILE * 4);
      tma_load_2d(sA, &mapA, &bar_full, kt * TK, rowA);
      tma_load_2d(sB, &mapB, &bar_full, kt * TK, rowB);
    }
    stage = 1;
    const bool landed = mbar_wait(&bar_full, phase);
    if (__syncthreads_or(!landed)) break;
    split_tf32(sA, sAl, TILE);
    // generic-proxy writes of the split tiles become visible to the MMA unit
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = idesc_tf32(TM, TN);
      const uint64_t dA[2] = {smem_desc_sw128(smem_u32(sA)), smem_desc_sw128(smem_u32(sAl))};
      const uint64_t dB[2] = {smem_desc_sw128(smem_u32(sB)), smem_desc_sw128(smem_u32(sBl))};
#pragma unroll
      for (int kk = 0; kk < TK / 8; ++kk) {
        // advance 8 TF32 values (32 bytes) along K inside the swizzle row
        const uint64_t off = (uint64_t)((kk * 32) >> 4);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          // t = 0: hi*hi, 1: lo*hi, 2: hi*lo
          const uint64_t da = dA[t == 1 ? 1 : 0] + off;
          const uint64_t db = dB[t == 2 ? 1 : 0] + off;
          const uint32_t acc = (kt > 0 || kk > 0 || t > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bar_mma))
          : "memory");
    }
    stage = 2;
    // every thread waits: the next copy and split overwrite the tiles the MMAs read
    const bool done = mbar_wait(&bar_mma, phase);
    if (__syncthreads_or(!done)) break;
    stage = 0;
    phase ^= 1u;
  }
  if (stage != 0 && threadIdx.x == 0) {
    fail = 1;
    atomicOr(b.err, 4);
    // let copies or MMAs still in flight land before the CTA leaves
    mbar_wait(&bar_full, phase);
    if (stage == 2) mbar_wait(&bar_mma, phase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31.  The tile
  // goes through shared memory (the operand tiles are free now; row stride
  // TN + 1 keeps a warp's per-row writes in distinct banks) and then to the
  // output row by row, so that consecutive threads store consecutive columns.
  float* St = (float*)base;
  constexpr int LDS = TN + 1;
  static_assert(TM * LDS * 4 <= 2 * (TM + TN) * TK * 4, "staging tile exceeds the operand tiles");
  if (!fail) {
    const int row = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32"
          " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q) St[row * LDS + c0 + q] = __uint_as_float(r[q]);
    }
  }
  __syncthreads();
  if (!fail) {
    const int64_t gbase = (int64_t)(a * p.r0 + l) * p.M * p.N;
    for (int e = threadIdx.x; e < TM * TN; e += TC_THREADS) {
      const int rr = e / TN, cc = e % TN;
      const int m = tm * TM + rr, n = tn * TN + cc;
      if (m < p.M && n < p.N) p.G[gbase + (int64_t)m * p.N + n] = St[rr * LDS + cc];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
  }
}

// Instruction descriptor for kind::f16 with BF16 operands: D F32, A and B
// BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)             // D format F32
         | (1u << 7)           // A format BF16
         | (1u << 10)          // B format BF16
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Split BF16 form of the same contraction (TT_MODE_BF16): every FP32 value x is
// split into hi = bf16(x) and lo = bf16(x - hi) (round to nearest; 8 + 8
// significant bits) and the MMAs accumulate hi*hi + hi*lo + lo*hi in FP32.  The
// dropped lo*lo term and the rounding of lo are about 2^-17 relative per
// product.  A 64-wide K chunk arrives as two 32-float TMA boxes per operand
// (the tensor maps of the TF32 kernel); the split writes the bf16 tiles in the
// 128-byte-swizzled K-major layout of 16-bit operands (64 values per 128-byte
// row: element (r, k) at r * 64 + ((k / 8) ^ (r % 8)) * 8 + k % 8), and each
// MMA (kind::f16, M = 128, N = 64) takes 16 of the chunk's K values.
constexpr int BK16 = 64;
__global__ void __launch_bounds__(TC_THREADS, 1)
matvec_bf16_kernel(const __grid_constant__ TcBatch b) {
  if ((int)blockIdx.z >= b.count) return;
  const TcCore& p = b.c[blockIdx.z];
  const CUtensorMap& mapA = p.mA;
  const CUtensorMap& mapB = p.mB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // FP32 boxes [A k0 | A k0+32 | B k0 | B k0+32], then bf16 [A hi | A lo | B hi | B lo]
  float* fA = (float*)base;                          // 2 x [TM][TK]
  float* fB = fA + 2 * TM * TK;                      // 2 x [TN][TK]
  uint16_t* hA = (uint16_t*)(fB + 2 * TN * TK);      // [TM][64]
  uint16_t* lA = hA + TM * BK16;
  uint16_t* hB = lA + TM * BK16;                     // [TN][64]
  uint16_t* lB = hB + TN * BK16;
  __shared__ __align__(8) uint64_t bar_full, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;

  const int tiles_m = (p.M + TM - 1) / TM, tiles_n = (p.N + TN - 1) / TN;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  if (tn >= tiles_n || (int)blockIdx.y >= p.R0 * p.r0) return;
  const int a = blockIdx.y / p.r0, l = blockIdx.y % p.r0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    fail = 0;
    mbar_init(&bar_full, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // one operand tile: rows x 64 FP32 values (two swizzled boxes) -> bf16 hi/lo;
  // each thread converts 4 consecutive K values (one 16-byte chunk of a box)
  auto split_tile = [&](const float* f, uint16_t* hi, uint16_t* lo, int rows) {
    for (int e = threadIdx.x; e < rows * (BK16 / 4); e += TC_THREADS) {
      const int r = e >> 4, kq = e & 15;            // 16 chunks of 4 per row
      const int bx = kq >> 3, c32 = kq & 7;
      const float4 v = *reinterpret_cast<const float4*>(f + bx * rows * TK + r * TK +
                                                         ((c32 ^ (r & 7)) << 2));
      const float xs[4] = {v.x, v.y, v.z, v.w};
      uint16_t hs[4], ls[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 h = __float2bfloat16_rn(xs[q]);
        const __nv_bfloat16 lo16 = __float2bfloat16_rn(xs[q] - __bfloat162float(h));
        hs[q] = __bfloat16_as_ushort(h);
        ls[q] = __bfloat16_as_ushort(lo16);
      }
      const int k = kq * 4;
      const int o = r * BK16 + ((((k >> 3) ^ (r & 7))) << 3) + (k & 7);
      *reinterpret_cast<uint2*>(hi + o) = make_uint2(hs[0] | ((uint32_t)hs[1] << 16),
                                                     hs[2] | ((uint32_t)hs[3] << 16));
      *reinterpret_cast<uint2*>(lo + o) = make_uint2(ls[0] | ((uint32_t)ls[1] << 16),
                                                     ls[2] | ((uint32_t)ls[3] << 16));
    }
  };

  const int ktiles = (p.K + BK16 - 1) / BK16;
  const int rowA = a * p.M + tm * TM;
  const int rowB = l * p.N + tn * TN;
  uint32_t phase = 0;
  int stage = 0;
  for (int kt = 0; kt < ktiles; ++kt) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bar_full, 2 * (TM + TN) * TK * 4);
      tma_load_2d(fA, &mapA, &bar_full, kt * BK16, rowA);
      tma_load_2d(fA + TM * TK, &mapA, &bar_full, kt * BK16 + TK, rowA);
      tma_load_2d(fB, &mapB, &bar_full, kt * BK16, rowB);
      tma_load_2d(fB + TN * TK, &mapB, &bar_full, kt * BK16 + TK, rowB);
    }
    stage = 1;
    const bool landed = mbar_wait(&bar_full, phase);
    if (__syncthreads_or(!landed)) break;
    split_tile(fA, hA, lA, TM);
    split_tile(fB, hB, lB, TN);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = idesc_bf16(TM, TN);
      const uint64_t dA[2] = {smem_desc_sw128(smem_u32(hA)), smem_desc_sw128(smem_u32(lA))};
      const uint64_t dB[2] = {smem_desc_sw128(smem_u32(hB)), smem_desc_sw128(smem_u32(lB))};
#pragma unroll
      for (int kk = 0; kk < BK16 / 16; ++kk) {
        // advance 16 BF16 values (32 bytes) along K inside the swizzle row
        const uint64_t off = (uint64_t)((kk * 32) >> 4);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          // t = 0: hi*hi, 1: lo*hi, 2: hi*lo
          const uint64_t da = dA[t == 1 ? 1 : 0] + off;
          const uint64_t db = dB[t == 2 ? 1 : 0] + off;
          const uint32_t acc = (kt > 0 || kk > 0 || t > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bar_mma))
          : "memory");
    }
    stage = 2;
    const bool done = mbar_wait(&bar_mma, phase);
    if (__syncthreads_or(!done)) break;
    stage = 0;
    phase ^= 1u;
  }
  if (stage != 0 && threadIdx.x == 0) {
    fail = 1;
    atomicOr(b.err, 4);
    mbar_wait(&bar_full, phase);
    if (stage == 2) mbar_wait(&bar_mma, phase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  float* St = (float*)base;
  constexpr int LDS = TN + 1;
  static_assert(TM * LDS * 4 <= 2 * (TM + TN) * TK * 4, "staging tile exceeds the FP32 boxes");
  if (!fail) {
    const int row = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32"
          " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q) St[row * LDS + c0 + q] = __uint_as_float(r[q]);
    }
  }
  __syncthreads();
  if (!fail) {
    const int64_t gbase = (int64_t)(a * p.r0 + l) * p.M * p.N;
    for (int e = threadIdx.x; e < TM * TN; e += TC_THREADS) {
      const int rr = e / TN, cc = e % TN;
      const int m = tm * TM + rr, n = tn * TN + cc;
      if (m < p.M && n < p.N) p.G[gbase + (int64_t)m * p.N + n] = St[rr * LDS + cc];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    TT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p)
      throw Error(TT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D FP32 tensor map: inner dimension K (contiguous), outer `rows` with row
// stride `ld` floats; box TK x box_rows, 128-byte swizzle, zero fill outside.
CUtensorMap make_map(const float* ptr, int64_t K, int64_t rows, int64_t ld, int box_rows) {
  if (((uintptr_t)ptr & 15) || ((ld * 4) & 15))
    throw Error(TT_ERR_UNSUPPORTED, "tensor map: base or row stride not 16-byte aligned");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(TT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

bool matvec_tc_supported(int64_t n, int64_t r1) {
  // K-major rows must be 16-byte multiples (n % 4 == 0) for the tensor maps
  return (n % 4) == 0 && n >= 8 && r1 >= 1;
}

// All tensor-core cores of one matvec: core k gives G_k (R0 r0 x n x R1 r1)
// from Dp_k ([R0][n R1][n]) and Ct_k ([r0][r1][n]); up to TC_MAXC cores per
// launch.
void matvec_tc_cores(const std::vector<TcCoreArgs>& cores, int* err, cudaStream_t st, bool bf16) {
  if (g_dry_run || cores.empty()) return;
  const size_t smem = (size_t)2 * (TM + TN) * TK * 4 + 1024;
  // split BF16: the FP32 boxes of a 64-wide chunk plus the bf16 hi/lo tiles
  const size_t smem16 = (size_t)2 * (TM + TN) * TK * 4 + (size_t)2 * (TM + TN) * BK16 * 2 + 1024;
  static const bool attr = [smem, smem16] {
    TT_CUDA(cudaFuncSetAttribute(matvec_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    TT_CUDA(cudaFuncSetAttribute(matvec_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem16));
    return true;
  }();
  (void)attr;
  for (size_t c0 = 0; c0 < cores.size(); c0 += TC_MAXC) {
    TcBatch bt;
    bt.count = 0;
    bt.err = err;
    int64_t max_tiles = 1, max_batch = 1;
    double flops = 0.0, bytes = 0.0;
    for (size_t i = c0; i < cores.size() && bt.count < TC_MAXC; ++i) {
      const TcCoreArgs& q = cores[i];
      const int64_t M = q.n * q.R1;
      TcCore& cc = bt.c[bt.count++];
      cc.mA = make_map(q.Dp, q.n, q.R0 * M, q.n, TM);
      cc.mB = make_map(q.Ct, q.n, q.r0 * q.r1, q.n, TN);
      cc.M = (int)M; cc.N = (int)q.r1; cc.K = (int)q.n; cc.r0 = (int)q.r0; cc.R0 = (int)q.R0;
      cc.G = q.G;
      max_tiles = std::max(max_tiles, ceil_div(M, (int64_t)TM) * ceil_div(q.r1, (int64_t)TN));
      max_batch = std::max(max_batch, q.R0 * q.r0);
      flops += 2.0 * M * q.r1 * q.n * q.R0 * q.r0;
      bytes += 4.0 * (q.R0 * M * q.n + q.r0 * q.r1 * q.n + q.R0 * q.r0 * M * q.r1);
    }
    if (max_batch > 65535) throw Error(TT_ERR_UNSUPPORTED, "matvec_tc: batch too large");
    const int tok = prof_begin(PROF_TC, st);
    if (bf16) {
      matvec_bf16_kernel<<<dim3((unsigned)max_tiles, (unsigned)max_batch, (unsigned)bt.count),
                           TC_THREADS, smem16, st>>>(bt);
      check_launch("matvec_bf16_kernel");
    } else {
      matvec_tc_kernel<<<dim3((unsigned)max_tiles, (unsigned)max_batch, (unsigned)bt.count),
                         TC_THREADS, smem, st>>>(bt);
      check_launch("matvec_tc_kernel");
    }
    // algorithmic flops and bytes (one product; the split adds two more on
    // the tensor pipe)
    prof_end(tok, st, flops, bytes);
  }
}

// Grouped GEMMs other than the matvec run on the FP32 CUDA-core kernel in
// TF32 mode (their operands are strided views the tensor maps do not cover).
void gemm_fp32_simt(const std::vector<GemmProblem>& probs, cudaStream_t st);
void gemm_tf32(const std::vector<GemmProblem>& probs, cudaStream_t st) {
  gemm_fp32_simt(probs, st);
}

}  // namespace ttsg
