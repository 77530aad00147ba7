// Shared definitions of the CUDA library: error handling, TT views, the
// grouped strided GEMM descriptor and the workspace bump allocator.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <stdexcept>
#include <cstdio>
#include "../../include/ttsg.h"

namespace ttsg {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
void set_last_error(const std::string& m);

#define TT_CHECK_ARG(cond, msg)                                   \
  do {                                                            \
    if (!(cond)) throw ::ttsg::Error(TT_ERR_ARG, (msg));          \
  } while (0)

#define TT_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t _e = (call);                                                       \
    if (_e != cudaSuccess)                                                         \
      throw ::ttsg::Error(TT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// When set, launch wrappers return without enqueuing work and host reads of
// device values return placeholders; used to measure workspace needs.
extern thread_local bool g_dry_run;

void count_launch();
inline void check_launch(const char* what) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(TT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- TT views
constexpr int MAXD = TT_MAX_D;

// Host-side view of a TT vector whose cores live on the device (compact
// [r_{k-1}][n_k][r_k] layout).
template <typename T>
struct TTv {
  int d = 0;
  int64_t n[MAXD] = {};
  int64_t r[MAXD + 1] = {};
  T* core[MAXD] = {};
  int64_t core_elems(int k) const { return r[k] * n[k] * r[k + 1]; }
  int64_t max_rank() const {
    int64_t m = 0;
    for (int k = 0; k <= d; ++k) m = r[k] > m ? r[k] : m;
    return m;
  }
};

// Host-side view of a TT operator in the permuted working layout
// [a][i][a'][j] (input column index j innermost, K-contiguous for the matvec).
template <typename T>
struct TTop {
  int d = 0;
  int64_t n[MAXD] = {};
  int64_t R[MAXD + 1] = {};
  T* core[MAXD] = {};
};

// ---------------------------------------------------------------- workspace
// Bump allocator over a caller-provided device buffer (256-byte aligned
// slices).  ``dry`` mode only counts bytes (used by the *_workspace queries).
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0, peak = 0;
  bool dry = false;
  Arena() = default;
  Arena(void* p, size_t n, bool dry_ = false) : base((char*)p), cap(n), dry(dry_) {}
  template <typename T>
  T* take(int64_t count) {
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    size_t start = (off + 255) & ~size_t(255);
    size_t end = start + bytes;
    if (!dry && end > cap)
      throw Error(TT_ERR_WORKSPACE, "workspace too small: need more than " + std::to_string(end) +
                                        " bytes, have " + std::to_string(cap));
    off = end;
    if (off > peak) peak = off;
    return dry ? nullptr : (T*)(base + start);
  }
  size_t mark() const { return off; }
  void release(size_t m) { off = m; }
};

// ---------------------------------------------------------------- GEMM
// One problem of a grouped strided batched GEMM:
//   C[b1,b2][m,n] = alpha * sum_k A[b1,b2][m,k] B[b1,b2][k,n] + beta * C[b1,b2][m,n]
// Element (m,k) of A is at A + b1*sAb1 + b2*sAb2 + m*sAm + k*sAk (same for B, C).
// alpha is multiplied by *alpha_dev when alpha_dev != nullptr.
// a_mode == 1 (Khatri-Rao operand): A[m,k] = Z[m, k / kr_n] * S[m, k % kr_n],
//   with Z = A (strides sAm, sAk) or Z == 1 when A == nullptr, and
//   S[m,i] at kr_S + m*kr_sS + i.
struct GemmProblem {
  int M = 0, N = 0, K = 0;
  int nb1 = 1, nb2 = 1;
  const void* A = nullptr;
  int64_t sAm = 0, sAk = 0, sAb1 = 0, sAb2 = 0;
  const void* B = nullptr;
  int64_t sBk = 0, sBn = 0, sBb1 = 0, sBb2 = 0;
  void* C = nullptr;
  int64_t sCm = 0, sCn = 0, sCb1 = 0, sCb2 = 0;
  double alpha = 1.0, beta = 0.0;
  const double* alpha_dev = nullptr;
  int a_mode = 0;
  const void* kr_S = nullptr;
  int kr_n = 1;
  int64_t kr_sS = 0;
};

constexpr int MAXG = 16;
struct GemmGroup {
  int count = 0;
  GemmProblem p[MAXG];
};

// Enqueue a grouped GEMM (any number of problems; split into launches of at
// most MAXG).  ``mode`` selects FP64 / FP32 SIMT or the TF32 tensor-core path.
void gemm(int mode, const std::vector<GemmProblem>& probs, cudaStream_t st);
// tcgen05 (TF32) contraction of one matvec core: G from the working-layout
// operator core Dp ([R0][n R1][n]) and the transposed vector core Ct
// ([r0][r1][n]); float data, n a multiple of 4 (tensor-map row alignment).
bool matvec_tc_supported(int64_t n, int64_t r1);
struct TcCoreArgs {
  const float* Dp;  // working-layout operator core [R0][n R1][n]
  const float* Ct;  // transposed vector core [r0][r1][n]
  float* G;         // output core
  int64_t n, R0, R1, r0, r1;
};
// bf16: the split-BF16 kernel (TT_MODE_BF16) instead of split TF32.
void matvec_tc_cores(const std::vector<TcCoreArgs>& cores, int* err, cudaStream_t st,
                     bool bf16 = false);
// Device scratch for split-K partial sums (set per API call; null disables split-K).
// GEMMs enqueued on another stream of the same call switch to a scratch of
// their own around their launches (the pointer is read at launch time).
void set_gemm_scratch(void* ws, size_t bytes);
void* gemm_split_ws();
size_t gemm_split_bytes();
constexpr size_t GEMM_SCRATCH_BYTES = size_t(48) << 20;

// Row-major plain helper: C (MxN, ldc) = alpha * A (MxK, lda) * B (KxN, ldb) + beta*C
inline GemmProblem gemm_rm(int M, int N, int K, const void* A, int64_t lda, const void* B,
                           int64_t ldb, void* C, int64_t ldc, double alpha = 1.0,
                           double beta = 0.0) {
  GemmProblem g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.sAm = lda; g.sAk = 1;
  g.B = B; g.sBk = ldb; g.sBn = 1;
  g.C = C; g.sCm = ldc; g.sCn = 1;
  g.alpha = alpha; g.beta = beta;
  return g;
}

template <typename T> struct ModeType;
inline int elem_size(int mode) { return mode == TT_MODE_FP64 ? 8 : 4; }

}  // namespace ttsg
