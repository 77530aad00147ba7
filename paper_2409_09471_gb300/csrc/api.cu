// extern "C" entry points declared in include/ttsg.h: argument validation,
// conversion of the plain C descriptors into device views, workspace carving,
// and translation of exceptions into status codes.
#include "solver.cuh"
#include <chrono>
#include <mutex>
#include <thread>
#include <cmath>

namespace ttsg {

thread_local bool g_dry_run = false;

namespace {
thread_local std::string g_last_error;

struct DryGuard {
  bool old;
  DryGuard() : old(g_dry_run) { g_dry_run = true; }
  ~DryGuard() { g_dry_run = old; }
};

template <typename F>
int guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return TT_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return TT_ERR_CUDA;
  }
}

int check_mode(int mode) {
  if (mode != TT_MODE_FP64 && mode != TT_MODE_FP32 && mode != TT_MODE_TF32 &&
      mode != TT_MODE_BF16)
    throw Error(TT_ERR_ARG, "unknown mode " + std::to_string(mode));
  return mode;
}

template <typename T>
TTv<T> view(const tt_vec* v, const char* what) {
  if (!v) throw Error(TT_ERR_ARG, std::string(what) + ": null descriptor");
  if (v->d < 1 || v->d > MAXD) throw Error(TT_ERR_ARG, std::string(what) + ": d out of range");
  if (!v->n || !v->rank || !v->core) throw Error(TT_ERR_ARG, std::string(what) + ": null array");
  TTv<T> t;
  t.d = v->d;
  for (int k = 0; k <= v->d; ++k) t.r[k] = v->rank[k];
  if (t.r[0] != 1 || t.r[v->d] != 1)
    throw Error(TT_ERR_ARG, std::string(what) + ": boundary ranks must be 1");
  for (int k = 0; k < v->d; ++k) {
    t.n[k] = v->n[k];
    if (t.n[k] < 1 || t.r[k + 1] < 1) throw Error(TT_ERR_ARG, std::string(what) + ": n, rank >= 1");
    if (!v->core[k]) throw Error(TT_ERR_ARG, std::string(what) + ": null core pointer");
    t.core[k] = (T*)v->core[k];
  }
  return t;
}

template <typename T>
TTv<T> view_out(const tt_vec_out* v, const char* what, int64_t* cap) {
  if (!v || !v->n || !v->cap || !v->rank || !v->core)
    throw Error(TT_ERR_ARG, std::string(what) + ": null descriptor or array");
  if (v->d < 1 || v->d > MAXD) throw Error(TT_ERR_ARG, std::string(what) + ": d out of range");
  TTv<T> t;
  t.d = v->d;
  for (int k = 0; k <= v->d; ++k) cap[k] = v->cap[k];
  for (int k = 0; k < v->d; ++k) {
    t.n[k] = v->n[k];
    t.core[k] = (T*)v->core[k];
    if (!t.core[k]) throw Error(TT_ERR_ARG, std::string(what) + ": null core pointer");
  }
  return t;
}

template <typename T>
TTop<T> view_op(const tt_op* A, int permute_expected) {
  (void)permute_expected;
  if (!A || !A->n || !A->rank || !A->core) throw Error(TT_ERR_ARG, "operator: null descriptor");
  if (A->d < 1 || A->d > MAXD) throw Error(TT_ERR_ARG, "operator: d out of range");
  TTop<T> o;
  o.d = A->d;
  for (int k = 0; k <= A->d; ++k) o.R[k] = A->rank[k];
  if (o.R[0] != 1 || o.R[A->d] != 1) throw Error(TT_ERR_ARG, "operator: boundary ranks must be 1");
  for (int k = 0; k < A->d; ++k) {
    o.n[k] = A->n[k];
    o.core[k] = (T*)A->core[k];
    if (!o.core[k]) throw Error(TT_ERR_ARG, "operator: null core pointer");
  }
  return o;
}

void same_modes(const int64_t* a, const int64_t* b, int d, const char* what) {
  for (int k = 0; k < d; ++k)
    if (a[k] != b[k]) throw Error(TT_ERR_ARG, std::string(what) + ": mode sizes differ");
}

// Workspace carving: a small header (error flag + reduction scratch) first.
struct Carved {
  Arena ar;
  Ctx ctx;
};
Carved carve(int mode, void* ws, size_t bytes, void* stream, bool dry, bool with_gemm = true) {
  Carved c;
  c.ar = Arena(ws, bytes, dry);
  if (!dry && !ws) throw Error(TT_ERR_WORKSPACE, "null workspace");
  c.ctx.mode = mode;
  c.ctx.st = (cudaStream_t)stream;
  c.ctx.err = c.ar.take<int>(64);
  c.ctx.scratch = c.ar.take<double>(512);
  if (with_gemm) set_gemm_scratch(c.ar.take<char>((int64_t)GEMM_SCRATCH_BYTES), GEMM_SCRATCH_BYTES);
  else set_gemm_scratch(nullptr, 0);
  return c;
}
void reset_flags(Carved& c) {
  if (!g_dry_run) TT_CUDA(cudaMemsetAsync(c.ctx.err, 0, 64 * sizeof(int), c.ctx.st));
}
void fix_ctx(Carved& c) { c.ctx.ar = &c.ar; }

template <typename T>
void permute_op(Carved& cv, const TTop<T>& in, TTop<T>& out) {
  out.d = in.d;
  std::vector<CopySeg> segs;
  for (int k = 0; k < in.d; ++k) {
    const int64_t R0 = in.R[k], R1 = in.R[k + 1], n = in.n[k];
    out.n[k] = n;
    out.R[k] = R0;
    out.core[k] = cv.ar.take<T>(R0 * n * n * R1);
    CopySeg s;
    s.src = in.core[k]; s.dst = out.core[k];
    s.A = R0 * n; s.B = R1; s.C = n; s.sa = n * R1; s.sb = 1; s.sc = R1;
    s.src_f64 = s.dst_f64 = sizeof(T) == 8;
    segs.push_back(s);
  }
  out.R[in.d] = 1;
  copy3d(segs, cv.ctx.st);
}

template <typename T>
void do_matvec(int mode, const tt_op* A, const tt_vec* x, const tt_vec* y, void* ws, size_t bytes,
               void* stream, bool dry) {
  TTop<T> a = view_op<T>(A, 0);
  TTv<T> xv = view<T>(x, "x");
  TTv<T> yv = view<T>(y, "y");
  if (a.d != xv.d || yv.d != xv.d) throw Error(TT_ERR_ARG, "matvec: d mismatch");
  same_modes(a.n, xv.n, xv.d, "matvec");
  same_modes(yv.n, xv.n, xv.d, "matvec");
  for (int k = 0; k <= xv.d; ++k)
    if (yv.r[k] != a.R[k] * xv.r[k]) throw Error(TT_ERR_ARG, "matvec: y ranks must be R_k r_k");
  Carved cv = carve(mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  TTop<T> ap;
  permute_op<T>(cv, a, ap);
  tt_matvec_dev<T>(cv.ctx, ap, xv, yv);
  if (dry) throw (size_t)cv.ar.peak;
}

// status of the last workspace query that failed (0 queries return 0 bytes)
thread_local int g_measure_code = TT_OK;

template <typename F>
size_t measure(F&& f, bool margin = true) {
  DryGuard g;
  try {
    f();
  } catch (size_t peak) {
    // margin for allocations whose size the dry run bounds from below
    g_measure_code = TT_OK;
    return margin ? peak + peak / 32 + (16u << 20) : peak;
  } catch (const Error& e) {
    g_last_error = e.what();
    g_measure_code = e.code;
    return 0;
  }
  g_measure_code = TT_ERR_ARG;
  return 0;
}

}  // namespace
}  // namespace ttsg

using namespace ttsg;

// The definitions below keep the C linkage of their declarations in ttsg.h.

const char* tt_version(void) { return "ttsg 0.1 (sm_103a)"; }
const char* tt_last_error(void) { return g_last_error.c_str(); }

size_t tt_matvec_workspace(int mode, const tt_op* A, const tt_vec* x) {
  return measure([&] {
    check_mode(mode);
    // y descriptor with the product ranks
    std::vector<int64_t> yr(x->d + 1);
    for (int k = 0; k <= x->d; ++k) yr[k] = A->rank[k] * x->rank[k];
    std::vector<void*> cores(x->d, (void*)1);
    tt_vec y{x->d, x->n, yr.data(), cores.data()};
    if (mode == TT_MODE_FP64) do_matvec<double>(mode, A, x, &y, nullptr, 0, nullptr, true);
    else do_matvec<float>(mode, A, x, &y, nullptr, 0, nullptr, true);
  });
}

int tt_matvec(int mode, const tt_op* A, const tt_vec* x, const tt_vec* y, void* ws,
              size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64) do_matvec<double>(mode, A, x, y, ws, ws_bytes, stream, false);
    else do_matvec<float>(mode, A, x, y, ws, ws_bytes, stream, false);
  });
}

namespace {
template <typename T>
void do_sketch(int mode, const tt_vec* x, int64_t s, void* const* S, double* out, void* ws,
               size_t bytes, void* stream, bool dry) {
  TTv<T> xv = view<T>(x, "x");
  if (s < 1) throw Error(TT_ERR_ARG, "sketch: s >= 1");
  if (!dry && (!S || !out)) throw Error(TT_ERR_ARG, "sketch: null S or out");
  Carved cv = carve(mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  std::vector<const T*> Sv(xv.d);
  for (int k = 0; k < xv.d; ++k) {
    Sv[k] = dry ? nullptr : (const T*)S[k];
    if (!dry && !Sv[k]) throw Error(TT_ERR_ARG, "sketch: null factor");
  }
  tt_sketch_dev<T>(cv.ctx, xv, s, Sv.data(), out);
  if (dry) throw (size_t)cv.ar.peak;
}

template <typename T>
void do_dot(int mode, const tt_vec* x, const tt_vec* y, double* out, void* ws, size_t bytes,
            void* stream, bool dry, bool with_gemm = true) {
  TTv<T> xv = view<T>(x, "x");
  TTv<T> yv = view<T>(y, "y");
  if (xv.d != yv.d) throw Error(TT_ERR_ARG, "dot: d mismatch");
  same_modes(xv.n, yv.n, xv.d, "dot");
  if (!dry && !out) throw Error(TT_ERR_ARG, "dot: null out");
  Carved cv = carve(mode, ws, bytes, stream, dry, with_gemm);
  fix_ctx(cv);
  tt_dot_dev<T>(cv.ctx, xv, yv, out);
  if (dry) throw (size_t)cv.ar.peak;
}

template <typename T>
void do_round(int mode, int nterms, const tt_vec* terms, const double* coef, double eps,
              int64_t rmax, int64_t p, uint64_t seed, void* const* drm, const int64_t* drm_rank,
              const tt_vec_out* y, void* ws, size_t bytes, void* stream, bool dry) {
  if (nterms < 1 || !terms) throw Error(TT_ERR_ARG, "round: nterms >= 1");
  if (!(eps >= 0.0) || rmax < 1 || p < 0) throw Error(TT_ERR_ARG, "round: eps >= 0, rmax >= 1, p >= 0");
  std::vector<Term<T>> tv(nterms);
  for (int b = 0; b < nterms; ++b) {
    tv[b].X = view<T>(&terms[b], "term");
    tv[b].coef = coef ? coef[b] : 1.0;
    if (tv[b].X.d != tv[0].X.d) throw Error(TT_ERR_ARG, "round: d mismatch");
    same_modes(tv[b].X.n, tv[0].X.n, tv[0].X.d, "round");
  }
  const int d = tv[0].X.d;
  if (d < 2) throw Error(TT_ERR_ARG, "round: d >= 2");
  int64_t ell[MAXD + 1];
  std::vector<const int64_t*> tr;
  for (auto& t : tv) tr.push_back(t.X.r);
  rto_ranks(tr, tv[0].X.n, d, rmax, p, ell);
  DRMSource<T> ds;
  ds.seed = seed;
  std::vector<const T*> dc(d);
  if (drm) {
    if (!drm_rank) throw Error(TT_ERR_ARG, "round: drm_rank required with drm");
    for (int k = 0; k < d; ++k) dc[k] = (const T*)drm[k];
    for (int k = 0; k <= d; ++k) ds.L[k] = drm_rank[k];
    ds.core = dc.data();
  } else {
    for (int k = 0; k <= d; ++k) ds.L[k] = (k == 0 || k == d) ? 1 : rmax + p;
  }
  TTv<T> yv;
  int64_t cap[MAXD + 1];
  if (dry) {
    yv.d = d;
    for (int k = 0; k < d; ++k) yv.n[k] = tv[0].X.n[k];
  } else {
    yv = view_out<T>(y, "y", cap);
    if (yv.d != d) throw Error(TT_ERR_ARG, "round: output d mismatch");
    // output ranks are at most min(rmax, l_mu); capacities must cover that
    for (int k = 1; k < d; ++k)
      if (cap[k] < std::min<int64_t>(rmax, ell[k]))
        throw Error(TT_ERR_ARG, "round: output capacity below min(rmax, sketch rank)");
  }
  Carved cv = carve(mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  reset_flags(cv);
  tt_round_rand_dev<T>(cv.ctx, tv, eps, rmax, p, ds, yv);
  if (dry) throw (size_t)cv.ar.peak;
  for (int k = 0; k <= d; ++k) y->rank[k] = yv.r[k];
}
}  // namespace

size_t tt_sketch_workspace(int mode, const tt_vec* x, int64_t s) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64) do_sketch<double>(mode, x, s, nullptr, nullptr, nullptr, 0, nullptr, true);
    else do_sketch<float>(mode, x, s, nullptr, nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_sketch(int mode, const tt_vec* x, int64_t s, void* const* S, double* out, void* ws,
              size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64) do_sketch<double>(mode, x, s, S, out, ws, ws_bytes, stream, false);
    else do_sketch<float>(mode, x, s, S, out, ws, ws_bytes, stream, false);
  });
}

size_t tt_dot_workspace(int mode, const tt_vec* x, const tt_vec* y) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64) do_dot<double>(mode, x, y, nullptr, nullptr, 0, nullptr, true);
    else do_dot<float>(mode, x, y, nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_dot(int mode, const tt_vec* x, const tt_vec* y, double* out, void* ws, size_t ws_bytes,
           void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64) do_dot<double>(mode, x, y, out, ws, ws_bytes, stream, false);
    else do_dot<float>(mode, x, y, out, ws, ws_bytes, stream, false);
  });
}

namespace ttsg {
// Inner product without split-K scratch, on a caller-chosen workspace; used by
// the allocation-free entry point (noalloc.cu).
size_t dot_bytes_without_splitk(int mode, const tt_vec* x, const tt_vec* y, int* code) {
  const size_t need = measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_dot<double>(mode, x, y, nullptr, nullptr, 0, nullptr, true, false);
    else
      do_dot<float>(mode, x, y, nullptr, nullptr, 0, nullptr, true, false);
  }, false);
  if (code) *code = need ? TT_OK : g_measure_code;
  return need;
}
int dot_on_workspace_without_splitk(int mode, const tt_vec* x, const tt_vec* y, double* out,
                                    void* ws, size_t bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64) do_dot<double>(mode, x, y, out, ws, bytes, stream, false, false);
    else do_dot<float>(mode, x, y, out, ws, bytes, stream, false, false);
  });
}
void set_last_error(const std::string& m) { g_last_error = m; }
}  // namespace ttsg

size_t tt_round_rand_workspace(int mode, int nterms, const tt_vec* terms, int64_t rmax,
                               int64_t oversample) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_round<double>(mode, nterms, terms, nullptr, 0.1, rmax, oversample, 0, nullptr, nullptr,
                       nullptr, nullptr, 0, nullptr, true);
    else
      do_round<float>(mode, nterms, terms, nullptr, 0.1, rmax, oversample, 0, nullptr, nullptr,
                      nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_round_rand(int mode, int nterms, const tt_vec* terms, const double* coef, double eps,
                  int64_t rmax, int64_t oversample, uint64_t seed, void* const* drm,
                  const int64_t* drm_rank, const tt_vec_out* y, void* ws, size_t ws_bytes,
                  void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_round<double>(mode, nterms, terms, coef, eps, rmax, oversample, seed, drm, drm_rank, y,
                       ws, ws_bytes, stream, false);
    else
      do_round<float>(mode, nterms, terms, coef, eps, rmax, oversample, seed, drm, drm_rank, y, ws,
                      ws_bytes, stream, false);
  });
}

namespace ttsg {
namespace {
template <typename T>
void do_stta_sketch(int mode, const tt_vec* x, double coef, int accumulate, const tt_vec* X,
                    const tt_vec* Y, double* const* psi, double* const* omega, void* ws,
                    size_t bytes, void* stream, bool dry) {
  TTv<T> xv = view<T>(x, "x");
  TTv<T> Xv = view<T>(X, "X (right DRM)");
  TTv<T> Yv = view<T>(Y, "Y (left DRM)");
  if (Xv.d != xv.d || Yv.d != xv.d) throw Error(TT_ERR_ARG, "stta_sketch: d mismatch");
  same_modes(Xv.n, xv.n, xv.d, "stta_sketch");
  same_modes(Yv.n, xv.n, xv.d, "stta_sketch");
  if (!dry) {
    if (!psi || (xv.d > 1 && !omega)) throw Error(TT_ERR_ARG, "stta_sketch: null psi or omega");
    for (int k = 0; k < xv.d; ++k)
      if (!psi[k] || (k + 1 < xv.d && !omega[k]))
        throw Error(TT_ERR_ARG, "stta_sketch: null sketch pointer");
  }
  Carved cv = carve(mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  std::vector<double*> none(MAXD, nullptr);  // placeholders of a dry run
  tt_stta_sketch_dev<T>(cv.ctx, xv, coef, accumulate, Xv, Yv, dry ? none.data() : psi,
                        dry ? none.data() : omega);
  if (dry) throw (size_t)cv.ar.peak;
}

void do_stta_recover(int d, const int64_t* n, const int64_t* r, const int64_t* l,
                     const double* const* psi, const double* const* omega, double rcond,
                     double* const* cores, void* ws, size_t bytes, void* stream, bool dry) {
  if (d < 1 || d > MAXD) throw Error(TT_ERR_ARG, "stta_recover: d out of range");
  if (!n || !r || !l) throw Error(TT_ERR_ARG, "stta_recover: null size array");
  if (r[0] != 1 || r[d] != 1 || l[0] != 1 || l[d] != 1)
    throw Error(TT_ERR_ARG, "stta_recover: boundary ranks must be 1");
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || r[k + 1] < 1 || l[k + 1] < 1)
      throw Error(TT_ERR_ARG, "stta_recover: n, ranks >= 1");
    if (l[k] < r[k]) throw Error(TT_ERR_ARG, "stta_recover: l_k >= r_k required");
  }
  if (!dry) {
    if (!psi || !cores || (d > 1 && !omega)) throw Error(TT_ERR_ARG, "stta_recover: null array");
    for (int k = 0; k < d; ++k)
      if (!psi[k] || !cores[k] || (k + 1 < d && !omega[k]))
        throw Error(TT_ERR_ARG, "stta_recover: null pointer");
  }
  Carved cv = carve(TT_MODE_FP64, ws, bytes, stream, dry);
  fix_ctx(cv);
  reset_flags(cv);
  std::vector<double*> none(MAXD, nullptr);  // placeholders of a dry run
  tt_stta_recover_dev(cv.ctx, d, n, r, l, dry ? none.data() : psi, dry ? none.data() : omega,
                      rcond > 0.0 ? rcond : 1e-12, dry ? none.data() : cores);
  if (dry) throw (size_t)cv.ar.peak;
}
}  // namespace
}  // namespace ttsg

size_t tt_stta_sketch_workspace(int mode, const tt_vec* x, const tt_vec* X, const tt_vec* Y) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_stta_sketch<double>(mode, x, 1.0, 0, X, Y, nullptr, nullptr, nullptr, 0, nullptr, true);
    else
      do_stta_sketch<float>(mode, x, 1.0, 0, X, Y, nullptr, nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_stta_sketch(int mode, const tt_vec* x, double coef, int accumulate, const tt_vec* X,
                   const tt_vec* Y, double* const* psi, double* const* omega, void* ws,
                   size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_stta_sketch<double>(mode, x, coef, accumulate, X, Y, psi, omega, ws, ws_bytes, stream,
                             false);
    else
      do_stta_sketch<float>(mode, x, coef, accumulate, X, Y, psi, omega, ws, ws_bytes, stream,
                            false);
  });
}

size_t tt_stta_recover_workspace(int d, const int64_t* n, const int64_t* r, const int64_t* l) {
  return measure([&] {
    do_stta_recover(d, n, r, l, nullptr, nullptr, 0.0, nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_stta_recover(int d, const int64_t* n, const int64_t* r, const int64_t* l,
                    const double* const* psi, const double* const* omega, double rcond,
                    double* const* cores, void* ws, size_t ws_bytes, void* stream) {
  return guarded([&] {
    do_stta_recover(d, n, r, l, psi, omega, rcond, cores, ws, ws_bytes, stream, false);
  });
}

int tt_sketch_factors(int mode, int d, const int64_t* n, int64_t s, uint64_t seed,
                      void* const* S, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (d < 1 || d > MAXD || !n || !S || s < 1) throw Error(TT_ERR_ARG, "sketch_factors: arguments");
    for (int k = 0; k < d; ++k) {
      if (n[k] < 1 || !S[k]) throw Error(TT_ERR_ARG, "sketch_factors: n[k] >= 1, S[k] non-null");
      // variance s^(-1/d): E ||S_odot x||^2 = ||x||^2 (Sec. 3.1)
      gaussian_fill(S[k], mode == TT_MODE_FP64, s * n[k], seed, 1024 + (uint64_t)k,
                    std::pow((double)s, -0.5 / d), (cudaStream_t)stream);
    }
  });
}

int tt_gaussian(int mode, void* out, int64_t count, uint64_t seed, uint64_t stream_id, double std_,
                void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (count < 0 || (count > 0 && !out)) throw Error(TT_ERR_ARG, "gaussian: bad output");
    gaussian_fill(out, mode == TT_MODE_FP64, count, seed, stream_id, std_, (cudaStream_t)stream);
  });
}

namespace {
template <typename T>
void do_dot_grad(int mode, const tt_vec* x, const tt_vec* y, void* const* g, void* const* M,
                 double* out, void* ws, size_t bytes, void* stream, bool dry) {
  TTv<T> xv = view<T>(x, "x");
  TTv<T> yv = view<T>(y, "y");
  if (xv.d != yv.d) throw Error(TT_ERR_ARG, "dot_grad: d mismatch");
  same_modes(xv.n, yv.n, xv.d, "dot_grad");
  const int d = xv.d;
  std::vector<T*> gp(d, nullptr);
  std::vector<const T*> mp(d, nullptr);
  if (!dry) {
    if (M) {
      if (!out) throw Error(TT_ERR_ARG, "local_dots: null out");
      for (int k = 0; k < d; ++k)
        if (!(mp[k] = (const T*)M[k])) throw Error(TT_ERR_ARG, "local_dots: null matrix");
    }
    if (g)
      for (int k = 0; k < d; ++k)
        if (!(gp[k] = (T*)g[k])) throw Error(TT_ERR_ARG, "dot_grad: null gradient core");
  }
  Carved cv = carve(mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  tt_dot_grad_dev<T>(cv.ctx, xv, yv, g ? gp.data() : nullptr, M ? mp.data() : nullptr, out);
  if (dry) throw (size_t)cv.ar.peak;
}
void* const kDryPtrs[1] = {nullptr};
}  // namespace

size_t tt_dot_grad_workspace(int mode, const tt_vec* x, const tt_vec* y) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_dot_grad<double>(mode, x, y, kDryPtrs, nullptr, nullptr, nullptr, 0, nullptr, true);
    else
      do_dot_grad<float>(mode, x, y, kDryPtrs, nullptr, nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_dot_grad(int mode, const tt_vec* x, const tt_vec* y, void* const* g, void* ws,
                size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (!g) throw Error(TT_ERR_ARG, "dot_grad: null gradient array");
    if (mode == TT_MODE_FP64)
      do_dot_grad<double>(mode, x, y, g, nullptr, nullptr, ws, ws_bytes, stream, false);
    else
      do_dot_grad<float>(mode, x, y, g, nullptr, nullptr, ws, ws_bytes, stream, false);
  });
}

size_t tt_local_dots_workspace(int mode, const tt_vec* x, const tt_vec* y) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_dot_grad<double>(mode, x, y, nullptr, kDryPtrs, nullptr, nullptr, 0, nullptr, true);
    else
      do_dot_grad<float>(mode, x, y, nullptr, kDryPtrs, nullptr, nullptr, 0, nullptr, true);
  });
}

int tt_local_dots(int mode, const tt_vec* x, const tt_vec* y, void* const* M, double* out,
                  void* ws, size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (!M) throw Error(TT_ERR_ARG, "local_dots: null matrix array");
    if (mode == TT_MODE_FP64)
      do_dot_grad<double>(mode, x, y, nullptr, M, out, ws, ws_bytes, stream, false);
    else
      do_dot_grad<float>(mode, x, y, nullptr, M, out, ws, ws_bytes, stream, false);
  });
}

int tt_kron_sum_op(int mode, int d, const int64_t* n, void* const* M, const double* theta,
                   void* const* cores, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (d < 1 || d > MAXD || !n || !M || !cores) throw Error(TT_ERR_ARG, "kron_sum_op: bad arguments");
    for (int k = 0; k < d; ++k)
      if (n[k] < 1 || !M[k] || !cores[k]) throw Error(TT_ERR_ARG, "kron_sum_op: bad mode " + std::to_string(k));
    if (mode == TT_MODE_FP64)
      tt_kron_sum_op_dev<double>((cudaStream_t)stream, d, n, (const double* const*)M, theta,
                                 (double* const*)cores);
    else
      tt_kron_sum_op_dev<float>((cudaStream_t)stream, d, n, (const float* const*)M, theta,
                                (float* const*)cores);
  });
}

int tt_op_transpose(int mode, const tt_op* A, void* const* cores, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (!cores) throw Error(TT_ERR_ARG, "op_transpose: null output");
    if (mode == TT_MODE_FP64) {
      TTop<double> a = view_op<double>(A, 0);
      for (int k = 0; k < a.d; ++k)
        if (!cores[k]) throw Error(TT_ERR_ARG, "op_transpose: null output core");
      tt_op_transpose_dev<double>((cudaStream_t)stream, a, (double* const*)cores);
    } else {
      TTop<float> a = view_op<float>(A, 0);
      for (int k = 0; k < a.d; ++k)
        if (!cores[k]) throw Error(TT_ERR_ARG, "op_transpose: null output core");
      tt_op_transpose_dev<float>((cudaStream_t)stream, a, (float* const*)cores);
    }
  });
}

size_t tt_qr_f64_workspace(int64_t m, int64_t l) { return qr_workspace(m, l) + 64 * 1024; }

int tt_qr_f64(int mode, const void* Y, int64_t m, int64_t l, int64_t sr, int64_t sc, void* Q,
              double* R, void* ws, size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (!Y || m < l || l < 1) throw Error(TT_ERR_ARG, "qr: need Y and m >= l >= 1");
    Carved cv = carve(mode, ws, ws_bytes, stream, false, false);
    fix_ctx(cv);
    reset_flags(cv);
    const size_t rest = ws_bytes - cv.ar.mark();
    void* qw = cv.ar.take<char>((int64_t)qr_workspace(m, l));
    const int f64 = mode == TT_MODE_FP64;
    qr_f64(Y, f64, m, l, sr, sc, Q, f64, l, R, qw, rest, cv.ctx.err, cv.ctx.st);
    check_device_flags(cv.ctx);
  });
}

size_t tt_lstsq_f64_workspace(int64_t s, int64_t k) { return lstsq_workspace(s, k) + 4096; }

int tt_lstsq_f64(const double* W, int64_t s, int64_t k, const double* c, double* y, double* res,
                 void* ws, size_t ws_bytes, void* stream) {
  return guarded([&] {
    if (!W || !c || !y || !res || !ws || s < 1 || k < 1 || k > s)
      throw Error(TT_ERR_ARG, "lstsq: bad arguments");
    if (ws_bytes < lstsq_workspace(s, k)) throw Error(TT_ERR_WORKSPACE, "lstsq: workspace");
    cudaStream_t st = (cudaStream_t)stream;
    lstsq_reset(c, s, k, ws, st);
    for (int64_t j = 0; j < k; ++j) lstsq_add_column(W, c, s, j, k, ws, y, res, st);
  });
}

namespace {
SolveParams to_params(const tt_solver_params* p) {
  if (!p) throw Error(TT_ERR_ARG, "solve: null params");
  SolveParams q;
  q.maxit = p->maxit; q.s = p->s; q.tol = p->tol; q.round_tol = p->round_tol; q.eta = p->eta;
  q.stop_safety = p->stop_safety; q.rmax = p->rmax; q.r_sol = p->r_sol;
  q.oversample = p->oversample; q.seed = p->seed; q.max_restarts = p->max_restarts;
  q.final_stta = p->final_stta;
  q.ell = p->ell > 0 ? p->ell : 1;
  if (q.maxit < 1 || q.tol <= 0 || q.rmax < 1 || q.oversample < 0 || q.max_restarts < 0 ||
      q.eta < 0 || q.stop_safety <= 0 || (q.final_stta != 0 && q.final_stta != 1))
    throw Error(TT_ERR_ARG, "solve: invalid parameters");
  return q;
}

PrecondArgs view_precond(const tt_precond* P, int d, bool dry) {
  if (!P) throw Error(TT_ERR_ARG, "precond: null descriptor");
  if (P->zeta < 1 || P->zeta > TT_MAX_PRECOND_TERMS)
    throw Error(TT_ERR_ARG, "precond: zeta out of range");
  if (!P->alpha || !P->beta || !P->A1d) throw Error(TT_ERR_ARG, "precond: null array");
  for (int i = 0; i < P->zeta; ++i)
    if (!(P->beta[i] > 0.0)) throw Error(TT_ERR_ARG, "precond: beta_i > 0 required");
  if (!dry)
    for (int k = 0; k < d; ++k)
      if (!P->A1d[k]) throw Error(TT_ERR_ARG, "precond: null matrix pointer");
  PrecondArgs a;
  a.zeta = P->zeta;
  a.alpha = P->alpha;
  a.beta = P->beta;
  a.A1d = P->A1d;
  return a;
}

void do_solve(const tt_op* A, const tt_vec* b, const tt_solver_params* p, const tt_vec_out* x,
              tt_solver_info* info, void* ws, size_t bytes, void* stream, bool dry,
              const tt_precond* P = nullptr) {
  SolveParams q = to_params(p);
  check_mode(p->mode);
  TTop<double> a = view_op<double>(A, 0);
  TTv<double> bv = view<double>(b, "b");
  if (a.d != bv.d) throw Error(TT_ERR_ARG, "solve: d mismatch");
  same_modes(a.n, bv.n, bv.d, "solve");
  PrecondArgs pa;
  if (P) {
    pa = view_precond(P, bv.d, dry);
    q.pre = &pa;
  }
  TTv<double> xv;
  int64_t cap[MAXD + 1];
  const int64_t r_sol = q.r_sol > 0 ? q.r_sol : q.rmax;
  if (!dry) {
    xv = view_out<double>(x, "x", cap);
    if (xv.d != bv.d) throw Error(TT_ERR_ARG, "solve: x d mismatch");
    for (int k = 1; k < bv.d; ++k)
      if (cap[k] < r_sol) throw Error(TT_ERR_ARG, "solve: x capacity below r_sol");
  } else {
    xv.d = bv.d;
  }
  Carved cv = carve(p->mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  reset_flags(cv);
  SolveResult r = p->mode == TT_MODE_FP64 ? sgmres_solve<double>(cv.ctx, a, bv, q, xv)
                                          : sgmres_solve<float>(cv.ctx, a, bv, q, xv);
  if (dry) throw (size_t)cv.ar.peak;
  for (int k = 0; k <= bv.d; ++k) x->rank[k] = xv.r[k];
  if (info) {
    info->iters = r.iters;
    info->cycles = r.cycles;
    info->sketched_res = r.sketched_res;
    info->true_res = r.true_res;
    info->max_rank = r.max_rank;
    info->status = r.status;
    info->seconds = r.seconds;
    info->svd_nonconverged = r.svd_nonconverged;
    info->svd_max_sweeps = r.svd_max_sweeps;
    info->svd_mean_sweeps = r.svd_mean_sweeps;
    info->breakdowns = r.breakdowns;
    for (int i = 0; i < info->hist_cap && i < (int)r.res_hist.size(); ++i) {
      if (info->res_hist) info->res_hist[i] = r.res_hist[i];
      if (info->rank_hist) info->rank_hist[i] = r.rank_hist[i];
    }
  }
  if (r.status != TT_OK)
    throw Error(r.status, "solve: true residual " + std::to_string(r.true_res) + " above tol after " +
                              std::to_string(r.cycles) + " cycles" +
                              (r.breakdowns ? " (the Krylov space became invariant)" : ""));
}
}  // namespace

size_t tt_spgmres_solve_workspace(const tt_op* A, const tt_precond* P, const tt_vec* b,
                                  const tt_solver_params* p) {
  return measure([&] { do_solve(A, b, p, nullptr, nullptr, nullptr, 0, nullptr, true, P); });
}

int tt_spgmres_solve(const tt_op* A, const tt_precond* P, const tt_vec* b,
                     const tt_solver_params* p, const tt_vec_out* x, tt_solver_info* info,
                     void* ws, size_t ws_bytes, void* stream) {
  return guarded([&] {
    if (!P) throw Error(TT_ERR_ARG, "spgmres: null preconditioner");
    do_solve(A, b, p, x, info, ws, ws_bytes, stream, false, P);
  });
}

int tt_exp_sum_coefficients(double a, double b, double tol, int cap, double* alpha,
                            double* beta) {
  return exp_sum_coefficients(a, b, tol, cap, alpha, beta);
}

namespace ttsg {
namespace {
template <typename T>
void do_precond_apply(int mode, const tt_precond* P, const tt_vec* x, double eps, int64_t rmax,
                      int64_t p, uint64_t seed, const tt_vec_out* y, void* ws, size_t bytes,
                      void* stream, bool dry) {
  TTv<T> xv = view<T>(x, "x");
  const int d = xv.d;
  if (d < 2) throw Error(TT_ERR_ARG, "precond: d >= 2");
  if (!(eps >= 0.0) || rmax < 1 || p < 0)
    throw Error(TT_ERR_ARG, "precond: eps >= 0, rmax >= 1, p >= 0");
  PrecondArgs pa = view_precond(P, d, dry);
  // sketch ranks of the zeta-term sum: the output capacity must cover them
  std::vector<const int64_t*> tr(pa.zeta, xv.r);
  int64_t ell[MAXD + 1];
  rto_ranks(tr, xv.n, d, rmax, p, ell);
  DRMSource<T> ds;
  ds.seed = seed;
  for (int k = 0; k <= d; ++k) ds.L[k] = (k == 0 || k == d) ? 1 : rmax + p;
  TTv<T> yv;
  int64_t cap[MAXD + 1];
  if (dry) {
    yv.d = d;
    for (int k = 0; k < d; ++k) yv.n[k] = xv.n[k];
  } else {
    yv = view_out<T>(y, "y", cap);
    if (yv.d != d) throw Error(TT_ERR_ARG, "precond: output d mismatch");
    for (int k = 1; k < d; ++k)
      if (cap[k] < std::min<int64_t>(rmax, ell[k]))
        throw Error(TT_ERR_ARG, "precond: output capacity below min(rmax, sketch rank)");
  }
  Carved cv = carve(mode, ws, bytes, stream, dry);
  fix_ctx(cv);
  reset_flags(cv);
  PrecondDev<T> pd;
  precond_setup<T>(cv.ctx, pa, d, xv.n, pd);
  std::vector<TTv<T>> bufs(pa.zeta);
  for (auto& b : bufs) {
    b.d = d;
    for (int k = 0; k <= d; ++k) b.r[k] = xv.r[k];
    for (int k = 0; k < d; ++k) {
      b.n[k] = xv.n[k];
      b.core[k] = cv.ar.take<T>(xv.core_elems(k));
    }
  }
  precond_apply_dev<T>(cv.ctx, pd, xv, eps, rmax, p, ds, bufs, yv);
  if (dry) throw (size_t)cv.ar.peak;
  if (!g_dry_run) TT_CUDA(cudaStreamSynchronize(cv.ctx.st));
  for (int k = 0; k <= d; ++k) y->rank[k] = yv.r[k];
}
}  // namespace
}  // namespace ttsg

size_t tt_precond_apply_workspace(int mode, const tt_precond* P, const tt_vec* x, int64_t rmax,
                                  int64_t oversample) {
  return measure([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_precond_apply<double>(mode, P, x, 0.1, rmax, oversample, 0, nullptr, nullptr, 0,
                               nullptr, true);
    else
      do_precond_apply<float>(mode, P, x, 0.1, rmax, oversample, 0, nullptr, nullptr, 0,
                              nullptr, true);
  });
}

int tt_precond_apply(int mode, const tt_precond* P, const tt_vec* x, double eps, int64_t rmax,
                     int64_t oversample, uint64_t seed, const tt_vec_out* y, void* ws,
                     size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (mode == TT_MODE_FP64)
      do_precond_apply<double>(mode, P, x, eps, rmax, oversample, seed, y, ws, ws_bytes, stream,
                               false);
    else
      do_precond_apply<float>(mode, P, x, eps, rmax, oversample, seed, y, ws, ws_bytes, stream,
                              false);
  });
}

size_t tt_sgmres_solve_workspace(const tt_op* A, const tt_vec* b, const tt_solver_params* p) {
  return measure([&] { do_solve(A, b, p, nullptr, nullptr, nullptr, 0, nullptr, true); });
}

int tt_sgmres_solve(const tt_op* A, const tt_vec* b, const tt_solver_params* p,
                    const tt_vec_out* x, tt_solver_info* info, void* ws, size_t ws_bytes,
                    void* stream) {
  return guarded([&] { do_solve(A, b, p, x, info, ws, ws_bytes, stream, false); });
}

// ------------------------------------------------------------ batched forms
namespace {
struct NarrowQR {
  bool old;
  NarrowQR() : old(g_qr_narrow) { g_qr_narrow = true; }
  ~NarrowQR() { g_qr_narrow = old; }
};
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Workspace of one solve whose QRs take the narrow form.
size_t solve_bytes_narrow(const tt_op* A, const tt_vec* b, const tt_solver_params* p) {
  NarrowQR f;
  return measure([&] { do_solve(A, b, p, nullptr, nullptr, nullptr, 0, nullptr, true); });
}

size_t batched_slice(const tt_op* A, int nrhs, const tt_vec* b, const tt_solver_params* p) {
  size_t mx = 0;
  for (int i = 0; i < nrhs; ++i) {
    const size_t s = solve_bytes_narrow(A, &b[i], p);
    if (s == 0) throw Error(TT_ERR_ARG, "rhs " + std::to_string(i) + ": " + g_last_error);
    mx = std::max(mx, s);
  }
  return align256(mx);
}
}  // namespace

size_t tt_qr_f64_batched_workspace(int count, const int64_t* m, const int64_t* l) {
  if (count < 1 || !m || !l) return 0;
  return qr_batch_workspace(count, m, l) + 64 * 1024;
}

int tt_qr_f64_batched(int mode, int count, void* const* Y, const int64_t* m, const int64_t* l,
                      void* const* Q, double* const* R, void* ws, size_t ws_bytes, void* stream) {
  return guarded([&] {
    check_mode(mode);
    if (count < 1 || !Y || !m || !l) throw Error(TT_ERR_ARG, "qr_batched: bad arguments");
    std::vector<QRProblem> pb(count);
    const int f64 = mode == TT_MODE_FP64;
    for (int i = 0; i < count; ++i) {
      if (!Y[i] || m[i] < l[i] || l[i] < 1)
        throw Error(TT_ERR_ARG, "qr_batched: problem " + std::to_string(i) + " needs Y and m >= l >= 1");
      pb[i] = QRProblem{Y[i], f64, m[i], l[i], l[i], 1, Q ? Q[i] : nullptr, f64, l[i],
                        R ? R[i] : nullptr};
    }
    Carved cv = carve(mode, ws, ws_bytes, stream, false, false);
    fix_ctx(cv);
    reset_flags(cv);
    const size_t need = qr_batch_workspace(count, m, l);
    void* qw = cv.ar.take<char>((int64_t)need);
    qr_f64_batched(count, pb.data(), qw, need, cv.ctx.err, cv.ctx.st);
    check_device_flags(cv.ctx);
  });
}

size_t tt_sgmres_solve_batched_workspace(const tt_op* A, int nrhs, const tt_vec* b,
                                         const tt_solver_params* p, int nworkers) {
  try {
    if (nrhs < 1 || !b) throw Error(TT_ERR_ARG, "solve_batched: nrhs >= 1 and b required");
    const int W = std::max(1, std::min(nworkers, nrhs));
    return (size_t)W * batched_slice(A, nrhs, b, p);
  } catch (const Error& e) {
    g_last_error = e.what();
    return 0;
  }
}

int tt_sgmres_solve_batched(const tt_op* A, int nrhs, const tt_vec* b, const tt_solver_params* p,
                            const tt_vec_out* x, tt_solver_info* info, int nworkers, void* ws,
                            size_t ws_bytes) {
  return guarded([&] {
    if (nrhs < 1 || !b || !x) throw Error(TT_ERR_ARG, "solve_batched: nrhs >= 1, b and x required");
    if (!ws) throw Error(TT_ERR_WORKSPACE, "null workspace");
    const int W = std::max(1, std::min(nworkers, nrhs));
    const size_t per = batched_slice(A, nrhs, b, p);
    if (ws_bytes < (size_t)W * per)
      throw Error(TT_ERR_WORKSPACE, "solve_batched: workspace below " + std::to_string(W * per));
    int dev = 0;
    TT_CUDA(cudaGetDevice(&dev));
    std::mutex mu;
    int first_err = 0, not_conv = 0;
    std::string msg;
    std::vector<std::thread> pool;
    for (int w = 0; w < W; ++w) {
      pool.emplace_back([&, w] {
        cudaSetDevice(dev);
        g_qr_narrow = true;
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
          std::lock_guard<std::mutex> lk(mu);
          if (!first_err) { first_err = TT_ERR_CUDA; msg = "solve_batched: stream creation failed"; }
          return;
        }
        char* slice = (char*)ws + (size_t)w * per;
        for (int i = w; i < nrhs; i += W) {
          const int rc = guarded([&] {
            do_solve(A, &b[i], p, &x[i], info ? &info[i] : nullptr, slice, per, st, false);
          });
          if (rc == TT_ERR_NOT_CONVERGED || rc == TT_ERR_BREAKDOWN) {
            std::lock_guard<std::mutex> lk(mu);
            ++not_conv;
          } else if (rc != TT_OK) {
            if (info) info[i].status = rc;
            std::lock_guard<std::mutex> lk(mu);
            if (!first_err) { first_err = rc; msg = "rhs " + std::to_string(i) + ": " + g_last_error; }
          }
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
      });
    }
    for (auto& t : pool) t.join();
    if (first_err) throw Error(first_err, msg);
    if (not_conv)
      throw Error(TT_ERR_NOT_CONVERGED, std::to_string(not_conv) + " of " + std::to_string(nrhs) +
                                            " right-hand sides stopped above tol");
  });
}

