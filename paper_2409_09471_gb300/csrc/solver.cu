// TT-sGMRES driver: Algorithm 4 with incomplete orthogonalisation l = 1 done
// explicitly in TT format (the Remark of Section 3.6 for l = 1), randomized
// rounding for the Gram-Schmidt update and for the final sum (Section 3.5),
// y_k = (S A V_k)^+ S r_0 (eq. pseudo_inv) by the incremental FP64 QR, and the
// restart loop of Section 3.4 driven by the exact FP64 true residual.
//
// Per iteration (all on the device; the host reads the new ranks and the
// sketched residual once):
//   w = A v_k (untruncated)
//   second stream: h = <w, v_k>, then W[:, k] = S w
//   v~ = Round(w - h v_k, round_tol, rmax) (its left sweep waits for h)
//     ->  v_{k+1} = v~ / ||v~||
//   y = argmin ||W y - S r0|| (after W[:, k]), stop when
//   ||W y - S r0|| <= inner_tol ||S r0||.
#include "solver.cuh"
#include <type_traits>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

namespace ttsg {

namespace {

template <typename T>
constexpr int f64_of() { return sizeof(T) == 8 ? 1 : 0; }

double read_double(cudaStream_t st, const double* dev) {
  if (g_dry_run) return 1.0;
  double h = 0.0;
  TT_CUDA(cudaMemcpyAsync(&h, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  return h;
}

// Mode-dependent floor of the per-cycle sketched tolerance: the accuracy the
// contractions of that precision can deliver before a restart is needed
// (TF32 mode: split-TF32 products, about 2^-20 relative each; BF16 mode:
// split-BF16 products, about 2^-17).
double inner_floor(int mode) {
  switch (mode) {
    case TT_MODE_FP64: return 0.0;
    case TT_MODE_FP32: return 1e-7;
    case TT_MODE_BF16: return 1e-5;
    default: return 1e-6;
  }
}

// Second stream of one solve, with the events that order it against the
// solver's own stream; released when the solve returns (pending work is not
// waited for by cudaStreamDestroy, it completes first).
struct SideStream {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, dots = nullptr, sketch = nullptr;
  void create() {
    TT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    TT_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    TT_CUDA(cudaEventCreateWithFlags(&dots, cudaEventDisableTiming));
    TT_CUDA(cudaEventCreateWithFlags(&sketch, cudaEventDisableTiming));
  }
  ~SideStream() {
    if (fork) cudaEventDestroy(fork);
    if (dots) cudaEventDestroy(dots);
    if (sketch) cudaEventDestroy(sketch);
    if (st) cudaStreamDestroy(st);
  }
};

template <typename T>
TTv<T> alloc_tt(Arena& ar, int d, const int64_t* n, const int64_t* cap) {
  TTv<T> v;
  v.d = d;
  for (int k = 0; k < d; ++k) {
    v.n[k] = n[k];
    v.core[k] = ar.take<T>(cap[k] * n[k] * cap[k + 1]);
    v.r[k] = cap[k];
  }
  v.r[d] = 1;
  return v;
}

}  // namespace

template <typename T>
SolveResult sgmres_solve(const Ctx& c0, const TTop<double>& A64in, const TTv<double>& b,
                         const SolveParams& p, TTv<double>& xout) {
  Ctx c = c0;
  Arena& ar = *c.ar;
  const int d = b.d;
  const int f64 = f64_of<T>();
  const auto t_start = std::chrono::steady_clock::now();
  TT_CHECK_ARG(d >= 2 && d <= MAXD, "solve: 2 <= d <= 64");
  TT_CHECK_ARG(p.maxit >= 1 && p.rmax >= 1 && p.tol > 0, "solve: maxit, rmax, tol");
  const int64_t s = p.s > 0 ? p.s : 2 * p.maxit;
  const int64_t r_sol = p.r_sol > 0 ? p.r_sol : p.rmax;
  const int64_t* n = b.n;
  SolveResult res;

  // ---- operator in the working layout [a][i][a'][j] (working and FP64 copies)
  TTop<T> A;
  TTop<double> A64;
  A.d = A64.d = d;
  int64_t Rmax = 1;
  {
    std::vector<CopySeg> segs;
    for (int k = 0; k < d; ++k) {
      const int64_t R0 = A64in.R[k], R1 = A64in.R[k + 1], nn = n[k];
      A.n[k] = A64.n[k] = nn;
      A.R[k] = A64.R[k] = R0;
      Rmax = std::max(Rmax, R0);
      A64.core[k] = ar.take<double>(R0 * nn * nn * R1);
      A.core[k] = f64 ? (T*)A64.core[k] : ar.take<T>(R0 * nn * nn * R1);
      CopySeg sg;
      sg.src = A64in.core[k]; sg.dst = A64.core[k];
      sg.A = R0 * nn; sg.B = R1; sg.C = nn; sg.sa = nn * R1; sg.sb = 1; sg.sc = R1;
      sg.src_f64 = 1; sg.dst_f64 = 1;
      segs.push_back(sg);
      if (!f64) {
        CopySeg s2 = sg;
        s2.dst = A.core[k];
        s2.dst_f64 = 0;
        segs.push_back(s2);
      }
    }
    A.R[d] = A64.R[d] = 1;
    copy3d(segs, c.st);
  }
  // ---- Khatri-Rao factors S_k: N(0, s^{-1/d}), Philox streams 1024 + k
  std::vector<T*> S(d);
  for (int k = 0; k < d; ++k) {
    S[k] = ar.take<T>(s * n[k]);
    gaussian_fill(S[k], f64, s * n[k], p.seed, 1024 + (uint64_t)k, std::pow((double)s, -0.5 / d),
                  c.st);
  }
  // Gaussian TT-DRM drawn once per solve (Philox streams 2048 + k) at the
  // capacity ranks; every rounding uses its leading sub-blocks
  DRMSource<T> drm;
  drm.seed = p.seed;
  drm.L[0] = drm.L[d] = 1;
  // capacity: every rounding's rank cap (basis rmax, solution r_sol, and the
  // right-hand side's own ranks, which cap the restart residual) plus p
  int64_t rb_drm = 1;
  for (int k = 0; k <= d; ++k) rb_drm = std::max(rb_drm, b.r[k]);
  for (int k = 1; k < d; ++k) drm.L[k] = std::max(std::max(p.rmax, r_sol), rb_drm) + p.oversample;
  std::vector<T*> drm_cores(d);
  std::vector<double*> drm64_cores(d);
  for (int k = 0; k < d; ++k) {
    const int64_t cnt = drm.L[k] * n[k] * drm.L[k + 1];
    const double sd = 1.0 / std::sqrt((double)cnt);
    drm64_cores[k] = ar.take<double>(cnt);
    gaussian_fill(drm64_cores[k], 1, cnt, p.seed, 2048 + (uint64_t)k, sd, c.st);
    if (f64) {
      drm_cores[k] = (T*)drm64_cores[k];
    } else {
      drm_cores[k] = ar.take<T>(cnt);
      CopySeg sg;
      sg.src = drm64_cores[k]; sg.dst = drm_cores[k]; sg.A = cnt; sg.sa = 1;
      sg.src_f64 = 1; sg.dst_f64 = 0;
      copy3d({sg}, c.st);
    }
  }
  drm.core = (const T* const*)drm_cores.data();

  // ---- persistent buffers
  int64_t rb = 1;
  for (int k = 0; k <= d; ++k) rb = std::max(rb, b.r[k]);
  const int64_t vcap_r = std::max(p.rmax, rb);
  std::vector<int64_t> vcap(d + 1, vcap_r), wcap(d + 1), xcap(d + 1, r_sol), bcap(d + 1);
  vcap[0] = vcap[d] = 1;
  xcap[0] = xcap[d] = 1;
  for (int k = 0; k <= d; ++k) {
    wcap[k] = A64.R[k] * std::max(vcap[k], xcap[k]);
    bcap[k] = b.r[k];
  }
  // Krylov basis.  With the STTA correction (final_stta) a basis vector is
  // sketched when it is formed and afterwards read only by the Gram-Schmidt
  // window of the next ell steps, so ell + 1 slots used as a ring hold all
  // that is live; the rounding form keeps the whole basis for Round(sum y_i v_i).
  const int ell = std::max(1, std::min(p.ell, p.maxit));
  const int nslots = p.final_stta ? ell + 1 : p.maxit + 1;
  std::vector<TTv<T>> V;
  for (int i = 0; i < nslots; ++i) V.push_back(alloc_tt<T>(ar, d, n, vcap.data()));
  auto VS = [&](int i) -> TTv<T>& { return V[i % nslots]; };
  TTv<T> w = alloc_tt<T>(ar, d, n, wcap.data());
  TTv<T> bT = f64 ? TTv<T>() : alloc_tt<T>(ar, d, n, bcap.data());
  TTv<T> rhs = alloc_tt<T>(ar, d, n, vcap.data());
  // the cycle's correction e is computed in the working precision; the
  // accumulated solution, the residual b - A x and its rounding stay in FP64
  // (mixed-precision iterative refinement)
  TTv<T> e = alloc_tt<T>(ar, d, n, xcap.data());
  TTv<double> x = alloc_tt<double>(ar, d, n, xcap.data());
  TTv<double> xn = alloc_tt<double>(ar, d, n, xcap.data());
  TTv<double> e64 = alloc_tt<double>(ar, d, n, xcap.data());
  TTv<double> w64 = alloc_tt<double>(ar, d, n, wcap.data());
  TTv<double> r64 = alloc_tt<double>(ar, d, n, vcap.data());
  Ctx c64 = c;
  c64.mode = TT_MODE_FP64;
  DRMSource<double> drm64;
  drm64.seed = drm.seed;
  for (int k = 0; k <= d; ++k) drm64.L[k] = drm.L[k];
  drm64.core = (const double* const*)drm64_cores.data();
  double* Wm = ar.take<double>(s * p.maxit);
  double* Sr0 = ar.take<double>(s);
  double* ydev = ar.take<double>(p.maxit);
  double* hcoef = ar.take<double>(p.maxit);  // h_{i,k} of the older vectors (ell > 1)
  double* scal = ar.take<double>(16);  // 0 beta, 1 h, 2 ||v~||^2, 3 ||v~||, 4 res, 5 ||Sr0||^2, 6 ||Sr0||
  double* lsws = (double*)ar.take<char>((int64_t)lstsq_workspace(s, p.maxit));
  if (f64) {
    bT.d = d;
    for (int k = 0; k < d; ++k) { bT.n[k] = n[k]; bT.core[k] = (T*)b.core[k]; }
    for (int k = 0; k <= d; ++k) bT.r[k] = b.r[k];
  } else {
    std::vector<CopySeg> segs;
    for (int k = 0; k < d; ++k) {
      CopySeg sg;
      sg.src = b.core[k]; sg.dst = bT.core[k]; sg.A = b.core_elems(k); sg.sa = 1;
      sg.src_f64 = 1; sg.dst_f64 = 0;
      segs.push_back(sg);
      bT.r[k] = b.r[k];
    }
    bT.r[d] = 1;
    copy3d(segs, c.st);
  }

  auto copy_tt = [&](const auto& src, auto& dst, const double* scale_dev, int inv) {
    std::vector<CopySeg> segs;
    for (int k = 0; k < d; ++k) {
      CopySeg sg;
      sg.src = src.core[k]; sg.dst = dst.core[k]; sg.A = src.core_elems(k); sg.sa = 1;
      sg.src_f64 = sizeof(*src.core[0]) == 8; sg.dst_f64 = sizeof(*dst.core[0]) == 8;
      if (k == 0) { sg.scale_dev = scale_dev; sg.scale_dev_inv = inv; }
      segs.push_back(sg);
      dst.r[k] = src.r[k];
    }
    dst.r[d] = 1;
    copy3d(segs, c.st);
  };

  // ---- STTA (Sec. 3.3, Alg. 4): each cycle's correction from one-pass
  // sketches of the basis vectors instead of a rounding of the stored basis.
  // Target ranks r_sol and left ranks r_sol + 20 (the paper's oversampling),
  // both capped by the mode-size products; Gaussian TT-DRMs from the Philox
  // streams 4096 + k (right) and 6144 + k (left).  The sketches are FP64 in
  // every mode: combined with the Krylov coefficients (a non-orthogonal basis,
  // so with cancellation) single-precision sketches left the correction too
  // inexact for the refinement to converge (FP32 mode stalled near 7e-5).
  const bool use_stta = p.final_stta != 0;
  int64_t rS[MAXD + 1], lS[MAXD + 1];
  TTv<double> Xv, Yv;
  TTv<double> vs64;        // FP64 copy of a basis vector in the float modes
  std::vector<int64_t> psi_off(d, 0), om_off(d, 0);
  int64_t ssz = 0;
  double* skb = nullptr;   // sketches of V[0..maxit-1], ssz doubles each
  double* comb = nullptr;  // their combination with y
  TTv<double> es;          // recovered correction (FP64, ranks rS)
  if (use_stta) {
    rS[0] = rS[d] = lS[0] = lS[d] = 1;
    double left = 1.0;
    for (int k = 1; k < d; ++k) {
      left *= (double)n[k - 1];
      double right = 1.0;
      for (int q = k; q < d; ++q) right *= (double)n[q];
      rS[k] = (int64_t)std::min<double>((double)r_sol, std::min(left, right));
      lS[k] = (int64_t)std::min<double>((double)(rS[k] + 20), left);
    }
    Xv.d = Yv.d = d;
    for (int k = 0; k <= d; ++k) { Xv.r[k] = rS[k]; Yv.r[k] = lS[k]; }
    for (int k = 0; k < d; ++k) {
      Xv.n[k] = Yv.n[k] = n[k];
      const int64_t cx = rS[k] * n[k] * rS[k + 1], cy = lS[k] * n[k] * lS[k + 1];
      Xv.core[k] = ar.take<double>(cx);
      Yv.core[k] = ar.take<double>(cy);
      gaussian_fill(Xv.core[k], 1, cx, p.seed, 4096 + (uint64_t)k, 1.0 / std::sqrt((double)cx),
                    c.st);
      gaussian_fill(Yv.core[k], 1, cy, p.seed, 6144 + (uint64_t)k, 1.0 / std::sqrt((double)cy),
                    c.st);
    }
    if (!f64) vs64 = alloc_tt<double>(ar, d, n, vcap.data());
    for (int k = 0; k < d; ++k) { psi_off[k] = ssz; ssz += lS[k] * n[k] * rS[k + 1]; }
    for (int k = 0; k + 1 < d; ++k) { om_off[k] = ssz; ssz += lS[k + 1] * rS[k + 1]; }
    skb = ar.take<double>(ssz * p.maxit);
    comb = ar.take<double>(ssz);
    es = alloc_tt<double>(ar, d, n, rS);
  }
  auto stta_sketch_basis = [&](int i) {
    std::vector<double*> ps(d), os(d, nullptr);
    for (int k = 0; k < d; ++k) ps[k] = skb + (int64_t)i * ssz + psi_off[k];
    for (int k = 0; k + 1 < d; ++k) os[k] = skb + (int64_t)i * ssz + om_off[k];
    if constexpr (std::is_same<T, double>::value) {
      tt_stta_sketch_dev<double>(c64, VS(i), 1.0, 0, Xv, Yv, ps.data(), os.data());
    } else {
      copy_tt(VS(i), vs64, nullptr, 0);
      tt_stta_sketch_dev<double>(c64, vs64, 1.0, 0, Xv, Yv, ps.data(), os.data());
    }
  };
  // x <- Round(x + Omega^+ Psi) in FP64, Psi and Omega combined with y
  auto stta_update_x = [&](int kdone, double final_tol, bool have) {
    stta_combine(skb, ssz, kdone, ydev, comb, c.st);
    std::vector<const double*> ps(d), os(d, nullptr);
    for (int k = 0; k < d; ++k) ps[k] = comb + psi_off[k];
    for (int k = 0; k + 1 < d; ++k) os[k] = comb + om_off[k];
    tt_stta_recover_dev(c64, d, n, rS, lS, ps.data(), os.data(), 1e-12, es.core);
    for (int q = 0; q <= d; ++q) es.r[q] = rS[q];
    std::vector<Term<double>> terms;
    if (have) { terms.emplace_back(); terms.back().X = x; }
    terms.emplace_back();
    terms.back().X = es;
    tt_round_rand_dev<double>(c64, terms, final_tol, r_sol, p.oversample, drm64, xn);
    copy_tt(xn, x, nullptr, 0);
  };

  // ---- right preconditioning (Algorithm 5): w = A P^{-1} v_k, and each
  // cycle's correction P^{-1} Round(sum_i y_i v_i); every application of
  // P^{-1} is rounded to the basis (or solution) rank cap
  const bool use_pre = p.pre != nullptr;
  TT_CHECK_ARG(!(use_pre && use_stta), "solve: preconditioning with final_stta is not supported");
  PrecondDev<T> pd;
  std::vector<TTv<T>> pbufs;
  TTv<T> z, e2;
  if (use_pre) {
    precond_setup<T>(c, *p.pre, d, n, pd);
    std::vector<int64_t> pcap(d + 1);
    for (int k = 0; k <= d; ++k) pcap[k] = std::max(vcap[k], xcap[k]);
    for (int i = 0; i < pd.zeta; ++i) pbufs.push_back(alloc_tt<T>(ar, d, n, pcap.data()));
    z = alloc_tt<T>(ar, d, n, vcap.data());
    e2 = alloc_tt<T>(ar, d, n, xcap.data());
  }

  // ---- side stream: an iteration's inner products <w, v_i> and its sketch
  // S w run on a second stream, concurrently with the rounding's
  // right-to-left partial contractions and its left-to-right QR sweep (FP64
  // latency-bound work that leaves most of the GPU idle).  They take their
  // temporaries from a slice of their own and their split-K sums from a
  // scratch of their own; events order them before the rounding's left sweep
  // (the coefficients) and before the least squares (the sketch column).
  int64_t wmax = 1, vmax = 1, nmax = 1;
  for (int k = 0; k <= d; ++k) {
    wmax = std::max(wmax, wcap[k]);
    vmax = std::max(vmax, vcap[k]);
  }
  for (int k = 0; k < d; ++k) nmax = std::max(nmax, n[k]);
  const size_t side_bytes =
      sizeof(T) * (size_t)(2 * s * wmax + wmax * nmax * vmax + 2 * wmax * vmax) + 8 * 256;
  Arena ar_side(ar.take<char>((int64_t)side_bytes), side_bytes, g_dry_run);
  void* side_split = ar.take<char>((int64_t)GEMM_SCRATCH_BYTES);
  // Not used when independent solves already share the GPU (the batched
  // worker pool): there the other solves fill it, and the extra streams only
  // add scheduling work.
  const bool use_side = !g_dry_run && !g_qr_narrow;
  SideStream side;
  if (use_side) side.create();
  Ctx cs = c;
  cs.ar = &ar_side;
  if (use_side) cs.st = side.st;

  if (g_dry_run) {
    // workspace query: run every scratch-using step once at capacity ranks
    for (auto& v : V) for (int q = 0; q <= d; ++q) v.r[q] = vcap[q];
    for (int q = 0; q <= d; ++q) { w.r[q] = wcap[q]; x.r[q] = e.r[q] = xcap[q]; }
    tt_dot_dev<double>(Ctx{TT_MODE_FP64, c.st, c.ar, c.err, c.scratch}, b, b, scal + 8);
    tt_sketch_dev<T>(c, w, s, (const T* const*)S.data(), Wm);
    tt_dot_dev<T>(c, w, V[0], scal + 1);
    std::vector<Term<T>> t2(1 + ell);
    t2[0].X = w;
    for (int i = 0; i < ell; ++i) t2[1 + i].X = V[i];
    tt_round_rand_dev<T>(c, t2, 0.1, p.rmax, p.oversample, drm, V[ell]);
    if (!use_stta) {
      std::vector<Term<T>> tk(p.maxit);
      for (int i = 0; i < p.maxit; ++i) tk[i].X = V[i];
      tt_round_rand_dev<T>(c, tk, 0.1, r_sol, p.oversample, drm, e);
    }
    for (int q = 0; q <= d; ++q) { e64.r[q] = xcap[q]; w64.r[q] = wcap[q]; }
    std::vector<Term<double>> u2(2);
    u2[0].X = x; u2[1].X = e64;
    tt_round_rand_dev<double>(c64, u2, 0.1, r_sol, p.oversample, drm64, xn);
    true_residual_norm<double>(c, A64, b, x);
    u2[0].X = b; u2[1].X = w64;
    tt_round_rand_dev<double>(c64, u2, 0.1, p.rmax, p.oversample, drm64, r64);
    if (use_stta) {
      stta_sketch_basis(0);
      stta_update_x(p.maxit, 0.1, true);
    }
    if (use_pre) {
      precond_apply_dev<T>(c, pd, V[0], 0.1, p.rmax, p.oversample, drm, pbufs, z);
      precond_apply_dev<T>(c, pd, e, 0.1, r_sol, p.oversample, drm, pbufs, e2);
    }
    return res;
  }
  // ||b|| in FP64 by the Gram sweep
  tt_dot_dev<double>(Ctx{TT_MODE_FP64, c.st, c.ar, c.err, c.scratch}, b, b, scal + 8);
  const double b2 = read_double(c.st, scal + 8);
  const double bn = std::sqrt(std::max(b2, 0.0));
  TT_CHECK_ARG(bn > 0.0, "solve: b is zero");

  double rel = 1.0;
  bool have_x = false;
  const TTv<T>* cur_rhs = &bT;
  for (int cyc = 0; cyc <= p.max_restarts; ++cyc) {
    double inner = std::min(0.5, p.stop_safety * p.tol / rel);
    inner = std::max(inner, inner_floor(c.mode));
    const double round_tol = p.round_tol > 0 ? p.round_tol : p.eta * inner;
    const double final_tol = 0.01 * p.tol;
    // v_1 = r0 / ||r0||, S r0, ||S r0||
    tt_dot_dev<T>(c, *cur_rhs, *cur_rhs, scal + 0);
    sqrt_scalar(scal + 0, scal + 0, c.st);
    copy_tt(*cur_rhs, V[0], scal + 0, 1);
    tt_sketch_dev<T>(c, *cur_rhs, s, (const T* const*)S.data(), Sr0);
    sumsq(Sr0, 1, s, scal + 5, c.scratch + 16, c.st);
    sqrt_scalar(scal + 5, scal + 6, c.st);
    lstsq_reset(Sr0, s, p.maxit, lsws, c.st);
    const double betaS = read_double(c.st, scal + 6);
    int kdone = 0;
    double sres = 1.0;
    for (int k = 0; k < p.maxit; ++k) {
      if (use_stta) stta_sketch_basis(k);
      // w = A v_k, or A P^{-1} v_k with P^{-1} v_k rounded to rmax
      const TTv<T>* av = &VS(k);
      if (use_pre) {
        precond_apply_dev<T>(c, pd, VS(k), round_tol, p.rmax, p.oversample, drm, pbufs, z);
        av = &z;
      }
      for (int q = 0; q <= d; ++q) w.r[q] = A64.R[q] * av->r[q];
      tt_matvec_dev<T>(c, A, *av, w);
      // side stream: h_{i,k} = <w, v_i> for the last ell basis vectors
      // (Sec. 3.4), then W[:, k] = S w
      if (use_side) {
        TT_CUDA(cudaEventRecord(side.fork, c.st));
        TT_CUDA(cudaStreamWaitEvent(side.st, side.fork, 0));
      }
      void* const main_split = gemm_split_ws();
      const size_t main_split_bytes = gemm_split_bytes();
      set_gemm_scratch(side_split, GEMM_SCRATCH_BYTES);
      const int first = std::max(0, k - ell + 1);
      std::vector<Term<T>> terms(1 + (k - first + 1));
      terms[0].X = w;
      for (int i = first; i <= k; ++i) {
        double* hi = i == k ? scal + 1 : hcoef + i;
        tt_dot_dev<T>(cs, w, VS(i), hi);
        Term<T>& t = terms[1 + i - first];
        t.X = VS(i);
        t.coef = -1.0;
        t.coef_dev = hi;
      }
      if (use_side) TT_CUDA(cudaEventRecord(side.dots, side.st));
      tt_sketch_dev<T>(cs, w, s, (const T* const*)S.data(), Wm + k * s);
      if (use_side) TT_CUDA(cudaEventRecord(side.sketch, side.st));
      set_gemm_scratch(main_split, main_split_bytes);
      // v~ = Round(w - sum_i h_{i,k} v_i): its partial contractions start at
      // once, its left sweep waits for the coefficients
      Ctx cr = c;
      cr.left_wait = use_side ? side.dots : nullptr;
      tt_round_rand_dev<T>(cr, terms, round_tol, p.rmax, p.oversample, drm, VS(k + 1));
      // h_{k+1,k} = ||v~||: the norm of core 1 when cores 2..d are
      // right-orthogonal (FP64 mode), otherwise the Gram sweep
      if (f64) sumsq(VS(k + 1).core[0], f64, VS(k + 1).core_elems(0), scal + 2, c.scratch + 16, c.st);
      else tt_dot_dev<T>(c, VS(k + 1), VS(k + 1), scal + 2);
      sqrt_scalar(scal + 2, scal + 3, c.st);
      {
        CopySeg sg;
        sg.src = VS(k + 1).core[0]; sg.dst = VS(k + 1).core[0]; sg.A = VS(k + 1).core_elems(0);
        sg.sa = 1; sg.src_f64 = f64; sg.dst_f64 = f64; sg.scale_dev = scal + 3; sg.scale_dev_inv = 1;
        copy3d({sg}, c.st);
      }
      if (use_side) TT_CUDA(cudaStreamWaitEvent(c.st, side.sketch, 0));
      lstsq_add_column(Wm, Sr0, s, k, p.maxit, lsws, ydev, scal + 4, c.st);
      // scal[1..4]: h_{k,k}, ||v~||^2, ||v~|| = h_{k+1,k}, sketched residual
      double hs4[4] = {0.0, 1.0, 1.0, 1.0};
      if (!g_dry_run) {
        TT_CUDA(cudaMemcpyAsync(hs4, scal + 1, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
        TT_CUDA(cudaStreamSynchronize(c.st));
      }
      const double hv[2] = {hs4[2], hs4[3]};
      sres = betaS > 0 ? hv[1] / betaS : 0.0;
      res.res_hist.push_back(sres);
      res.rank_hist.push_back(VS(k + 1).max_rank());
      res.max_rank = std::max(res.max_rank, VS(k + 1).max_rank());
      kdone = k + 1;
      ++res.iters;
      // h_{k+1,k} = 0 to working precision: ||v~|| at the rounding level of
      // ||w|| = sqrt(h_{k,k}^2 + h_{k+1,k}^2) (the d core contractions of A v_k
      // and its rounding each contribute a few units of roundoff).  The Krylov
      // space is then invariant under A, so the least-squares solution of this
      // cycle is exact in it (a breakdown), and the new direction would be
      // rounding noise.
      const double u_work = f64 ? 0x1p-53 : 0x1p-24;
      const double wn = std::sqrt(hs4[0] * hs4[0] + hv[0] * hv[0]);
      if (hv[0] <= 16.0 * d * u_work * wn) {
        ++res.breakdowns;
        break;
      }
      if (hv[1] <= inner * betaS) break;
      // stagnation: less than 10% progress over the last 10 iterations ends the
      // cycle (the restart continues from the true residual)
      const size_t nh = res.res_hist.size();
      if (kdone >= 20 && res.res_hist[nh - 1] > 0.9 * res.res_hist[nh - 11]) break;
    }
    if (use_stta) {
      stta_update_x(kdone, final_tol, have_x);
      have_x = true;
    } else {
    // e = Round(sum_i y_i v_i)
    {
      std::vector<Term<T>> terms(kdone);
      for (int i = 0; i < kdone; ++i) {
        terms[i].X = V[i];
        terms[i].coef = 1.0;
        terms[i].coef_dev = ydev + i;
      }
      tt_round_rand_dev<T>(c, terms, final_tol, r_sol, p.oversample, drm, e);
    }
    // right preconditioning: the correction is P^{-1} e
    TTv<T>* ec = &e;
    if (use_pre) {
      precond_apply_dev<T>(c, pd, e, final_tol, r_sol, p.oversample, drm, pbufs, e2);
      ec = &e2;
    }
    // x <- Round(x + e) in FP64
    if (!have_x) {
      copy_tt(*ec, x, nullptr, 0);
      have_x = true;
    } else {
      copy_tt(*ec, e64, nullptr, 0);
      std::vector<Term<double>> terms(2);
      terms[0].X = x;
      terms[1].X = e64;
      tt_round_rand_dev<double>(c64, terms, final_tol, r_sol, p.oversample, drm64, xn);
      copy_tt(xn, x, nullptr, 0);
    }
    }
    res.cycles = cyc + 1;
    res.sketched_res = sres;
    rel = true_residual_norm<double>(c, A64, b, x) / bn;
    res.true_res = rel;
    if (std::getenv("TTSG_DEBUG"))
      std::fprintf(stderr, "[ttsg] cycle %d: %d its, sketched %.3e (target %.1e), true %.3e, "
                   "x max rank %lld\n", cyc, kdone, sres, inner, rel, (long long)x.max_rank());
    if (rel <= p.tol) break;
    // next right-hand side: Round(b - A x), formed and rounded in FP64
    for (int q = 0; q <= d; ++q) w64.r[q] = A64.R[q] * x.r[q];
    tt_matvec_dev<double>(c64, A64, x, w64);
    std::vector<Term<double>> terms(2);
    terms[0].X = b;
    terms[1].X = w64;
    terms[1].coef = -1.0;
    const double next_inner = std::max(std::min(0.5, p.stop_safety * p.tol / rel),
                                       inner_floor(c.mode));
    tt_round_rand_dev<double>(c64, terms, std::max(0.1 * next_inner, 1e-14), vcap_r,
                              p.oversample, drm64, r64);
    copy_tt(r64, rhs, nullptr, 0);
    cur_rhs = &rhs;
  }
  // output in FP64
  {
    std::vector<CopySeg> segs;
    xout.d = d;
    for (int k = 0; k < d; ++k) {
      CopySeg sg;
      sg.src = x.core[k]; sg.dst = xout.core[k]; sg.A = x.core_elems(k); sg.sa = 1;
      sg.src_f64 = 1; sg.dst_f64 = 1;
      segs.push_back(sg);
      xout.r[k] = x.r[k];
      xout.n[k] = n[k];
    }
    xout.r[d] = 1;
    copy3d(segs, c.st);
    if (!g_dry_run) TT_CUDA(cudaStreamSynchronize(c.st));
  }
  if (!g_dry_run) {
    int flags[6] = {0, 0, 0, 0, 0, 0};
    TT_CUDA(cudaMemcpy(flags, c.err, sizeof(flags), cudaMemcpyDeviceToHost));
    res.svd_nonconverged = flags[1];
    res.svd_max_sweeps = flags[3];
    res.svd_mean_sweeps = flags[5] > 0 ? (double)flags[4] / flags[5] : 0.0;
  }
  res.status = res.true_res <= p.tol ? TT_OK
               : (res.breakdowns > 0 ? TT_ERR_BREAKDOWN : TT_ERR_NOT_CONVERGED);
  res.seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return res;
}

template SolveResult sgmres_solve<float>(const Ctx&, const TTop<double>&, const TTv<double>&,
                                         const SolveParams&, TTv<double>&);
template SolveResult sgmres_solve<double>(const Ctx&, const TTop<double>&, const TTv<double>&,
                                          const SolveParams&, TTv<double>&);

}  // namespace ttsg
