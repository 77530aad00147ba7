// TT operations of one TT-sGMRES iteration mapped onto grouped GEMMs, the
// FP64 Householder QR and the small Jacobi SVD.
//
// Index conventions: cores are compact [r_{k-1}][n_k][r_k]; the working
// operator layout is [a][i][a'][j] (input index innermost).  An implicit sum
// of terms is never materialised: every sweep processes the terms' cores block
// by block, and the blocks of a bond are concatenated along the rank index
// (offset off_b of term b).
#include "tt_ops.cuh"

namespace ttsg {

namespace {
template <typename T>
constexpr int f64_of() { return sizeof(T) == 8 ? 1 : 0; }

// Truncation factors from the Jacobi output V (l x l, row-major, columns =
// left singular vectors) and sigma: A = diag(1/sigma_r) V[:, :r]^T (r x l) and
// B = V[:, :r] diag(sigma_r) (l x r); B A is the projector on the kept directions.
template <typename T>
__global__ void trunc_factors_kernel(const double* V, const double* sigma, int l, int r, T* A,
                                     T* B) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * r; e += gridDim.x * blockDim.x) {
    const int i = e / r, j = e % r;
    const double v = V[(size_t)i * l + j], sg = sigma[j];
    A[(size_t)j * l + i] = (T)(sg > 0.0 ? v / sg : 0.0);
    B[(size_t)i * r + j] = (T)(v * sg);
  }
}

int read_int(const Ctx& c, const int* dev) {
  if (g_dry_run) return 1;
  int h = 0;
  TT_CUDA(cudaMemcpyAsync(&h, dev, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  TT_CUDA(cudaStreamSynchronize(c.st));
  return h;
}
}  // namespace

void check_device_flags(const Ctx& c) {
  if (g_dry_run) return;
  const int h = read_int(c, c.err);
  if (h & 1) throw Error(TT_ERR_TIMEOUT, "a grid barrier of the FP64 QR timed out");
  if (h & 4) throw Error(TT_ERR_TIMEOUT, "an mbarrier wait of a tensor-core kernel timed out");
}

// ------------------------------------------------------------------ matvec
// G_k[(a,l), i, (a',l')] = sum_j D_k[a,i,j,a'] C_k[l,j,l'] as a GEMM per
// (a, l): rows (i, a'), columns l', reduction over j.
template <typename T>
void tt_matvec_dev(const Ctx& c, const TTop<T>& A, const TTv<T>& x, const TTv<T>& y) {
  std::vector<GemmProblem> ps;
  if ((c.mode == TT_MODE_TF32 || c.mode == TT_MODE_BF16) && sizeof(T) == 4) {
    // tensor cores: Ct_k[l][l'][j] = C_k[l][j][l'] for every core (one copy
    // launch), then one tcgen05 launch for all of them
    const size_t mk = c.ar->mark();
    std::vector<CopySeg> segs;
    std::vector<TcCoreArgs> tc;
    for (int k = 0; k < x.d; ++k) {
      const int64_t n = x.n[k], R0 = A.R[k], R1 = A.R[k + 1], r0 = x.r[k], r1 = x.r[k + 1];
      if (!matvec_tc_supported(n, r1)) continue;
      float* Ct = c.ar->take<float>(r0 * r1 * n);
      CopySeg sg;
      sg.src = x.core[k]; sg.dst = Ct; sg.A = r0; sg.B = r1; sg.C = n;
      sg.sa = n * r1; sg.sb = 1; sg.sc = r1;
      segs.push_back(sg);
      tc.push_back(TcCoreArgs{(const float*)A.core[k], Ct, (float*)y.core[k], n, R0, R1, r0, r1});
    }
    copy3d(segs, c.st);
    matvec_tc_cores(tc, c.err, c.st, c.mode == TT_MODE_BF16);
    c.ar->release(mk);
    for (int k = 0; k < x.d; ++k) {
      if (matvec_tc_supported(x.n[k], x.r[k + 1])) continue;
      const int64_t n = x.n[k], R0 = A.R[k], R1 = A.R[k + 1], r0 = x.r[k], r1 = x.r[k + 1];
      GemmProblem g;
      g.M = (int)(n * R1); g.N = (int)r1; g.K = (int)n; g.nb1 = (int)R0; g.nb2 = (int)r0;
      g.A = A.core[k]; g.sAm = n; g.sAk = 1; g.sAb1 = n * R1 * n; g.sAb2 = 0;
      g.B = x.core[k]; g.sBk = r1; g.sBn = 1; g.sBb1 = 0; g.sBb2 = n * r1;
      g.C = y.core[k]; g.sCm = r1; g.sCn = 1; g.sCb1 = r0 * n * R1 * r1; g.sCb2 = n * R1 * r1;
      ps.push_back(g);
    }
    gemm(c.mode, ps, c.st);
    return;
  }
  for (int k = 0; k < x.d; ++k) {
    const int64_t n = x.n[k], R0 = A.R[k], R1 = A.R[k + 1], r0 = x.r[k], r1 = x.r[k + 1];
    GemmProblem g;
    g.M = (int)(n * R1); g.N = (int)r1; g.K = (int)n; g.nb1 = (int)R0; g.nb2 = (int)r0;
    g.A = A.core[k]; g.sAm = n; g.sAk = 1; g.sAb1 = n * R1 * n; g.sAb2 = 0;
    g.B = x.core[k]; g.sBk = r1; g.sBn = 1; g.sBb1 = 0; g.sBb2 = n * r1;
    g.C = y.core[k]; g.sCm = r1; g.sCn = 1; g.sCb1 = r0 * n * R1 * r1; g.sCb2 = n * R1 * r1;
    ps.push_back(g);
  }
  gemm(c.mode, ps, c.st);
}

// ------------------------------------------------------------------ sketch
// Z_k[j, :] = sum_{p,i} (Z_{k-1}[j,p] S_k[j,i]) C_k[p,i,:]: a GEMM whose
// A operand is the row-wise Khatri-Rao product of Z_{k-1} and S_k.
template <typename T>
void tt_sketch_dev(const Ctx& c, const TTv<T>& x, int64_t s, const T* const* S, double* out) {
  const size_t mk = c.ar->mark();
  const int64_t rmax = x.max_rank();
  T* Z[2] = {c.ar->take<T>(s * rmax), c.ar->take<T>(s * rmax)};
  const T* Zprev = nullptr;
  for (int k = 0; k < x.d; ++k) {
    GemmProblem g;
    g.M = (int)s; g.N = (int)x.r[k + 1]; g.K = (int)(x.r[k] * x.n[k]);
    g.a_mode = 1; g.A = Zprev; g.sAm = x.r[k]; g.sAk = 1;
    g.kr_S = S[k]; g.kr_n = (int)x.n[k]; g.kr_sS = x.n[k];
    g.B = x.core[k]; g.sBk = x.r[k + 1]; g.sBn = 1;
    g.C = Z[k & 1]; g.sCm = x.r[k + 1]; g.sCn = 1;
    gemm(c.mode, {g}, c.st);
    Zprev = Z[k & 1];
  }
  CopySeg cs;
  cs.src = Zprev; cs.dst = out; cs.A = s; cs.sa = 1; cs.src_f64 = f64_of<T>(); cs.dst_f64 = 1;
  copy3d({cs}, c.st);
  c.ar->release(mk);
}

// --------------------------------------------------------------------- dot
// Gram sweep Z_k = sum_i X_k[:,i,:]^T Z_{k-1} Y_k[:,i,:]:
// U = Z_{k-1} Y_k (t x n q'), then Z_k = X_k^T U with reduction over (p, i).
template <typename T>
void tt_dot_dev(const Ctx& c, const TTv<T>& x, const TTv<T>& y, double* out) {
  const size_t mk = c.ar->mark();
  int64_t tmax = x.max_rank(), qmax = y.max_rank(), nmax = 0;
  for (int k = 0; k < x.d; ++k) nmax = std::max(nmax, x.n[k]);
  T* U = c.ar->take<T>(tmax * nmax * qmax);
  T* Z[2] = {c.ar->take<T>(tmax * qmax), c.ar->take<T>(tmax * qmax)};
  const T* Zc = nullptr;
  for (int k = 0; k < x.d; ++k) {
    const int64_t t0 = x.r[k], t1 = x.r[k + 1], q0 = y.r[k], q1 = y.r[k + 1], n = x.n[k];
    const T* Uk = y.core[k];
    if (k > 0) {
      GemmProblem g = gemm_rm((int)t0, (int)(n * q1), (int)q0, Zc, q0, y.core[k], n * q1, U, n * q1);
      gemm(c.mode, {g}, c.st);
      Uk = U;
    }
    GemmProblem g;
    g.M = (int)t1; g.N = (int)q1; g.K = (int)(t0 * n);
    g.A = x.core[k]; g.sAm = 1; g.sAk = t1;
    g.B = Uk; g.sBk = q1; g.sBn = 1;
    g.C = Z[k & 1]; g.sCm = q1; g.sCn = 1;
    gemm(c.mode, {g}, c.st);
    Zc = Z[k & 1];
  }
  CopySeg cs;
  cs.src = Zc; cs.dst = out; cs.A = 1; cs.src_f64 = f64_of<T>(); cs.dst_f64 = 1;
  copy3d({cs}, c.st);
  c.ar->release(mk);
}

// ------------------------------------------------------ randomized rounding
void rto_ranks(const std::vector<const int64_t*>& term_ranks, const int64_t* n, int d,
               int64_t rmax, int64_t oversample, int64_t* ells) {
  ells[0] = 1;
  for (int mu = 1; mu < d; ++mu) {
    int64_t t = 0;
    for (auto r : term_ranks) t += r[mu];
    double right = 1.0;
    for (int k = mu; k < d; ++k) right *= (double)n[k];
    int64_t l = std::min<int64_t>(rmax + oversample, t);
    l = std::min<int64_t>(l, ells[mu - 1] * n[mu - 1]);
    if (right < (double)l) l = (int64_t)right;
    ells[mu] = l;
  }
  ells[d] = 1;
}

template <typename T>
void tt_round_rand_dev(const Ctx& c, const std::vector<Term<T>>& terms, double eps, int64_t rmax,
                       int64_t oversample, const DRMSource<T>& drm, TTv<T>& y) {
  const int d = terms[0].X.d;
  const int nb = (int)terms.size();
  TT_CHECK_ARG(d >= 2, "tt_round_rand: d >= 2 required");
  TT_CHECK_ARG(rmax >= 1 && oversample >= 0, "tt_round_rand: rmax >= 1, oversample >= 0");
  const int64_t* n = terms[0].X.n;
  std::vector<const int64_t*> tr;
  for (auto& t : terms) tr.push_back(t.X.r);
  int64_t ell[MAXD + 1];
  rto_ranks(tr, n, d, rmax, oversample, ell);
  // concatenated rank per bond and the term offsets
  std::vector<std::vector<int64_t>> off(nb, std::vector<int64_t>(d + 1, 0));
  std::vector<int64_t> Ts(d + 1, 0);
  for (int mu = 0; mu <= d; ++mu) {
    int64_t o = 0;
    for (int b = 0; b < nb; ++b) { off[b][mu] = o; o += terms[b].X.r[mu]; }
    Ts[mu] = o;
  }
  const size_t mk = c.ar->mark();
  const int f64 = f64_of<T>();
  Arena& ar = *c.ar;

  // 1. compact DRM cores R_k: [ell_k][n_k][ell_{k+1}]
  std::vector<T*> R(d);
  for (int k = 0; k < d; ++k) R[k] = ar.take<T>(ell[k] * n[k] * ell[k + 1]);
  if (drm.core) {
    std::vector<CopySeg> segs;
    for (int k = 0; k < d; ++k) {
      TT_CHECK_ARG(drm.L[k] >= ell[k] && drm.L[k + 1] >= ell[k + 1],
                   "tt_round_rand: DRM ranks smaller than the sketch ranks");
      CopySeg s;
      s.src = drm.core[k]; s.dst = R[k]; s.A = ell[k]; s.B = n[k]; s.C = ell[k + 1];
      s.sa = n[k] * drm.L[k + 1]; s.sb = drm.L[k + 1]; s.sc = 1; s.src_f64 = f64; s.dst_f64 = f64;
      segs.push_back(s);
    }
    copy3d(segs, c.st);
  } else {
    for (int k = 0; k < d; ++k) {
      TT_CHECK_ARG(drm.L[k] >= ell[k] && drm.L[k + 1] >= ell[k + 1],
                   "tt_round_rand: DRM capacity smaller than the sketch ranks");
      const double sd = 1.0 / std::sqrt((double)drm.L[k] * n[k] * drm.L[k + 1]);
      gaussian_subblock(R[k], f64, ell[k], n[k], ell[k + 1], drm.L[k + 1], drm.seed,
                        2048 + (uint64_t)k, sd, c.st);
    }
  }

  // 2. right partial contractions, stacked per bond: Wc[mu] is Ts[mu] x ell[mu]
  std::vector<T*> Wc(d + 1, nullptr);
  for (int mu = 1; mu < d; ++mu) Wc[mu] = ar.take<T>(Ts[mu] * ell[mu]);
  std::vector<T*> T1(nb);
  for (int b = 0; b < nb; ++b) {
    int64_t mx = 1;
    for (int mu = 2; mu < d; ++mu)
      mx = std::max(mx, terms[b].X.r[mu - 1] * n[mu - 1] * ell[mu]);
    T1[b] = ar.take<T>(mx);
  }
  for (int mu = d; mu >= 2; --mu) {  // core mu (1-based) -> W at bond mu-1
    const int k = mu - 1;
    const int64_t nn = n[k];
    if (mu == d) {
      std::vector<GemmProblem> ps;
      for (int b = 0; b < nb; ++b) {
        const TTv<T>& X = terms[b].X;
        GemmProblem g;
        g.M = (int)X.r[k]; g.K = (int)nn; g.N = (int)ell[k];
        g.A = X.core[k]; g.sAm = nn; g.sAk = 1;
        g.B = R[k]; g.sBk = 1; g.sBn = nn;
        g.C = Wc[k] + off[b][k] * ell[k]; g.sCm = ell[k]; g.sCn = 1;
        ps.push_back(g);
      }
      gemm(c.mode, ps, c.st);
    } else {
      std::vector<GemmProblem> p1, p2;
      for (int b = 0; b < nb; ++b) {
        const TTv<T>& X = terms[b].X;
        const int64_t t0 = X.r[k], t1 = X.r[k + 1];
        p1.push_back(gemm_rm((int)(t0 * nn), (int)ell[mu], (int)t1, X.core[k], t1,
                             Wc[mu] + off[b][mu] * ell[mu], ell[mu], T1[b], ell[mu]));
        GemmProblem g;
        g.M = (int)t0; g.K = (int)(nn * ell[mu]); g.N = (int)ell[k];
        g.A = T1[b]; g.sAm = nn * ell[mu]; g.sAk = 1;
        g.B = R[k]; g.sBk = 1; g.sBn = nn * ell[mu];
        g.C = Wc[k] + off[b][k] * ell[k]; g.sCm = ell[k]; g.sCn = 1;
        p2.push_back(g);
      }
      gemm(c.mode, p1, c.st);
      gemm(c.mode, p2, c.st);
    }
    // The rounding's result does not depend on the scale of any W: rescale the
    // stacked contractions of this bond by an exact power of two.  Over many
    // cores the Gaussian DRM factors (entries ~ 1/sqrt(l n l)) would otherwise
    // shrink W geometrically, into the subnormal range of FP32 at d = 20.
    pow2_normalize(Wc[k], f64, Ts[k] * ell[k], c.scratch + 256, c.st);
  }

  // 3. left sweep: Z = M x_1 X, Y = Z W, Y = Q R, core <- Q, M = Q^T Z
  if (c.left_wait && !g_dry_run) TT_CUDA(cudaStreamWaitEvent(c.st, c.left_wait, 0));
  int64_t zmax = 1, mmax = 1, ymax = 1;
  for (int mu = 1; mu < d; ++mu) {
    zmax = std::max(zmax, ell[mu - 1] * n[mu - 1] * Ts[mu]);
    mmax = std::max(mmax, ell[mu] * Ts[mu]);
    ymax = std::max(ymax, ell[mu - 1] * n[mu - 1] * ell[mu]);
  }
  T* Zc = ar.take<T>(zmax);
  T* Mc = ar.take<T>(mmax);
  T* Y = ar.take<T>(ymax);
  T* Xs = ar.take<T>(Ts[d - 1] * n[d - 1]);
  std::vector<T*> H(d);
  for (int k = 0; k < d; ++k) H[k] = ar.take<T>(ell[k] * n[k] * ell[k + 1]);
  size_t qws = 0;
  for (int mu = 1; mu < d; ++mu) qws = std::max(qws, qr_workspace(ell[mu - 1] * n[mu - 1], ell[mu]));
  void* qw = ar.take<char>((int64_t)qws);

  for (int mu = 1; mu < d; ++mu) {
    const int k = mu - 1;
    const int64_t nn = n[k], m = ell[k] * nn, Tm = Ts[mu];
    if (mu == 1) {
      std::vector<CopySeg> segs;
      for (int b = 0; b < nb; ++b) {
        const TTv<T>& X = terms[b].X;
        CopySeg s;
        s.src = X.core[0]; s.dst = Zc + off[b][1];
        s.A = nn; s.B = X.r[1]; s.C = 1; s.sa = X.r[1]; s.sb = 1; s.sc = 0;
        s.da = Tm; s.db = 1; s.dc = 0;
        s.scale = terms[b].coef; s.scale_dev = terms[b].coef_dev;
        s.src_f64 = f64; s.dst_f64 = f64;
        segs.push_back(s);
      }
      copy3d(segs, c.st);
    } else {
      std::vector<GemmProblem> ps;
      for (int b = 0; b < nb; ++b) {
        const TTv<T>& X = terms[b].X;
        const int64_t t0 = X.r[k], t1 = X.r[k + 1];
        GemmProblem g;
        g.M = (int)ell[k]; g.K = (int)t0; g.N = (int)t1; g.nb1 = (int)nn;
        g.A = Mc + off[b][k]; g.sAm = Ts[k]; g.sAk = 1; g.sAb1 = 0;
        g.B = X.core[k]; g.sBk = nn * t1; g.sBn = 1; g.sBb1 = t1;
        g.C = Zc + off[b][mu]; g.sCm = nn * Tm; g.sCn = 1; g.sCb1 = Tm;
        ps.push_back(g);
      }
      gemm(c.mode, ps, c.st);
    }
    gemm(c.mode, {gemm_rm((int)m, (int)ell[mu], (int)Tm, Zc, Tm, Wc[mu], ell[mu], Y, ell[mu])},
         c.st);
    qr_f64(Y, f64, m, ell[mu], ell[mu], 1, H[k], f64, ell[mu], nullptr, qw, qws, c.err, c.st);
    GemmProblem g;
    g.M = (int)ell[mu]; g.K = (int)m; g.N = (int)Tm;
    g.A = H[k]; g.sAm = 1; g.sAk = ell[mu];
    g.B = Zc; g.sBk = Tm; g.sBn = 1;
    g.C = Mc; g.sCm = Tm; g.sCn = 1;
    gemm(c.mode, {g}, c.st);
  }
  {  // last core: sum over terms of M^b X^b_d, as one GEMM over the stacked cores
    const int k = d - 1;
    std::vector<CopySeg> segs;
    for (int b = 0; b < nb; ++b) {
      const TTv<T>& X = terms[b].X;
      CopySeg s;
      s.src = X.core[k]; s.dst = Xs + off[b][k] * n[k];
      s.A = X.r[k] * n[k]; s.sa = 1; s.src_f64 = f64; s.dst_f64 = f64;
      segs.push_back(s);
    }
    copy3d(segs, c.st);
    gemm(c.mode, {gemm_rm((int)ell[k], (int)n[k], (int)Ts[k], Mc, Ts[k], Xs, n[k], H[k], n[k])},
         c.st);
  }

  // 4. truncation sweep (right to left) or plain copy
  bool trunc = eps > 0.0;
  for (int mu = 1; mu < d; ++mu) trunc = trunc || ell[mu] > rmax;
  y.d = d;
  for (int k = 0; k < d; ++k) y.n[k] = n[k];
  if (!trunc) {
    std::vector<CopySeg> segs;
    for (int k = 0; k < d; ++k) {
      CopySeg s;
      s.src = H[k]; s.dst = y.core[k]; s.A = ell[k] * n[k] * ell[k + 1]; s.sa = 1;
      s.src_f64 = f64; s.dst_f64 = f64;
      segs.push_back(s);
      y.r[k] = ell[k];
    }
    y.r[d] = 1;
    copy3d(segs, c.st);
    check_device_flags(c);
    ar.release(mk);
    return;
  }
  if (!f64) {
    // Float modes: all bonds truncated from the same left-orthogonal tensor.
    // Right Gram matrices G_b = C_{>b}^T C_{>b} (one sweep), their
    // eigenvectors W_b by batched FP64 Cholesky + Jacobi (one CTA per bond),
    // then core k <- W_k^T H_k W_{k+1}.  The error is at most the sum of the
    // dropped tails, so each bond uses delta = eps ||T|| / (d - 1).
    std::vector<T*> Gk(d + 1, nullptr);
    std::vector<double*> Gd(d + 1, nullptr), Rd(d + 1, nullptr), Vd(d + 1, nullptr),
        GVd(d + 1, nullptr), sg(d + 1, nullptr);
    int64_t t1max = 1;
    for (int b = 1; b < d; ++b) {
      Gk[b] = ar.take<T>(ell[b] * ell[b]);
      Gd[b] = ar.take<double>(ell[b] * ell[b]);
      Rd[b] = ar.take<double>(ell[b] * ell[b]);
      Vd[b] = ar.take<double>(ell[b] * ell[b]);
      GVd[b] = ar.take<double>(ell[b] * ell[b]);
      sg[b] = ar.take<double>(ell[b]);
      if (b < d - 1) t1max = std::max(t1max, ell[b] * n[b] * ell[b + 1]);
    }
    T* T1g = ar.take<T>(t1max);
    int* rks = ar.take<int>(d + 1);
    {  // G_{d-1} = H_{d-1} H_{d-1}^T
      const int b = d - 1;
      GemmProblem g;
      g.M = (int)ell[b]; g.N = (int)ell[b]; g.K = (int)n[b];
      g.A = H[b]; g.sAm = n[b]; g.sAk = 1;
      g.B = H[b]; g.sBk = 1; g.sBn = n[b];
      g.C = Gk[b]; g.sCm = ell[b]; g.sCn = 1;
      gemm(c.mode, {g}, c.st);
    }
    for (int b = d - 2; b >= 1; --b) {
      const int64_t nb = n[b], l0 = ell[b], l1 = ell[b + 1];
      gemm(c.mode, {gemm_rm((int)(l0 * nb), (int)l1, (int)l1, H[b], l1, Gk[b + 1], l1, T1g, l1)},
           c.st);
      GemmProblem g;
      g.M = (int)l0; g.N = (int)l0; g.K = (int)(nb * l1);
      g.A = T1g; g.sAm = nb * l1; g.sAk = 1;
      g.B = H[b]; g.sBk = 1; g.sBn = nb * l1;
      g.C = Gk[b]; g.sCm = l0; g.sCn = 1;
      gemm(c.mode, {g}, c.st);
    }
    {
      std::vector<CopySeg> segs;
      for (int b = 1; b < d; ++b) {
        CopySeg sgm;
        sgm.src = Gk[b]; sgm.dst = Gd[b]; sgm.A = ell[b] * ell[b]; sgm.sa = 1;
        sgm.src_f64 = 0; sgm.dst_f64 = 1;
        segs.push_back(sgm);
      }
      copy3d(segs, c.st);
    }
    chol_f64_batched(d - 1, (const double* const*)&Gd[1], &ell[1], 1e-14, &Rd[1], c.err + 2,
                     c.st);
    JacobiBatchArgs ja;
    ja.count = d - 1; ja.trans = 0; ja.f32 = 1; ja.eps = eps;
    ja.dm1 = (int64_t)(d - 1) * (d - 1);  // delta = eps ||T|| / (d - 1)
    ja.rmax = rmax; ja.err = c.err + 1;
    for (int b = 1; b < d; ++b) {
      ja.G[b - 1] = Rd[b]; ja.l[b - 1] = ell[b]; ja.GV[b - 1] = GVd[b]; ja.V[b - 1] = Vd[b];
      ja.sigma[b - 1] = sg[b]; ja.rank_out[b - 1] = rks + b;
      ja.vtmp[b - 1] = Gd[b];  // the FP64 Gram is consumed by the Cholesky factorisation
    }
    jacobi_svd_batched(ja, c.st);
    // one host read for the ranks and the error word (only the QRs and the
    // tensor-core kernels set error bits, and they have all run by now)
    std::vector<int> rh(d + 1, 1);
    int flags = 0;
    if (!g_dry_run) {
      TT_CUDA(cudaMemcpyAsync(rh.data() + 1, rks + 1, sizeof(int) * (d - 1), cudaMemcpyDeviceToHost,
                              c.st));
      TT_CUDA(cudaMemcpyAsync(&flags, c.err, sizeof(int), cudaMemcpyDeviceToHost, c.st));
      TT_CUDA(cudaStreamSynchronize(c.st));
    }
    if (flags & 1) throw Error(TT_ERR_TIMEOUT, "a grid barrier of the FP64 QR timed out");
    if (flags & 4) throw Error(TT_ERR_TIMEOUT, "an mbarrier wait of a tensor-core kernel timed out");
    rh[0] = rh[d] = 1;
    // W_b = V_b[:, :r_b] in the working precision
    // (buffers sized by the rank caps min(l_b, rmax), so that the workspace
    // query, which cannot see the ranks, reserves the same bytes)
    std::vector<T*> W(d + 1, nullptr);
    {
      std::vector<CopySeg> segs;
      for (int b = 1; b < d; ++b) {
        W[b] = ar.take<T>(ell[b] * std::min(ell[b], rmax));
        CopySeg sgm;
        sgm.src = Vd[b]; sgm.dst = W[b]; sgm.A = ell[b]; sgm.B = rh[b]; sgm.C = 1;
        sgm.sa = ell[b]; sgm.sb = 1; sgm.src_f64 = 1; sgm.dst_f64 = 0;
        segs.push_back(sgm);
      }
      copy3d(segs, c.st);
    }
    // U_k = H_k W_{k+1} ((ell_k n_k) x r_{k+1}); core k = W_k^T U_k
    std::vector<T*> U(d, nullptr);
    std::vector<GemmProblem> p1, p2;
    for (int k = 0; k < d - 1; ++k) {
      U[k] = (k == 0) ? y.core[0] : ar.take<T>(ell[k] * n[k] * std::min(ell[k + 1], rmax));
      p1.push_back(gemm_rm((int)(ell[k] * n[k]), rh[k + 1], (int)ell[k + 1], H[k], ell[k + 1],
                           W[k + 1], rh[k + 1], U[k], rh[k + 1]));
    }
    for (int k = 1; k < d; ++k) {
      const T* Uk = (k == d - 1) ? H[d - 1] : U[k];
      const int64_t cols = n[k] * rh[k + 1];
      GemmProblem g;
      g.M = rh[k]; g.N = (int)cols; g.K = (int)ell[k];
      g.A = W[k]; g.sAm = 1; g.sAk = rh[k];
      g.B = Uk; g.sBk = cols; g.sBn = 1;
      g.C = y.core[k]; g.sCm = cols; g.sCn = 1;
      p2.push_back(g);
    }
    gemm(c.mode, p1, c.st);
    gemm(c.mode, p2, c.st);
    for (int k = 0; k <= d; ++k) y.r[k] = rh[k];
    ar.release(mk);
    return;
  }
  int64_t lmax = 1, hmax = 1, qtmax = 1;
  for (int k = 0; k <= d; ++k) lmax = std::max(lmax, ell[k]);
  for (int k = 0; k < d; ++k) hmax = std::max(hmax, ell[k] * n[k] * ell[k + 1]);
  for (int k = 0; k < d; ++k) qtmax = std::max(qtmax, n[k] * ell[k + 1] * ell[k]);
  double* Rf = ar.take<double>(lmax * lmax);
  double* GV = ar.take<double>(lmax * lmax);
  double* Vd = ar.take<double>(lmax * lmax);
  double* sig = ar.take<double>(lmax);
  T* GVt = ar.take<T>(lmax * lmax);
  T* Vt = ar.take<T>(lmax * lmax);
  T* Qt = ar.take<T>(qtmax);
  T* Pb = ar.take<T>(lmax * lmax);
  T* cur2[2] = {ar.take<T>(hmax), ar.take<T>(hmax)};
  double* nrm = ar.take<double>(1);
  int* rk = ar.take<int>(1);
  size_t qws2 = 0;
  for (int k = 1; k < d; ++k) {
    const int64_t a = ell[k], bcols = n[k] * ell[k + 1];
    qws2 = std::max(qws2, qr_workspace(std::max(a, bcols), std::min(a, bcols)));
  }
  void* qw2 = ar.take<char>((int64_t)qws2);
  const int f32svd = f64 ? 0 : 1;
  // float modes: Gram X X^T + shifted Cholesky replace the QR of the truncation
  double* Gb = ar.take<double>(lmax * lmax);
  size_t gws = 0;
  for (int k = 1; k < d; ++k) gws = std::max(gws, gram_workspace(n[k] * ell[k + 1], ell[k]));
  void* gw = f64 ? nullptr : ar.take<char>((int64_t)gws);
  double* Vs = ar.take<double>(lmax * lmax);  // Jacobi V scratch for large bonds
  double* Pre = ar.take<double>(4 * lmax * lmax);  // FP32 pre-pass of the FP64 Jacobi

  const T* cur = H[d - 1];
  int64_t rr = 1;
  y.r[d] = 1;
  for (int mu = d; mu >= 2; --mu) {
    const int k = mu - 1;
    const int64_t L = ell[k], cc = n[k] * rr;
    const int64_t rows_prev = ell[k - 1] * n[k - 1];
    T* next = (mu - 1 == 1) ? y.core[0] : cur2[mu & 1];
    int r = 0;
    if (!f64) {
      gram_f64(cur, 0, cc, L, 1, cc, Gb, gw, gws, c.st);
      chol_f64(Gb, L, 1e-14, Rf, c.err + 2, c.st);
      jacobi_svd(Rf, L, 0, 1, GV, Vd, sig, eps, d - 1, rmax, mu == d ? nullptr : nrm,
                 mu == d ? nrm : nullptr, rk, c.err + 1, c.st, Vs, Pre);
      r = read_int(c, rk);
      if (!g_dry_run) {
        trunc_factors_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(
                                      ceil_div(L * r, 256), 256)), 256, 0, c.st>>>(
            Vd, sig, (int)L, r, Vt, GVt);
        check_launch("trunc_factors_kernel");
      }
      // core mu = diag(1/sigma_r) U_r^T X (r x cc); core mu-1 = H_{mu-1} U_r diag(sigma_r)
      GemmProblem g = gemm_rm(r, (int)cc, (int)L, Vt, L, cur, cc, y.core[k], cc);
      GemmProblem g2 = gemm_rm((int)rows_prev, r, (int)L, H[k - 1], L, GVt, r, next, r);
      gemm(c.mode, {g, g2}, c.st);
    } else if (cc >= L) {
      // X = cur (L x cc); X^T = Qt R  (Qt: cc x L)
      qr_f64(cur, f64, cc, L, 1, cc, Qt, f64, L, Rf, qw2, qws2, c.err, c.st);
      jacobi_svd(Rf, L, 1, f32svd, GV, Vd, sig, eps, d - 1, rmax, mu == d ? nullptr : nrm,
                 mu == d ? nrm : nullptr, rk, c.err + 1, c.st, Vs, Pre);
      r = read_int(c, rk);
      CopySeg s1, s2;
      s1.src = Vd; s1.dst = Vt; s1.A = L * L; s1.sa = 1; s1.src_f64 = 1; s1.dst_f64 = f64;
      s2 = s1; s2.src = GV; s2.dst = GVt;
      copy3d({s1, s2}, c.st);
      // core mu = U_R[:, :r]^T Qt^T  (r x cc)
      GemmProblem g;
      g.M = r; g.K = (int)L; g.N = (int)cc;
      g.A = Vt; g.sAm = 1; g.sAk = L;
      g.B = Qt; g.sBk = 1; g.sBn = L;
      g.C = y.core[k]; g.sCm = cc; g.sCn = 1;
      // core mu-1 = H_{mu-1} (rows_prev x L) GV[:, :r]
      GemmProblem g2 = gemm_rm((int)rows_prev, r, (int)L, H[k - 1], L, GVt, L, next, r);
      gemm(c.mode, {g, g2}, c.st);
    } else {
      // X = Q2 R2 (Q2: L x cc), R2 V2 = U2 Sigma
      qr_f64(cur, f64, L, cc, cc, 1, Qt, f64, cc, Rf, qw2, qws2, c.err, c.st);
      jacobi_svd(Rf, cc, 0, f32svd, GV, Vd, sig, eps, d - 1, rmax, mu == d ? nullptr : nrm,
                 mu == d ? nrm : nullptr, rk, c.err + 1, c.st, Vs, Pre);
      r = read_int(c, rk);
      CopySeg s1, s2;
      s1.src = Vd; s1.dst = y.core[k]; s1.A = r; s1.B = cc; s1.sa = 1; s1.sb = cc;
      s1.src_f64 = 1; s1.dst_f64 = f64;
      s2.src = GV; s2.dst = GVt; s2.A = cc * cc; s2.sa = 1; s2.src_f64 = 1; s2.dst_f64 = f64;
      copy3d({s1, s2}, c.st);
      // P = Q2 GV[:, :r] (L x r); core mu-1 = H_{mu-1} P
      gemm(c.mode, {gemm_rm((int)L, r, (int)cc, Qt, cc, GVt, cc, Pb, r)}, c.st);
      gemm(c.mode, {gemm_rm((int)rows_prev, r, (int)L, H[k - 1], L, Pb, r, next, r)}, c.st);
    }
    y.r[k] = r;
    rr = r;
    cur = next;
    // the next step reads H[k-1] replaced by ``next``
    H[k - 1] = next;
  }
  y.r[0] = 1;
  check_device_flags(c);
  ar.release(mk);
}

// ------------------------------------------------------------ true residual
template <typename T>
double true_residual_norm(const Ctx& c0, const TTop<double>& A, const TTv<double>& b,
                          const TTv<T>& x) {
  Ctx c = c0;
  c.mode = TT_MODE_FP64;
  Arena& ar = *c.ar;
  const size_t mk = ar.mark();
  const int d = b.d;
  // x in FP64
  TTv<double> xd;
  xd.d = d;
  std::vector<CopySeg> segs;
  for (int k = 0; k < d; ++k) {
    xd.n[k] = x.n[k];
    xd.r[k] = x.r[k];
    xd.core[k] = ar.take<double>(x.core_elems(k));
    CopySeg s;
    s.src = x.core[k]; s.dst = xd.core[k]; s.A = x.core_elems(k); s.sa = 1;
    s.src_f64 = f64_of<T>(); s.dst_f64 = 1;
    segs.push_back(s);
  }
  xd.r[d] = 1;
  copy3d(segs, c.st);
  TTv<double> ax;
  ax.d = d;
  for (int k = 0; k <= d; ++k) ax.r[k] = A.R[k] * xd.r[k];
  for (int k = 0; k < d; ++k) {
    ax.n[k] = b.n[k];
    ax.core[k] = ar.take<double>(ax.core_elems(k));
  }
  tt_matvec_dev(c, A, xd, ax);
  // QR sweep of the explicit sum [b, -Ax]; only R factors are propagated
  const TTv<double>* X[2] = {&b, &ax};
  const double coef[2] = {1.0, -1.0};
  int64_t Ts[MAXD + 1], off[2][MAXD + 1];
  for (int k = 0; k <= d; ++k) {
    off[0][k] = 0;
    off[1][k] = b.r[k];
    Ts[k] = b.r[k] + ax.r[k];
  }
  int64_t zmax = 1;
  for (int k = 0; k < d; ++k) zmax = std::max(zmax, Ts[k] * b.n[k] * Ts[k + 1]);
  double* Zc = ar.take<double>(zmax);
  double* Rm = ar.take<double>(zmax);
  size_t qws = 0;
  for (int k = 0; k < d; ++k) qws = std::max(qws, qr_workspace(Ts[k] * b.n[k], Ts[k + 1]));
  void* qw = ar.take<char>((int64_t)qws);
  int64_t rows = 1;  // row count of the current R factor
  for (int k = 0; k < d; ++k) {
    const int64_t nn = b.n[k];
    const int64_t Tn = (k == d - 1) ? 1 : Ts[k + 1];
    if (k == 0) {
      std::vector<CopySeg> sg;
      for (int t = 0; t < 2; ++t) {
        CopySeg s;
        s.src = X[t]->core[0]; s.dst = Zc + off[t][1];
        s.A = nn; s.B = X[t]->r[1]; s.C = 1; s.sa = X[t]->r[1]; s.sb = 1;
        s.da = Tn; s.db = 1; s.dc = 0; s.scale = coef[t]; s.src_f64 = 1; s.dst_f64 = 1;
        sg.push_back(s);
      }
      copy3d(sg, c.st);
    } else if (k < d - 1) {
      std::vector<GemmProblem> ps;
      for (int t = 0; t < 2; ++t) {
        const int64_t t0 = X[t]->r[k], t1 = X[t]->r[k + 1];
        GemmProblem g;
        g.M = (int)rows; g.K = (int)t0; g.N = (int)t1; g.nb1 = (int)nn;
        g.A = Rm + off[t][k]; g.sAm = Ts[k]; g.sAk = 1;
        g.B = X[t]->core[k]; g.sBk = nn * t1; g.sBn = 1; g.sBb1 = t1;
        g.C = Zc + off[t][k + 1]; g.sCm = nn * Tn; g.sCn = 1; g.sCb1 = Tn;
        ps.push_back(g);
      }
      gemm(c.mode, ps, c.st);
    } else {
      // last core: Z = sum_t R[:, block t] X_t (rows x n)
      GemmProblem g0 = gemm_rm((int)rows, (int)nn, (int)X[0]->r[k], Rm + off[0][k], Ts[k],
                               X[0]->core[k], nn, Zc, nn);
      gemm(c.mode, {g0}, c.st);
      GemmProblem g1 = gemm_rm((int)rows, (int)nn, (int)X[1]->r[k], Rm + off[1][k], Ts[k],
                               X[1]->core[k], nn, Zc, nn, 1.0, 1.0);
      gemm(c.mode, {g1}, c.st);
      sumsq(Zc, 1, rows * nn, c.scratch + 8, c.scratch + 16, c.st);
      break;
    }
    const int64_t m = rows * nn;
    if (m > Tn) {
      qr_f64(Zc, 1, m, Tn, Tn, 1, nullptr, 1, Tn, Rm, qw, qws, c.err, c.st);
      rows = Tn;
    } else {
      // Q = I: the factor is Z itself (m x Tn)
      CopySeg s;
      s.src = Zc; s.dst = Rm; s.A = m * Tn; s.sa = 1; s.src_f64 = 1; s.dst_f64 = 1;
      copy3d({s}, c.st);
      rows = m;
    }
  }
  double h = 0.0;
  if (g_dry_run) { ar.release(mk); return 0.0; }
  TT_CUDA(cudaMemcpyAsync(&h, c.scratch + 8, sizeof(double), cudaMemcpyDeviceToHost, c.st));
  TT_CUDA(cudaStreamSynchronize(c.st));
  check_device_flags(c);
  ar.release(mk);
  return std::sqrt(std::max(h, 0.0));
}

#define INST(T)                                                                                 \
  template void tt_matvec_dev<T>(const Ctx&, const TTop<T>&, const TTv<T>&, const TTv<T>&);     \
  template void tt_sketch_dev<T>(const Ctx&, const TTv<T>&, int64_t, const T* const*, double*);  \
  template void tt_dot_dev<T>(const Ctx&, const TTv<T>&, const TTv<T>&, double*);                \
  template void tt_round_rand_dev<T>(const Ctx&, const std::vector<Term<T>>&, double, int64_t,   \
                                     int64_t, const DRMSource<T>&, TTv<T>&);                     \
  template double true_residual_norm<T>(const Ctx&, const TTop<double>&, const TTv<double>&,     \
                                        const TTv<T>&);
INST(float)
INST(double)

}  // namespace ttsg
