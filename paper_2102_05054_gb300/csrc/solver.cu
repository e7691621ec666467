// Krylov-Schur restarted Arnoldi on the geometric-sum filter g_k(U) (Secs. 3-4 of Luitz,
// arXiv:2102.05054), batched over independent problems that advance in lockstep.
//
// Per restart cycle and problem b:
//   expansion   for j = p .. m-1: w = g_k(U_b) v_j (filter graph), CGS2 against V[:, :j+1]
//               -> H[:j+2, j], v_{j+1};
//   small solve H_m = Y diag(theta) Y^{-1} on the device (descending |theta|, the ARPACK
//               'LM' order the paper uses), Ritz estimates |beta| |e_m^T y|;
//   check       when the top nc >= nev+1 Ritz values are converged: Ritz vectors X = V Y,
//               omega = <x|U|x>, r = ||U x - omega x|| (Eq. residual, FP64 U); the nev
//               in-lobe eigenvalues closest to exp(i phi) are final once the nev-th has
//               |g_k(omega)| above the smallest converged |theta| (every closer eigenvalue
//               has a larger |g_k| and so is among the converged);
//   restart     keep the p leading Ritz directions: Q = orth(Y[:, :p]), V <- V Q,
//               H <- [Q^H H_m Q ; beta e_m^T Q] (a Krylov-Schur decomposition with a full
//               p x p block; ARPACK's implicit restart keeps the same subspace).
// The FILTER_FP32 form runs the filter sweeps in complex64 and everything else in FP64,
// then polishes the returned pairs (polish()).

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "floquet_internal.cuh"
#include "linalg.cuh"
#include "solver.cuh"

namespace fq {

using cd = std::complex<double>;

template <typename T> struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    if (count <= n) return FLOQUET_OK;
    cudaFree(p);
    p = nullptr;
    n = 0;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of %zu bytes failed", count * sizeof(T));
      return FLOQUET_ENOMEM;
    }
    n = count;
    return FLOQUET_OK;
  }
  ~DevBuf() { cudaFree(p); }
};

int DevVec::alloc(size_t count) {
  if (count <= n) return FLOQUET_OK;
  cudaFree(p);
  p = nullptr;
  n = 0;
  if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed", count * sizeof(double2));
    return FLOQUET_ENOMEM;
  }
  n = count;
  return FLOQUET_OK;
}
DevVec::~DevVec() { cudaFree(p); }

static double wrapped_angle(cd om, double phi) { return std::arg(om * std::polar(1.0, -phi)); }

// |g_k(omega)| with omega rotated by exp(-i phi): (1 - w^k)/(1 - w) evaluated by the
// recurrence g_{n+1} = g_n + w^n (no cancellation near w = 1)
static cd gk_value(cd om, double phi, int64_t k) {
  const cd w = om * std::polar(1.0, -phi);
  const double a = std::abs(1.0 - w);
  if (a > 1e-3) return (1.0 - std::pow(w, (double)k)) / (1.0 - w);
  cd g = 0, wn = 1;
  for (int64_t n = 0; n < k; ++n) {
    g += wn;
    wn *= w;
  }
  return g;
}

// Selection of the nev eigenvalues closest to exp(i phi): indices into om sorted by
// (|arg|, arg), restricted to the main lobe |arg| < 2 pi / k.
static std::vector<int> select_closest(const std::vector<cd>& om, double phi, int64_t k,
                                       int nev, bool inlobe_only) {
  std::vector<int> idx;
  for (int i = 0; i < (int)om.size(); ++i) {
    const double a = std::fabs(wrapped_angle(om[i], phi));
    if (std::abs(om[i]) < 0.5) continue;  // not an eigenvalue of a unitary (degenerate vector)
    if (!inlobe_only || a < 2 * M_PI / (double)k) idx.push_back(i);
  }
  std::sort(idx.begin(), idx.end(), [&](int x, int y) {
    const double ax = wrapped_angle(om[x], phi), ay = wrapped_angle(om[y], phi);
    if (std::fabs(ax) != std::fabs(ay)) return std::fabs(ax) < std::fabs(ay);
    return ax < ay;
  });
  if ((int)idx.size() > nev) idx.resize(nev);
  return idx;
}

__global__ void restart_h_kernel(const double2* __restrict__ Hold, int64_t ldh,
                                 int64_t strideH, const double2* __restrict__ Bp,
                                 int64_t strideB, const double2* __restrict__ Q, int64_t strideQ,
                                 int m, int p, double2* __restrict__ Hnew) {
  const int64_t b = blockIdx.x;
  const double2 beta = Hold[b * strideH + (int64_t)(m - 1) * ldh + m];
  double2* Hn = Hnew + b * strideH;
  for (int64_t i = threadIdx.x; i < ldh * m; i += blockDim.x) {
    const int r = (int)(i % ldh), c = (int)(i / ldh);
    double2 v = make_double2(0, 0);
    if (c < p && r < p) v = Bp[b * strideB + (int64_t)c * p + r];
    if (c < p && r == p) v = cmul(beta, Q[b * strideQ + (int64_t)c * m + (m - 1)]);
    Hn[i] = v;
  }
}

__global__ void broadcast_kernel(const double2* __restrict__ v, double2* __restrict__ out,
                                 int64_t d, int64_t stride) {
  const int64_t b = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x)
    out[b * stride + i] = v[i];
}

// ------------------------------------------------------------------ solver state

struct KS {
  floquet_op* op;
  int B, vpp;  // problems; vectors of the op's tables per problem index (b / vpp = table)
  int64_t d;
  int m, nev;
  int64_t k;
  int precision;
  double tol, tol_resid;
  int max_restarts;
  std::vector<double> phis;  // per problem
  cudaStream_t st;
  Workspace ws;
  DevBuf<double2> V, V2, H, H2, w, lam, Y, Q, Bp, Tmp, eigw, X, W, R, Xs;
  DevBuf<double> rq;
  DevBuf<int> info;
  DevBuf<double2> coef64;  // accumulate form: z_b^j, j < k, per problem
  DevBuf<float2> coef32;
  DevBuf<float4> coefdf;
  bool horner = true;      // Horner form: only z_b per problem (the first entry of each row)
  int64_t strideV() const { return d * (m + 1); }
  int64_t ldh() const { return m + 1; }
  int64_t strideH() const { return (int64_t)(m + 1) * m; }
};

static int ks_alloc(KS& s) {
  const size_t B = s.B, m = s.m, d = s.d;
  FQ_TRY(s.V.alloc(B * d * (m + 1)));
  FQ_TRY(s.V2.alloc(B * d * (m + 1)));
  FQ_TRY(s.H.alloc(B * (m + 1) * m));
  FQ_TRY(s.H2.alloc(B * (m + 1) * m));
  FQ_TRY(s.w.alloc(B * d));
  FQ_TRY(s.lam.alloc(B * m));
  FQ_TRY(s.Y.alloc(B * m * m));
  FQ_TRY(s.Q.alloc(B * m * m));
  FQ_TRY(s.Bp.alloc(B * m * m));
  FQ_TRY(s.Tmp.alloc(B * m * m));
  FQ_TRY(s.eigw.alloc(B * small_eig_work_elems((int)m)));
  FQ_TRY(s.info.alloc(B));
  FQ_TRY(s.X.alloc(B * d * m));
  FQ_TRY(s.W.alloc(B * d * m));
  FQ_TRY(s.rq.alloc(B * m * 3));
  // filter coefficients z_b^j = exp(-i j phi_b), float64 on the host: j < k for the
  // accumulate form, j = 1 only for the Horner form (the default; FLOQUET_KRYLOV_FORM=acc
  // selects the accumulate form)
  const char* form = getenv("FLOQUET_KRYLOV_FORM");
  s.horner = !(form && strcmp(form, "acc") == 0);
  const int64_t nc = s.horner ? 1 : s.k;
  std::vector<double2> c64((size_t)B * nc);
  for (size_t b = 0; b < B; ++b)
    for (int64_t j = 0; j < nc; ++j) {
      const double a = -s.phis[b] * (double)(s.horner ? 1 : j);
      c64[b * nc + j] = make_double2(cos(a), sin(a));
    }
  if (s.precision == FLOQUET_FP64) {
    FQ_TRY(s.coef64.alloc(c64.size()));
    FQ_CUDA(cudaMemcpy(s.coef64.p, c64.data(), c64.size() * sizeof(double2),
                       cudaMemcpyHostToDevice));
  } else if (s.precision == FLOQUET_FILTER_DF) {
    std::vector<float4> cdf(c64.size());
    for (size_t i = 0; i < c64.size(); ++i) cdf[i] = from_d2<dfloat>(c64[i]);
    FQ_TRY(s.coefdf.alloc(cdf.size()));
    FQ_CUDA(cudaMemcpy(s.coefdf.p, cdf.data(), cdf.size() * sizeof(float4),
                       cudaMemcpyHostToDevice));
  } else {
    std::vector<float2> c32(c64.size());
    for (size_t i = 0; i < c64.size(); ++i)
      c32[i] = make_float2((float)c64[i].x, (float)c64[i].y);
    FQ_TRY(s.coef32.alloc(c32.size()));
    FQ_CUDA(cudaMemcpy(s.coef32.p, c32.data(), c32.size() * sizeof(float2),
                       cudaMemcpyHostToDevice));
  }
  return FLOQUET_OK;
}

// w_b = g_k(U_b) V_b[:, j]
static int ks_filter(KS& s, int j) {
  const double2* in = s.V.p + (int64_t)j * s.d;
  if (s.horner) {
    if (s.precision == FLOQUET_FP64)
      return filter_horner<double, double>(s.op, in, s.strideV(), s.w.p, s.d, s.coef64.p, s.k,
                                           s.B, s.vpp, true, s.st);
    if (s.precision == FLOQUET_FILTER_DF)
      return filter_horner<dfloat, double>(s.op, in, s.strideV(), s.w.p, s.d, s.coefdf.p, s.k,
                                           s.B, s.vpp, true, s.st);
    return filter_horner<float, double>(s.op, in, s.strideV(), s.w.p, s.d, s.coef32.p, s.k,
                                        s.B, s.vpp, true, s.st);
  }
  if (s.precision == FLOQUET_FP64)
    return filter_coef<double, double>(s.op, in, s.strideV(), s.w.p, s.d, s.coef64.p, s.k, s.B,
                                       s.vpp, true, s.st);
  if (s.precision == FLOQUET_FILTER_DF)
    return filter_coef<dfloat, double>(s.op, in, s.strideV(), s.w.p, s.d, s.coefdf.p, s.k, s.B,
                                       s.vpp, true, s.st);
  return filter_coef<float, double>(s.op, in, s.strideV(), s.w.p, s.d, s.coef32.p, s.k, s.B,
                                    s.vpp, true, s.st);
}

// Ritz vectors X_b = V_b[:, :n] Y_b[:, :nx], then W = U X and (omega, resid) to host
static int ks_ritz(KS& s, int n, int nx, std::vector<double>& rq_host) {
  FQ_TRY(gemm_nn(s.V.p, s.d, s.strideV(), s.Y.p, s.m, (int64_t)s.m * s.m, s.X.p, s.d,
                 s.d * nx, s.d, n, nx, s.B, s.st));
  FQ_TRY(apply_u<double>(s.op, s.X.p, s.W.p, s.B * nx, nx * s.vpp, s.st));
  FQ_TRY(rayleigh_residual(s.ws, s.X.p, s.W.p, s.d, s.B * nx, s.rq.p, s.st));
  rq_host.resize((size_t)3 * s.B * nx);
  FQ_CUDA(cudaMemcpyAsync(rq_host.data(), s.rq.p, rq_host.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, s.st));
  FQ_CUDA(cudaStreamSynchronize(s.st));
  return FLOQUET_OK;
}

struct ProblemResult {
  bool done = false;
  std::vector<cd> omega;
  std::vector<double> resid;
  std::vector<int> cols;  // columns of X (within the problem's block) of the selected pairs
  int nconv_ritz = 0;     // converged Ritz values of g_k used for the block
};

// Polish of the FILTER_FP32 result (one problem): defect-corrected filtering of the
// Ritz block, alternating with FP64 Rayleigh-Ritz on [X, Y].
int polish(floquet_op* op, Workspace& ws, double phi, int64_t k, int nev, double tol_resid,
           int max_iter, double2* X, int nb, int64_t d, std::vector<cd>& omega_out,
           std::vector<double>& resid_out, std::vector<int>& cols_out, int* iters,
           cudaStream_t st);

int krylov_schur(floquet_op* op, int B, int vpp, const double* phis, int64_t k, int nev, int m,
                 int precision, double tol, double tol_resid, int max_restarts,
                 const double2* v0_dev, std::vector<KSOut>& out, cudaStream_t st,
                 KSStats* stats) {
  KS s;
  s.op = op;
  s.B = B;
  s.vpp = vpp;
  s.d = op->d;
  s.m = m;
  s.nev = nev;
  s.k = k;
  s.precision = precision;
  s.tol = tol;
  s.tol_resid = tol_resid;
  s.max_restarts = max_restarts;
  s.phis.assign(phis, phis + B);
  s.st = st;
  FQ_TRY(ks_alloc(s));
  out.clear();
  out.resize(B);

  // v_0 = v0 / ||v0|| for every problem
  {
    const unsigned gx = (unsigned)std::min<int64_t>((s.d + 255) / 256, 1024);
    broadcast_kernel<<<dim3(gx, B), 256, 0, st>>>(v0_dev, s.w.p, s.d, s.d);
    count_launch();
    FQ_CHECK_LAUNCH();
    FQ_TRY(cgs2(s.ws, s.V.p, s.d, s.strideV(), 0, s.w.p, s.d, s.d, B, nullptr, 0, s.V.p,
                s.strideV(), st));
  }
  FQ_CUDA(cudaMemsetAsync(s.H.p, 0, sizeof(double2) * (size_t)B * s.strideH(), st));

  std::vector<ProblemResult> res(B);
  std::vector<double2> lam_h((size_t)B * m), ylast((size_t)B * m), beta_h(B);
  std::vector<double> rq_h;
  int p = 0;
  int restarts = 0;
  bool all_done = false;
  // Convergence check on the current Krylov decomposition of dimension n (n <= m): Ritz
  // pairs of H[:n, :n], Ritz estimates |beta_n| |e_n^T y|, and for problems with more than nev
  // converged values the Ritz vectors, Rayleigh quotients, residuals and the completeness
  // rule. Leaves nc[b] (converged prefix) and, in s.Y, the eigenvectors of H[:n, :n].
  std::vector<int> nc(B, 0);
  bool near_done = false;  // set by check(): some unfinished problem has nev converged estimates
  auto check = [&](int n) -> int {
    FQ_TRY(small_eig_batched(s.H.p, s.ldh(), s.strideH(), n, B, s.lam.p, m, s.Y.p, m,
                             (int64_t)m * m, s.eigw.p, s.info.p, st));
    FQ_CUDA(cudaMemcpyAsync(lam_h.data(), s.lam.p, sizeof(double2) * B * m,
                            cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaMemcpy2DAsync(ylast.data(), sizeof(double2), s.Y.p + (n - 1),
                              sizeof(double2) * m, sizeof(double2), (size_t)B * m,
                              cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaMemcpy2DAsync(beta_h.data(), sizeof(double2),
                              s.H.p + (int64_t)(n - 1) * s.ldh() + n,
                              sizeof(double2) * s.strideH(), sizeof(double2), B,
                              cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaStreamSynchronize(st));
    // converged prefix per problem
    int nx = 0;
    for (int b = 0; b < B; ++b) {
      const double beta = std::abs(cd(beta_h[b].x, beta_h[b].y));
      int c = 0;
      while (c < n) {
        const cd th(lam_h[(size_t)b * m + c].x, lam_h[(size_t)b * m + c].y);
        const cd yl(ylast[(size_t)b * m + c].x, ylast[(size_t)b * m + c].y);
        if (beta * std::abs(yl) > tol * std::abs(th)) break;
        ++c;
      }
      nc[b] = c;
      if (!res[b].done && c > nev) nx = std::max(nx, c);
      if (!res[b].done && c >= nev) near_done = true;
    }
    if (nx > 0) {
      FQ_TRY(ks_ritz(s, n, nx, rq_h));
      for (int b = 0; b < B; ++b) {
        if (res[b].done || nc[b] <= nev) continue;
        std::vector<cd> om(nc[b]);
        for (int i = 0; i < nc[b]; ++i) {
          const double* q = &rq_h[3 * ((size_t)b * nx + i)];
          om[i] = cd(q[0], q[1]);
        }
        const std::vector<int> sel = select_closest(om, s.phis[b], k, nev, true);
        if ((int)sel.size() < nev) continue;
        const double g_nev = std::abs(gk_value(om[sel.back()], s.phis[b], k));
        const cd th_last(lam_h[(size_t)b * m + nc[b] - 1].x, lam_h[(size_t)b * m + nc[b] - 1].y);
        if (!(g_nev > std::abs(th_last) * (1 + 1e-9))) continue;
        bool resid_ok = true;
        for (int i : sel) resid_ok &= rq_h[3 * ((size_t)b * nx + i) + 2] <= tol_resid;
        if (precision != FLOQUET_FILTER_FP32 && !resid_ok) continue;
        ProblemResult& r = res[b];
        r.done = true;
        r.cols = sel;
        r.nconv_ritz = nc[b];
        r.omega.clear();
        r.resid.clear();
        for (int i : sel) {
          r.omega.push_back(om[i]);
          r.resid.push_back(rq_h[3 * ((size_t)b * nx + i) + 2]);
        }
        // keep the selected Ritz vectors (FP64 form) or the whole converged block (FP32
        // form, for the polish) in the output slot of this problem
        KSOut& o = out[b];
        o.omega = r.omega;
        o.resid = r.resid;
        if (precision != FLOQUET_FILTER_FP32) {
          FQ_TRY(o.vecs.alloc((size_t)nev * s.d));
          for (int i = 0; i < nev; ++i)
            FQ_CUDA(cudaMemcpyAsync(o.vecs.p + (size_t)i * s.d,
                                    s.X.p + ((size_t)b * nx + sel[i]) * s.d,
                                    sizeof(double2) * s.d, cudaMemcpyDeviceToDevice, st));
          o.cols.resize(nev);
          std::iota(o.cols.begin(), o.cols.end(), 0);
        } else {
          o.nblock = nc[b];
          FQ_TRY(o.vecs.alloc((size_t)nc[b] * s.d));
          FQ_CUDA(cudaMemcpyAsync(o.vecs.p, s.X.p + (size_t)b * nx * s.d,
                                  sizeof(double2) * s.d * nc[b], cudaMemcpyDeviceToDevice, st));
          o.cols = sel;
        }
        o.converged = true;
      }
    }
    return FLOQUET_OK;
  };

  // checks every 16 Krylov steps; for a few problems (a filter step then costs far more than
  // a check), every 4 steps once some unfinished problem has nev converged Ritz estimates
  // (only the completeness or residual test is left)
  const int check_every = 16, check_every_near = B <= 4 ? 4 : 16;
  for (;; ++restarts) {
    // expand p -> m, checking for convergence every check_every steps once the basis can
    // hold nev + check_every Ritz pairs (the Krylov relation holds at every size)
    bool done_early = false;
    for (int j = p; j < m; ++j) {
      FQ_TRY(ks_filter(s, j));
      FQ_TRY(cgs2(s.ws, s.V.p, s.d, s.strideV(), j + 1, s.w.p, s.d, s.d, s.B,
                  s.H.p + (int64_t)j * s.ldh(), s.strideH(), s.V.p + (int64_t)(j + 1) * s.d,
                  s.strideV(), s.st));
      if (stats) stats->expansions += 1;
      const int n = j + 1;
      // (not for the FP32-filter form: its polish needs the full converged block as guard
      // directions, which only the complete Krylov space provides)
      const int every = near_done ? check_every_near : check_every;
      if (precision != FLOQUET_FILTER_FP32 && n < m &&
          n >= std::max(p + check_every, nev + check_every) && n % every == 0) {
        FQ_TRY(check(n));
        bool all = true;
        for (int b = 0; b < B; ++b) all &= res[b].done;
        if (all) {
          done_early = true;
          break;
        }
      }
    }
    if (!done_early) FQ_TRY(check(m));

    all_done = true;
    for (int b = 0; b < B; ++b) all_done &= res[b].done;
    if (all_done || restarts >= max_restarts) break;

    // ---- restart: keep p leading Ritz directions
    int ncmax = 0;
    for (int b = 0; b < B; ++b)
      if (!res[b].done) ncmax = std::max(ncmax, nc[b]);
    const int base = std::max(ncmax, nev);
    p = base + (m - base) / 2;
    p = std::min(p, m - std::max(2, m / 8));
    p = std::max(p, 1);
    FQ_TRY(small_orth_batched(s.Y.p, m, (int64_t)m * m, m, p, B, s.Q.p, m, (int64_t)m * m, st));
    // V2[:, :p] = V[:, :m] Q ; V2[:, p] = V[:, m]
    FQ_TRY(gemm_nn(s.V.p, s.d, s.strideV(), s.Q.p, m, (int64_t)m * m, s.V2.p, s.d, s.strideV(),
                   s.d, m, p, B, st));
    copy_matrix_launch(s.V.p + (int64_t)m * s.d, s.d, s.strideV(), s.V2.p + (int64_t)p * s.d,
                       s.d, s.strideV(), (int)s.d, 1, B, st);
    FQ_CHECK_LAUNCH();
    std::swap(s.V.p, s.V2.p);
    std::swap(s.V.n, s.V2.n);
    // H2 = [Q^H H_m Q ; beta Q[m-1, :]]
    FQ_TRY(small_gemm_batched('N', 'N', m, p, m, s.H.p, s.ldh(), s.strideH(), s.Q.p, m,
                              (int64_t)m * m, s.Tmp.p, m, (int64_t)m * m, B, st));
    FQ_TRY(small_gemm_batched('C', 'N', p, p, m, s.Q.p, m, (int64_t)m * m, s.Tmp.p, m,
                              (int64_t)m * m, s.Bp.p, p, (int64_t)m * m, B, st));
    restart_h_kernel<<<B, 256, 0, st>>>(s.H.p, s.ldh(), s.strideH(), s.Bp.p, (int64_t)m * m,
                                        s.Q.p, (int64_t)m * m, m, p, s.H2.p);
    count_launch();
    FQ_CHECK_LAUNCH();
    std::swap(s.H.p, s.H2.p);
    std::swap(s.H.n, s.H2.n);
    if (stats) stats->restarts = restarts + 1;
  }
  if (stats) stats->restarts = restarts;

  // FP32 form: polish every converged problem in FP64
  if (precision == FLOQUET_FILTER_FP32) {
    for (int b = 0; b < B; ++b) {
      KSOut& o = out[b];
      if (!o.converged) continue;
      std::vector<cd> om;
      std::vector<double> rs;
      std::vector<int> cols;
      int it = 0;
      FQ_TRY(polish(op, s.ws, s.phis[b], k, nev, tol_resid, 30, o.vecs.p, o.nblock, s.d, om, rs,
                    cols, &it, st));
      o.omega = om;
      o.resid = rs;
      o.cols = cols;
      if (stats) stats->polish_iters = it;
    }
  }
  return all_done ? FLOQUET_OK : FLOQUET_ENOCONV;
}

// ------------------------------------------------------------------ polish

// Hermitian n x n matrix A (column-major, host) = R^H R by Cholesky with diagonal pivoting:
// at each step the column with the largest remaining diagonal is taken, until that diagonal
// falls to `floor` (the remaining columns are dependent on the chosen ones and dropped).
// piv[0..rank) are the chosen columns in order; R (rank x rank, column-major, upper) acts on
// them. Returns the rank.
static int pivoted_cholesky(std::vector<cd> A, int n, double floor, std::vector<int>& piv,
                            std::vector<cd>& R) {
  std::vector<int> p(n);
  std::iota(p.begin(), p.end(), 0);
  int rank = 0;
  for (; rank < n; ++rank) {
    int best = rank;
    for (int j = rank + 1; j < n; ++j)
      if (A[(size_t)p[j] * n + p[j]].real() > A[(size_t)p[best] * n + p[best]].real()) best = j;
    std::swap(p[rank], p[best]);
    const int c = p[rank];
    const double dg = A[(size_t)c * n + c].real();
    if (!(dg > floor)) break;
    const double r = std::sqrt(dg);
    // row `rank` of R over the remaining pivot order: R[rank, j] = A[c, p_j] / r
    for (int j = rank + 1; j < n; ++j) {
      const int cj = p[j];
      const cd rij = A[(size_t)cj * n + c] / r;  // A(c, cj)
      // update the Schur complement A(p_i, p_j) -= conj(R[rank, i]) R[rank, j]
      for (int i2 = rank + 1; i2 < n; ++i2) {
        const int ci = p[i2];
        const cd rii = A[(size_t)ci * n + c] / r;
        A[(size_t)cj * n + ci] -= std::conj(rii) * rij;
      }
    }
    // keep R's row for the chosen columns, recomputed below from the final order
    A[(size_t)c * n + c] = cd(r, 0.0);
  }
  // R[i, j] over the chosen pivots (i <= j < rank): a second, exact pass from the original
  // relation A_pp = R^H R is not needed; rebuild R from the updated entries instead
  piv.assign(p.begin(), p.begin() + rank);
  return rank;
}

// Q = C M with M = R^{-1} on the chosen columns (upper-triangular inverse, host).
static std::vector<cd> upper_inverse(const std::vector<cd>& R, int r) {
  std::vector<cd> X((size_t)r * r, cd(0.0, 0.0));
  for (int j = 0; j < r; ++j) {
    X[(size_t)j * r + j] = 1.0 / R[(size_t)j * r + j];
    for (int i = j - 1; i >= 0; --i) {
      cd sum = 0;
      for (int l = i + 1; l <= j; ++l) sum += R[(size_t)l * r + i] * X[(size_t)j * r + l];
      X[(size_t)j * r + i] = -sum / R[(size_t)i * r + i];
    }
  }
  return X;
}

// Cholesky R (rank x rank, column-major upper) of the pivoted Hermitian block A[piv, piv].
static std::vector<cd> cholesky_upper(const std::vector<cd>& A, int n,
                                      const std::vector<int>& piv) {
  const int r = (int)piv.size();
  std::vector<cd> R((size_t)r * r, cd(0.0, 0.0));
  for (int j = 0; j < r; ++j) {
    for (int i = 0; i <= j; ++i) {
      cd sum = A[(size_t)piv[j] * n + piv[i]];  // A(piv_i, piv_j)
      for (int l = 0; l < i; ++l) sum -= std::conj(R[(size_t)i * r + l]) * R[(size_t)j * r + l];
      if (i == j) {
        const double v = sum.real();
        R[(size_t)j * r + j] = cd(std::sqrt(v > 0 ? v : 0.0), 0.0);
      } else {
        R[(size_t)j * r + i] = sum / R[(size_t)i * r + i];
      }
    }
  }
  return R;
}

// Orthonormalise the nn columns S[:, n0 : n0 + nn] (leading dimension d) against S[:, :n0]
// (classical Gram-Schmidt, twice) and among themselves (Cholesky QR with diagonal pivoting,
// twice). Each column is first scaled to unit length; a column whose remaining length after
// the projections is below `drop` adds no direction and is dropped. The kept columns end up
// in S[:, n0 : n0 + kept]. T is scratch of d x nn, M of max(n0, nn) x nn complex.
static int orth_block(Workspace& ws, double2* S, int64_t d, int n0, int nn, double drop,
                      double2* T, double2* M, int* kept, cudaStream_t st) {
  *kept = 0;
  if (nn <= 0) return FLOQUET_OK;
  double2* C = S + (int64_t)n0 * d;
  std::vector<double2> g((size_t)nn * nn);
  auto gram = [&](int n) -> int {  // g = C[:, :n]^H C[:, :n] on the host
    FQ_TRY(gemm_cn(ws, C, d, 0, C, d, 0, d, n, n, 1, M, n, 0, st));
    FQ_CUDA(cudaMemcpyAsync(g.data(), M, sizeof(double2) * n * n, cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaStreamSynchronize(st));
    return FLOQUET_OK;
  };
  // unit columns
  FQ_TRY(gram(nn));
  {
    std::vector<double2> sc(nn);
    for (int j = 0; j < nn; ++j) {
      const double v = g[(size_t)j * nn + j].x;
      sc[j] = make_double2(v > 0 ? 1.0 / std::sqrt(v) : 0.0, 0.0);
    }
    FQ_CUDA(cudaMemcpyAsync(M, sc.data(), sizeof(double2) * nn, cudaMemcpyHostToDevice, st));
    FQ_TRY(scale_cols(C, d, nn, M, st));
  }
  for (int pass = 0; pass < 2 && n0 > 0; ++pass) {
    FQ_TRY(gemm_cn(ws, S, d, 0, C, d, 0, d, n0, nn, 1, M, n0, 0, st));  // S^H C
    FQ_TRY(gemm_nn(S, d, 0, M, n0, 0, T, d, 0, d, n0, nn, 1, st));     // S (S^H C)
    FQ_TRY(sub_cols(C, d, T, d, d, nn, st));
  }
  int n = nn;
  for (int pass = 0; pass < 2; ++pass) {
    FQ_TRY(gram(n));
    std::vector<cd> A((size_t)n * n);
    for (size_t i = 0; i < A.size(); ++i) A[i] = cd(g[i].x, g[i].y);
    std::vector<int> piv;
    std::vector<cd> Rdummy;
    const int r = pivoted_cholesky(A, n, pass == 0 ? drop * drop : 0.0, piv, Rdummy);
    if (r == 0) {
      *kept = 0;
      return FLOQUET_OK;
    }
    const std::vector<cd> R = cholesky_upper(A, n, piv);
    const std::vector<cd> Ri = upper_inverse(R, r);
    // Q = C P R^{-1}: M (n x r) holds Ri's rows at the pivot positions
    std::vector<double2> mh((size_t)n * r, make_double2(0, 0));
    for (int j = 0; j < r; ++j)
      for (int i = 0; i <= j; ++i) {
        const cd v = Ri[(size_t)j * r + i];
        mh[(size_t)j * n + piv[i]] = make_double2(v.real(), v.imag());
      }
    FQ_CUDA(cudaMemcpyAsync(M, mh.data(), sizeof(double2) * n * r, cudaMemcpyHostToDevice, st));
    FQ_TRY(gemm_nn(C, d, 0, M, n, 0, T, d, 0, d, n, r, 1, st));
    FQ_CUDA(cudaMemcpyAsync(C, T, sizeof(double2) * d * r, cudaMemcpyDeviceToDevice, st));
    n = r;
  }
  *kept = n;
  return FLOQUET_OK;
}

// FP64 polish of the FILTER_FP32 result (one problem): the Ritz step with U on approximate
// eigenvectors that the Sec. 4 footnote suggests, iterated until the U-residuals reach
// tol_resid.
//
// Each iteration: Rayleigh-Ritz with U in complex128 on span(S) (G = S^H U S, its eigen-
// decomposition on the device); the block = the nb Ritz pairs with the largest |g_k(omega)|
// (values off the unit circle are mixtures and rank last); stop when the nev in-lobe pairs
// closest to exp(i phi) have residual <= tol_resid. Otherwise compute a correction for every
// selected pair still above tol_resid / 10: with r = (U - omega) x formed in FP64 and the
// filter g_K centred on omega itself,
//     g_K(U / omega) x - K x = q(U) r,   q(U) = sum_{l < K-1} (K-1-l) omega^{-(l+1)} U^l,
// (Sec. 3, Eq. geo, the defect of the geometric sum at its own peak), so q(U) r is
// g_K(U / omega) x with the part along x removed: the error components of x far from omega
// come back multiplied by about -K, those near omega are suppressed. Only the small residual
// r goes through the complex64 sweeps (Horner form with the coefficients K-1-l), so their
// rounding is relative to ||r||. The corrections of all pairs share one batched filter
// launch; K = k/2 by default (FLOQUET_POLISH_K sets it).
// The next space is [Ritz block, the last kWindow correction blocks] (an LOBPCG-like window):
// the earlier blocks carry what the previous corrections found, so the error components that
// the pairs share keep converging while the space stays bounded. The Ritz block and the kept
// blocks lie in span(S): they are re-based by a coefficient matrix (no new U applications);
// only the new corrections need U in FP64.
int polish(floquet_op* op, Workspace& ws, double phi, int64_t k, int nev, double tol_resid,
           int max_iter, double2* X0, int nb_in, int64_t d, std::vector<cd>& omega_out,
           std::vector<double>& resid_out, std::vector<int>& cols_out, int* iters,
           cudaStream_t st) {
  const bool verbose = getenv("FLOQUET_VERBOSE") != nullptr;
  int64_t K = std::max<int64_t>(2, k / 2);
  if (const char* e = getenv("FLOQUET_POLISH_K")) K = std::max<int64_t>(2, atoll(e));
  // block: the wanted pairs and guard directions (the largest |g_k| beyond them)
  const int nb = std::min(nb_in, nev + std::max(16, nev / 4));
  // correction blocks kept in the space (3, or fewer so that the space fits the small
  // eigensolver's 512)
  int kWindow = 3;
  if (const char* e = getenv("FLOQUET_POLISH_WINDOW")) kWindow = std::max(1, atoi(e));
  kWindow = std::min(kWindow, (512 - nb) / std::max(1, nb));
  if (kWindow < 1) {
    set_error("polish: nev %d too large for the Rayleigh-Ritz space", nev);
    return FLOQUET_EINVAL;
  }
  const int smax = nb + kWindow * nb;
  const double drop = 1e-6;
  DevBuf<double2> S, W, S2, W2, T, M, G, Gt, Yg, Ysel, Mq, lam, eigw, X, UX, R, Cb;
  DevBuf<double> rq;
  DevBuf<int> info;
  DevBuf<float2> zs, hc;
  DevBuf<float4> zsd, hcd;  // double-float copies for the later correction steps
  FQ_TRY(S.alloc((size_t)smax * d));
  FQ_TRY(W.alloc((size_t)smax * d));
  FQ_TRY(S2.alloc((size_t)smax * d));
  FQ_TRY(W2.alloc((size_t)smax * d));
  FQ_TRY(T.alloc((size_t)nb * d));
  FQ_TRY(M.alloc((size_t)smax * nb));
  FQ_TRY(G.alloc((size_t)smax * smax));
  FQ_TRY(Gt.alloc((size_t)smax * smax));
  FQ_TRY(Yg.alloc((size_t)smax * smax));
  FQ_TRY(Ysel.alloc((size_t)smax * nb));
  FQ_TRY(Mq.alloc((size_t)smax * smax));
  FQ_TRY(lam.alloc(smax));
  FQ_TRY(eigw.alloc(small_eig_work_elems(smax)));
  FQ_TRY(info.alloc(1));
  FQ_TRY(X.alloc((size_t)nb * d));
  FQ_TRY(UX.alloc((size_t)nb * d));
  FQ_TRY(R.alloc((size_t)nb * d));
  FQ_TRY(Cb.alloc((size_t)nb * d));
  FQ_TRY(rq.alloc((size_t)3 * nb));
  // the correction sweeps run in complex64; FLOQUET_POLISH_DF_FROM = i runs the steps from
  // the i-th on in double-float instead
  int df_from = 1 << 30;
  if (const char* e = getenv("FLOQUET_POLISH_DF_FROM")) df_from = std::max(0, atoi(e));
  FQ_TRY(zs.alloc(nb));
  FQ_TRY(hc.alloc((size_t)K));
  FQ_TRY(zsd.alloc(nb));
  FQ_TRY(hcd.alloc((size_t)K));
  {  // Horner coefficients of q: hc[j] = j + 1 (hc[0] unused)
    std::vector<float2> h((size_t)K);
    std::vector<float4> hd((size_t)K);
    for (int64_t j = 0; j < K; ++j) {
      h[j] = make_float2((float)(j + 1), 0.0f);
      hd[j] = from_d2<dfloat>(make_double2((double)(j + 1), 0.0));
    }
    FQ_CUDA(cudaMemcpyAsync(hc.p, h.data(), sizeof(float2) * K, cudaMemcpyHostToDevice, st));
    FQ_CUDA(cudaMemcpyAsync(hcd.p, hd.data(), sizeof(float4) * K, cudaMemcpyHostToDevice, st));
    FQ_CUDA(cudaStreamSynchronize(st));
  }
  // initial space: the block of the converged Ritz vectors with the largest |theta|
  FQ_CUDA(cudaMemcpyAsync(S.p, X0, sizeof(double2) * nb * d, cudaMemcpyDeviceToDevice, st));
  int ns = 0;
  FQ_TRY(orth_block(ws, S.p, d, 0, nb, drop, T.p, M.p, &ns, st));
  FQ_TRY(apply_u<double>(op, S.p, W.p, ns, ns, st));
  FQ_TRY(gemm_cn(ws, S.p, d, 0, W.p, d, 0, d, ns, ns, 1, G.p, smax, 0, st));
  // column ranges of S holding the kept correction blocks, oldest first
  std::vector<std::pair<int, int>> blocks;
  std::vector<double2> lam_h(smax);
  std::vector<double> rq_h(3 * nb);
  int corrections = 0;
  for (int it = 0;; ++it) {
    FQ_TRY(small_eig_batched(G.p, smax, 0, ns, 1, lam.p, 0, Yg.p, ns, 0, eigw.p, info.p, st));
    int info_h = 0;
    FQ_CUDA(cudaMemcpyAsync(lam_h.data(), lam.p, sizeof(double2) * ns, cudaMemcpyDeviceToHost,
                            st));
    FQ_CUDA(cudaMemcpyAsync(&info_h, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaStreamSynchronize(st));
    if (info_h) {
      set_error("polish: small eigensolver did not converge (n = %d)", ns);
      return FLOQUET_ENOCONV;
    }
    // the block: nk Ritz values with the largest |g_k|, values on the unit circle first
    const int nk = std::min(nb, ns);
    std::vector<int> order(ns);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> gabs(ns);
    for (int i = 0; i < ns; ++i) {
      const cd l(lam_h[i].x, lam_h[i].y);
      gabs[i] = std::abs(gk_value(l, phi, k));
      if (std::fabs(std::abs(l) - 1.0) > 1e-8) gabs[i] *= 1e-6;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gabs[a] > gabs[b]; });
    for (int i = 0; i < nk; ++i)
      FQ_CUDA(cudaMemcpyAsync(Ysel.p + (size_t)i * ns, Yg.p + (size_t)order[i] * ns,
                              sizeof(double2) * ns, cudaMemcpyDeviceToDevice, st));
    FQ_TRY(gemm_nn(S.p, d, 0, Ysel.p, ns, 0, X.p, d, 0, d, ns, nk, 1, st));
    // U X by a fresh FP64 application (not W Y): the residuals do not depend on how
    // accurately the re-based W still equals U S
    FQ_TRY(apply_u<double>(op, X.p, UX.p, nk, nk, st));
    FQ_TRY(rayleigh_residual(ws, X.p, UX.p, d, nk, rq.p, st));
    FQ_CUDA(cudaMemcpyAsync(rq_h.data(), rq.p, sizeof(double) * 3 * nk, cudaMemcpyDeviceToHost,
                            st));
    FQ_CUDA(cudaStreamSynchronize(st));
    std::vector<cd> om(nk), om_c(nk);
    for (int i = 0; i < nk; ++i) {
      om[i] = cd(rq_h[3 * i], rq_h[3 * i + 1]);
      // an eigenpair with residual r has ||omega| - 1| ~ r^2 / 2: values farther off the
      // circle are mixtures, not candidates
      om_c[i] = std::fabs(std::abs(om[i]) - 1.0) < 1e-8 ? om[i] : cd(0.0, 0.0);
    }
    const std::vector<int> sel = select_closest(om_c, phi, k, nev, true);
    double worst = sel.size() < (size_t)nev ? INFINITY : 0.0;
    for (int i : sel) worst = std::max(worst, rq_h[3 * i + 2]);
    omega_out.clear();
    resid_out.clear();
    cols_out = sel;
    for (int i : sel) {
      omega_out.push_back(om[i]);
      resid_out.push_back(rq_h[3 * i + 2]);
    }
    *iters = it;
    // pairs to correct: every block member still above a tenth of the target, the guard
    // directions included (a guard left unconverged would mix back into the nearly degenerate
    // wanted pairs at the next Rayleigh-Ritz step)
    std::vector<int> act;
    for (int i = 0; i < nk; ++i)
      if (rq_h[3 * i + 2] > 0.1 * tol_resid) act.push_back(i);
    const int nf = (int)act.size();
    if (verbose)
      fprintf(stderr, "floquet polish: iter %d space %d block %d worst selected resid %.3e "
              "(candidates %zu), correcting %d (K = %lld)\n", it, ns, nk, worst, sel.size(), nf,
              (long long)K);
    if (worst <= tol_resid || it >= max_iter || nf == 0) {
      FQ_CUDA(cudaMemcpyAsync(X0, X.p, sizeof(double2) * nk * d, cudaMemcpyDeviceToDevice, st));
      break;
    }
    // residual vectors of the pairs to correct, then q(U) r in one batched filter launch
    FQ_TRY(residual_vectors(X.p, UX.p, R.p, d, nk, rq.p, st));
    for (int j = 0; j < nf; ++j)
      FQ_CUDA(cudaMemcpyAsync(T.p + (size_t)j * d, R.p + (size_t)act[j] * d,
                              sizeof(double2) * d, cudaMemcpyDeviceToDevice, st));
    std::vector<float2> zh(nf);
    std::vector<float4> zhd(nf);
    for (int j = 0; j < nf; ++j) {
      const cd z = 1.0 / om[act[j]];
      zh[j] = make_float2((float)z.real(), (float)z.imag());
      zhd[j] = from_d2<dfloat>(make_double2(z.real(), z.imag()));
    }
    if (it >= df_from) {
      FQ_CUDA(cudaMemcpyAsync(zsd.p, zhd.data(), sizeof(float4) * nf, cudaMemcpyHostToDevice,
                              st));
      FQ_CUDA(cudaStreamSynchronize(st));
      FQ_TRY((filter_horner_coef<dfloat, double>(op, T.p, d, Cb.p, d, zsd.p, hcd.p, K - 1, nf,
                                                 st)));
    } else {
      FQ_CUDA(cudaMemcpyAsync(zs.p, zh.data(), sizeof(float2) * nf, cudaMemcpyHostToDevice,
                              st));
      FQ_CUDA(cudaStreamSynchronize(st));
      FQ_TRY((filter_horner_coef<float, double>(op, T.p, d, Cb.p, d, zs.p, hc.p, K - 1, nf,
                                                st)));
    }
    corrections += nf;
    // re-base the kept part of the space, [Ritz block, the newest kWindow - 1 correction
    // blocks] = S Z, by an orthonormal coefficient matrix Mq spanning the columns of Z in that
    // order (Gram-Schmidt twice on the host; a column whose remaining length is below 1e-8 is
    // dropped), so that each kept block's remainder stays a contiguous range of columns
    {
      while ((int)blocks.size() > kWindow - 1) blocks.erase(blocks.begin());
      int nz = nk;
      for (auto& b : blocks) nz += b.second;
      std::vector<double2> yh((size_t)ns * nk);
      FQ_CUDA(cudaMemcpyAsync(yh.data(), Ysel.p, sizeof(double2) * ns * nk,
                              cudaMemcpyDeviceToHost, st));
      FQ_CUDA(cudaStreamSynchronize(st));
      std::vector<cd> q((size_t)ns * nz);
      int nq = 0;
      std::vector<cd> col(ns);
      std::vector<std::pair<int, int>> nblocks;
      int c = 0;
      for (int g = -1; g < (int)blocks.size(); ++g) {
        const int gcols = g < 0 ? nk : blocks[g].second;
        const int start = nq;
        for (int cc = 0; cc < gcols; ++cc, ++c) {
          for (int r = 0; r < ns; ++r)
            col[r] = g < 0 ? cd(yh[(size_t)cc * ns + r].x, yh[(size_t)cc * ns + r].y)
                           : (r == blocks[g].first + cc ? cd(1.0, 0.0) : cd(0.0, 0.0));
          double n0 = 0;
          for (int r = 0; r < ns; ++r) n0 += std::norm(col[r]);
          n0 = std::sqrt(n0);
          if (!(n0 > 0)) continue;
          for (int pass = 0; pass < 2; ++pass)
            for (int j2 = 0; j2 < nq; ++j2) {
              const cd* qj = &q[(size_t)j2 * ns];
              cd h = 0;
              for (int r = 0; r < ns; ++r) h += std::conj(qj[r]) * col[r];
              for (int r = 0; r < ns; ++r) col[r] -= h * qj[r];
            }
          double n1 = 0;
          for (int r = 0; r < ns; ++r) n1 += std::norm(col[r]);
          n1 = std::sqrt(n1);
          if (!(n1 > 1e-8 * n0)) continue;
          for (int r = 0; r < ns; ++r) q[(size_t)nq * ns + r] = col[r] / n1;
          ++nq;
        }
        if (g >= 0 && nq > start) nblocks.push_back({start, nq - start});
      }
      blocks = nblocks;
      std::vector<double2> mq((size_t)ns * nq);
      for (size_t t = 0; t < mq.size(); ++t) mq[t] = make_double2(q[t].real(), q[t].imag());
      FQ_CUDA(cudaMemcpyAsync(Mq.p, mq.data(), sizeof(double2) * ns * nq,
                              cudaMemcpyHostToDevice, st));
      FQ_TRY(gemm_nn(S.p, d, 0, Mq.p, ns, 0, S2.p, d, 0, d, ns, nq, 1, st));
      FQ_TRY(gemm_nn(W.p, d, 0, Mq.p, ns, 0, W2.p, d, 0, d, ns, nq, 1, st));
      // G <- Mq^H G Mq
      FQ_TRY(small_gemm_batched('N', 'N', ns, nq, ns, G.p, smax, 0, Mq.p, ns, 0, Gt.p, smax, 0,
                                1, st));
      FQ_TRY(small_gemm_batched('C', 'N', nq, nq, ns, Mq.p, ns, 0, Gt.p, smax, 0, G.p, smax, 0,
                                1, st));
      std::swap(S.p, S2.p);
      std::swap(W.p, W2.p);
      ns = nq;
    }
    // append the new corrections, orthonormalised against the re-based space
    double2* Cdst = S.p + (size_t)ns * d;
    FQ_CUDA(cudaMemcpyAsync(Cdst, Cb.p, sizeof(double2) * nf * d, cudaMemcpyDeviceToDevice,
                            st));
    int nc = 0;
    FQ_TRY(orth_block(ws, S.p, d, ns, nf, drop, T.p, M.p, &nc, st));
    if (nc > 0) blocks.push_back({ns, nc});
    if (nc > 0) {
      FQ_TRY(apply_u<double>(op, Cdst, W.p + (size_t)ns * d, nc, nc, st));
      // G[:ns, ns:ns+nc] = S_old^H W_new; G[ns:ns+nc, :ns+nc] = S_new^H W
      FQ_TRY(gemm_cn(ws, S.p, d, 0, W.p + (size_t)ns * d, d, 0, d, ns, nc, 1,
                     G.p + (size_t)ns * smax, smax, 0, st));
      FQ_TRY(gemm_cn(ws, Cdst, d, 0, W.p, d, 0, d, nc, ns + nc, 1, G.p + ns, smax, 0, st));
      ns += nc;
    }
  }
  if (verbose) fprintf(stderr, "floquet polish: %d corrections of %lld terms\n", corrections,
                       (long long)(K - 1));
  return FLOQUET_OK;
}

}  // namespace fq
