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

// a_l(omega) = z^{l+1} g_{k-1-l}(z omega), l = 0..k-2: the polynomial q with
// g_k(U) - g_k(omega) = q(U) (U - omega), so that g_k(U) x = g_k(omega) x + q(U) r for
// r = (U - omega) x. The FP32 sweeps then act on the small residual r only.
static void defect_coefficients(cd omega, double phi, int64_t k, cd* out, cd* g_at_omega) {
  const cd z = std::polar(1.0, -phi);
  const cd w = z * omega;
  // g_n(w) for n = 1 .. k by g_{n} = g_{n-1} + w^{n-1}
  std::vector<cd> g(k + 1);
  g[0] = 0;
  cd wn = 1;
  for (int64_t n = 1; n <= k; ++n) {
    g[n] = g[n - 1] + wn;
    wn *= w;
  }
  *g_at_omega = g[k];
  for (int64_t l = 0; l + 1 < k; ++l) {
    out[l] = std::polar(1.0, -phi * (double)(l + 1)) * g[k - 1 - l];
  }
}

// out_j = q_j(U) r_j for j < n, q_j the defect polynomial of omega_j above with filter length
// K and target phi: the correction step of the polish, and the C ABI's
// floquet_polish_correction. Sweeps in complex64 (df = false) or double-float (df = true),
// the coefficients rounded to that precision; r_j at R + j d, out_j at out + j d (complex128).
int polish_correction(floquet_op* op, double phi, int64_t K, const cd* omega, const double2* R,
                      double2* out, int n, bool df, cudaStream_t st) {
  const int64_t d = op->d;
  const size_t nc = (size_t)n * (K - 1);
  std::vector<cd> a((size_t)(K - 1));
  cd gv;
  if (df) {
    std::vector<float4> h(nc);
    for (int j = 0; j < n; ++j) {
      defect_coefficients(omega[j], phi, K, a.data(), &gv);
      for (int64_t l = 0; l + 1 < K; ++l)
        h[(size_t)j * (K - 1) + l] = from_d2<dfloat>(make_double2(a[l].real(), a[l].imag()));
    }
    DevBuf<float4> c;
    FQ_TRY(c.alloc(nc));
    FQ_CUDA(cudaMemcpyAsync(c.p, h.data(), sizeof(float4) * nc, cudaMemcpyHostToDevice, st));
    FQ_TRY((filter_coef<dfloat, double>(op, R, d, out, d, c.p, K - 1, n, n, true, st)));
    FQ_CUDA(cudaStreamSynchronize(st));  // c is freed on return
  } else {
    std::vector<float2> h(nc);
    for (int j = 0; j < n; ++j) {
      defect_coefficients(omega[j], phi, K, a.data(), &gv);
      for (int64_t l = 0; l + 1 < K; ++l)
        h[(size_t)j * (K - 1) + l] = make_float2((float)a[l].real(), (float)a[l].imag());
    }
    DevBuf<float2> c;
    FQ_TRY(c.alloc(nc));
    FQ_CUDA(cudaMemcpyAsync(c.p, h.data(), sizeof(float2) * nc, cudaMemcpyHostToDevice, st));
    FQ_TRY((filter_coef<float, double>(op, R, d, out, d, c.p, K - 1, n, n, true, st)));
    FQ_CUDA(cudaStreamSynchronize(st));
  }
  return FLOQUET_OK;
}

// Orthonormalise the columns of X in place, one at a time: each column is normalised, then
// projected twice against the columns kept so far (CGS2); a column whose new component is
// below `drop` of its length adds no direction and is dropped (later columns move up).
// Without the drop, nearly dependent columns would leave the basis non-orthogonal at the
// drop level / eps ratio and the Rayleigh-Ritz step would mix eigenvectors.
static int orthonormalize(Workspace& ws, double2* X, int n, int64_t d, double drop, int* kept,
                          cudaStream_t st) {
  int w = 0;
  double beta = 0;
  for (int j = 0; j < n; ++j) {
    double2* col = X + (int64_t)w * d;
    if (j != w)
      FQ_CUDA(cudaMemcpyAsync(col, X + (int64_t)j * d, sizeof(double2) * d,
                              cudaMemcpyDeviceToDevice, st));
    // normalise (no projection), then project against the kept columns
    FQ_TRY(cgs2(ws, X, d, 0, 0, col, 0, d, 1, nullptr, 0, col, 0, st));
    FQ_CUDA(cudaMemcpyAsync(&beta, ws.last_betas, sizeof(double), cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaStreamSynchronize(st));
    if (!(beta > 0)) continue;
    if (w > 0) {
      FQ_TRY(cgs2(ws, X, d, 0, w, col, 0, d, 1, nullptr, 0, col, 0, st));
      FQ_CUDA(cudaMemcpyAsync(&beta, ws.last_betas, sizeof(double), cudaMemcpyDeviceToHost, st));
      FQ_CUDA(cudaStreamSynchronize(st));
      if (!(beta > drop)) continue;
    }
    ++w;
  }
  *kept = w;
  return FLOQUET_OK;
}

// FP64 polish of the FILTER_FP32 result (Sec. 4 footnote: a Ritz step with U on approximate
// eigenvectors, here iterated). Each iteration: Rayleigh-Ritz with U on span(S); keep the nb
// Ritz pairs with the largest |g_k(omega)| (the block the filter enhances); stop when the nev
// closest in-lobe pairs have residuals <= tol_resid; otherwise extend S by the
// defect-corrected filter directions q(U) r of the unconverged pairs, where
// g_k(U) x = g_k(omega) x + q(U) r and r = (U - omega) x is computed in FP64, so the
// complex64 sweeps only act on the small residual.
int polish(floquet_op* op, Workspace& ws, double phi, int64_t k, int nev, double tol_resid,
           int max_iter, double2* X0, int nb, int64_t d, std::vector<cd>& omega_out,
           std::vector<double>& resid_out, std::vector<int>& cols_out, int* iters,
           cudaStream_t st) {
  const int n2 = 2 * nb;
  const bool verbose = getenv("FLOQUET_VERBOSE") != nullptr;
  DevBuf<double2> S, WS, Xn, G, Yg, lam, eigw, R, corr;
  // the correction filter q(U) r sums k terms of size up to k |r|: complex64 sweeps round it
  // at ~u32 k relative to the useful part, double-float sweeps at ~2^-48 k. The polish starts
  // with complex64 (cheaper) and switches to double-float once the worst selected residual
  // has not halved over three iterations (both values finite: a shortfall of candidates is
  // not a stall); FLOQUET_POLISH_SWEEP=c64 or =df fixes the choice, and
  // FLOQUET_POLISH_DF_FROM=i switches at iteration i.
  const char* psw = getenv("FLOQUET_POLISH_SWEEP");
  const bool forced = psw && (strcmp(psw, "c64") == 0 || strcmp(psw, "df") == 0);
  bool df_corr = forced && strcmp(psw, "df") == 0;
  int df_from = -1;
  if (const char* e = getenv("FLOQUET_POLISH_DF_FROM")) df_from = std::max(0, atoi(e));
  std::vector<double> worst_hist;
  DevBuf<double> rq;
  DevBuf<int> info;
  FQ_TRY(S.alloc((size_t)n2 * d));
  FQ_TRY(WS.alloc((size_t)n2 * d));
  FQ_TRY(Xn.alloc((size_t)n2 * d));
  FQ_TRY(G.alloc((size_t)n2 * n2));
  FQ_TRY(Yg.alloc((size_t)n2 * n2));
  FQ_TRY(lam.alloc(n2));
  FQ_TRY(eigw.alloc(small_eig_work_elems(n2)));
  FQ_TRY(info.alloc(1));
  FQ_TRY(R.alloc((size_t)nb * d));
  FQ_TRY(corr.alloc((size_t)nb * d));
  FQ_TRY(rq.alloc((size_t)3 * n2));
  const double drop = 1e-6;
  FQ_CUDA(cudaMemcpyAsync(S.p, X0, sizeof(double2) * nb * d, cudaMemcpyDeviceToDevice, st));
  int ns = 0;
  FQ_TRY(orthonormalize(ws, S.p, nb, d, drop, &ns, st));
  std::vector<double> rq_h(3 * n2);
  std::vector<double2> lam_h(n2);
  int nk = 0;
  for (int it = 0;; ++it) {
    // Rayleigh-Ritz with U on span(S): G = S^H U S = Yg diag(lam) Yg^{-1}
    FQ_TRY(apply_u<double>(op, S.p, WS.p, ns, ns, st));
    FQ_TRY(gemm_cn(ws, S.p, d, 0, WS.p, d, 0, d, ns, ns, 1, G.p, ns, 0, st));
    FQ_TRY(small_eig_batched(G.p, ns, 0, ns, 1, lam.p, 0, Yg.p, ns, 0, eigw.p, info.p, st));
    int info_h = 0;
    FQ_CUDA(cudaMemcpyAsync(lam_h.data(), lam.p, sizeof(double2) * ns, cudaMemcpyDeviceToHost,
                            st));
    FQ_CUDA(cudaMemcpyAsync(&info_h, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaStreamSynchronize(st));
    if (info_h) {
      set_error("polish: small eigensolver did not converge (n = %d)", ns);
      return FLOQUET_ENOCONV;
    }
    // keep the nk = min(nb, ns) Ritz values with the largest |g_k(omega)|
    nk = std::min(nb, ns);
    std::vector<int> order(ns);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> gabs(ns);
    // Ritz values off the unit circle are mixtures (a converged pair with ||omega| - 1|
    // ~ resid^2 / 2 is far closer to it); rank them after every value on the circle
    for (int i = 0; i < ns; ++i) {
      const cd l(lam_h[i].x, lam_h[i].y);
      gabs[i] = std::abs(gk_value(l, phi, k));
      if (std::fabs(std::abs(l) - 1.0) > 1e-8) gabs[i] *= 1e-6;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gabs[a] > gabs[b]; });
    order.resize(nk);
    for (int i = 0; i < nk; ++i)
      FQ_CUDA(cudaMemcpyAsync(G.p + (size_t)i * ns, Yg.p + (size_t)order[i] * ns,
                              sizeof(double2) * ns, cudaMemcpyDeviceToDevice, st));
    FQ_TRY(gemm_nn(S.p, d, 0, G.p, ns, 0, Xn.p, d, 0, d, ns, nk, 1, st));
    FQ_TRY(gemm_nn(WS.p, d, 0, G.p, ns, 0, corr.p, d, 0, d, ns, nk, 1, st));  // U Xn
    FQ_TRY(rayleigh_residual(ws, Xn.p, corr.p, d, nk, rq.p, st));
    FQ_CUDA(cudaMemcpyAsync(rq_h.data(), rq.p, sizeof(double) * 3 * nk, cudaMemcpyDeviceToHost,
                            st));
    FQ_CUDA(cudaStreamSynchronize(st));
    std::vector<cd> om(nk);
    for (int i = 0; i < nk; ++i) om[i] = cd(rq_h[3 * i], rq_h[3 * i + 1]);
    // Rayleigh-Ritz over an extended space also yields mixtures of eigenvectors whose
    // Rayleigh quotients sit inside the unit disk; an eigenpair with residual r has
    // ||omega| - 1| ~ r^2 / 2, so only values within 1e-8 of the circle (residual below
    // ~1e-4) inside the main lobe are candidates.
    std::vector<cd> om_c(nk);
    for (int i = 0; i < nk; ++i)
      om_c[i] = std::fabs(std::abs(om[i]) - 1.0) < 1e-8 ? om[i] : cd(0.0, 0.0);
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
    // residual vectors of the pairs still above a tenth of the target (the others are
    // locked: they stay in the Rayleigh-Ritz space but are not filtered again)
    std::vector<int> act;
    for (int i = 0; i < nk; ++i)
      if (rq_h[3 * i + 2] > 0.1 * tol_resid) act.push_back(i);
    const int nf = (int)act.size();
    if (verbose) {
      fprintf(stderr, "floquet polish: iter %d space %d block %d worst selected resid %.3e, "
              "filtering %d\n", it, ns, nk, worst, nf);
      int wi = -1;
      for (int i : sel)
        if (wi < 0 || rq_h[3 * i + 2] > rq_h[3 * wi + 2]) wi = i;
      if (wi >= 0)
        fprintf(stderr, "  worst pair: block index %d |omega|-1 %.2e angle %.4e |g| %.4e "
                "(block |g| range %.4e .. %.4e), candidates %d\n", wi,
                std::abs(om[wi]) - 1.0, wrapped_angle(om[wi], phi),
                std::abs(gk_value(om[wi], phi, k)), gabs[order[0]], gabs[order[nk - 1]],
                (int)sel.size());
    }
    worst_hist.push_back(worst);
    const bool stalled = it >= 3 && std::isfinite(worst) && std::isfinite(worst_hist[it - 3]) &&
                         !(worst < 0.5 * worst_hist[it - 3]);
    if (!forced && !df_corr && (stalled || (df_from >= 0 && it >= df_from))) {
      df_corr = true;  // complex64 corrections have stalled (or the switch is requested)
      if (verbose)
        fprintf(stderr, "floquet polish: switching to double-float corrections at iteration %d\n",
                it);
    }
    if (worst <= tol_resid || it >= max_iter || nf == 0) {
      FQ_CUDA(cudaMemcpyAsync(X0, Xn.p, sizeof(double2) * nk * d, cudaMemcpyDeviceToDevice, st));
      break;
    }
    FQ_TRY(residual_vectors(Xn.p, corr.p, R.p, d, nk, rq.p, st));
    std::vector<cd> om_act(nf);
    for (int j = 0; j < nf; ++j) {
      const int i = act[j];
      if (i != j)
        FQ_CUDA(cudaMemcpyAsync(R.p + (size_t)j * d, R.p + (size_t)i * d, sizeof(double2) * d,
                                cudaMemcpyDeviceToDevice, st));
      om_act[j] = om[i];
    }
    FQ_TRY(polish_correction(op, phi, k, om_act.data(), R.p, corr.p, nf, df_corr, st));
    // span(S) = span(Xn, g_k(U) Xn_active) = span(Xn, corr_active)
    FQ_CUDA(cudaMemcpyAsync(S.p, Xn.p, sizeof(double2) * nk * d, cudaMemcpyDeviceToDevice, st));
    FQ_CUDA(cudaMemcpyAsync(S.p + (size_t)nk * d, corr.p, sizeof(double2) * nf * d,
                            cudaMemcpyDeviceToDevice, st));
    FQ_TRY(orthonormalize(ws, S.p, nk + nf, d, drop, &ns, st));
  }
  return FLOQUET_OK;
}

}  // namespace fq
