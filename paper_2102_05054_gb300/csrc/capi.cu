// C ABI entry points (include/floquet.h): argument checking, pointer classification and the
// calls into the operator, filter and eigensolver code.

#include <cmath>
#include <complex>
#include <algorithm>
#include <cstring>
#include <vector>

#include "floquet_internal.cuh"
#include "linalg.cuh"
#include "solver.cuh"

namespace fq {
int64_t launch_count();
void reset_launch_count();
int profile_enable(int on);
int profile_read(double* ms, int64_t* apps, double* bytes);
}  // namespace fq

using namespace fq;

#define FQ_GUARD_BEGIN try {
#define FQ_GUARD_END                                   \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    set_error("host allocation failed");               \
    return FLOQUET_ENOMEM;                             \
  }                                                    \
  catch (...) {                                        \
    set_error("unexpected C++ exception");             \
    return FLOQUET_ECUDA;                              \
  }

static int clear_and(int rc) {
  if (rc == FLOQUET_OK) set_error("%s", "");
  return rc;
}

template <typename Real> static int dtype_code();
template <> int dtype_code<float>() { return FLOQUET_C64; }
template <> int dtype_code<double>() { return FLOQUET_C128; }
template <> int dtype_code<dfloat>() { return FLOQUET_C128_DF; }

// Coefficients z^j = exp(-i j phi) in float64 (no recurrence), then rounded to Real.
template <typename Real>
static int upload_geometric_coef(floquet_op* op, double phi, int64_t k, int nvec,
                                 cudaStream_t st) {
  const size_t bytes = (size_t)k * nvec * sizeof(cplx<Real>);
  const int dt = dtype_code<Real>();
  if (op->coef && op->coef_bytes >= bytes && op->coef_phi == phi && op->coef_k == k &&
      op->coef_dtype == dt && op->coef_nvec == nvec && op->coef_form == FLOQUET_FORM_ACC)
    return FLOQUET_OK;
  if (op->coef_bytes < bytes) {
    FQ_CUDA(cudaStreamSynchronize(st));
    cudaFree(op->coef);
    op->coef = nullptr;
    op->coef_bytes = 0;
    FQ_CUDA(cudaMalloc(&op->coef, bytes));
    op->coef_bytes = bytes;
  }
  std::vector<cplx<Real>> h((size_t)k * nvec);
  for (int64_t j = 0; j < k; ++j) {
    const double ang = -phi * (double)j;
    const cplx<Real> z = from_d2<Real>(make_double2(cos(ang), sin(ang)));
    for (int v = 0; v < nvec; ++v) h[(size_t)v * k + j] = z;
  }
  FQ_CUDA(cudaStreamSynchronize(st));
  FQ_CUDA(cudaMemcpy(op->coef, h.data(), bytes, cudaMemcpyHostToDevice));
  op->coef_phi = phi;
  op->coef_k = k;
  op->coef_dtype = dt;
  op->coef_nvec = nvec;
  op->coef_form = FLOQUET_FORM_ACC;
  return FLOQUET_OK;
}

template <typename Real>
static int upload_horner_z(floquet_op* op, double phi, int nvec, cudaStream_t st) {
  const size_t bytes = (size_t)nvec * sizeof(cplx<Real>);
  const int dt = dtype_code<Real>();
  if (op->coef && op->coef_bytes >= bytes && op->coef_phi == phi && op->coef_dtype == dt &&
      op->coef_nvec == nvec && op->coef_form == FLOQUET_FORM_HORNER)
    return FLOQUET_OK;
  if (op->coef_bytes < bytes) {
    FQ_CUDA(cudaStreamSynchronize(st));
    cudaFree(op->coef);
    op->coef = nullptr;
    op->coef_bytes = 0;
    FQ_CUDA(cudaMalloc(&op->coef, bytes));
    op->coef_bytes = bytes;
  }
  std::vector<cplx<Real>> h(nvec, from_d2<Real>(make_double2(cos(-phi), sin(-phi))));
  FQ_CUDA(cudaStreamSynchronize(st));
  FQ_CUDA(cudaMemcpy(op->coef, h.data(), bytes, cudaMemcpyHostToDevice));
  op->coef_phi = phi;
  op->coef_k = -1;
  op->coef_dtype = dt;
  op->coef_nvec = nvec;
  op->coef_form = FLOQUET_FORM_HORNER;
  return FLOQUET_OK;
}

template <typename Real, typename Rio>
static int filter_apply_t(floquet_t op, double phi, int64_t k, const void* in, void* out,
                          int nvec, int form, cudaStream_t st) {
  using C = cplx<Real>;
  using CIO = cplx<Rio>;
  if (form == FLOQUET_FORM_ACC) {
    FQ_TRY(upload_geometric_coef<Real>(op, phi, k, nvec, st));
    return filter_coef<Real, Rio>(op, (const CIO*)in, op->d, (CIO*)out, op->d,
                                  (const C*)op->coef, k, nvec, nvec, true, st);
  }
  FQ_TRY(upload_horner_z<Real>(op, phi, nvec, st));
  return filter_horner<Real, Rio>(op, (const CIO*)in, op->d, (CIO*)out, op->d,
                                  (const C*)op->coef, k, nvec, nvec, true, st);
}

// U applied with double-float sweeps to complex128 states (through a float4 copy)
static int apply_u_df(floquet_t op, const double2* in, double2* out, int nvec, cudaStream_t st);


// True if p is device (or managed) memory of some device; false for host memory.
static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Owning device buffer for the C ABI's temporaries.
struct Tmp {
  void* p = nullptr;
  int alloc(size_t bytes) {
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("cudaMalloc of %zu bytes failed", bytes);
      return FLOQUET_ENOMEM;
    }
    return FLOQUET_OK;
  }
  ~Tmp() { cudaFree(p); }
};

// Copy `bytes` from host-or-device `src` into a device buffer.
static int to_device(const void* src, size_t bytes, Tmp& dst, cudaStream_t st) {
  FQ_TRY(dst.alloc(bytes));
  FQ_CUDA(cudaMemcpyAsync(dst.p, src, bytes,
                          is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          st));
  return FLOQUET_OK;
}

static int copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t st) {
  FQ_CUDA(cudaMemcpyAsync(dst, src_dev, bytes,
                          is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          st));
  return FLOQUET_OK;
}

static int solve_and_copy(floquet_op* op, int B, int vpp, const double* phis, int64_t k, int nev,
                          int m, int precision, double tol, double tol_resid, int max_restarts,
                          const void* v0, double* evals, void* evecs, double* resid,
                          int* n_conv, cudaStream_t st) {
  const int64_t d = op->d;
  Tmp v0d;
  FQ_TRY(to_device(v0, sizeof(double2) * d, v0d, st));
  std::vector<KSOut> out;
  const int rc = krylov_schur(op, B, vpp, phis, k, nev, m, precision, tol, tol_resid,
                              max_restarts, (const double2*)v0d.p, out, st, nullptr);
  if (rc != FLOQUET_OK && rc != FLOQUET_ENOCONV) return rc;
  for (int b = 0; b < B; ++b) {
    const KSOut& o = out[b];
    int nc = 0;
    for (int i = 0; i < nev; ++i) {
      const bool have = o.converged && i < (int)o.omega.size();
      evals[2 * ((size_t)b * nev + i)] = have ? o.omega[i].real() : 0.0;
      evals[2 * ((size_t)b * nev + i) + 1] = have ? o.omega[i].imag() : 0.0;
      resid[(size_t)b * nev + i] = have ? o.resid[i] : INFINITY;
      if (have && o.resid[i] <= tol_resid) ++nc;
      if (have && evecs && B == 1)
        FQ_TRY(copy_out((double2*)evecs + (size_t)i * d, o.vecs.p + (size_t)o.cols[i] * d,
                        sizeof(double2) * d, st));
    }
    n_conv[b] = nc;
  }
  FQ_CUDA(cudaStreamSynchronize(st));
  return rc;
}

static int apply_u_df(floquet_t op, const double2* in, double2* out, int nvec, cudaStream_t st) {
  const int64_t n = (int64_t)nvec * op->d;
  Tmp buf;
  FQ_TRY(buf.alloc(sizeof(float4) * n));
  float4* b = (float4*)buf.p;
  FQ_TRY((launch_convert<double, dfloat>(in, b, n, st)));
  FQ_TRY(apply_u<dfloat>(op, b, b, nvec, nvec, st));
  FQ_TRY((launch_convert<dfloat, double>(b, out, n, st)));
  FQ_CUDA(cudaStreamSynchronize(st));  // the scratch is freed on return
  return FLOQUET_OK;
}

extern "C" {

int floquet_create(int L, double J, double g, const double* h, floquet_t* out) {
  FQ_GUARD_BEGIN
  if (!out || !h) {
    set_error("floquet_create: NULL argument");
    return FLOQUET_EINVAL;
  }
  *out = nullptr;
  if (L < 3 || L > 24) {
    set_error("floquet_create: L = %d outside [3, 24]", L);
    return FLOQUET_EINVAL;
  }
  if (!std::isfinite(J) || !std::isfinite(g)) {
    set_error("floquet_create: J and g must be finite");
    return FLOQUET_EINVAL;
  }
  for (int i = 0; i < L; ++i)
    if (!std::isfinite(h[i])) {
      set_error("floquet_create: h[%d] is not finite", i);
      return FLOQUET_EINVAL;
    }
  floquet_op* op = new floquet_op();
  const int rc = op_init(op, L, J, g, h, 1);
  if (rc != FLOQUET_OK) {
    op_free(op);
    delete op;
    return rc;
  }
  *out = op;
  return clear_and(FLOQUET_OK);
  FQ_GUARD_END
}

int brickwork_create(int L, const double* g2, const double* g1, floquet_t* out) {
  FQ_GUARD_BEGIN
  if (!out || !g2 || !g1) {
    set_error("brickwork_create: NULL argument");
    return FLOQUET_EINVAL;
  }
  *out = nullptr;
  if (L < 4 || L > 24 || (L & 1)) {
    set_error("brickwork_create: L = %d must be even and in [4, 24]", L);
    return FLOQUET_EINVAL;
  }
  for (int i = 0; i < 32 * (L - 1); ++i)
    if (!std::isfinite(g2[i])) {
      set_error("brickwork_create: g2[%d] is not finite", i);
      return FLOQUET_EINVAL;
    }
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(g1[i])) {
      set_error("brickwork_create: g1[%d] is not finite", i);
      return FLOQUET_EINVAL;
    }
  floquet_op* op = new floquet_op();
  const int rc = brick_init(op, L, g2, g1);
  if (rc != FLOQUET_OK) {
    op_free(op);
    delete op;
    return rc;
  }
  *out = op;
  return clear_and(FLOQUET_OK);
  FQ_GUARD_END
}

int floquet_destroy(floquet_t op) {
  if (!op) return FLOQUET_OK;
  op_free(op);
  delete op;
  return FLOQUET_OK;
}

int floquet_dim(floquet_t op, int64_t* d) {
  if (!op || !d) {
    set_error("floquet_dim: NULL argument");
    return FLOQUET_EINVAL;
  }
  *d = op->d;
  return FLOQUET_OK;
}

int floquet_apply_u(floquet_t op, const void* psi_in, void* psi_out, int nvec, int dtype,
                    void* stream) {
  FQ_GUARD_BEGIN
  if (!op || !psi_in || !psi_out || nvec < 1) {
    set_error("floquet_apply_u: NULL pointer or nvec < 1");
    return FLOQUET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if (dtype == FLOQUET_C128)
    rc = apply_u<double>(op, (const double2*)psi_in, (double2*)psi_out, nvec, nvec, st);
  else if (dtype == FLOQUET_C64)
    rc = apply_u<float>(op, (const float2*)psi_in, (float2*)psi_out, nvec, nvec, st);
  else if (dtype == FLOQUET_C128_DF)
    rc = apply_u_df(op, (const double2*)psi_in, (double2*)psi_out, nvec, st);
  else {
    set_error("floquet_apply_u: bad dtype %d", dtype);
    return FLOQUET_EINVAL;
  }
  return clear_and(rc);
  FQ_GUARD_END
}

int filter_apply(floquet_t op, double phi, int64_t k, const void* psi_in, void* psi_out,
                 int nvec, int dtype, int form, void* stream) {
  FQ_GUARD_BEGIN
  if (!op || !psi_in || !psi_out || nvec < 1 || k < 1) {
    set_error("filter_apply: NULL pointer, nvec < 1 or k < 1");
    return FLOQUET_EINVAL;
  }
  if (!std::isfinite(phi)) {
    set_error("filter_apply: phi must be finite");
    return FLOQUET_EINVAL;
  }
  if (form != FLOQUET_FORM_ACC && form != FLOQUET_FORM_HORNER) {
    set_error("filter_apply: bad form %d", form);
    return FLOQUET_EINVAL;
  }
  const size_t esz = dtype == FLOQUET_C64 ? 8 : 16;
  const char* a = (const char*)psi_in;
  const char* b = (const char*)psi_out;
  const size_t bytes = (size_t)nvec * op->d * esz;
  if (a < b + bytes && b < a + bytes) {
    set_error("filter_apply: psi_in and psi_out overlap");
    return FLOQUET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if (dtype == FLOQUET_C128)
    rc = filter_apply_t<double, double>(op, phi, k, psi_in, psi_out, nvec, form, st);
  else if (dtype == FLOQUET_C64)
    rc = filter_apply_t<float, float>(op, phi, k, psi_in, psi_out, nvec, form, st);
  else if (dtype == FLOQUET_C128_DF)
    rc = filter_apply_t<dfloat, double>(op, phi, k, psi_in, psi_out, nvec, form, st);
  else {
    set_error("filter_apply: bad dtype %d", dtype);
    return FLOQUET_EINVAL;
  }
  return clear_and(rc);
  FQ_GUARD_END
}

int floquet_polish_correction(floquet_t op, double phi, int64_t K, const double* omega,
                              const void* R, void* out, int n, int sweep, void* stream) {
  FQ_GUARD_BEGIN
  if (!op || !omega || !R || !out || n < 1 || K < 2) {
    set_error("floquet_polish_correction: NULL pointer, n < 1 or K < 2");
    return FLOQUET_EINVAL;
  }
  if (op->brick) {
    set_error("floquet_polish_correction: kicked-Ising operators only");
    return FLOQUET_EINVAL;
  }
  if (sweep != FLOQUET_C64 && sweep != FLOQUET_C128_DF) {
    set_error("floquet_polish_correction: sweep must be FLOQUET_C64 or FLOQUET_C128_DF");
    return FLOQUET_EINVAL;
  }
  if (!std::isfinite(phi)) {
    set_error("floquet_polish_correction: phi not finite");
    return FLOQUET_EINVAL;
  }
  const char* a = (const char*)R;
  const char* b = (const char*)out;
  const size_t bytes = (size_t)n * op->d * 16;
  if (a < b + bytes && b < a + bytes) {
    set_error("floquet_polish_correction: R and out overlap");
    return FLOQUET_EINVAL;
  }
  std::vector<std::complex<double>> om(n);
  for (int j = 0; j < n; ++j) {
    om[j] = std::complex<double>(omega[2 * j], omega[2 * j + 1]);
    if (!std::isfinite(om[j].real()) || !std::isfinite(om[j].imag())) {
      set_error("floquet_polish_correction: omega %d not finite", j);
      return FLOQUET_EINVAL;
    }
  }
  const int rc = polish_correction(op, phi, K, om.data(), (const double2*)R, (double2*)out, n,
                                   sweep == FLOQUET_C128_DF, (cudaStream_t)stream);
  return clear_and(rc);
  FQ_GUARD_END
}

int gram_schmidt(int64_t d, const void* V, int n, void* w, double* h, void* stream) {
  FQ_GUARD_BEGIN
  if (d < 1 || n < 0 || !w || !h || (n > 0 && !V)) {
    set_error("gram_schmidt: bad arguments");
    return FLOQUET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  Tmp hcol;
  FQ_TRY(hcol.alloc(sizeof(double2) * (n + 1)));
  FQ_TRY(cgs2(ws, (const double2*)V, d, 0, n, (double2*)w, 0, d, 1, (double2*)hcol.p, 0,
              (double2*)w, 0, st));
  FQ_CUDA(cudaMemcpyAsync(h, hcol.p, sizeof(double2) * (n + 1), cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaStreamSynchronize(st));
  return clear_and(FLOQUET_OK);
  FQ_GUARD_END
}

int small_eig(int n, const void* A, double* lambda, void* Y, void* stream) {
  FQ_GUARD_BEGIN
  if (n < 1 || n > 512 || !A || !lambda) {
    set_error("small_eig: n = %d outside [1, 512] or NULL pointer", n);
    return FLOQUET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t mb = sizeof(double2) * n * n;
  Tmp Ad, Yd, lam, work, info;
  FQ_TRY(to_device(A, mb, Ad, st));
  FQ_TRY(Yd.alloc(mb));
  FQ_TRY(lam.alloc(sizeof(double2) * n));
  FQ_TRY(work.alloc(sizeof(double2) * small_eig_work_elems(n)));
  FQ_TRY(info.alloc(sizeof(int)));
  FQ_TRY(small_eig_batched((const double2*)Ad.p, n, 0, n, 1, (double2*)lam.p, 0, (double2*)Yd.p,
                           n, 0, (double2*)work.p, (int*)info.p, st));
  FQ_CUDA(cudaMemcpyAsync(lambda, lam.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
  if (Y) FQ_TRY(copy_out(Y, Yd.p, mb, st));
  int inf = 0;
  FQ_CUDA(cudaMemcpyAsync(&inf, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaStreamSynchronize(st));
  if (inf) {
    set_error("small_eig: QR iteration did not converge");
    return FLOQUET_ENOCONV;
  }
  return clear_and(FLOQUET_OK);
  FQ_GUARD_END
}

int ritz_residuals(floquet_t op, const void* X, int nvec, double* omega, double* resid,
                   void* stream) {
  FQ_GUARD_BEGIN
  if (!op || !X || nvec < 1 || !omega || !resid) {
    set_error("ritz_residuals: bad arguments");
    return FLOQUET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t d = op->d;
  Tmp W, out;
  Workspace ws;
  FQ_TRY(W.alloc(sizeof(double2) * d * nvec));
  FQ_TRY(out.alloc(sizeof(double) * 3 * nvec));
  FQ_TRY(apply_u<double>(op, (const double2*)X, (double2*)W.p, nvec, nvec, st));
  FQ_TRY(rayleigh_residual(ws, (const double2*)X, (const double2*)W.p, d, nvec, (double*)out.p,
                           st));
  std::vector<double> h(3 * (size_t)nvec);
  FQ_CUDA(cudaMemcpyAsync(h.data(), out.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < nvec; ++i) {
    omega[2 * i] = h[3 * i];
    omega[2 * i + 1] = h[3 * i + 1];
    resid[i] = h[3 * i + 2];
  }
  return clear_and(FLOQUET_OK);
  FQ_GUARD_END
}

static int check_eig_args(int64_t d, int64_t k, int nev, int m, int precision, int max_restarts) {
  if (k < 2 || nev < 1 || m <= nev || m > 512 || (int64_t)m > d || max_restarts < 0 ||
      (precision != FLOQUET_FP64 && precision != FLOQUET_FILTER_FP32 &&
       precision != FLOQUET_FILTER_DF) ||
      k > (1LL << 24)) {
    set_error("eigensolver: need 2 <= k <= 2^24, 1 <= nev < m <= min(d, 512), max_restarts >= "
              "0, valid precision (k=%lld nev=%d m=%d precision=%d)",
              (long long)k, nev, m, precision);
    return FLOQUET_EINVAL;
  }
  return FLOQUET_OK;
}

int arnoldi_eigs(floquet_t op, double phi, int64_t k, int nev, int m, int precision, double tol,
                 double tol_resid, int max_restarts, const void* v0, double* evals, void* evecs,
                 double* resid, int* n_conv, void* stream) {
  FQ_GUARD_BEGIN
  if (!op || !v0 || !evals || !resid || !n_conv || !std::isfinite(phi)) {
    set_error("arnoldi_eigs: NULL pointer or non-finite phi");
    return FLOQUET_EINVAL;
  }
  FQ_TRY(check_eig_args(op->d, k, nev, m, precision, max_restarts));
  if (tol <= 0) tol = precision == FLOQUET_FILTER_FP32 ? 1e-6 : 1e-12;
  if (tol_resid <= 0) tol_resid = 1e-10;
  const int rc = solve_and_copy(op, 1, 1, &phi, k, nev, m, precision, tol, tol_resid,
                                max_restarts, v0, evals, evecs, resid, n_conv,
                                (cudaStream_t)stream);
  if (rc == FLOQUET_ENOCONV) set_error("arnoldi_eigs: max_restarts reached");
  return rc == FLOQUET_OK ? clear_and(rc) : rc;
  FQ_GUARD_END
}

int arnoldi_eigs_batched(int L, double J, double g, const double* h, int R, const double* phis,
                         int P, int64_t k, int nev, int m, int precision, double tol,
                         double tol_resid, int max_restarts, const void* v0, double* evals,
                         double* resid, int* n_conv, void* stream) {
  FQ_GUARD_BEGIN
  if (!h || !phis || !v0 || !evals || !resid || !n_conv || R < 1 || P < 1 || L < 3 || L > 24 ||
      (int64_t)R * P > 65535) {
    set_error("arnoldi_eigs_batched: bad arguments");
    return FLOQUET_EINVAL;
  }
  if (precision != FLOQUET_FP64 && precision != FLOQUET_FILTER_DF) {
    set_error("arnoldi_eigs_batched: precision must be FLOQUET_FP64 or FLOQUET_FILTER_DF");
    return FLOQUET_EINVAL;
  }
  FQ_TRY(check_eig_args((int64_t)1 << L, k, nev, m, precision, max_restarts));
  if (tol <= 0) tol = 1e-12;
  if (tol_resid <= 0) tol_resid = 1e-10;
  floquet_op op;
  int rc = op_init(&op, L, J, g, h, R);
  if (rc == FLOQUET_OK) {
    std::vector<double> ph((size_t)R * P);
    for (int r = 0; r < R; ++r)
      for (int p = 0; p < P; ++p) ph[(size_t)r * P + p] = phis[p];
    rc = solve_and_copy(&op, R * P, P, ph.data(), k, nev, m, precision, tol, tol_resid,
                        max_restarts, v0, evals, nullptr, resid, n_conv, (cudaStream_t)stream);
  }
  op_free(&op);
  if (rc == FLOQUET_ENOCONV) set_error("arnoldi_eigs_batched: max_restarts reached");
  return rc == FLOQUET_OK ? clear_and(rc) : rc;
  FQ_GUARD_END
}

int floquet_profile_enable(int on) { return profile_enable(on); }
int floquet_profile_read(double* sweep_ms, int64_t* u_applications, double* alg_bytes) {
  return profile_read(sweep_ms, u_applications, alg_bytes);
}

int64_t floquet_launch_count(void) { return launch_count(); }
void floquet_reset_launch_count(void) { reset_launch_count(); }

const char* floquet_last_error(void) { return get_error(); }

}  // extern "C"

// ------------------------------------------------------------------ parameter rule (Secs. 4-5)

extern "C" int floquet_suggest_params(int L, int nev, int max_m, int64_t* k, int* m) {
  if (L < 3 || L > 24 || nev < 1 || !k || !m) {
    set_error("floquet_suggest_params: need 3 <= L <= 24, nev >= 1 and output pointers");
    return FLOQUET_EINVAL;
  }
  const int64_t d = (int64_t)1 << L;
  const int64_t cap = std::min<int64_t>(max_m, d - 1);
  if ((int64_t)2 * nev + 1 > cap) {
    set_error("floquet_suggest_params: 2 nev + 1 = %d exceeds min(max_m, d - 1) = %lld",
              2 * nev + 1, (long long)cap);
    return FLOQUET_EINVAL;
  }
  // floor(2^(L/2 + 1)) = integer square root of 2^(L + 2)
  const int64_t sq = (int64_t)1 << (L + 2);
  int64_t r = (int64_t)std::sqrt((double)sq);
  while (r * r > sq) --r;
  while ((r + 1) * (r + 1) <= sq) ++r;
  int64_t mm = std::max<int64_t>(r, (int64_t)2 * nev + 1);
  mm = std::min<int64_t>(mm, cap);
  // round(2^(L+3) / (5 m)) = floor((2^(L+4) + 5 m) / (10 m))
  int64_t kk = (((int64_t)1 << (L + 4)) + 5 * mm) / (10 * mm);
  if (kk < 2) kk = 2;
  *k = kk;
  *m = (int)mm;
  return FLOQUET_OK;
}

// ------------------------------------------------------------------ entanglement entropy (Sec. 5)

namespace fq {
int entanglement_entropy_run(int L, const double2* X, int nvec, const int* cuts, int ncut,
                             double* S, cudaStream_t st);
}

extern "C" int entanglement_entropy(int L, const void* X, int nvec, const int* cuts, int ncut,
                                    double* S, void* stream) {
  if (L < 1 || L > 24 || !X || nvec < 1 || nvec > 65535 || !cuts || ncut < 1 || !S) {
    set_error("entanglement_entropy: need 1 <= L <= 24, 1 <= nvec <= 65535, ncut >= 1 and "
              "non-NULL pointers");
    return FLOQUET_EINVAL;
  }
  for (int c = 0; c < ncut; ++c) {
    if (cuts[c] < 0 || cuts[c] > L) {
      set_error("entanglement_entropy: cut %d = %d outside [0, L]", c, cuts[c]);
      return FLOQUET_EINVAL;
    }
    // the Householder reduction runs in one CTA per matrix of side 2^min(L_A, L - L_A)
    if (std::min(cuts[c], L - cuts[c]) > 11) {
      set_error("entanglement_entropy: cut %d = %d needs a reduced density matrix of side "
                "2^%d > 2048", c, cuts[c], std::min(cuts[c], L - cuts[c]));
      return FLOQUET_EINVAL;
    }
  }
  if (!is_device_ptr(X)) {
    set_error("entanglement_entropy: X must be device memory");
    return FLOQUET_EINVAL;
  }
  return fq::entanglement_entropy_run(L, (const double2*)X, nvec, cuts, ncut, S,
                                      (cudaStream_t)stream);
}
