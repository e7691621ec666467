// Krylov-Schur eigensolver on g_k(U) (solver.cu).
#pragma once

#include <complex>
#include <vector>

#include "floquet_internal.cuh"

namespace fq {

// Owning device buffer of the solver's results.
struct DevVec {
  double2* p = nullptr;
  size_t n = 0;
  int alloc(size_t count);
  DevVec() = default;
  DevVec(const DevVec&) = delete;
  DevVec& operator=(const DevVec&) = delete;
  DevVec(DevVec&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevVec& operator=(DevVec&& o) noexcept {
    std::swap(p, o.p);
    std::swap(n, o.n);
    return *this;
  }
  ~DevVec();
};

struct KSOut {
  bool converged = false;
  std::vector<std::complex<double>> omega;  // nev, closest first
  std::vector<double> resid;                // nev
  DevVec vecs;                              // d x nblock (or d x nev) complex128
  std::vector<int> cols;                    // columns of vecs holding the nev pairs
  int nblock = 0;
};

struct KSStats {
  int restarts = 0;
  int64_t expansions = 0;
  int polish_iters = 0;
};

// B problems in lockstep; problem b uses the op's phase tables b / vpp and target phis[b].
int krylov_schur(floquet_op* op, int B, int vpp, const double* phis, int64_t k, int nev, int m,
                 int precision, double tol, double tol_resid, int max_restarts,
                 const double2* v0_dev, std::vector<KSOut>& out, cudaStream_t st,
                 KSStats* stats);

// The polish's correction step: out_j = q_j(U) r_j with q_j the defect polynomial of the
// k-term filter at target phi and Ritz value omega[j] (g_k(U) - g_k(omega_j) = q_j(U)(U - omega_j)),
// in complex64 (df = false) or double-float (df = true) sweeps; R and out are d x n complex128.
int polish_correction(floquet_op* op, double phi, int64_t K, const std::complex<double>* omega,
                      const double2* R, double2* out, int n, bool df, cudaStream_t st);

}  // namespace fq
