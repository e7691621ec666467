// Declarations of the complex128 Krylov-basis kernels (linalg.cu) and the small dense
// eigensolver (smalleig.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fq {

// Device scratch reused across calls (grown on demand, freed with the owner).
struct Workspace {
  double2* part = nullptr;
  size_t part_cap = 0;
  double2* small = nullptr;
  size_t small_cap = 0;
  double* npart = nullptr;
  size_t npart_cap = 0;
  // results of the last cgs2 call (point into `small`)
  double* last_betas = nullptr;
  double2* last_h1 = nullptr;
  double2* last_h2 = nullptr;
  int reserve_part(size_t n_complex);
  int reserve_small(size_t n_complex);
  int reserve_npart(size_t n_double);
  ~Workspace();

 private:
  static int grow(void** p, size_t* cap, size_t bytes);
};

// CGS2 for B problems: w_b <- w_b - V_b V_b^H w_b twice (n columns of V_b, leading dimension
// ldv, problem stride strideV). Writes the summed coefficients to Hcol_b[0..n) and the norm
// to Hcol_b[n] (if Hcol), and vnext_b = w_b / beta_b (if vnext).
int cgs2(Workspace& ws, const double2* V, int64_t ldv, int64_t strideV, int n, double2* w,
         int64_t strideW, int64_t d, int B, double2* Hcol, int64_t strideH, double2* vnext,
         int64_t strideVn, cudaStream_t st);

void add_kernel_launch(const double2* a, const double2* b, int n, int B, double2* out,
                       int64_t ostride, cudaStream_t st);
void copy_matrix_launch(const double2* a, int64_t lda, int64_t sa, double2* b, int64_t ldb,
                        int64_t sb, int rows, int cols, int batch, cudaStream_t st);

// C_b = A_b B_b (A: d x m tall-skinny, B: m x p small), column-major.
int gemm_nn(const double2* A, int64_t lda, int64_t strideA, const double2* B, int64_t ldb,
            int64_t strideB, double2* C, int64_t ldc, int64_t strideC, int64_t d, int m, int p,
            int batch, cudaStream_t st);

// G_b = A_b^H B_b (n1 x n2), reduced over the d rows.
int gemm_cn(Workspace& ws, const double2* A, int64_t lda, int64_t strideA, const double2* B,
            int64_t ldb, int64_t strideB, int64_t d, int n1, int n2, int batch, double2* G,
            int64_t ldg, int64_t strideG, cudaStream_t st);

// out[3j..3j+2] = (Re omega_j, Im omega_j, resid_j), omega_j = <x_j|w_j>/<x_j|x_j>,
// resid_j = ||w_j - omega_j x_j|| / ||x_j||, for W = U X (device output).
int rayleigh_residual(Workspace& ws, const double2* X, const double2* W, int64_t d, int n,
                      double* out, cudaStream_t st);

int scale_cols(double2* X, int64_t d, int n, const double2* s, cudaStream_t st);
int axpy_cols(const double2* X, double2* Y, int64_t d, int n, const double2* a,
              cudaStream_t st);
int residual_vectors(const double2* X, const double2* W, double2* R, int64_t d, int n,
                     const double* om3, cudaStream_t st);
// C[:, j] -= T[:, j] for j < n (d rows; leading dimensions ldc, ldt).
int sub_cols(double2* C, int64_t ldc, const double2* T, int64_t ldt, int64_t d, int n,
             cudaStream_t st);

// Small dense eigensolver (one CTA per matrix): A_b (n x n, lda) = Y_b diag(lam_b) Y_b^{-1}.
// Y has unit-norm columns; eigenvalues in descending modulus. `work` must hold
// small_eig_work_elems(n) complex per matrix. info_b = 0, or the QR sweep count limit hit.
__host__ __device__ size_t small_eig_work_elems(int n);
int small_eig_batched(const double2* A, int64_t lda, int64_t strideA, int n, int batch,
                      double2* lam, int64_t strideLam, double2* Y, int64_t ldy,
                      int64_t strideY, double2* work, int* info, cudaStream_t st);

// Q_b (n x p) = orthonormal basis of the columns of Y_b (n x p), by twice-iterated
// modified Gram-Schmidt in one CTA per matrix.
int small_orth_batched(const double2* Y, int64_t ldy, int64_t strideY, int n, int p, int batch,
                       double2* Q, int64_t ldq, int64_t strideQ, cudaStream_t st);

// C_b = op(A_b) * op(B_b) for small matrices; opA/opB: 'N' or 'C' (conjugate transpose).
int small_gemm_batched(char opA, char opB, int M, int N, int K, const double2* A, int64_t lda,
                       int64_t strideA, const double2* B, int64_t ldb, int64_t strideB,
                       double2* C, int64_t ldc, int64_t strideC, int batch, cudaStream_t st);

}  // namespace fq
