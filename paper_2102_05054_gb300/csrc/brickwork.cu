// The paper's own Floquet operator: a two-layer brickwork circuit of two-qubit gates (Luitz,
// arXiv:2102.05054, Sec. 2, Eqs. U, unitary), applied as two dense matrix products
// (Eq. matvec).
//
// Circuit (0-based qubits, L even, qubit i = bit i): U = U_a U_b, U_b = u_0 u_{1,2} u_{3,4}
// ... u_{L-3,L-2} u_{L-1} acting first, U_a = u_{0,1} u_{2,3} ... u_{L-2,L-1}. Bond gate
// indices are b_i + 2 b_{i+1}.
//
// Split. For an odd qubit q, the gates on qubits <= q (U_a bonds i <= q - 1, U_b bonds
// i <= q - 2 and u_0) form U_L on the q + 1 low qubits, the others (U_a bonds i >= q + 1,
// U_b bonds i >= q and u_{L-1}) form U_R on the L - q high qubits; the two parts share qubit
// q only through the U_b gate (q, q+1) (in U_R, applied first) and the U_a gate (q-1, q) (in
// U_L, applied second), and every other pair commutes, so U = (U_L x 1)(1 x U_R). With
// psi as a column-major 2^q x d_R matrix (rows: the q low bits) the first product is
// psi U_R^T, and with psi as a d_L x (d / d_L) matrix the second is U_L psi: two complex
// GEMMs on two reshapes of the same buffer, no data movement. q is the odd value that
// minimises d_L + d_R = 2^(q+1) + 2^(L-q) (about 2 sqrt(2d), as the paper advises).
//
// U_L and U_R are built on the host in float64 (gate by gate on the unit vectors) when the
// operator is created; the products run in cuBLAS ZGEMM (plain library GEMMs, float64).
#include <cublas_v2.h>

#include <cmath>
#include <complex>
#include <vector>

#include "floquet_internal.cuh"

namespace fq {

using cd = std::complex<double>;

#define FQ_CUBLAS(call)                                                                   \
  do {                                                                                    \
    cublasStatus_t _s = (call);                                                           \
    if (_s != CUBLAS_STATUS_SUCCESS) {                                                    \
      ::fq::set_error("%s failed: cuBLAS status %d (%s:%d)", #call, (int)_s, __FILE__,    \
                      __LINE__);                                                          \
      return FLOQUET_ECUDA;                                                               \
    }                                                                                     \
  } while (0)

// u (4 x 4, row-major, indices b_i + 2 b_{i+1}) on qubits (i, i+1) of an n-qubit vector
static void host_gate2(std::vector<cd>& x, int n, int i, const cd* u) {
  const int64_t dim = (int64_t)1 << n, lo = (int64_t)1 << i, hi = (int64_t)1 << (i + 1);
  for (int64_t s = 0; s < dim; ++s) {
    if (s & (lo | hi)) continue;  // s: both bits zero
    const int64_t idx[4] = {s, s | lo, s | hi, s | lo | hi};  // local index b_i + 2 b_{i+1}
    cd in[4], out[4];
    for (int c = 0; c < 4; ++c) in[c] = x[idx[c]];
    for (int r = 0; r < 4; ++r) {
      out[r] = 0;
      for (int c = 0; c < 4; ++c) out[r] += u[4 * r + c] * in[c];
    }
    for (int r = 0; r < 4; ++r) x[idx[r]] = out[r];
  }
}

// u (2 x 2, row-major) on qubit q
static void host_gate1(std::vector<cd>& x, int n, int q, const cd* u) {
  const int64_t dim = (int64_t)1 << n, b = (int64_t)1 << q;
  for (int64_t s = 0; s < dim; ++s) {
    if (s & b) continue;
    const cd a0 = x[s], a1 = x[s | b];
    x[s] = u[0] * a0 + u[1] * a1;
    x[s | b] = u[2] * a0 + u[3] * a1;
  }
}

struct Gate {
  int kind;   // 1 or 2 qubits
  int qubit;  // local qubit (the bond's low qubit for two-qubit gates)
  const cd* u;
};

// dense column-major matrix of the gate sequence (applied in order) on n qubits
static std::vector<double2> host_dense(int n, const std::vector<Gate>& gates) {
  const int64_t dim = (int64_t)1 << n;
  std::vector<double2> M((size_t)(dim * dim));
  std::vector<cd> x((size_t)dim);
  for (int64_t c = 0; c < dim; ++c) {
    std::fill(x.begin(), x.end(), cd(0, 0));
    x[(size_t)c] = 1;
    for (const Gate& g : gates) {
      if (g.kind == 1) host_gate1(x, n, g.qubit, g.u);
      else host_gate2(x, n, g.qubit, g.u);
    }
    for (int64_t r = 0; r < dim; ++r) M[(size_t)(c * dim + r)] = make_double2(x[r].real(), x[r].imag());
  }
  return M;
}

static int choose_split(int L) {
  int best = 1;
  int64_t cost = INT64_MAX;
  for (int q = 1; q <= L - 1; q += 2) {
    const int64_t c = ((int64_t)1 << (q + 1)) + ((int64_t)1 << (L - q));
    if (c < cost) {
      cost = c;
      best = q;
    }
  }
  return best;
}

int brick_init(floquet_op* op, int L, const double* g2, const double* g1) {
  BrickOp* b = new BrickOp();
  op->brick = b;
  op->L = L;
  op->d = (int64_t)1 << L;
  op->nprob = 1;
  op->J = op->g = op->tau = 0;
  op->swap = false;
  const int q = choose_split(L);
  b->L = L;
  b->q = q;
  b->dL = (int64_t)1 << (q + 1);
  b->dR = (int64_t)1 << (L - q);
  std::vector<cd> G2((size_t)(L - 1) * 16), G1(8);
  for (size_t i = 0; i < G2.size(); ++i) G2[i] = cd(g2[2 * i], g2[2 * i + 1]);
  for (size_t i = 0; i < G1.size(); ++i) G1[i] = cd(g1[2 * i], g1[2 * i + 1]);
  // U_L = A_left B_left on qubits 0..q: B_left (u_0, odd bonds i <= q-2) first
  std::vector<Gate> left, right;
  left.push_back({1, 0, &G1[0]});
  for (int i = 1; i <= q - 2; i += 2) left.push_back({2, i, &G2[16 * i]});
  for (int i = 0; i <= q - 1; i += 2) left.push_back({2, i, &G2[16 * i]});
  // U_R = A_right B_right on qubits q..L-1 (local qubit = global - q): B_right (odd bonds
  // i >= q, u_{L-1}) first
  for (int i = q; i <= L - 3; i += 2) right.push_back({2, i - q, &G2[16 * i]});
  right.push_back({1, L - 1 - q, &G1[4]});
  for (int i = q + 1; i <= L - 2; i += 2) right.push_back({2, i - q, &G2[16 * i]});
  const std::vector<double2> UL = host_dense(q + 1, left), UR = host_dense(L - q, right);
  FQ_CUDA(cudaMalloc(&b->UL, UL.size() * sizeof(double2)));
  FQ_CUDA(cudaMalloc(&b->UR, UR.size() * sizeof(double2)));
  FQ_CUDA(cudaMemcpy(b->UL, UL.data(), UL.size() * sizeof(double2), cudaMemcpyHostToDevice));
  FQ_CUDA(cudaMemcpy(b->UR, UR.data(), UR.size() * sizeof(double2), cudaMemcpyHostToDevice));
  const double2 consts[2] = {make_double2(1, 0), make_double2(0, 0)};
  FQ_CUDA(cudaMalloc(&b->consts, sizeof(consts)));
  FQ_CUDA(cudaMemcpy(b->consts, consts, sizeof(consts), cudaMemcpyHostToDevice));
  cublasHandle_t h;
  FQ_CUBLAS(cublasCreate(&h));
  b->cublas = h;
  // a fixed workspace, so that no GEMM allocates (also inside a captured filter graph)
  b->ws_bytes = (size_t)32 << 20;
  FQ_CUDA(cudaMalloc(&b->ws, b->ws_bytes));
  FQ_CUBLAS(cublasSetWorkspace(h, b->ws, b->ws_bytes));
  return FLOQUET_OK;
}

void brick_free(BrickOp* b) {
  if (!b) return;
  if (b->cublas) cublasDestroy((cublasHandle_t)b->cublas);
  cudaFree(b->UL);
  cudaFree(b->UR);
  cudaFree(b->tmp);
  cudaFree(b->apply_tmp);
  cudaFree(b->consts);
  cudaFree(b->ws);
  delete b;
}

static int grow(double2** p, size_t* elems, size_t need) {
  if (*elems >= need) return FLOQUET_OK;
  cudaFree(*p);
  *p = nullptr;
  *elems = 0;
  if (cudaMalloc(p, need * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    set_error("brickwork: cudaMalloc of %zu bytes failed", need * sizeof(double2));
    return FLOQUET_ENOMEM;
  }
  *elems = need;
  return FLOQUET_OK;
}

int brick_reserve(BrickOp* b, int nvec) {
  return grow(&b->tmp, &b->tmp_elems, (size_t)nvec << b->L);
}

// tmp_v = psi_v U_R^T for every vector (psi_v as a column-major 2^q x d_R matrix)
static int gemm_right(BrickOp* b, const double2* in, double2* tmp, int nvec, cudaStream_t st) {
  cublasHandle_t h = (cublasHandle_t)b->cublas;
  const int64_t d = (int64_t)1 << b->L, m = (int64_t)1 << b->q;
  const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
  FQ_CUBLAS(cublasSetStream(h, st));
  FQ_CUBLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
  FQ_CUBLAS(cublasZgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_T, (int)m, (int)b->dR,
                                      (int)b->dR, &one, (const cuDoubleComplex*)in, (int)m, d,
                                      (const cuDoubleComplex*)b->UR, (int)b->dR, 0, &zero,
                                      (cuDoubleComplex*)tmp, (int)m, d, nvec));
  count_launch();
  return FLOQUET_OK;
}

// out_v = U_L tmp_v (tmp_v as a column-major d_L x (d / d_L) matrix)
static int gemm_left(BrickOp* b, const double2* tmp, double2* out, int nvec, cudaStream_t st) {
  cublasHandle_t h = (cublasHandle_t)b->cublas;
  const int64_t d = (int64_t)1 << b->L, n = d / b->dL;
  const cuDoubleComplex one = make_cuDoubleComplex(1, 0), zero = make_cuDoubleComplex(0, 0);
  FQ_CUBLAS(cublasSetStream(h, st));
  FQ_CUBLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
  FQ_CUBLAS(cublasZgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)b->dL, (int)n,
                                      (int)b->dL, &one, (const cuDoubleComplex*)b->UL,
                                      (int)b->dL, 0, (const cuDoubleComplex*)tmp,
                                      (int)b->dL, d, &zero, (cuDoubleComplex*)out,
                                      (int)b->dL, d, nvec));
  count_launch();
  return FLOQUET_OK;
}

int brick_apply(BrickOp* b, const double2* in, double2* out, int nvec, cudaStream_t st) {
  FQ_TRY(grow(&b->apply_tmp, &b->apply_tmp_elems, (size_t)nvec << b->L));
  FQ_TRY(gemm_right(b, in, b->apply_tmp, nvec, st));
  return gemm_left(b, b->apply_tmp, out, nvec, st);
}

// Horner step: acc_v = psi_in_v + z_v U acc_v (z_v: device, one per vector)
int brick_horner_step(BrickOp* b, double2* acc, const double2* psi_in, const double2* zs,
                      int nvec, cudaStream_t st) {
  cublasHandle_t h = (cublasHandle_t)b->cublas;
  const int64_t d = (int64_t)1 << b->L, n = d / b->dL;
  FQ_TRY(gemm_right(b, acc, b->tmp, nvec, st));
  FQ_CUDA(cudaMemcpyAsync(acc, psi_in, sizeof(double2) * d * nvec, cudaMemcpyDeviceToDevice,
                          st));
  FQ_CUBLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_DEVICE));
  for (int v = 0; v < nvec; ++v) {
    FQ_CUBLAS(cublasZgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)b->dL, (int)n, (int)b->dL,
                          (const cuDoubleComplex*)(zs + v), (const cuDoubleComplex*)b->UL,
                          (int)b->dL, (const cuDoubleComplex*)(b->tmp + v * d), (int)b->dL,
                          (const cuDoubleComplex*)b->consts, (cuDoubleComplex*)(acc + v * d),
                          (int)b->dL));
    count_launch();
  }
  FQ_CUBLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
  return FLOQUET_OK;
}

// accumulate step: work_v = U work_v; acc_v += coef[v * coef_stride + j] work_v
int brick_acc_step(BrickOp* b, double2* work, double2* acc, const double2* coef,
                   int64_t coef_stride, int j, int nvec, cudaStream_t st) {
  cublasHandle_t h = (cublasHandle_t)b->cublas;
  const int64_t d = (int64_t)1 << b->L;
  FQ_TRY(gemm_right(b, work, b->tmp, nvec, st));
  FQ_TRY(gemm_left(b, b->tmp, work, nvec, st));
  FQ_CUBLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_DEVICE));
  for (int v = 0; v < nvec; ++v) {
    FQ_CUBLAS(cublasZaxpy(h, (int)d, (const cuDoubleComplex*)(coef + v * coef_stride + j),
                          (const cuDoubleComplex*)(work + v * d), 1,
                          (cuDoubleComplex*)(acc + v * d), 1));
    count_launch();
  }
  FQ_CUBLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
  return FLOQUET_OK;
}

}  // namespace fq
