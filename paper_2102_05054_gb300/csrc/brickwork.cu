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
// operator is created. The complex128 products run in cuBLAS ZGEMM (plain library GEMMs); the
// double-float sweeps of the filter (FLOQUET_C128_DF) run in this file's own split-K complex
// GEMM on the FP32 pipes (each real an unevaluated sum of two floats, error-free
// transformations), since the part's FP64 rate is 1/58 of its FP32 rate.
#include <cublas_v2.h>

#include <cmath>
#include <complex>
#include <vector>

#include "pass_kernel.cuh"

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
  std::vector<float4> ULd(UL.size()), URd(UR.size());
  for (size_t i = 0; i < UL.size(); ++i) ULd[i] = from_d2<dfloat>(UL[i]);
  for (size_t i = 0; i < UR.size(); ++i) URd[i] = from_d2<dfloat>(UR[i]);
  FQ_CUDA(cudaMalloc(&b->ULdf, ULd.size() * sizeof(float4)));
  FQ_CUDA(cudaMalloc(&b->URdf, URd.size() * sizeof(float4)));
  FQ_CUDA(cudaMemcpy(b->ULdf, ULd.data(), ULd.size() * sizeof(float4), cudaMemcpyHostToDevice));
  FQ_CUDA(cudaMemcpy(b->URdf, URd.data(), URd.size() * sizeof(float4), cudaMemcpyHostToDevice));
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
  cudaFree(b->ULdf);
  cudaFree(b->URdf);
  cudaFree(b->part);
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


// ------------------------------------------------------------------ double-float GEMM

namespace {
constexpr int kTM = 32, kTN = 32, kTK = 16, kGemmThreads = 128;

// acc += a * b for double-float complex values (float4: re.hi, re.lo, im.hi, im.lo); the
// pairs are left unnormalised (see df_fma_lazy) and renormalised once per K chunk
__device__ __forceinline__ void df_cmac(float4& acc, float4 a, float4 b) {
  const float2 ar = make_float2(a.x, a.y), ai = make_float2(a.z, a.w);
  const float2 br = make_float2(b.x, b.y), bi = make_float2(b.z, b.w);
  float2 re = df_fma_lazy(ar, br, make_float2(acc.x, acc.y));
  re = df_fma_lazy(df_neg(ai), bi, re);
  float2 im = df_fma_lazy(ar, bi, make_float2(acc.z, acc.w));
  im = df_fma_lazy(ai, br, im);
  acc = make_float4(re.x, re.y, im.x, im.y);
}
}  // namespace

// Partial products P[s][v] (M x N column-major) = sum over l in split s of A_v(i, l) B_v(l, j),
// A_v(i, l) = A[v * sa + i * a_i + l * a_l], B_v(l, j) = B[v * sb + l * b_l + j * b_j].
// One CTA per 32 x 32 output tile, vector and K split; each thread keeps 2 x 4 outputs.
__global__ void __launch_bounds__(kGemmThreads) df_gemm_partial_kernel(
    const float4* __restrict__ A, int64_t sa, int64_t a_i, int64_t a_l,
    const float4* __restrict__ B, int64_t sb, int64_t b_l, int64_t b_j, int M, int N, int K,
    int kslab, int nvec, float4* __restrict__ P) {
  __shared__ float4 As[kTK][kTM + 1];
  __shared__ float4 Bs[kTK][kTN + 1];
  const int tilesM = (M + kTM - 1) / kTM;
  const int i0 = (blockIdx.x % tilesM) * kTM, j0 = (blockIdx.x / tilesM) * kTN;
  const int v = blockIdx.y, s = blockIdx.z;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;  // outputs rows 2tx..2tx+1, cols 4ty..4ty+3
  const float4* Av = A + (int64_t)v * sa;
  const float4* Bv = B + (int64_t)v * sb;
  float4 acc[2][4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float4(0, 0, 0, 0);
  const int l_begin = s * kslab, l_end = min(K, l_begin + kslab);
  for (int l0 = l_begin; l0 < l_end; l0 += kTK) {
    // A chunk: 32 rows x 16 k; lanes along whichever index has unit stride
    for (int q = 0; q < (kTM * kTK) / kGemmThreads; ++q) {
      const int e = t + q * kGemmThreads;
      int i, l;
      if (a_i == 1) {
        i = e % kTM;
        l = e / kTM;
      } else {
        l = e % kTK;
        i = e / kTK;
      }
      const int gi = i0 + i, gl = l0 + l;
      As[l][i] = (gi < M && gl < l_end) ? Av[gi * a_i + gl * a_l] : make_float4(0, 0, 0, 0);
    }
    for (int q = 0; q < (kTN * kTK) / kGemmThreads; ++q) {
      const int e = t + q * kGemmThreads;
      int j, l;
      if (b_j == 1) {
        j = e % kTN;
        l = e / kTN;
      } else {
        l = e % kTK;
        j = e / kTK;
      }
      const int gj = j0 + j, gl = l0 + l;
      Bs[l][j] = (gj < N && gl < l_end) ? Bv[gl * b_l + gj * b_j] : make_float4(0, 0, 0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < kTK; ++l) {
      const float4 a0 = As[l][2 * tx], a1 = As[l][2 * tx + 1];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float4 bb = Bs[l][4 * ty + b];
        df_cmac(acc[0][b], a0, bb);
        df_cmac(acc[1][b], a1, bb);
      }
    }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 4; ++b) acc[a][b] = df_renorm(acc[a][b]);
    __syncthreads();
  }
  float4* Pv = P + ((int64_t)s * nvec + v) * (int64_t)M * N;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 4; ++b) {
      const int gi = i0 + 2 * tx + a, gj = j0 + 4 * ty + b;
      if (gi < M && gj < N) Pv[gi + (int64_t)gj * M] = acc[a][b];
    }
}

__device__ __forceinline__ float4 df_cadd(float4 a, float4 b) {
  const float2 r = df_two_sum(a.x, b.x), i = df_two_sum(a.z, b.z);
  const float2 rr = df_quick_two_sum(r.x, r.y + (a.y + b.y));
  const float2 ii = df_quick_two_sum(i.x, i.y + (a.w + b.w));
  return make_float4(rr.x, rr.y, ii.x, ii.y);
}

// C_v = sum_s P[s][v] (splits added in order); horner: C_v = pin_v + z_v * sum. C_v is
// column-major M x N with leading dimension M at C + v * sc.
__global__ void df_gemm_finish_kernel(const float4* __restrict__ P, int nsplit, int M, int N,
                                      int nvec, float4* __restrict__ C, int64_t sc,
                                      const float4* __restrict__ pin, const float4* __restrict__ zs) {
  const int64_t per = (int64_t)M * N;
  const int v = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per;
       e += (int64_t)gridDim.x * blockDim.x) {
    float4 sum = P[(int64_t)v * per + e];
    for (int s = 1; s < nsplit; ++s) sum = df_cadd(sum, P[((int64_t)s * nvec + v) * per + e]);
    if (zs) sum = zfma(zs[v], sum, pin[(int64_t)v * sc + e]);
    C[(int64_t)v * sc + e] = sum;
  }
}

// K splits of a double-float GEMM: enough CTAs for the GPU (~4 per SM), at least 64 of K per
// split.
static int df_splits(int M, int N, int K, int nvec) {
  const int64_t tiles = (int64_t)((M + kTM - 1) / kTM) * ((N + kTN - 1) / kTN) * nvec;
  int64_t s = (152 * 4 + tiles - 1) / tiles;
  s = std::min<int64_t>(s, std::max(1, K / 64));
  return (int)std::max<int64_t>(1, s);
}

// C_v = A_v B_v (store) or pin_v + z_v A_v B_v (horner: pin, zs non-null), double-float
static int df_gemm(BrickOp* b, const float4* A, int64_t sa, int64_t a_i, int64_t a_l,
                   const float4* B, int64_t sb, int64_t b_l, int64_t b_j, int M, int N, int K,
                   int nvec, float4* C, int64_t sc, const float4* pin, const float4* zs,
                   cudaStream_t st) {
  const int ns = df_splits(M, N, K, nvec);
  if ((size_t)ns * nvec * M * N > b->part_elems) {
    set_error("brickwork: double-float GEMM scratch not reserved");
    return FLOQUET_EINVAL;
  }
  const int kslab = ((K + ns - 1) / ns + kTK - 1) / kTK * kTK;
  const int tiles = ((M + kTM - 1) / kTM) * ((N + kTN - 1) / kTN);
  df_gemm_partial_kernel<<<dim3(tiles, nvec, ns), kGemmThreads, 0, st>>>(
      A, sa, a_i, a_l, B, sb, b_l, b_j, M, N, K, kslab, nvec, b->part);
  count_launch();
  FQ_CHECK_LAUNCH();
  const int64_t per = (int64_t)M * N;
  const unsigned gx = (unsigned)std::min<int64_t>((per + 255) / 256, 1024);
  df_gemm_finish_kernel<<<dim3(gx, nvec), 256, 0, st>>>(b->part, ns, M, N, nvec, C, sc, pin, zs);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

int brick_reserve_df(BrickOp* b, int nvec) {
  FQ_TRY(brick_reserve(b, nvec));  // the intermediate T (reinterpreted as double-float)
  const int64_t d = (int64_t)1 << b->L, m = (int64_t)1 << b->q;
  const int sr = df_splits((int)m, (int)b->dR, (int)b->dR, nvec);
  const int sl = df_splits((int)b->dL, (int)(d / b->dL), (int)b->dL, nvec);
  const size_t need = (size_t)std::max(sr, sl) * nvec * d;
  if (b->part_elems >= need) return FLOQUET_OK;
  cudaFree(b->part);
  b->part = nullptr;
  b->part_elems = 0;
  if (cudaMalloc(&b->part, need * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    set_error("brickwork: cudaMalloc of %zu bytes failed", need * sizeof(float4));
    return FLOQUET_ENOMEM;
  }
  b->part_elems = need;
  return FLOQUET_OK;
}

// acc_v = psi_in_v + z_v U acc_v in double-float: T_v = acc_v U_R^T (acc_v as 2^q x d_R),
// then acc_v = psi_in_v + z_v U_L T_v (T_v as d_L x d / d_L)
int brick_horner_step_df(BrickOp* b, float4* acc, const float4* psi_in, const float4* zs,
                         int nvec, cudaStream_t st) {
  const int64_t d = (int64_t)1 << b->L, m = (int64_t)1 << b->q;
  float4* T = reinterpret_cast<float4*>(b->tmp);
  // T(i, j) = sum_l acc(i + l m) U_R(j, l) = sum_l acc(i, l) U_R(j + l dR)
  FQ_TRY(df_gemm(b, acc, d, 1, m, b->URdf, 0, b->dR, 1, (int)m, (int)b->dR, (int)b->dR, nvec,
                 T, d, nullptr, nullptr, st));
  // acc(i, j) = pin + z sum_l U_L(i + l dL) T(l + j dL)
  FQ_TRY(df_gemm(b, b->ULdf, 0, 1, b->dL, T, d, 1, b->dL, (int)b->dL, (int)(d / b->dL),
                 (int)b->dL, nvec, acc, d, psi_in, zs, st));
  return FLOQUET_OK;
}

}  // namespace fq
