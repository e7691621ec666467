// Small dense complex eigensolver on the device: the Ritz pairs of the projected matrix
// H_m = V^H g_k(U) V of Sec. 4 (Eq. arnoldi) of Luitz, arXiv:2102.05054, where the paper
// relies on ARPACK's dense routines. One CTA per matrix, matrices in global memory (they are
// small and stay in L1/L2):
//   1. Householder reduction to upper Hessenberg form, Q accumulated;
//   2. implicit single-shift complex QR sweeps with Wilkinson shifts and deflation, giving
//      the Schur form T = Z^H A Z;
//   3. eigenvectors of T by back substitution, Y = Z X, unit-norm columns;
//   4. eigenvalues sorted by descending modulus (the 'LM' order used for g_k(U)).
// Also: twice-iterated classical Gram-Schmidt of a few columns and small batched GEMMs.

#include <cfloat>

#include "floquet_internal.cuh"
#include "linalg.cuh"

namespace fq {

static constexpr int kEigThreads = 512;

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 conj_(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  const double r = b.x / b.y, den = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
__device__ double2 csqrt_(double2 z) {
  const double m = cabs_(z);
  if (m == 0) return make_double2(0, 0);
  const double re = sqrt(0.5 * (m + fabs(z.x)));
  const double t = z.y / (2 * re);
  if (z.x >= 0) return make_double2(re, t);
  return make_double2(fabs(t), z.y >= 0 ? re : -re);
}

template <typename T> __device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

__host__ __device__ size_t small_eig_work_elems(int n) { return (size_t)3 * n * n + 2 * (size_t)n; }

// work layout per matrix: T (n*n), Z (n*n), X (n*n), v (n), tmp (n)
__global__ void __launch_bounds__(kEigThreads) small_eig_kernel(
    const double2* __restrict__ A, int64_t lda, int64_t strideA, int n, double2* lam,
    int64_t strideLam, double2* Y, int64_t ldy, int64_t strideY, double2* work, int* info) {
  __shared__ double red[kEigThreads / 32];
  __shared__ double2 rot_s;
  __shared__ double rot_c;
  __shared__ int sh_lo, sh_hi, sh_done;
  __shared__ double2 sh_mu;
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  double2* T = work + b * (int64_t)small_eig_work_elems(n);
  double2* Z = T + (int64_t)n * n;
  double2* X = Z + (int64_t)n * n;
  double2* v = X + (int64_t)n * n;
  double2* tmp = v + n;
  const double2* Ab = A + b * strideA;
#define TT(r, c) T[(int64_t)(c) * n + (r)]
#define ZZ(r, c) Z[(int64_t)(c) * n + (r)]
#define XX(r, c) X[(int64_t)(c) * n + (r)]
  for (int64_t i = tid; i < (int64_t)n * n; i += nt) {
    const int r = (int)(i % n), c = (int)(i / n);
    TT(r, c) = Ab[(int64_t)c * lda + r];
    ZZ(r, c) = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();

  // ---- 1. Householder reduction to Hessenberg form
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;
    double sq = 0;
    for (int i = tid; i < len; i += nt) sq += cabs2(TT(j + 1 + i, j));
    const double xnorm2 = block_sum(sq, red);
    const double2 x0 = TT(j + 1, j);
    const double tail = xnorm2 - cabs2(x0);
    if (tail <= 1e-300) {  // nothing below the subdiagonal
      __syncthreads();
      continue;
    }
    const double xn = sqrt(xnorm2);
    const double ax0 = cabs_(x0);
    const double2 ph = ax0 > 0 ? cscale(x0, 1.0 / ax0) : make_double2(1, 0);
    const double2 alpha = cscale(ph, -xn);  // x -> alpha e1
    for (int i = tid; i < len; i += nt) v[i] = TT(j + 1 + i, j);
    __syncthreads();
    if (tid == 0) v[0] = make_double2(x0.x - alpha.x, x0.y - alpha.y);
    __syncthreads();
    double vv = 0;
    for (int i = tid; i < len; i += nt) vv += cabs2(v[i]);
    const double vnorm2 = block_sum(vv, red);
    const double beta = 2.0 / vnorm2;
    // left: T[j+1:, c] -= beta v (v^H T[j+1:, c]), columns c >= j
    for (int c = j + tid; c < n; c += nt) {
      double2 s = make_double2(0, 0);
      for (int i = 0; i < len; ++i) s = cfma(conj_(v[i]), TT(j + 1 + i, c), s);
      s = cscale(s, beta);
      for (int i = 0; i < len; ++i) {
        const double2 p = cmul(v[i], s);
        TT(j + 1 + i, c).x -= p.x;
        TT(j + 1 + i, c).y -= p.y;
      }
    }
    __syncthreads();
    // right: T[r, j+1:] -= beta (T[r, j+1:] v) v^H for all rows; same for Z
    for (int r = tid; r < 2 * n; r += nt) {
      double2* M = r < n ? T : Z;
      const int rr = r < n ? r : r - n;
      double2 s = make_double2(0, 0);
      for (int i = 0; i < len; ++i) s = cfma(M[(int64_t)(j + 1 + i) * n + rr], v[i], s);
      s = cscale(s, beta);
      for (int i = 0; i < len; ++i) {
        const double2 p = cmul(s, conj_(v[i]));
        M[(int64_t)(j + 1 + i) * n + rr].x -= p.x;
        M[(int64_t)(j + 1 + i) * n + rr].y -= p.y;
      }
    }
    __syncthreads();
    if (tid == 0) {
      TT(j + 1, j) = alpha;
      for (int i = j + 2; i < n; ++i) TT(i, j) = make_double2(0, 0);
    }
    __syncthreads();
  }

  // ---- 2. shifted QR to Schur form
  double fro = 0;
  for (int64_t i = tid; i < (int64_t)n * n; i += nt) fro += cabs2(T[i]);
  fro = sqrt(block_sum(fro, red));
  const double small_abs = DBL_EPSILON * fro + 1e-300;
  int its = 0, total = 0;
  const int max_total = 60 * n + 100;
  if (tid == 0) {
    sh_hi = n - 1;
    sh_done = 0;
  }
  __syncthreads();
  while (true) {
    if (tid == 0) {
      int hi = sh_hi;
      int lo = 0;
      while (hi > 0) {
        int l = hi;
        for (; l > 0; --l) {
          const double sub = cabs_(TT(l, l - 1));
          const double dsum = cabs_(TT(l - 1, l - 1)) + cabs_(TT(l, l));
          if (sub <= DBL_EPSILON * dsum || sub <= small_abs) {
            TT(l, l - 1) = make_double2(0, 0);
            break;
          }
        }
        if (l == hi) {
          --hi;
          its = 0;
          continue;
        }
        lo = l;
        break;
      }
      sh_hi = hi;
      sh_lo = lo;
      if (hi <= 0 || total >= max_total) {
        sh_done = 1;
      } else {
        // Wilkinson shift from the trailing 2x2 of the active block
        const double2 a = TT(hi - 1, hi - 1), bb = TT(hi - 1, hi), c = TT(hi, hi - 1),
                      dd = TT(hi, hi);
        double2 mu;
        if (its > 0 && its % 11 == 0) {
          // exceptional shift
          const double e = cabs_(c) + (hi >= 2 ? cabs_(TT(hi - 1, hi - 2)) : 0.0);
          mu = make_double2(dd.x + 0.75 * e, dd.y);
        } else {
          const double2 p = cscale(make_double2(a.x - dd.x, a.y - dd.y), 0.5);
          const double2 disc = csqrt_(cadd(cmul(p, p), cmul(bb, c)));
          const double2 m1 = cadd(dd, cadd(p, disc)), m2 = cadd(dd, csub(p, disc));
          const double d1 = cabs2(csub(m1, dd)), d2 = cabs2(csub(m2, dd));
          mu = d1 < d2 ? m1 : m2;
        }
        sh_mu = mu;
        ++its;
        ++total;
      }
    }
    __syncthreads();
    if (sh_done) break;
    const int lo = sh_lo, hi = sh_hi;
    const double2 mu = sh_mu;
    for (int k = lo; k < hi; ++k) {
      if (tid == 0) {
        double2 x, y;
        if (k == lo) {
          x = csub(TT(lo, lo), mu);
          y = TT(lo + 1, lo);
        } else {
          x = TT(k, k - 1);
          y = TT(k + 1, k - 1);
        }
        const double ax = cabs_(x), ay = cabs_(y);
        double c;
        double2 s;
        if (ay == 0) {
          c = 1;
          s = make_double2(0, 0);
        } else if (ax == 0) {
          c = 0;
          s = cscale(conj_(y), 1.0 / ay);
        } else {
          const double r = hypot(ax, ay);
          c = ax / r;
          s = cscale(cmul(cscale(x, 1.0 / ax), conj_(y)), 1.0 / r);
        }
        rot_c = c;
        rot_s = s;
      }
      __syncthreads();
      const double c = rot_c;
      const double2 s = rot_s;
      // rows k, k+1: [c s; -conj(s) c], columns max(k-1, lo) .. n-1
      for (int col = (k > lo ? k - 1 : lo) + tid; col < n; col += nt) {
        const double2 t1 = TT(k, col), t2 = TT(k + 1, col);
        TT(k, col) = cadd(cscale(t1, c), cmul(s, t2));
        TT(k + 1, col) = csub(cscale(t2, c), cmul(conj_(s), t1));
      }
      if (tid == 0 && k > lo) TT(k + 1, k - 1) = make_double2(0, 0);
      __syncthreads();
      // columns k, k+1 of T (rows 0 .. min(k+2, hi)) and of Z (all rows): M G^H
      const int rmax = min(k + 2, hi);
      for (int r = tid; r <= rmax + n; r += nt) {
        double2* M;
        int rr;
        if (r <= rmax) {
          M = T;
          rr = r;
        } else {
          M = Z;
          rr = r - rmax - 1;
          if (rr >= n) continue;
        }
        const double2 t1 = M[(int64_t)k * n + rr], t2 = M[(int64_t)(k + 1) * n + rr];
        M[(int64_t)k * n + rr] = cadd(cscale(t1, c), cmul(conj_(s), t2));
        M[(int64_t)(k + 1) * n + rr] = csub(cscale(t2, c), cmul(s, t1));
      }
      __syncthreads();
    }
  }
  if (tid == 0 && info) info[b] = (sh_hi > 0) ? 1 : 0;

  // ---- 3. eigenvectors of T by back substitution (one thread per eigenvector)
  const double smin = fmax(DBL_EPSILON * fro, 1e-300);
  for (int i = tid; i < n; i += nt) {
    const double2 ti = TT(i, i);
    for (int r = i + 1; r < n; ++r) XX(r, i) = make_double2(0, 0);
    XX(i, i) = make_double2(1, 0);
    for (int r = i - 1; r >= 0; --r) {
      double2 s = make_double2(0, 0);
      for (int c2 = r + 1; c2 <= i; ++c2) s = cfma(TT(r, c2), XX(c2, i), s);
      double2 den = csub(TT(r, r), ti);
      if (cabs_(den) < smin) den = make_double2(smin, 0);
      XX(r, i) = cdiv(make_double2(-s.x, -s.y), den);
    }
  }
  __syncthreads();

  // ---- 4. order by descending |lambda| (selection by rank, one thread per eigenvalue)
  int* rank = reinterpret_cast<int*>(tmp);  // n ints fit in n double2
  for (int i = tid; i < n; i += nt) {
    const double mi = cabs2(TT(i, i));
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double mj = cabs2(TT(j, j));
      if (mj > mi || (mj == mi && j < i)) ++rk;
    }
    rank[i] = rk;
  }
  __syncthreads();
  // Y[:, rank[i]] = Z X[:, i], normalised; lam[rank[i]] = T[i, i]
  double2* Yb = Y + b * strideY;
  double2* lb = lam + b * strideLam;
  for (int i = 0; i < n; ++i) {
    const int col = rank[i];
    double sq = 0;
    for (int r = tid; r < n; r += nt) {
      double2 s = make_double2(0, 0);
      for (int c2 = 0; c2 <= i; ++c2) s = cfma(ZZ(r, c2), XX(c2, i), s);
      v[r] = s;
      sq += cabs2(s);
    }
    const double nrm = sqrt(block_sum(sq, red));
    const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
    for (int r = tid; r < n; r += nt) Yb[(int64_t)col * ldy + r] = cscale(v[r], inv);
    if (tid == 0) lb[col] = TT(i, i);
    __syncthreads();
  }
#undef TT
#undef ZZ
#undef XX
}

int small_eig_batched(const double2* A, int64_t lda, int64_t strideA, int n, int batch,
                      double2* lam, int64_t strideLam, double2* Y, int64_t ldy,
                      int64_t strideY, double2* work, int* info, cudaStream_t st) {
  if (n < 1 || n > 1024 || batch < 1) {
    set_error("small_eig: n = %d outside [1, 1024]", n);
    return FLOQUET_EINVAL;
  }
  small_eig_kernel<<<batch, kEigThreads, 0, st>>>(A, lda, strideA, n, lam, strideLam, Y, ldy,
                                                  strideY, work, info);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// -------------------------------------------------------------- small orthonormalisation

// Q = orth(Y[:, :p]) column by column; each column is projected twice against the previous
// ones (classical Gram-Schmidt, all coefficients at once), then normalised.
__global__ void __launch_bounds__(256) small_orth_kernel(const double2* __restrict__ Y,
                                                         int64_t ldy, int64_t strideY, int n,
                                                         int p, double2* Q, int64_t ldq,
                                                         int64_t strideQ) {
  extern __shared__ double2 coef[];  // p
  __shared__ double red[8];
  const int64_t b = blockIdx.x;
  const double2* Yb = Y + b * strideY;
  double2* Qb = Q + b * strideQ;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < p; ++j) {
    for (int r = tid; r < n; r += nt) Qb[(int64_t)j * ldq + r] = Yb[(int64_t)j * ldy + r];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = tid; i < j; i += nt) {
        double2 s = make_double2(0, 0);
        for (int r = 0; r < n; ++r)
          s = cfma(conj_(Qb[(int64_t)i * ldq + r]), Qb[(int64_t)j * ldq + r], s);
        coef[i] = s;
      }
      __syncthreads();
      for (int r = tid; r < n; r += nt) {
        double2 s = Qb[(int64_t)j * ldq + r];
        for (int i = 0; i < j; ++i) s = csub(s, cmul(Qb[(int64_t)i * ldq + r], coef[i]));
        Qb[(int64_t)j * ldq + r] = s;
      }
      __syncthreads();
    }
    double sq = 0;
    for (int r = tid; r < n; r += nt) sq += cabs2(Qb[(int64_t)j * ldq + r]);
    const double nrm = sqrt(block_sum(sq, red));
    const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
    for (int r = tid; r < n; r += nt) Qb[(int64_t)j * ldq + r] = cscale(Qb[(int64_t)j * ldq + r], inv);
    __syncthreads();
  }
}

int small_orth_batched(const double2* Y, int64_t ldy, int64_t strideY, int n, int p, int batch,
                       double2* Q, int64_t ldq, int64_t strideQ, cudaStream_t st) {
  if (p < 1) return FLOQUET_OK;
  small_orth_kernel<<<batch, 256, (size_t)p * sizeof(double2), st>>>(Y, ldy, strideY, n, p, Q,
                                                                     ldq, strideQ);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// -------------------------------------------------------------- small GEMM

__global__ void small_gemm_kernel(bool ca, bool cb, int M, int N, int K,
                                  const double2* __restrict__ A, int64_t lda, int64_t strideA,
                                  const double2* __restrict__ B, int64_t ldb, int64_t strideB,
                                  double2* __restrict__ C, int64_t ldc, int64_t strideC) {
  const int64_t z = blockIdx.y;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  const double2* Ab = A + z * strideA;
  const double2* Bb = B + z * strideB;
  double2 s = make_double2(0, 0);
  for (int k = 0; k < K; ++k) {
    const double2 a = ca ? conj_(Ab[(int64_t)i * lda + k]) : Ab[(int64_t)k * lda + i];
    const double2 bb = cb ? conj_(Bb[(int64_t)k * ldb + j]) : Bb[(int64_t)j * ldb + k];
    s = cfma(a, bb, s);
  }
  C[z * strideC + (int64_t)j * ldc + i] = s;
}

int small_gemm_batched(char opA, char opB, int M, int N, int K, const double2* A, int64_t lda,
                       int64_t strideA, const double2* B, int64_t ldb, int64_t strideB,
                       double2* C, int64_t ldc, int64_t strideC, int batch, cudaStream_t st) {
  if (M < 1 || N < 1) return FLOQUET_OK;
  const int64_t n = (int64_t)M * N;
  small_gemm_kernel<<<dim3((unsigned)((n + 127) / 128), batch), 128, 0, st>>>(
      opA == 'C', opB == 'C', M, N, K, A, lda, strideA, B, ldb, strideB, C, ldc, strideC);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

}  // namespace fq
