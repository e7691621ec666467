// Entanglement entropy of eigenstates (Luitz, arXiv:2102.05054, Sec. 5, Eq. ee): cut the chain
// into A = qubits 0 .. L_A - 1 (the low bits of the amplitude index) and B = the rest;
// S_A = -sum_i lambda_i ln lambda_i over the eigenvalues of the reduced density matrix, which
// are the squared singular values of the state as a 2^{L_A} x 2^{L - L_A} matrix
// M[a, b] = psi[a + 2^{L_A} b].
//
// GPU route, per cut and state, all in float64:
//   1. G = X^H X, the Gram matrix of the smaller side (n = 2^{min(L_A, L - L_A)}): for the
//      smaller A, X[b, a] = M[a, b] and G = conj(rho_A); for the smaller B, X = M and
//      G = M^H M = rho_B^T. Both are Hermitian with the nonzero spectrum of rho_A.
//      Tiled 32 x 32 output tiles, the reduction over the other side split into slabs
//      whose partial sums are added in a fixed order (deterministic).
//   2. Householder reduction of G to a Hermitian tridiagonal matrix (one CTA per matrix):
//      for column k, v = x - alpha e_1 with alpha = -e^{i arg x_0} |x|, p = A v, K = v^H p,
//      w = 2 p - 2 K v, A <- A - v w^H - w v^H. The eigenvalues equal those of the real
//      symmetric tridiagonal with diagonal Re A_kk and off-diagonal |A_{k+1,k}|.
//   3. Every eigenvalue by bisection on Sturm counts (one thread per eigenvalue index),
//      then S = -sum lambda ln lambda over lambda > 0, summed in a fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "floquet_internal.cuh"

namespace fq {

static constexpr int kGramTile = 32;

// part[s][vec] (n x n, column-major) = sum over rows i in slab s of conj(X[i, c1]) X[i, c2],
// X[i, c] = psi_vec[i * rs + c * cs], rows i in [0, r).
__global__ void __launch_bounds__(256) gram_slab_kernel(const double2* __restrict__ X,
                                                        int64_t d, int64_t rs, int64_t cs,
                                                        int n, int64_t r, int64_t slab,
                                                        int nvec, double2* __restrict__ part) {
  __shared__ double2 A[kGramTile][kGramTile + 1];  // [row in chunk][column]
  __shared__ double2 B[kGramTile][kGramTile + 1];
  const int ntile = (n + kGramTile - 1) / kGramTile;
  const int t1 = blockIdx.x % ntile, t2 = blockIdx.x / ntile;
  const int vec = blockIdx.y, s = blockIdx.z;
  const double2* psi = X + (int64_t)vec * d;
  const int c1 = t1 * kGramTile, c2 = t2 * kGramTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in [0, 8)
  double2 acc[4];
  for (int q = 0; q < 4; ++q) acc[q] = make_double2(0, 0);
  const int64_t i0 = (int64_t)s * slab, i1 = (i0 + slab < r) ? i0 + slab : r;
  for (int64_t ib = i0; ib < i1; ib += kGramTile) {
    // load 32 rows x 32 columns of both column tiles; the lane index runs along the
    // unit-stride direction so that the loads are coalesced
    for (int q = 0; q < 4; ++q) {
      const int u = ty + 8 * q;
      int row, col;
      if (cs == 1) {
        row = u;
        col = tx;
      } else {
        row = tx;
        col = u;
      }
      const int64_t i = ib + row;
      double2 va = make_double2(0, 0), vb = make_double2(0, 0);
      if (i < i1) {
        if (c1 + col < n) va = psi[i * rs + (int64_t)(c1 + col) * cs];
        if (c2 + col < n) vb = psi[i * rs + (int64_t)(c2 + col) * cs];
      }
      A[row][col] = va;
      B[row][col] = vb;
    }
    __syncthreads();
    // thread (tx, ty) accumulates G[c1 + tx, c2 + ty + 8 q]
#pragma unroll 4
    for (int j = 0; j < kGramTile; ++j) {
      const double2 a = A[j][tx];
      for (int q = 0; q < 4; ++q) {
        const double2 b = B[j][ty + 8 * q];
        acc[q].x += a.x * b.x + a.y * b.y;  // conj(a) * b
        acc[q].y += a.x * b.y - a.y * b.x;
      }
    }
    __syncthreads();
  }
  double2* out = part + ((int64_t)s * nvec + vec) * n * n;
  for (int q = 0; q < 4; ++q) {
    const int row = c1 + tx, col = c2 + ty + 8 * q;
    if (row < n && col < n) out[(int64_t)col * n + row] = acc[q];
  }
}

// G[vec] = sum_s part[s][vec], slabs added in order
__global__ void gram_sum_kernel(const double2* __restrict__ part, int nsplit, int64_t per,
                                double2* __restrict__ G) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per;
       i += (int64_t)gridDim.x * blockDim.x) {
    double2 s = part[i];
    for (int k = 1; k < nsplit; ++k) {
      const double2 v = part[(int64_t)k * per + i];
      s.x += v.x;
      s.y += v.y;
    }
    G[i] = s;
  }
}

static constexpr int kTriThreads = 512;

__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

// Householder reduction of the Hermitian matrices G[vec] (n x n, column-major, overwritten)
// to tridiagonal form; writes diag[vec][k] = Re A_kk and off2[vec][k] = |A_{k+1,k}|^2.
// work: 2 n complex per matrix (v and p / w).
__global__ void __launch_bounds__(kTriThreads) hermitian_tridiag_kernel(
    double2* __restrict__ G, int n, double2* __restrict__ work, double* __restrict__ diag,
    double* __restrict__ off2) {
  __shared__ double red[kTriThreads / 32];
  const int vec = blockIdx.x;
  double2* A = G + (int64_t)vec * n * n;
  double2* v = work + (int64_t)vec * 2 * n;
  double2* p = v + n;
  double* dg = diag + (int64_t)vec * n;
  double* e2 = off2 + (int64_t)vec * n;
  const int t = threadIdx.x;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // trailing rows/columns k+1 .. n-1
    double2* col = A + (int64_t)k * n + (k + 1);
    double s = 0;
    for (int i = t; i < m; i += blockDim.x) s += col[i].x * col[i].x + col[i].y * col[i].y;
    const double norm2 = block_sum_d(s, red);
    const double2 x0 = col[0];
    const double ax0 = hypot(x0.x, x0.y);
    const double tail2 = norm2 - ax0 * ax0;
    if (!(tail2 > 1e-300 * (norm2 + 1e-300)) || norm2 == 0.0) {
      // column already reduced (tail zero): no reflection
      if (t == 0) e2[k] = ax0 * ax0;
      __syncthreads();
      continue;
    }
    const double nrm = sqrt(norm2);
    // alpha = -e^{i arg x0} |x|
    const double2 ph = ax0 > 0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
    const double2 alpha = make_double2(-ph.x * nrm, -ph.y * nrm);
    // v = x - alpha e_1 normalised; |x0 - alpha| = |x0| + |x|
    const double vn = sqrt(tail2 + (ax0 + nrm) * (ax0 + nrm));
    for (int i = t; i < m; i += blockDim.x) {
      double2 xi = col[i];
      if (i == 0) xi = make_double2(xi.x - alpha.x, xi.y - alpha.y);
      v[i] = make_double2(xi.x / vn, xi.y / vn);
    }
    __syncthreads();
    // p = A22 v, A22 = A[k+1:, k+1:]
    for (int i = t; i < m; i += blockDim.x) {
      double2 acc = make_double2(0, 0);
#pragma unroll 4
      for (int j = 0; j < m; ++j) {
        const double2 a = A[(int64_t)(k + 1 + j) * n + (k + 1 + i)];
        const double2 vj = v[j];
        acc.x += a.x * vj.x - a.y * vj.y;
        acc.y += a.x * vj.y + a.y * vj.x;
      }
      p[i] = acc;
    }
    __syncthreads();
    // K = v^H p (real for Hermitian A)
    double kk = 0;
    for (int i = t; i < m; i += blockDim.x) kk += v[i].x * p[i].x + v[i].y * p[i].y;
    const double K = block_sum_d(kk, red);
    // w = 2 p - 2 K v (in place of p)
    for (int i = t; i < m; i += blockDim.x)
      p[i] = make_double2(2 * p[i].x - 2 * K * v[i].x, 2 * p[i].y - 2 * K * v[i].y);
    __syncthreads();
    // A22 -= v w^H + w v^H
    for (int i = t; i < m; i += blockDim.x) {
      const double2 vi = v[i], wi = p[i];
#pragma unroll 4
      for (int j = 0; j < m; ++j) {
        const double2 vj = v[j], wj = p[j];
        double2& a = A[(int64_t)(k + 1 + j) * n + (k + 1 + i)];
        // vi conj(wj) + wi conj(vj)
        a.x -= vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
        a.y -= vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
      }
    }
    if (t == 0) e2[k] = nrm * nrm;  // the new subdiagonal is alpha, |alpha| = |x|
    __syncthreads();
  }
  for (int i = t; i < n; i += blockDim.x) dg[i] = A[(int64_t)i * n + i].x;
  if (t == 0 && n >= 2) {
    const double2 last = A[(int64_t)(n - 2) * n + (n - 1)];
    e2[n - 2] = last.x * last.x + last.y * last.y;
  }
}

// Number of eigenvalues of the symmetric tridiagonal (diag dg, squared off-diagonal e2) that
// are smaller than x (Sturm count through the LDL^T pivots).
__device__ int sturm_count(const double* dg, const double* e2, int n, double x) {
  int cnt = 0;
  double q = dg[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    if (q == 0) q = 1e-300;
    q = dg[i] - x - e2[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// S[vec * ncut + cut] = -sum lambda ln lambda over the eigenvalues (bisection) of the
// tridiagonal of matrix vec.
__global__ void __launch_bounds__(kTriThreads) tridiag_entropy_kernel(
    const double* __restrict__ diag, const double* __restrict__ off2, int n, double* S,
    int ncut, int cut) {
  __shared__ double red[kTriThreads / 32];
  const int vec = blockIdx.x;
  const double* dg = diag + (int64_t)vec * n;
  const double* e2 = off2 + (int64_t)vec * n;
  // Gershgorin interval
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < n ? sqrt(e2[i]) : 0.0);
    lo = fmin(lo, dg[i] - r);
    hi = fmax(hi, dg[i] + r);
  }
  const double span = fmax(hi - lo, 1e-300);
  lo -= 1e-14 * span;
  hi += 1e-14 * span;
  double s = 0;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    // the idx-th smallest eigenvalue: the x where the count passes idx
    // to an absolute width of 1e-16 of the spectral span: an eigenvalue lambda enters the
    // entropy as -lambda ln lambda, so one below that width changes S by < 1e-14
    double a = lo, b = hi;
    const double width = 1e-16 * fmax(span, 1.0);
    for (int it = 0; it < 100 && b - a > width; ++it) {
      const double mid = 0.5 * (a + b);
      if (sturm_count(dg, e2, n, mid) > idx) b = mid;
      else a = mid;
    }
    const double lam = 0.5 * (a + b);
    if (lam > 1e-300) s -= lam * log(lam);
  }
  const double tot = block_sum_d(s, red);
  if (threadIdx.x == 0) S[(int64_t)vec * ncut + cut] = tot;
}

// ------------------------------------------------------------------ driver

namespace {
struct DBuf {
  void* p = nullptr;
  ~DBuf() { cudaFree(p); }
  int alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("entanglement_entropy: cudaMalloc of %zu bytes failed", bytes);
      return FLOQUET_ENOMEM;
    }
    return FLOQUET_OK;
  }
};
}  // namespace

// S (host, nvec * ncut) for states X (device, nvec x d complex128, column-major)
int entanglement_entropy_run(int L, const double2* X, int nvec, const int* cuts, int ncut,
                             double* S, cudaStream_t st) {
  const int64_t d = (int64_t)1 << L;
  DBuf Sd;
  FQ_TRY(Sd.alloc(sizeof(double) * nvec * ncut));
  FQ_CUDA(cudaMemsetAsync(Sd.p, 0, sizeof(double) * nvec * ncut, st));
  for (int c = 0; c < ncut; ++c) {
    const int LA = cuts[c], LB = L - LA;
    if (LA == 0 || LB == 0) continue;  // a pure state: S = 0
    const int nb = std::min(LA, LB);
    const int n = 1 << nb;
    const int64_t r = d / n;
    // smaller A: X[b, a] = psi[a + 2^LA b] (rows b, stride 2^LA; columns a, unit stride);
    // smaller B: X = M (rows a, unit stride; columns b, stride 2^LA)
    const int64_t rs = LA <= LB ? ((int64_t)1 << LA) : 1;
    const int64_t cs = LA <= LB ? 1 : ((int64_t)1 << LA);
    const int ntile = (n + kGramTile - 1) / kGramTile;
    const int64_t per = (int64_t)n * n;
    // vectors per chunk so that the Gram matrices and slab partials stay below ~4 GiB
    int nsplit = 1;
    {
      const int64_t ctas = (int64_t)ntile * ntile * nvec;
      while (ctas * nsplit < 2 * 152 && r / (2 * nsplit) >= 4 * kGramTile) nsplit *= 2;
    }
    const int64_t slab = ((r + nsplit - 1) / nsplit + kGramTile - 1) / kGramTile * kGramTile;
    const int64_t bytes_per_vec = per * (int64_t)sizeof(double2) * (nsplit + 1);
    int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nvec, ((int64_t)4 << 30) / bytes_per_vec));
    DBuf part, G, work, diag, off2;
    FQ_TRY(part.alloc(sizeof(double2) * per * nsplit * chunk));
    FQ_TRY(G.alloc(sizeof(double2) * per * chunk));
    FQ_TRY(work.alloc(sizeof(double2) * 2 * n * chunk));
    FQ_TRY(diag.alloc(sizeof(double) * n * chunk));
    FQ_TRY(off2.alloc(sizeof(double) * n * chunk));
    for (int v0 = 0; v0 < nvec; v0 += chunk) {
      const int nv = std::min(chunk, nvec - v0);
      gram_slab_kernel<<<dim3((unsigned)(ntile * ntile), (unsigned)nv, (unsigned)nsplit), 256,
                         0, st>>>(X + (int64_t)v0 * d, d, rs, cs, n, r, slab, nv,
                                  (double2*)part.p);
      count_launch();
      FQ_CHECK_LAUNCH();
      const int64_t tot = per * nv;
      gram_sum_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, st>>>(
          (const double2*)part.p, nsplit, tot, (double2*)G.p);
      count_launch();
      FQ_CHECK_LAUNCH();
      hermitian_tridiag_kernel<<<(unsigned)nv, kTriThreads, 0, st>>>(
          (double2*)G.p, n, (double2*)work.p, (double*)diag.p, (double*)off2.p);
      count_launch();
      FQ_CHECK_LAUNCH();
      tridiag_entropy_kernel<<<(unsigned)nv, kTriThreads, 0, st>>>(
          (const double*)diag.p, (const double*)off2.p, n, (double*)Sd.p + (int64_t)v0 * ncut,
          ncut, c);
      count_launch();
      FQ_CHECK_LAUNCH();
    }
    // the chunk buffers are freed (DBuf) after the stream has used them
    FQ_CUDA(cudaStreamSynchronize(st));
  }
  FQ_CUDA(cudaMemcpyAsync(S, Sd.p, sizeof(double) * nvec * ncut, cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaStreamSynchronize(st));
  return FLOQUET_OK;
}

}  // namespace fq
