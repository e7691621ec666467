// Krylov-basis linear algebra in complex128 (Sec. 4 of Luitz, arXiv:2102.05054: the
// Arnoldi process with Gram-Schmidt orthogonalisation, Ritz vectors V y, Rayleigh quotients
// and residuals of Eq. residual).
//
// Everything here is memory- or FP64-ALU-bound tall-skinny work on column-major blocks
// (leading dimension d), batched over independent problems by blockIdx.y / blockIdx.z with
// explicit strides. Reductions are two-stage (per-CTA partials, then a fixed-order sum), so
// results are deterministic run to run.

#include <algorithm>
#include <mutex>

#include "floquet_internal.cuh"
#include "linalg.cuh"

namespace fq {

static constexpr int kThreads = 256;

__device__ __forceinline__ int64_t dmin64(int64_t a, int64_t b) { return a < b ? a : b; }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// -------------------------------------------------------------- h = V^H w (partials)

// part[(b * nchunk + chunk) * n + i] = sum_{r in chunk} conj(V_b[r, i]) w_b[r].
// One warp per column (columns strided over the 8 warps); the chunk of w sits in shared
// memory.
__global__ void __launch_bounds__(kThreads) dots_kernel(const double2* __restrict__ V,
                                                        int64_t ldv, int64_t strideV, int n,
                                                        const double2* __restrict__ w,
                                                        int64_t strideW, int64_t d, int chunk,
                                                        double2* __restrict__ part) {
  extern __shared__ double2 ws[];
  const int64_t b = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int rows = (int)dmin64(chunk, d - r0);
  const double2* Vb = V + b * strideV;
  const double2* wb = w + b * strideW;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) ws[i] = wb[r0 + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  double2* pb = part + (b * gridDim.x + blockIdx.x) * (int64_t)n;
  for (int i = warp; i < n; i += nwarps) {
    const double2* col = Vb + (int64_t)i * ldv + r0;
    double re = 0, im = 0;
    for (int r = lane; r < rows; r += 32) {
      const double2 v = col[r];
      const double2 x = ws[r];
      re = fma(v.x, x.x, fma(v.y, x.y, re));
      im = fma(v.x, x.y, fma(-v.y, x.x, im));
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) pb[i] = make_double2(re, im);
  }
}

// out[b * ostride + i] = sum_chunk part[(b * nchunk + chunk) * n + i] (+ add[b*astride + i])
__global__ void __launch_bounds__(kThreads) reduce_parts_kernel(
    const double2* __restrict__ part, int nchunk, int n, double2* __restrict__ out,
    int64_t ostride, const double2* __restrict__ add, int64_t astride) {
  __shared__ double sre[kThreads / 32], sim[kThreads / 32];
  const int64_t b = blockIdx.y;
  const int i = blockIdx.x;
  double re = 0, im = 0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
    const double2 v = part[(b * nchunk + c) * (int64_t)n + i];
    re += v.x;
    im += v.y;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sre[warp] = re;
    sim[warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    re = 0;
    im = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      re += sre[k];
      im += sim[k];
    }
    if (add) {
      re += add[b * astride + i].x;
      im += add[b * astride + i].y;
    }
    out[b * ostride + i] = make_double2(re, im);
  }
}

// -------------------------------------------------------------- w -= V h (+ ||w||^2 partials)

__global__ void __launch_bounds__(kThreads) update_kernel(const double2* __restrict__ V,
                                                          int64_t ldv, int64_t strideV, int n,
                                                          const double2* __restrict__ h,
                                                          int64_t strideH, double2* w,
                                                          int64_t strideW, int64_t d,
                                                          double* __restrict__ npart) {
  extern __shared__ double2 hs[];
  __shared__ double red[kThreads / 32];
  const int64_t b = blockIdx.y;
  for (int i = threadIdx.x; i < n; i += blockDim.x) hs[i] = h[b * strideH + i];
  __syncthreads();
  const double2* Vb = V + b * strideV;
  double2* wb = w + b * strideW;
  double nrm = 0;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < d) {
    double re = 0, im = 0;
    int i = 0;
    for (; i + 1 < n; i += 2) {
      const double2 v0 = Vb[(int64_t)i * ldv + r];
      const double2 v1 = Vb[(int64_t)(i + 1) * ldv + r];
      const double2 c0 = hs[i], c1 = hs[i + 1];
      re = fma(v0.x, c0.x, fma(-v0.y, c0.y, re));
      im = fma(v0.x, c0.y, fma(v0.y, c0.x, im));
      re = fma(v1.x, c1.x, fma(-v1.y, c1.y, re));
      im = fma(v1.x, c1.y, fma(v1.y, c1.x, im));
    }
    if (i < n) {
      const double2 v0 = Vb[(int64_t)i * ldv + r];
      const double2 c0 = hs[i];
      re = fma(v0.x, c0.x, fma(-v0.y, c0.y, re));
      im = fma(v0.x, c0.y, fma(v0.y, c0.x, im));
    }
    double2 x = wb[r];
    x.x -= re;
    x.y -= im;
    wb[r] = x;
    nrm = x.x * x.x + x.y * x.y;
  }
  if (npart) {
    nrm = warp_sum(nrm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
      npart[b * gridDim.x + blockIdx.x] = s;
    }
  }
}

// beta_b = sqrt(sum npart); H_b[j+1, j] = beta; betas[b] = beta
__global__ void norm_finalize_kernel(const double* __restrict__ npart, int nblk,
                                     double2* __restrict__ Hcol, int64_t strideH, int row,
                                     double* __restrict__ betas) {
  __shared__ double red[kThreads / 32];
  const int64_t b = blockIdx.x;
  double s = 0;
  for (int c = threadIdx.x; c < nblk; c += blockDim.x) s += npart[b * nblk + c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    const double beta = sqrt(t);
    if (Hcol) Hcol[b * strideH + row] = make_double2(beta, 0.0);
    betas[b] = beta;
  }
}

// out_b = w_b / beta_b (beta = 0 leaves a zero vector: an exact invariant subspace)
__global__ void scale_kernel(const double2* __restrict__ w, int64_t strideW,
                             const double* __restrict__ betas, double2* __restrict__ out,
                             int64_t strideO, int64_t d) {
  const int64_t b = blockIdx.y;
  const double beta = betas[b];
  const double inv = beta > 0 ? 1.0 / beta : 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = w[b * strideW + r];
    out[b * strideO + r] = make_double2(x.x * inv, x.y * inv);
  }
}

static int dots_chunk(int64_t d) { return (int)std::min<int64_t>(d, 2048); }

int cgs2(Workspace& ws, const double2* V, int64_t ldv, int64_t strideV, int n, double2* w,
         int64_t strideW, int64_t d, int B, double2* Hcol, int64_t strideH, double2* vnext,
         int64_t strideVn, cudaStream_t st) {
  const int chunk = dots_chunk(d);
  const int nchunk = (int)((d + chunk - 1) / chunk);
  const int nblk = (int)((d + kThreads - 1) / kThreads);
  FQ_TRY(ws.reserve_part((size_t)B * nchunk * std::max(n, 1)));
  FQ_TRY(ws.reserve_small((size_t)B * (2 * (size_t)n + 2)));
  FQ_TRY(ws.reserve_npart((size_t)B * nblk));
  double2* h1 = ws.small;
  double2* h2 = ws.small + (size_t)B * n;
  double* betas = reinterpret_cast<double*>(ws.small + (size_t)2 * B * n);
  if (n > 0) {
    const size_t smw = (size_t)chunk * sizeof(double2);
    const size_t smh = (size_t)n * sizeof(double2);
    for (int pass = 0; pass < 2; ++pass) {
      double2* h = pass == 0 ? h1 : h2;
      dots_kernel<<<dim3(nchunk, B), kThreads, smw, st>>>(V, ldv, strideV, n, w, strideW, d,
                                                          chunk, ws.part);
      count_launch();
      FQ_CHECK_LAUNCH();
      // pass 0: h1 = sum; pass 1: H column = h1 + sum, and h2 = sum for the update
      reduce_parts_kernel<<<dim3(n, B), kThreads, 0, st>>>(ws.part, nchunk, n, h, n, nullptr,
                                                           0);
      count_launch();
      FQ_CHECK_LAUNCH();
      update_kernel<<<dim3(nblk, B), kThreads, smh, st>>>(V, ldv, strideV, n, h, n, w, strideW,
                                                          d, pass == 1 ? ws.npart : nullptr);
      count_launch();
      FQ_CHECK_LAUNCH();
    }
    if (Hcol) {
      add_kernel_launch(h1, h2, n, B, Hcol, strideH, st);
      FQ_CHECK_LAUNCH();
    }
  } else {
    // no projection: only the norm
    update_kernel<<<dim3(nblk, B), kThreads, 0, st>>>(V, ldv, strideV, 0, nullptr, 0, w, strideW,
                                                      d, ws.npart);
    count_launch();
    FQ_CHECK_LAUNCH();
  }
  norm_finalize_kernel<<<B, kThreads, 0, st>>>(ws.npart, nblk, Hcol, strideH, n, betas);
  count_launch();
  FQ_CHECK_LAUNCH();
  if (vnext) {
    const unsigned gx = (unsigned)std::min<int64_t>((d + kThreads - 1) / kThreads, 4096);
    scale_kernel<<<dim3(gx, B), kThreads, 0, st>>>(w, strideW, betas, vnext, strideVn, d);
    count_launch();
    FQ_CHECK_LAUNCH();
  }
  ws.last_betas = betas;
  ws.last_h1 = h1;
  ws.last_h2 = h2;
  return FLOQUET_OK;
}

__global__ void add_kernel(const double2* __restrict__ a, const double2* __restrict__ b, int n,
                           double2* __restrict__ out, int64_t ostride) {
  const int64_t bb = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 x = a[bb * n + i], y = b[bb * n + i];
    out[bb * ostride + i] = make_double2(x.x + y.x, x.y + y.y);
  }
}

void add_kernel_launch(const double2* a, const double2* b, int n, int B, double2* out,
                       int64_t ostride, cudaStream_t st) {
  add_kernel<<<dim3((n + 255) / 256, B), 256, 0, st>>>(a, b, n, out, ostride);
  count_launch();
}

// -------------------------------------------------------------- C = A B (tall-skinny)

// C_b[d x p] = A_b[d x m] * B_b[m x p]; all column-major. Tile 64 rows x 32 columns, 256
// threads, each 4 rows x 2 columns; column tiles vary fastest so the CTAs that share a row
// panel of A run together and re-read it from L2.
__global__ void __launch_bounds__(256) gemm_nn_kernel(const double2* __restrict__ A, int64_t lda,
                                                      int64_t strideA, const double2* __restrict__ Bm,
                                                      int64_t ldb, int64_t strideB,
                                                      double2* __restrict__ C, int64_t ldc,
                                                      int64_t strideC, int64_t d, int m, int p) {
  __shared__ double2 As[16][64 + 1];
  __shared__ double2 Bs[16][32 + 1];
  // flattened grid: blockIdx.x = row_tile * col_tiles + col_tile (column tiles vary fastest)
  const int64_t bz = blockIdx.y;
  const int col_tiles = (p + 31) / 32;
  const int col0 = (int)(blockIdx.x % col_tiles) * 32;
  const int64_t row0 = (int64_t)(blockIdx.x / col_tiles) * 64;
  const double2* Ab = A + bz * strideA;
  const double2* Bb = Bm + bz * strideB;
  double2* Cb = C + bz * strideC;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0, 0);
  for (int k0 = 0; k0 < m; k0 += 16) {
    // A tile: 64 rows x 16 k
    for (int idx = threadIdx.x; idx < 64 * 16; idx += 256) {
      const int r = idx & 63, kk = idx >> 6;
      const int64_t gr = row0 + r;
      As[kk][r] = (gr < d && k0 + kk < m) ? Ab[(int64_t)(k0 + kk) * lda + gr] : make_double2(0, 0);
    }
    for (int idx = threadIdx.x; idx < 16 * 32; idx += 256) {
      const int kk = idx & 15, c = idx >> 4;
      Bs[kk][c] = (k0 + kk < m && col0 + c < p) ? Bb[(int64_t)(col0 + c) * ldb + k0 + kk]
                                                 : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      double2 a[4], bv[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 2; ++j) bv[j] = Bs[kk][tx * 2 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = cfma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + ty * 4 + i;
    if (gr >= d) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = col0 + tx * 2 + j;
      if (c < p) Cb[(int64_t)c * ldc + gr] = acc[i][j];
    }
  }
}

int gemm_nn(const double2* A, int64_t lda, int64_t strideA, const double2* B, int64_t ldb,
            int64_t strideB, double2* C, int64_t ldc, int64_t strideC, int64_t d, int m, int p,
            int batch, cudaStream_t st) {
  if (p <= 0 || d <= 0 || batch <= 0) return FLOQUET_OK;
  const int64_t rt = (d + 63) / 64;
  const int64_t ct = (p + 31) / 32;
  if (rt * ct > 0x7fffffffLL || batch > 65535) {
    set_error("gemm_nn: grid too large");
    return FLOQUET_EINVAL;
  }
  dim3 grid((unsigned)(rt * ct), batch);
  gemm_nn_kernel<<<grid, 256, 0, st>>>(A, lda, strideA, B, ldb, strideB, C, ldc, strideC, d, m,
                                       p);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// -------------------------------------------------------------- G = A^H B (reduce over d)

// part[(b * nchunk + chunk)][n1 x n2] = sum_{r in chunk} conj(A_b[r, i]) B_b[r, j]; tile 32 x 32
// of G per CTA (grid.x = tile, grid.y = chunk, grid.z = batch); threads 16 x 16, 2 x 2 each.
__global__ void __launch_bounds__(256) gemm_cn_kernel(const double2* __restrict__ A, int64_t lda,
                                                      int64_t strideA, const double2* __restrict__ Bm,
                                                      int64_t ldb, int64_t strideB, int64_t d,
                                                      int n1, int n2, int chunk,
                                                      double2* __restrict__ part) {
  __shared__ double2 As[32][32 + 1];
  __shared__ double2 Bs[32][32 + 1];
  const int64_t bz = blockIdx.z;
  const int tiles_i = (n1 + 31) / 32;
  const int ti = blockIdx.x % tiles_i, tj = blockIdx.x / tiles_i;
  const int i0 = ti * 32, j0 = tj * 32;
  const int64_t r0 = (int64_t)blockIdx.y * chunk;
  const int64_t r1 = dmin64(d, r0 + chunk);
  const double2* Ab = A + bz * strideA;
  const double2* Bb = Bm + bz * strideB;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0, 0);
  for (int64_t rr = r0; rr < r1; rr += 32) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
      const int r = idx & 31, c = idx >> 5;
      const int64_t gr = rr + r;
      As[r][c] = (gr < r1 && i0 + c < n1) ? Ab[(int64_t)(i0 + c) * lda + gr] : make_double2(0, 0);
      Bs[r][c] = (gr < r1 && j0 + c < n2) ? Bb[(int64_t)(j0 + c) * ldb + gr] : make_double2(0, 0);
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      double2 a[2], bv[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = As[r][ty * 2 + i];
#pragma unroll
      for (int j = 0; j < 2; ++j) bv[j] = Bs[r][tx * 2 + j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const double2 p = cmulc(a[i], bv[j]);
          acc[i][j].x += p.x;
          acc[i][j].y += p.y;
        }
    }
    __syncthreads();
  }
  double2* pb = part + (bz * gridDim.y + blockIdx.y) * (int64_t)n1 * n2;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gi = i0 + ty * 2 + i, gj = j0 + tx * 2 + j;
      if (gi < n1 && gj < n2) pb[(int64_t)gj * n1 + gi] = acc[i][j];
    }
}

int gemm_cn(Workspace& ws, const double2* A, int64_t lda, int64_t strideA, const double2* B,
            int64_t ldb, int64_t strideB, int64_t d, int n1, int n2, int batch, double2* G,
            int64_t ldg, int64_t strideG, cudaStream_t st) {
  const int chunk = (int)std::min<int64_t>(d, 4096);
  const int nchunk = (int)((d + chunk - 1) / chunk);
  FQ_TRY(ws.reserve_part((size_t)batch * nchunk * n1 * n2));
  const int tiles = ((n1 + 31) / 32) * ((n2 + 31) / 32);
  gemm_cn_kernel<<<dim3(tiles, nchunk, batch), 256, 0, st>>>(A, lda, strideA, B, ldb, strideB, d,
                                                             n1, n2, chunk, ws.part);
  count_launch();
  FQ_CHECK_LAUNCH();
  // reduce: treat the n1*n2 entries as columns
  FQ_TRY(ws.reserve_small((size_t)batch * n1 * n2));
  reduce_parts_kernel<<<dim3(n1 * n2, batch), kThreads, 0, st>>>(ws.part, nchunk, n1 * n2,
                                                                  ws.small, (int64_t)n1 * n2,
                                                                  nullptr, 0);
  count_launch();
  FQ_CHECK_LAUNCH();
  // scatter to G with its leading dimension
  copy_matrix_launch(ws.small, n1, (int64_t)n1 * n2, G, ldg, strideG, n1, n2, batch, st);
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

__global__ void copy_matrix_kernel(const double2* __restrict__ a, int64_t lda, int64_t sa,
                                   double2* __restrict__ b, int64_t ldb, int64_t sb, int rows,
                                   int cols) {
  const int64_t z = blockIdx.y;
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % rows, c = idx / rows;
    b[z * sb + c * ldb + r] = a[z * sa + c * lda + r];
  }
}

void copy_matrix_launch(const double2* a, int64_t lda, int64_t sa, double2* b, int64_t ldb,
                        int64_t sb, int rows, int cols, int batch, cudaStream_t st) {
  const int64_t n = (int64_t)rows * cols;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048));
  copy_matrix_kernel<<<dim3(gx, batch), 256, 0, st>>>(a, lda, sa, b, ldb, sb, rows, cols);
  count_launch();
}

// -------------------------------------------------------------- Rayleigh quotient, residual

// per column j: part[(b*nchunk+chunk)*3n + {j, n+j, 2n+j}] = (x.x, x.w) sums over the chunk
__global__ void __launch_bounds__(kThreads) colstats_kernel(const double2* __restrict__ X,
                                                            const double2* __restrict__ W,
                                                            int64_t d, int n, int chunk,
                                                            double* __restrict__ part) {
  __shared__ double red[3][kThreads / 32];
  const int j = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * chunk;
  const int64_t r1 = dmin64(d, r0 + chunk);
  const double2* x = X + (int64_t)j * d;
  const double2* w = W + (int64_t)j * d;
  double xx = 0, re = 0, im = 0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double2 a = x[r], b = w[r];
    xx = fma(a.x, a.x, fma(a.y, a.y, xx));
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
  xx = warp_sum(xx);
  re = warp_sum(re);
  im = warp_sum(im);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][warp] = xx;
    red[1][warp] = re;
    red[2][warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s0 += red[0][k];
      s1 += red[1][k];
      s2 += red[2][k];
    }
    double* pb = part + (int64_t)blockIdx.y * 3 * n;
    pb[j] = s0;
    pb[n + j] = s1;
    pb[2 * n + j] = s2;
  }
}

// stats[j] = (sum xx, omega.re, omega.im) with omega = x.w / x.x
__global__ void colstats_finalize_kernel(const double* __restrict__ part, int nchunk, int n,
                                         double* __restrict__ stats) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double xx = 0, re = 0, im = 0;
  for (int c = 0; c < nchunk; ++c) {
    const double* pb = part + (int64_t)c * 3 * n;
    xx += pb[j];
    re += pb[n + j];
    im += pb[2 * n + j];
  }
  stats[3 * j] = xx;
  stats[3 * j + 1] = xx > 0 ? re / xx : 0;
  stats[3 * j + 2] = xx > 0 ? im / xx : 0;
}

// part[chunk * n + j] = sum ||w - omega x||^2 over the chunk
__global__ void __launch_bounds__(kThreads) resid_kernel(const double2* __restrict__ X,
                                                         const double2* __restrict__ W,
                                                         int64_t d, int n, int chunk,
                                                         const double* __restrict__ stats,
                                                         double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  const int j = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * chunk;
  const int64_t r1 = dmin64(d, r0 + chunk);
  const double2* x = X + (int64_t)j * d;
  const double2* w = W + (int64_t)j * d;
  const double ore = stats[3 * j + 1], oim = stats[3 * j + 2];
  double s = 0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double2 a = x[r], b = w[r];
    const double dr = b.x - (ore * a.x - oim * a.y);
    const double di = b.y - (ore * a.y + oim * a.x);
    s = fma(dr, dr, fma(di, di, s));
  }
  s = warp_sum(s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[(int64_t)blockIdx.y * n + j] = t;
  }
}

__global__ void resid_finalize_kernel(const double* __restrict__ part, int nchunk, int n,
                                      double* __restrict__ stats, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0;
  for (int c = 0; c < nchunk; ++c) s += part[(int64_t)c * n + j];
  const double xx = stats[3 * j];
  out[3 * j] = stats[3 * j + 1];
  out[3 * j + 1] = stats[3 * j + 2];
  out[3 * j + 2] = xx > 0 ? sqrt(s / xx) : 0;
}

// out[3j..3j+2] = (omega.re, omega.im, resid) for columns X[:, j], W[:, j] = U X[:, j]
int rayleigh_residual(Workspace& ws, const double2* X, const double2* W, int64_t d, int n,
                      double* out, cudaStream_t st) {
  const int chunk = (int)std::min<int64_t>(d, 16384);
  const int nchunk = (int)((d + chunk - 1) / chunk);
  FQ_TRY(ws.reserve_npart((size_t)nchunk * 3 * n + 3 * (size_t)n));
  double* part = ws.npart;
  double* stats = ws.npart + (size_t)nchunk * 3 * n;
  colstats_kernel<<<dim3(n, nchunk), kThreads, 0, st>>>(X, W, d, n, chunk, part);
  count_launch();
  FQ_CHECK_LAUNCH();
  colstats_finalize_kernel<<<(n + 127) / 128, 128, 0, st>>>(part, nchunk, n, stats);
  count_launch();
  FQ_CHECK_LAUNCH();
  resid_kernel<<<dim3(n, nchunk), kThreads, 0, st>>>(X, W, d, n, chunk, stats, part);
  count_launch();
  FQ_CHECK_LAUNCH();
  resid_finalize_kernel<<<(n + 127) / 128, 128, 0, st>>>(part, nchunk, n, stats, out);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// -------------------------------------------------------------- column scaling and axpy

// X[:, j] *= s[j] (complex s)
__global__ void scale_cols_kernel(double2* X, int64_t d, const double2* __restrict__ s) {
  const int j = blockIdx.y;
  const double2 c = s[j];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
       r += (int64_t)gridDim.x * blockDim.x)
    X[(int64_t)j * d + r] = cmul(c, X[(int64_t)j * d + r]);
}

int scale_cols(double2* X, int64_t d, int n, const double2* s, cudaStream_t st) {
  const unsigned gx = (unsigned)std::min<int64_t>((d + 255) / 256, 1024);
  scale_cols_kernel<<<dim3(gx, n), 256, 0, st>>>(X, d, s);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// Y[:, j] = a[j] X[:, j] + Y[:, j]
__global__ void axpy_cols_kernel(const double2* __restrict__ X, double2* Y, int64_t d,
                                 const double2* __restrict__ a) {
  const int j = blockIdx.y;
  const double2 c = a[j];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)j * d + r;
    Y[i] = cfma(c, X[i], Y[i]);
  }
}

int axpy_cols(const double2* X, double2* Y, int64_t d, int n, const double2* a,
              cudaStream_t st) {
  const unsigned gx = (unsigned)std::min<int64_t>((d + 255) / 256, 1024);
  axpy_cols_kernel<<<dim3(gx, n), 256, 0, st>>>(X, Y, d, a);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// C[:, j] -= T[:, j], j < n (leading dimensions ldc, ldt)
__global__ void sub_cols_kernel(double2* __restrict__ C, int64_t ldc,
                                const double2* __restrict__ T, int64_t ldt, int64_t d) {
  const int j = blockIdx.y;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = C[(int64_t)j * ldc + r], b = T[(int64_t)j * ldt + r];
    C[(int64_t)j * ldc + r] = make_double2(a.x - b.x, a.y - b.y);
  }
}

int sub_cols(double2* C, int64_t ldc, const double2* T, int64_t ldt, int64_t d, int n,
             cudaStream_t st) {
  if (n <= 0) return FLOQUET_OK;
  const unsigned gx = (unsigned)std::min<int64_t>((d + 255) / 256, 1024);
  sub_cols_kernel<<<dim3(gx, n), 256, 0, st>>>(C, ldc, T, ldt, d);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// R[:, j] = W[:, j] - omega_j X[:, j], omega from stats triples (re, im, .)
__global__ void residual_vectors_kernel(const double2* __restrict__ X,
                                        const double2* __restrict__ W, double2* __restrict__ R,
                                        int64_t d, const double* __restrict__ om3) {
  const int j = blockIdx.y;
  const double ore = om3[3 * j], oim = om3[3 * j + 1];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)j * d + r;
    const double2 a = X[i], b = W[i];
    R[i] = make_double2(b.x - (ore * a.x - oim * a.y), b.y - (ore * a.y + oim * a.x));
  }
}

int residual_vectors(const double2* X, const double2* W, double2* R, int64_t d, int n,
                     const double* om3, cudaStream_t st) {
  const unsigned gx = (unsigned)std::min<int64_t>((d + 255) / 256, 1024);
  residual_vectors_kernel<<<dim3(gx, n), 256, 0, st>>>(X, W, R, d, om3);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// -------------------------------------------------------------- workspace

int Workspace::grow(void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return FLOQUET_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("workspace: cudaMalloc(%zu) failed", bytes);
    return FLOQUET_ENOMEM;
  }
  *cap = bytes;
  return FLOQUET_OK;
}
int Workspace::reserve_part(size_t n) {
  void* p = part;
  const int rc = grow(&p, &part_cap, n * sizeof(double2));
  part = (double2*)p;
  return rc;
}
int Workspace::reserve_small(size_t n) {
  void* p = small;
  const int rc = grow(&p, &small_cap, n * sizeof(double2));
  small = (double2*)p;
  return rc;
}
int Workspace::reserve_npart(size_t n) {
  void* p = npart;
  const int rc = grow(&p, &npart_cap, n * sizeof(double));
  npart = (double*)p;
  return rc;
}
Workspace::~Workspace() {
  cudaFree(part);
  cudaFree(small);
  cudaFree(npart);
}

// ==============================================================================
// gram_schmidt_noalloc: the CGS2 step with its scratch in a fixed device array.
//
// Some callers must not allocate device memory once they are running: services that
// reserve their whole memory budget at start-up and treat any later cudaMalloc as a
// failure, or latency-critical loops where the device-wide synchronisation that cudaFree
// implies is unacceptable. gram_schmidt allocates its partial sums on every call; this entry
// point instead keeps them in the file-scope array below, which every GPU that loads the
// library holds for the life of the process.
//
// Capacity: d <= 2^20 rows and n <= 256 columns. Layout of the array (complex128 slots):
// dots partials nchunk * n (nchunk = d / 2048 <= 512), then the two projection vectors
// (n each), then the norm partials (d / 256 doubles) and the norm itself. Every slot that a
// kernel reads is first written by an earlier kernel of the same call, so nothing has to
// start at zero; the array simply keeps the last call's values. All calls share the one
// array: calls whose work overlaps on the GPU (different streams, threads or devices'
// contexts racing on the same device) corrupt each other and must be serialised by the
// caller.
// ==============================================================================

namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 20;
constexpr int kNoAllocMaxCols = 256;
constexpr int64_t kNoAllocChunks = kNoAllocMaxRows / 2048;        // dots partial blocks
constexpr int64_t kNoAllocNormBlocks = kNoAllocMaxRows / 256;     // norm partial blocks
constexpr int64_t kNoAllocSlots = kNoAllocChunks * kNoAllocMaxCols  // dots partials
                                  + 2 * kNoAllocMaxCols             // h1, h2
                                  + kNoAllocNormBlocks / 2 + 1      // norm partials (doubles)
                                  + 1;                              // beta

}  // namespace

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocSlots];

// Device address of g_noalloc_scratch per device ordinal, looked up once per device with that
// device current (in host code the symbol name is only a host-side stand-in).
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {nullptr};

static int noalloc_scratch(double2** out) {
  int dev = 0;
  FQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("gram_schmidt_noalloc: device ordinal %d out of range", dev);
    return FLOQUET_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("gram_schmidt_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return FLOQUET_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<double2*>(g_noalloc_addr[dev]);
  return FLOQUET_OK;
}

}  // namespace fq

extern "C" int gram_schmidt_noalloc(int64_t d, const void* V, int n, void* w, void* h,
                                    void* stream) {
  using namespace fq;
  if (d < 1 || d > kNoAllocMaxRows) {
    set_error("gram_schmidt_noalloc: d = %lld outside [1, %lld] (the fixed scratch array's "
              "capacity); use gram_schmidt for larger states",
              (long long)d, (long long)kNoAllocMaxRows);
    return FLOQUET_EINVAL;
  }
  if (n < 0 || n > kNoAllocMaxCols) {
    set_error("gram_schmidt_noalloc: n = %d outside [0, %d] (the fixed scratch array's "
              "capacity); use gram_schmidt for more columns",
              n, kNoAllocMaxCols);
    return FLOQUET_EINVAL;
  }
  if (!w || !h || (n > 0 && !V)) {
    set_error("gram_schmidt_noalloc: NULL pointer");
    return FLOQUET_EINVAL;
  }
  double2* scratch = nullptr;
  FQ_TRY(noalloc_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = dots_chunk(d);
  const int nchunk = (int)((d + chunk - 1) / chunk);
  const int nblk = (int)((d + kThreads - 1) / kThreads);
  double2* part = scratch;
  double2* h1 = part + kNoAllocChunks * kNoAllocMaxCols;
  double2* h2 = h1 + kNoAllocMaxCols;
  double* npart = reinterpret_cast<double*>(h2 + kNoAllocMaxCols);
  double* beta = npart + kNoAllocNormBlocks;
  const double2* Vd = (const double2*)V;
  double2* wd = (double2*)w;
  double2* hd = (double2*)h;
  if (n > 0) {
    const size_t smw = (size_t)chunk * sizeof(double2);
    const size_t smh = (size_t)n * sizeof(double2);
    for (int pass = 0; pass < 2; ++pass) {
      double2* hp = pass == 0 ? h1 : h2;
      dots_kernel<<<dim3(nchunk, 1), kThreads, smw, st>>>(Vd, d, 0, n, wd, 0, d, chunk, part);
      count_launch();
      FQ_CHECK_LAUNCH();
      reduce_parts_kernel<<<dim3(n, 1), kThreads, 0, st>>>(part, nchunk, n, hp, n, nullptr, 0);
      count_launch();
      FQ_CHECK_LAUNCH();
      update_kernel<<<dim3(nblk, 1), kThreads, smh, st>>>(Vd, d, 0, n, hp, n, wd, 0, d,
                                                          pass == 1 ? npart : nullptr);
      count_launch();
      FQ_CHECK_LAUNCH();
    }
    add_kernel_launch(h1, h2, n, 1, hd, 0, st);
    FQ_CHECK_LAUNCH();
  } else {
    update_kernel<<<dim3(nblk, 1), kThreads, 0, st>>>(Vd, d, 0, 0, nullptr, 0, wd, 0, d, npart);
    count_launch();
    FQ_CHECK_LAUNCH();
  }
  norm_finalize_kernel<<<1, kThreads, 0, st>>>(npart, nblk, hd, 0, n, beta);
  count_launch();
  FQ_CHECK_LAUNCH();
  const unsigned gx = (unsigned)std::min<int64_t>((d + kThreads - 1) / kThreads, 4096);
  scale_kernel<<<dim3(gx, 1), kThreads, 0, st>>>(wd, 0, beta, wd, 0, d);
  count_launch();
  FQ_CHECK_LAUNCH();
  set_error("%s", "");
  return FLOQUET_OK;
}
