// Internal declarations shared by the CUDA translation units of libfloquet.
//
// Model (Sec. 2 of Luitz, arXiv:2102.05054, with the kicked-Ising operator of this library):
//   U = D K, K = prod_q exp(-i g X_q), D_s = exp(-i theta_s),
//   theta_s = J sum_i z_i z_{i+1 mod L} + sum_i h_i z_i, z_i = 1 - 2 b_i(s).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/floquet.h"

namespace fq {

// ------------------------------------------------------------------ complex helpers

// Sweep precisions: float (complex64), double (complex128) and dfloat, a tag for
// double-float arithmetic: each real number is an unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi)/2), about 48 significant bits, computed on the FP32 pipes with
// error-free transformations. A complex dfloat is a float4 (re.hi, re.lo, im.hi, im.lo).
struct dfloat {};

template <typename Real> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<dfloat> { using type = float4; };
template <typename Real> using cplx = typename cplx_of<Real>::type;

// Real scalars of each sweep precision (the butterfly multiplier tau).
template <typename Real> struct scal_of { using type = Real; };
template <> struct scal_of<dfloat> { using type = float2; };
template <typename Real> using scal = typename scal_of<Real>::type;

// complex value <-> (double re, double im)
__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_d2(float4 a) {
  return make_double2((double)a.x + (double)a.y, (double)a.z + (double)a.w);
}
template <typename Real> __host__ __device__ __forceinline__ cplx<Real> from_d2(double2 a);
template <> __host__ __device__ __forceinline__ float2 from_d2<float>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}
template <> __host__ __device__ __forceinline__ double2 from_d2<double>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float4 from_d2<dfloat>(double2 a) {
  const float rh = (float)a.x, ih = (float)a.y;
  return make_float4(rh, (float)(a.x - (double)rh), ih, (float)(a.y - (double)ih));
}
template <typename Real> __host__ __device__ __forceinline__ scal<Real> scal_from(double t);
template <> __host__ __device__ __forceinline__ float scal_from<float>(double t) { return (float)t; }
template <> __host__ __device__ __forceinline__ double scal_from<double>(double t) { return t; }
template <> __host__ __device__ __forceinline__ float2 scal_from<dfloat>(double t) {
  const float h = (float)t;
  return make_float2(h, (float)(t - (double)h));
}

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
  C r;
  r.x = re;
  r.y = im;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
  C r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
  C r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
// a + b * c
template <typename C> __host__ __device__ __forceinline__ C cfma(C b, C c, C a) {
  C r;
  r.x = a.x + b.x * c.x - b.y * c.y;
  r.y = a.y + b.x * c.y + b.y * c.x;
  return r;
}

// ------------------------------------------------------------------ errors

void set_error(const char* fmt, ...);
const char* get_error();
extern thread_local int last_status;

#define FQ_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::fq::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, \
                      __LINE__);                                                       \
      return FLOQUET_ECUDA;                                                            \
    }                                                                                  \
  } while (0)

#define FQ_CHECK_LAUNCH()                                                             \
  do {                                                                                \
    cudaError_t _e = cudaGetLastError();                                              \
    if (_e != cudaSuccess) {                                                          \
      ::fq::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e),     \
                      __FILE__, __LINE__);                                            \
      return FLOQUET_ECUDA;                                                           \
    }                                                                                 \
  } while (0)

#define FQ_TRY(expr)            \
  do {                          \
    int _s = (expr);            \
    if (_s != FLOQUET_OK) return _s; \
  } while (0)

void count_launch(int64_t n = 1);

// ------------------------------------------------------------------ U application passes

// One pass over a state: the tile of 2^NB amplitudes is formed by global bits
// [0, c) (coalesced "column" bits) and [start, start + NB - c); the CTA index supplies the
// other bits, [c, start) then [start + NB - c, L). The pass applies the X kick of every
// qubit in tile bits [kick_from, NB), i.e. qubits [0, NB) for the first pass
// (kick_from = 0, c = NB) and qubits [start, start + NB - c) for a later pass (kick_from = c).
struct Pass {
  int NB, c, start, kick_from;
};

enum Epilogue {
  EPI_STORE = 0,        // dst = K_pass src
  EPI_PHASE = 1,        // dst = D K_pass src (last pass of U)
  EPI_PHASE_ACC = 2,    // dst = D K_pass src; acc += coef[j] * dst
  EPI_PHASE_HORNER = 3  // dst = psi_in + (z D) K_pass src (src = dst = acc; z is folded into
                        // the per-vector tab_lo)
};

// Everything a pass kernel needs, passed by value.
template <typename Real> struct PassArgs {
  const cplx<Real>* src;
  cplx<Real>* dst;
  int64_t d;          // state length 2^L (stride between vectors)
  int L, NB, c, start, kick_from, midbits, topshift;
  scal<Real> tau;     // butterfly multiplier, |tau| <= 1
  // diagonal phase: D_s * scale = tab_lo[s & (2^a - 1)] * tab_hi[((s >> (a-1)) << 1) | (s & 1)]
  const cplx<Real>* tab_lo;
  const cplx<Real>* tab_hi;
  int a;
  int64_t tab_lo_stride, tab_hi_stride;  // per problem
  int vec_per_prob;
  int lo_by_vec;      // tab_lo holds one table per vector (Horner: z folded in) instead of per problem
  // accumulate / Horner epilogue
  cplx<Real>* acc;
  const cplx<Real>* coef;  // per vector: coef[vec * coef_stride + jstep]
  int64_t coef_stride;
  int jstep;
  const cplx<Real>* psi_in;
  // general Horner coefficients (nullable): the Horner epilogue adds hcoef[vec * hcoef_stride
  // + jstep] * psi_in instead of psi_in
  const cplx<Real>* hcoef;
  int64_t hcoef_stride;
};

// Launch shapes of the pass kernel that the autotuner chooses from, per sweep precision: the
// tile of 2^NB amplitudes (the plan's pass structure follows from it), 2^RB amplitudes per
// thread, the column bits later passes keep (0: the precision's default) and whether the
// persistent pipelined kernel (pass_pipe.cuh) runs the passes it has been compiled for.
struct PassVariant {
  int NB, RB;
  int cols = 0;
  bool pipe = false;
  bool pair = false;  // the tile is split over a two-CTA cluster (pass_pair.cuh)
};
template <typename Real> int num_variants();
template <typename Real> PassVariant variant_info(int v);
// Launch one pass for `nvec` vectors with launch shape `v` (tiles smaller than the variant's
// use the generic kernel). `swap` selects the cot form of the butterfly.
template <typename Real>
int launch_pass_variant(int v, const PassArgs<Real>& a, int epi, bool swap, int nvec,
                        cudaStream_t st);

// Elementwise helpers (uapply.cu)
template <typename Rin, typename Rout>
int launch_convert(const cplx<Rin>* in, cplx<Rout>* out, int64_t n, cudaStream_t st);
// work = in (converted); acc = coef[vec*stride + 0] * in (converted), per vector of length d
template <typename Rin, typename Rout>
int launch_filter_init(const cplx<Rin>* in, int64_t in_stride, cplx<Rout>* work,
                       cplx<Rout>* acc, const cplx<Rout>* coef, int64_t coef_stride, int64_t d,
                       int nvec, cudaStream_t st);

// ------------------------------------------------------------------ operator

struct FilterGraph {
  int64_t k;
  int nvec, dtype, form;
  const void* key_in;
  void* key_out;
  const void* key_coef;
  cudaGraphExec_t exec;
};

struct BatchTables {
  // phase tables for P problems (device), both precisions
  double2* lo64 = nullptr;
  double2* hi64 = nullptr;
  float2* lo32 = nullptr;
  float2* hi32 = nullptr;
  float4* lodf = nullptr;
  float4* hidf = nullptr;
  int64_t lo_n = 0, hi_n = 0;
  int a = 0;
  int P = 0;
};

struct Plan {
  std::vector<Pass> passes;  // first pass kicks [0, NB); the last applies the epilogue
};

// The brickwork random-circuit operator (brickwork.cu): U = (U_L x 1)(1 x U_R) split at the
// odd qubit q, applied as two complex GEMMs (cuBLAS), complex128 only.
struct BrickOp {
  int L = 0, q = 0;
  int64_t dL = 0, dR = 0;          // 2^(q+1), 2^(L-q)
  double2* UL = nullptr;           // dL x dL, column-major
  double2* UR = nullptr;           // dR x dR, column-major
  double2* tmp = nullptr;          // GEMM intermediate of the filter loops (captured in
  size_t tmp_elems = 0;            // graphs: grown only with the graphs dropped)
  double2* apply_tmp = nullptr;    // GEMM intermediate of plain U applications
  size_t apply_tmp_elems = 0;
  float4* ULdf = nullptr;          // U_L and U_R in double-float, for the double-float sweeps
  float4* URdf = nullptr;
  float4* part = nullptr;          // split-K partial sums of the double-float GEMMs (captured
  size_t part_elems = 0;           // in graphs like tmp: grown only with the graphs dropped)
  double2* consts = nullptr;       // device (1, 0) for the device-pointer GEMMs
  void* cublas = nullptr;          // cublasHandle_t
  void* ws = nullptr;              // cuBLAS workspace (fixed, so no GEMM allocates)
  size_t ws_bytes = 0;
};

}  // namespace fq

struct floquet_op {
  fq::BrickOp* brick = nullptr;  // non-null: the brickwork operator instead of kicked Ising
  int L;
  double J, g;
  std::vector<double> h;  // L (or R*L for a batch)
  int64_t d;
  int nprob;              // problems sharing L, J, g (1 for floquet_create)
  double tau;             // butterfly multiplier
  bool swap;              // cot form
  fq::BatchTables tabs;
  // per sweep precision, indexed by floquet_dtype (C128, C64, C128_DF): chosen launch shape,
  // its pass plan, and whether the autotuner has run
  fq::Plan plan[3];
  int variant[3] = {0, 0, 0};
  bool tuned[3] = {false, false, false};
  int gshape[3] = {-1, -1, -1};  // shape of the persistent Horner kernel (-1: per-pass kernels)
  // filter workspace (lazily sized)
  void* work = nullptr;
  void* acc = nullptr;
  void* psi_in_copy = nullptr;
  size_t work_bytes = 0;
  void* zlo = nullptr;  // Horner: per-vector tab_lo with the filter's z folded in
  size_t zlo_bytes = 0;
  void* coef = nullptr;
  size_t coef_bytes = 0;
  double coef_phi = 0;
  int64_t coef_k = -1;
  int coef_dtype = -1, coef_nvec = -1, coef_form = -1;
  std::vector<fq::FilterGraph> graphs;
  cudaStream_t cap_stream = nullptr;  // capture/replay stream of the filter graphs
  unsigned* bar = nullptr;  // grid-barrier counter and error word of the persistent filter
  void* ptab = nullptr;     // full phase table z D_s per vector (double-float persistent filter)
  size_t ptab_bytes = 0;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace fq {

// Builds tables and plans for `nprob` problems (h: nprob * L doubles).
int op_init(floquet_op* op, int L, double J, double g, const double* h, int nprob);
void op_free(floquet_op* op);

// Brickwork operator (brickwork.cu). g2: (L-1) row-major 4 x 4 complex bond gates, g1: two
// row-major 2 x 2 boundary gates, interleaved (re, im) doubles.
int brick_init(floquet_op* op, int L, const double* g2, const double* g1);
void brick_free(BrickOp* b);
int brick_reserve(BrickOp* b, int nvec);
int brick_apply(BrickOp* b, const double2* in, double2* out, int nvec, cudaStream_t st);
int brick_horner_step(BrickOp* b, double2* acc, const double2* psi_in, const double2* zs,
                      int nvec, cudaStream_t st);
// double-float sweeps: reserve (outside any capture) and one Horner step
int brick_reserve_df(BrickOp* b, int nvec);
int brick_horner_step_df(BrickOp* b, float4* acc, const float4* psi_in, const float4* zs,
                         int nvec, cudaStream_t st);
int brick_acc_step(BrickOp* b, double2* work, double2* acc, const double2* coef,
                   int64_t coef_stride, int j, int nvec, cudaStream_t st);

// U application on nvec vectors (vector v belongs to problem v / vec_per_prob).
template <typename Real>
int apply_u(floquet_op* op, const cplx<Real>* in, cplx<Real>* out, int nvec, int vec_per_prob,
            cudaStream_t st);

// Polynomial filter in the accumulate form, out_v = sum_{j<k} coef[v*k + j] U^j in_v, for
// nvec vectors (in_v at in + v*in_stride, out_v at out + v*out_stride, type Rio); the
// sweeps run in Real in the op's internal workspace. `use_graph` captures the k-step loop
// once and replays it.
template <typename Real, typename Rio>
int filter_coef(floquet_op* op, const cplx<Rio>* in, int64_t in_stride, cplx<Rio>* out,
                int64_t out_stride, const cplx<Real>* coef, int64_t k, int nvec,
                int vec_per_prob, bool use_graph, cudaStream_t st);

// Horner form with one z per vector (zs: device, nvec complex of Real).
template <typename Real, typename Rio>
int filter_horner(floquet_op* op, const cplx<Rio>* in, int64_t in_stride, cplx<Rio>* out,
                  int64_t out_stride, const cplx<Real>* zs, int64_t k, int nvec,
                  int vec_per_prob, bool use_graph, cudaStream_t st);

}  // namespace fq
