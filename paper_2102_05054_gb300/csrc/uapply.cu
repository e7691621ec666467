// Matrix-free application of the kicked-Ising Floquet operator U = D K and of the
// geometric-sum filter g_k(U) (Luitz, arXiv:2102.05054: Sec. 2 matrix-free product, Sec. 3
// Eq. geo).
//
// Kick layer. exp(-i g X_q) = c I - i s X_q acts on the amplitude pair (s, s xor 2^q).
// Factoring out c (when |c| >= |s|) gives the butterfly
//     x' = x - i tau y,  y' = y - i tau x,   tau = tan g,
// two fused multiply-adds per real output; factoring out -i s instead (|s| > |c|) gives the
// same butterfly with tau = -cot g and the two outputs exchanged. The L factors (c^L or
// (-i s)^L) are folded into the diagonal-phase table, so each butterfly has |tau| <= 1 and
// one rounding per real output.
//
// Tiling. A CTA owns a tile of 2^NB amplitudes (Pass). Each thread holds R = 2^RB of them
// in registers; the RB register bits are kicked in registers, then the tile is transposed
// through padded shared memory so that the next group of RB tile bits becomes the register
// bits. Loads and stores use the mapping whose lane bits are the tile's lowest bits, which
// are contiguous global bits, so global accesses are coalesced.
//
// Last pass. The diagonal phase D_s (times the kick scale) is the product of two table
// entries built on the host in float64: tab_lo over bits [0, a) and tab_hi over bits
// [a-1, L) plus bit 0 (the two bonds crossing the split and the periodic bond are placed in
// tab_hi by giving it the neighbouring bits). The geometric accumulate acc += coef_j psi_j
// (or the Horner update acc = psi_in + z U acc) is fused into the same pass.

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "floquet_internal.cuh"
#include "horner_grid.cuh"

namespace fq {

// ------------------------------------------------------------------ error state

thread_local int last_status = 0;
static thread_local char g_err[1024] = {0};
static int64_t g_launches = 0;
static std::mutex g_launch_mu;

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* get_error() { return g_err; }

// ------------------------------------------------------------------ sweep profiling

struct SweepEvent {
  cudaEvent_t a, b;
  int kind;  // 0 complex128, 1 complex64
  int64_t u_apps;
  double bytes;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<SweepEvent> g_prof_pending;
static double g_prof_ms[3] = {0, 0, 0};
static int64_t g_prof_apps[3] = {0, 0, 0};
static double g_prof_bytes[3] = {0, 0, 0};

int profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& e : g_prof_pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g_prof_pending.clear();
  g_prof_on = on != 0;
  for (int i = 0; i < 3; ++i) {
    g_prof_ms[i] = 0;
    g_prof_apps[i] = 0;
    g_prof_bytes[i] = 0;
  }
  return FLOQUET_OK;
}

int profile_read(double* ms, int64_t* apps, double* bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& e : g_prof_pending) {
    FQ_CUDA(cudaEventSynchronize(e.b));
    float t = 0;
    FQ_CUDA(cudaEventElapsedTime(&t, e.a, e.b));
    g_prof_ms[e.kind] += t;
    g_prof_apps[e.kind] += e.u_apps;
    g_prof_bytes[e.kind] += e.bytes;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g_prof_pending.clear();
  for (int i = 0; i < 3; ++i) {
    if (ms) ms[i] = g_prof_ms[i];
    if (apps) apps[i] = g_prof_apps[i];
    if (bytes) bytes[i] = g_prof_bytes[i];
  }
  return FLOQUET_OK;
}

static bool profile_begin(cudaStream_t s, cudaEvent_t* a) {
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return false;
  }
  if (cudaEventCreate(a) != cudaSuccess) return false;
  cudaEventRecord(*a, s);
  return true;
}

static void profile_end(cudaStream_t s, cudaEvent_t a, int kind, int64_t u_apps,
                        double bytes) {
  cudaEvent_t b;
  if (cudaEventCreate(&b) != cudaSuccess) return;
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_pending.push_back(SweepEvent{a, b, kind, u_apps, bytes});
}

void count_launch(int64_t n) {
  std::lock_guard<std::mutex> lk(g_launch_mu);
  g_launches += n;
}
int64_t launch_count() {
  std::lock_guard<std::mutex> lk(g_launch_mu);
  return g_launches;
}
void reset_launch_count() {
  std::lock_guard<std::mutex> lk(g_launch_mu);
  g_launches = 0;
}

// The pass kernel itself is in pass_kernel.cuh, instantiated per sweep precision in
// pass_f32.cu, pass_f64.cu and pass_df.cu.

// ------------------------------------------------------------------ elementwise kernels

template <typename Rin, typename Rout>
__global__ void convert_kernel(const cplx<Rin>* __restrict__ in, cplx<Rout>* __restrict__ out,
                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = from_d2<Rout>(to_d2(in[i]));
}

static unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename Rin, typename Rout>
int launch_convert(const cplx<Rin>* in, cplx<Rout>* out, int64_t n, cudaStream_t st) {
  convert_kernel<Rin, Rout><<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}
template int launch_convert<double, float>(const double2*, float2*, int64_t, cudaStream_t);
template int launch_convert<float, double>(const float2*, double2*, int64_t, cudaStream_t);
template int launch_convert<double, double>(const double2*, double2*, int64_t, cudaStream_t);
template int launch_convert<float, float>(const float2*, float2*, int64_t, cudaStream_t);
template int launch_convert<double, dfloat>(const double2*, float4*, int64_t, cudaStream_t);
template int launch_convert<dfloat, double>(const float4*, double2*, int64_t, cudaStream_t);

template <typename Rin, typename Rout>
__global__ void filter_init_kernel(const cplx<Rin>* __restrict__ in, int64_t in_stride,
                                   cplx<Rout>* __restrict__ work, cplx<Rout>* __restrict__ acc,
                                   const cplx<Rout>* __restrict__ coef, int64_t coef_stride,
                                   int64_t d) {
  const int64_t vec = blockIdx.y;
  const double2 c0 = coef ? to_d2(coef[vec * coef_stride]) : make_double2(1, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = to_d2(in[vec * in_stride + i]);
    if (work) work[vec * d + i] = from_d2<Rout>(x);
    acc[vec * d + i] = from_d2<Rout>(cmul(c0, x));
  }
}

template <typename Rin, typename Rout>
int launch_filter_init(const cplx<Rin>* in, int64_t in_stride, cplx<Rout>* work,
                       cplx<Rout>* acc, const cplx<Rout>* coef, int64_t coef_stride, int64_t d,
                       int nvec, cudaStream_t st) {
  unsigned gx = grid_for(d, 256);
  if ((int64_t)gx * nvec > 152 * 64) gx = (unsigned)std::max<int64_t>(1, 152 * 64 / nvec);
  dim3 grid(gx, nvec);
  filter_init_kernel<Rin, Rout><<<grid, 256, 0, st>>>(in, in_stride, work, acc, coef,
                                                      coef_stride, d);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}
template int launch_filter_init<double, float>(const double2*, int64_t, float2*, float2*,
                                               const float2*, int64_t, int64_t, int,
                                               cudaStream_t);
template int launch_filter_init<double, double>(const double2*, int64_t, double2*, double2*,
                                                const double2*, int64_t, int64_t, int,
                                                cudaStream_t);
template int launch_filter_init<float, float>(const float2*, int64_t, float2*, float2*,
                                              const float2*, int64_t, int64_t, int, cudaStream_t);
template int launch_filter_init<double, dfloat>(const double2*, int64_t, float4*, float4*,
                                                const float4*, int64_t, int64_t, int,
                                                cudaStream_t);

// out[vec * out_stride + i] = in[vec * d + i] (converted)
template <typename Rin, typename Rout>
__global__ void convert_strided_kernel(const cplx<Rin>* __restrict__ in,
                                       cplx<Rout>* __restrict__ out, int64_t out_stride,
                                       int64_t d) {
  const int64_t vec = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[vec * out_stride + i] = from_d2<Rout>(to_d2(in[vec * d + i]));
  }
}

template <typename Rin, typename Rout>
static int launch_convert_strided(const cplx<Rin>* in, cplx<Rout>* out, int64_t out_stride,
                                  int64_t d, int nvec, cudaStream_t st) {
  unsigned gx = grid_for(d, 256);
  if ((int64_t)gx * nvec > 152 * 64) gx = (unsigned)std::max<int64_t>(1, 152 * 64 / nvec);
  convert_strided_kernel<Rin, Rout><<<dim3(gx, nvec), 256, 0, st>>>(in, out, out_stride, d);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// ------------------------------------------------------------------ operator set-up


template <typename Real> static int sweep_dtype();
template <> int sweep_dtype<float>() { return FLOQUET_C64; }
template <> int sweep_dtype<double>() { return FLOQUET_C128; }
template <> int sweep_dtype<dfloat>() { return FLOQUET_C128_DF; }

// Split the L qubits into passes: the first kicks the NB lowest qubits in contiguous tiles;
// each later pass keeps at least `min_cols` low (contiguous) bits in its tile for coalescing
// and kicks up to NB - min_cols further qubits.
static Plan make_plan(int L, int NBmax, int min_cols) {
  Plan p;
  if (L <= NBmax) {
    p.passes.push_back(Pass{L, L, L, 0});
    return p;
  }
  p.passes.push_back(Pass{NBmax, NBmax, NBmax, 0});
  int q0 = NBmax;
  while (q0 < L) {
    const int nq = std::min(L - q0, NBmax - min_cols);
    const int c = NBmax - nq;
    p.passes.push_back(Pass{NBmax, c, q0, c});
    q0 += nq;
  }
  return p;
}

}  // namespace fq

// Host-only query of the pass plan (C ABI): the passes make_plan forms and the two derived
// index fields the kernels receive (midbits = start - c, topshift = start + NB - c; for a
// single pass 0 and L).
extern "C" int floquet_pass_plan(int L, int NB, int min_cols, int* out, int max_passes,
                                 int* n_passes) {
  using namespace fq;
  if (L < 1 || L > 30 || NB < 1 || min_cols < 0 || min_cols >= NB || !out || !n_passes ||
      max_passes < 1) {
    set_error("floquet_pass_plan: invalid arguments");
    return FLOQUET_EINVAL;
  }
  const Plan p = make_plan(L, NB, min_cols);
  *n_passes = (int)p.passes.size();
  if ((int)p.passes.size() > max_passes) {
    set_error("floquet_pass_plan: %d passes, room for %d", (int)p.passes.size(), max_passes);
    return FLOQUET_EINVAL;
  }
  for (size_t i = 0; i < p.passes.size(); ++i) {
    const Pass& ps = p.passes[i];
    const bool single = ps.NB == L;
    int* o = out + 6 * i;
    o[0] = ps.NB;
    o[1] = ps.c;
    o[2] = ps.start;
    o[3] = ps.kick_from;
    o[4] = single ? 0 : ps.start - ps.c;
    o[5] = single ? L : ps.start + ps.NB - ps.c;
  }
  set_error("%s", "");
  return FLOQUET_OK;
}

namespace fq {

template <typename Real>
static PassArgs<Real> make_args(const floquet_op* op, const Pass& ps, const cplx<Real>* tlo,
                                const cplx<Real>* thi) {
  PassArgs<Real> a;
  memset(&a, 0, sizeof(a));
  a.d = op->d;
  a.L = op->L;
  a.NB = ps.NB;
  a.c = ps.c;
  a.start = ps.start;
  a.kick_from = ps.kick_from;
  a.midbits = ps.start - ps.c;
  a.topshift = ps.start + ps.NB - ps.c;
  if (ps.NB == op->L) {  // single pass: the whole state is one tile
    a.midbits = 0;
    a.topshift = op->L;
  }
  a.tau = scal_from<Real>(op->tau);
  a.tab_lo = tlo;
  a.tab_hi = thi;
  a.a = op->tabs.a;
  a.tab_lo_stride = op->tabs.lo_n;
  a.tab_hi_stride = op->tabs.hi_n;
  a.vec_per_prob = 1;
  return a;
}

// Column bits kept in the later passes' tiles: 4 complex64 (32-byte row segments) or 3
// wider elements (48-byte segments).
template <typename Real> static int min_cols() { return sizeof(cplx<Real>) == 8 ? 4 : 3; }

template <typename Real> static void set_variant(floquet_op* op, int v) {
  const int t = sweep_dtype<Real>();
  op->variant[t] = v;
  const PassVariant pv = variant_info<Real>(v);
  op->plan[t] = make_plan(op->L, pv.NB, pv.cols > 0 ? pv.cols : min_cols<Real>());
}

int op_init(floquet_op* op, int L, double J, double g, const double* h, int nprob) {
  op->L = L;
  op->J = J;
  op->g = g;
  op->d = (int64_t)1 << L;
  op->nprob = nprob;
  op->h.assign(h, h + (size_t)L * nprob);
  const double c = cos(g), s = sin(g);
  // scale of the kick layer after factoring each 2x2 rotation
  double sc_re, sc_im;
  if (fabs(c) >= fabs(s)) {
    op->swap = false;
    op->tau = s / c;  // x' = x - i tan(g) y
    sc_re = pow(c, L);
    sc_im = 0;
  } else {
    op->swap = true;
    op->tau = -c / s;  // outputs exchanged, tau = -cot g
    // (-i s)^L
    const double mag = pow(fabs(s), L) * ((s < 0 && (L & 1)) ? -1.0 : 1.0);
    const int ph = L & 3;  // (-i)^L
    const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, -1, 0, 1};
    sc_re = mag * pr[ph];
    sc_im = mag * pi[ph];
  }
  const int a = (L + 2) / 2;
  BatchTables& T = op->tabs;
  T.a = a;
  T.P = nprob;
  T.lo_n = (int64_t)1 << a;
  T.hi_n = (int64_t)1 << (L - a + 2);
  std::vector<double2> lo((size_t)T.lo_n * nprob), hi((size_t)T.hi_n * nprob);
  std::vector<float2> lo32(lo.size()), hi32(hi.size());
  for (int p = 0; p < nprob; ++p) {
    const double* hp = h + (size_t)p * L;
    for (int64_t x = 0; x < T.lo_n; ++x) {  // bits [0, a): fields and internal bonds
      double th = 0;
      for (int i = 0; i < a; ++i) {
        const int zi = ((x >> i) & 1) ? -1 : 1;
        th += hp[i] * zi;
        if (i + 1 < a) th += J * zi * ((((x >> (i + 1)) & 1)) ? -1 : 1);
      }
      const double cr = cos(th), ci = -sin(th);  // exp(-i theta) * scale
      lo[p * T.lo_n + x] = mk<double2>(cr * sc_re - ci * sc_im, cr * sc_im + ci * sc_re);
    }
    for (int64_t y = 0; y < T.hi_n; ++y) {
      // y = (u << 1) | b0, u = bits [a-1, L) of s
      const int b0 = (int)(y & 1);
      const int64_t u = y >> 1;
      auto z = [&](int i) -> int {  // z_i for i in [a-1, L) from u
        return ((u >> (i - (a - 1))) & 1) ? -1 : 1;
      };
      double th = 0;
      for (int i = a; i < L; ++i) th += hp[i] * z(i);
      for (int i = a - 1; i + 1 < L; ++i) th += J * z(i) * z(i + 1);
      th += J * z(L - 1) * (b0 ? -1 : 1);  // periodic bond (L-1, 0)
      hi[p * T.hi_n + y] = mk<double2>(cos(th), -sin(th));
    }
  }
  std::vector<float4> lodf(lo.size()), hidf(hi.size());
  for (size_t i = 0; i < lo.size(); ++i) lodf[i] = from_d2<dfloat>(lo[i]);
  for (size_t i = 0; i < hi.size(); ++i) hidf[i] = from_d2<dfloat>(hi[i]);
  FQ_CUDA(cudaMalloc(&T.lodf, lo.size() * sizeof(float4)));
  FQ_CUDA(cudaMalloc(&T.hidf, hi.size() * sizeof(float4)));
  FQ_CUDA(cudaMemcpy(T.lodf, lodf.data(), lo.size() * sizeof(float4), cudaMemcpyHostToDevice));
  FQ_CUDA(cudaMemcpy(T.hidf, hidf.data(), hi.size() * sizeof(float4), cudaMemcpyHostToDevice));
  for (size_t i = 0; i < lo.size(); ++i) lo32[i] = mk<float2>((float)lo[i].x, (float)lo[i].y);
  for (size_t i = 0; i < hi.size(); ++i) hi32[i] = mk<float2>((float)hi[i].x, (float)hi[i].y);
  FQ_CUDA(cudaMalloc(&T.lo64, lo.size() * sizeof(double2)));
  FQ_CUDA(cudaMalloc(&T.hi64, hi.size() * sizeof(double2)));
  FQ_CUDA(cudaMalloc(&T.lo32, lo.size() * sizeof(float2)));
  FQ_CUDA(cudaMalloc(&T.hi32, hi.size() * sizeof(float2)));
  FQ_CUDA(cudaMemcpy(T.lo64, lo.data(), lo.size() * sizeof(double2), cudaMemcpyHostToDevice));
  FQ_CUDA(cudaMemcpy(T.hi64, hi.data(), hi.size() * sizeof(double2), cudaMemcpyHostToDevice));
  FQ_CUDA(cudaMemcpy(T.lo32, lo32.data(), lo.size() * sizeof(float2), cudaMemcpyHostToDevice));
  FQ_CUDA(cudaMemcpy(T.hi32, hi32.data(), hi.size() * sizeof(float2), cudaMemcpyHostToDevice));
  set_variant<float>(op, 0);
  set_variant<double>(op, 0);
  set_variant<dfloat>(op, 0);
  return FLOQUET_OK;
}

static void destroy_graphs(floquet_op* op) {
  for (auto& g : op->graphs) cudaGraphExecDestroy(g.exec);
  op->graphs.clear();
}

void op_free(floquet_op* op) {
  destroy_graphs(op);
  brick_free(op->brick);
  op->brick = nullptr;
  if (op->cap_stream) cudaStreamDestroy(op->cap_stream);
  if (op->ev_in) cudaEventDestroy(op->ev_in);
  if (op->ev_out) cudaEventDestroy(op->ev_out);
  cudaFree(op->tabs.lo64);
  cudaFree(op->tabs.hi64);
  cudaFree(op->tabs.lo32);
  cudaFree(op->tabs.lodf);
  cudaFree(op->tabs.hidf);
  cudaFree(op->tabs.hi32);
  cudaFree(op->work);
  cudaFree(op->acc);
  cudaFree(op->psi_in_copy);
  cudaFree(op->zlo);
  cudaFree(op->coef);
  cudaFree(op->bar);
  cudaFree(op->ptab);
}

template <typename Real> static const Plan& plan_of(const floquet_op* op);
template <typename Real> const Plan& plan_of(const floquet_op* op) {
  return op->plan[sweep_dtype<Real>()];
}
template <typename Real> static const cplx<Real>* tlo_of(const floquet_op* op);
template <> const float2* tlo_of<float>(const floquet_op* op) { return op->tabs.lo32; }
template <> const double2* tlo_of<double>(const floquet_op* op) { return op->tabs.lo64; }
template <> const float4* tlo_of<dfloat>(const floquet_op* op) { return op->tabs.lodf; }
template <typename Real> static const cplx<Real>* thi_of(const floquet_op* op);
template <> const float2* thi_of<float>(const floquet_op* op) { return op->tabs.hi32; }
template <> const double2* thi_of<double>(const floquet_op* op) { return op->tabs.hi64; }
template <> const float4* thi_of<dfloat>(const floquet_op* op) { return op->tabs.hidf; }

// One U application (all passes) from `in` to `out` (in place allowed), with the last
// pass's epilogue `epi`.
template <typename Real>
static int u_passes(floquet_op* op, const cplx<Real>* in, cplx<Real>* out, int nvec,
                    int vec_per_prob, int epi, cplx<Real>* acc, const cplx<Real>* coef,
                    int64_t coef_stride, int jstep, const cplx<Real>* psi_in, cudaStream_t st,
                    const cplx<Real>* lo_per_vec = nullptr,
                    const cplx<Real>* hcoef = nullptr, int64_t hcoef_stride = 0) {
  const Plan& pl = plan_of<Real>(op);
  const int np = (int)pl.passes.size();
  for (int i = 0; i < np; ++i) {
    PassArgs<Real> a = make_args<Real>(op, pl.passes[i], tlo_of<Real>(op), thi_of<Real>(op));
    a.src = (i == 0) ? in : out;
    a.dst = out;
    a.vec_per_prob = vec_per_prob;
    const bool last = (i == np - 1);
    if (last) {
      a.acc = acc;
      a.coef = coef;
      a.coef_stride = coef_stride;
      a.jstep = jstep;
      a.psi_in = psi_in;
      a.hcoef = hcoef;
      a.hcoef_stride = hcoef_stride;
      if (lo_per_vec) {  // one tab_lo per vector (Horner, z folded in)
        a.tab_lo = lo_per_vec;
        a.lo_by_vec = 1;
      }
    }
    FQ_TRY(launch_pass_variant<Real>(op->variant[sweep_dtype<Real>()], a,
                                     last ? epi : EPI_STORE, op->swap, nvec, st));
  }
  return FLOQUET_OK;
}

static void destroy_graphs(floquet_op* op);

// out[v * d + s] = zs[v] * D_s (times the kick scale; zs null: z = 1), the product of the two
// chunk tables formed in float64, for the persistent kernel's full phase table
template <typename Real>
__global__ void phase_table_kernel(const double2* __restrict__ tlo, const double2* __restrict__ thi,
                                   int a, int vpp, int64_t lo_n, int64_t hi_n,
                                   const cplx<Real>* __restrict__ zs, cplx<Real>* __restrict__ out,
                                   int64_t d) {
  const int64_t v = blockIdx.y;
  const int64_t prob = v / vpp;
  const double2 z = zs ? to_d2(zs[v]) : make_double2(1.0, 0.0);
  const uint32_t lomask = (1u << a) - 1u;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < d;
       s += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t u = (uint32_t)s;
    const double2 p = cmul(tlo[prob * lo_n + (u & lomask)],
                           thi[prob * hi_n + (((u >> (a - 1)) << 1) | (u & 1u))]);
    out[v * d + s] = from_d2<Real>(cmul(z, p));
  }
}

// The full phase table z D_s per vector for double-float sweeps with up to 2^23 table entries
// (*out stays null otherwise, and for the other precisions, whose sweeps are bound by data
// movement rather than arithmetic). Cached filter graphs hold the table's address: a
// reallocation drops them.
template <typename Real>
static int build_phase_table(floquet_op* op, const cplx<Real>* zs, int nvec, int vpp,
                             cudaStream_t st, const cplx<Real>** out) {
  *out = nullptr;
  const int64_t d = op->d;
  if (!std::is_same<Real, dfloat>::value || (int64_t)nvec * d > (int64_t(1) << 23))
    return FLOQUET_OK;
  const size_t pbytes = (size_t)nvec * d * sizeof(cplx<Real>);
  if (op->ptab_bytes < pbytes) {
    destroy_graphs(op);
    cudaFree(op->ptab);
    op->ptab = nullptr;
    op->ptab_bytes = 0;
    if (cudaMalloc(&op->ptab, pbytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("filter workspace: cudaMalloc of %zu bytes failed", pbytes);
      return FLOQUET_ENOMEM;
    }
    op->ptab_bytes = pbytes;
  }
  phase_table_kernel<Real><<<dim3(grid_for(d, 256), nvec), 256, 0, st>>>(
      op->tabs.lo64, op->tabs.hi64, op->tabs.a, vpp, op->tabs.lo_n, op->tabs.hi_n, zs,
      reinterpret_cast<cplx<Real>*>(op->ptab), d);
  count_launch();
  FQ_CHECK_LAUNCH();
  *out = reinterpret_cast<const cplx<Real>*>(op->ptab);
  return FLOQUET_OK;
}

// Live test data for the autotuner: a normalised state with varied amplitudes.
template <typename Real>
__global__ void tune_fill_kernel(cplx<Real>* __restrict__ x, int64_t n, double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = from_d2<Real>(make_double2(scale * cos(0.1 * (double)i), scale * sin(0.37 * (double)i)));
}

static int ensure_bar(floquet_op* op);

// Persistent Horner kernel arguments for nvec vectors of the operator's own tables (z = 1,
// vec_per_prob = nvec: one problem).
template <typename Real>
static HornerGridArgs<Real> grid_args(floquet_op* op, const cplx<Real>* pin, cplx<Real>* acc,
                                      const cplx<Real>* tlo, int64_t lo_stride, int64_t k,
                                      int nvec, int vec_per_prob) {
  HornerGridArgs<Real> ga;
  memset(&ga, 0, sizeof(ga));
  ga.psi_in = pin;
  ga.t = acc;
  ga.d = op->d;
  ga.L = op->L;
  ga.nvec = nvec;
  ga.vec_per_prob = vec_per_prob;
  ga.a = op->tabs.a;
  ga.tau = scal_from<Real>(op->tau);
  ga.tab_lo = tlo;
  ga.lo_stride = lo_stride;
  ga.tab_hi = thi_of<Real>(op);
  ga.hi_stride = op->tabs.hi_n;
  ga.nsteps = k;
  ga.bar = op->bar;
  return ga;
}

// Autotuner: the first U application or filter in a sweep precision on an operator with
// L >= 13 times the launch choices on the hot path's own work, Horner filter steps
// acc <- psi_in + z U acc on a live (non-zero) state with the caller's batch width: every
// per-pass launch shape of the precision (3 warm-up and 10 timed steps) and, where the chain
// length has one, the persistent kernel (10 steps in one launch after a warm-up launch).
// The fastest launch shape serves plain U applications and per-pass filters; the persistent
// kernel serves the Horner filters if it beats that shape. CUDA events on the caller's
// stream. It runs before any filter graph of the operator is captured and drops the
// operator's cached graphs when it changes the plan. FLOQUET_PASS_VARIANT=<i> pins a shape
// and FLOQUET_FILTER_KERNEL=grid|pass the filter kernel, with FLOQUET_GRID_SHAPE=<i> the
// persistent kernel's shape (profiling, tests).
// Process-wide memory of the tuner's choices per (device, L, sweep precision, timed batch
// width): operators of the same geometry take the stored choice instead of timing again (the
// choice depends on the launch geometry, not on the field values), which also keeps the
// choice stable from one operator to the next.
struct TuneKey {
  int dev, L, dtype, nt;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, L, dtype, nt) < std::tie(o.dev, o.L, o.dtype, o.nt);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune_memo;  // -> (pass variant, grid shape)

template <typename Real> static int tune(floquet_op* op, int nvec, cudaStream_t st) {
  const int t = sweep_dtype<Real>();
  if (op->tuned[t]) return FLOQUET_OK;
  op->tuned[t] = true;
  const std::vector<HornerGridShape<Real>> gs = horner_grid_shapes<Real>(op->L);
  const bool has_grid = !gs.empty();
  op->gshape[t] = has_grid ? 0 : -1;
  const char* fk = getenv("FLOQUET_FILTER_KERNEL");
  const bool grid_forced = fk && (strcmp(fk, "grid") == 0 || strcmp(fk, "pass") == 0);
  if (grid_forced) op->gshape[t] = (has_grid && strcmp(fk, "grid") == 0) ? 0 : -1;
  if (const char* fs = getenv("FLOQUET_GRID_SHAPE")) {  // pin a persistent shape (tests)
    const int i = atoi(fs);
    if (grid_forced && op->gshape[t] >= 0 && i >= 0 && i < (int)gs.size()) op->gshape[t] = i;
  }
  const int nv = num_variants<Real>();
  const char* forced = getenv("FLOQUET_PASS_VARIANT");  // fixed shape, e.g. to profile
  if (forced) {
    const int v = atoi(forced);
    if (v >= 0 && v < nv && variant_info<Real>(v).NB <= op->L) {
      set_variant<Real>(op, v);
      destroy_graphs(op);
    }
  }
  if (op->L < 13 || (forced && (grid_forced || !has_grid)) || (nv < 2 && !has_grid))
    return FLOQUET_OK;
  // time with the caller's batch width (capped), since the best tile depends on how many
  // CTAs the whole launch has
  const int nt = std::max(1, std::min(nvec, std::max(1, (int)((int64_t(64) << 20) / op->d))));
  int dev = 0;
  FQ_CUDA(cudaGetDevice(&dev));
  const TuneKey key{dev, op->L, t, nt};
  const bool memo_ok = !forced && !grid_forced;
  if (memo_ok) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune_memo.find(key);
    if (it != g_tune_memo.end()) {
      set_variant<Real>(op, it->second.first);
      op->gshape[t] = it->second.second;
      destroy_graphs(op);
      return FLOQUET_OK;
    }
  }
  cplx<Real>* buf = nullptr;
  FQ_CUDA(cudaMalloc(&buf, 2 * sizeof(cplx<Real>) * op->d * nt));
  cplx<Real>* pin = buf;
  cplx<Real>* acc = buf + op->d * nt;
  tune_fill_kernel<Real><<<grid_for(op->d * nt, 256), 256, 0, st>>>(
      pin, op->d * nt, 1.0 / std::sqrt((double)op->d));
  tune_fill_kernel<Real><<<grid_for(op->d * nt, 256), 256, 0, st>>>(
      acc, op->d * nt, 1.0 / std::sqrt((double)op->d));
  count_launch(2);
  cudaEvent_t e0, e1;
  FQ_CUDA(cudaEventCreate(&e0));
  FQ_CUDA(cudaEventCreate(&e1));
  const bool verbose = getenv("FLOQUET_VERBOSE") != nullptr;
  float best = 3.0e38f;
  int bestv = op->variant[t];
  int rc = FLOQUET_OK;
  for (int v = 0; v < nv && rc == FLOQUET_OK && !forced; ++v) {
    set_variant<Real>(op, v);
    if (variant_info<Real>(v).NB > op->L) continue;
    for (int i = 0; i < 3 && rc == FLOQUET_OK; ++i)
      rc = u_passes<Real>(op, acc, acc, nt, nt, EPI_PHASE_HORNER, nullptr, nullptr, 0, 0, pin,
                          st);
    cudaEventRecord(e0, st);
    for (int i = 0; i < 10 && rc == FLOQUET_OK; ++i)
      rc = u_passes<Real>(op, acc, acc, nt, nt, EPI_PHASE_HORNER, nullptr, nullptr, 0, 0, pin,
                          st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = FLOQUET_ECUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (verbose)
      fprintf(stderr, "floquet tune: L=%d dtype=%d nvec=%d shape (NB=%d, RB=%d): %.2f us per "
              "Horner step\n", op->L, t, nt, variant_info<Real>(v).NB, variant_info<Real>(v).RB,
              1000.0 * ms / 10);
    if (rc == FLOQUET_OK && ms < best) {
      best = ms;
      bestv = v;
    }
  }
  if (!forced) set_variant<Real>(op, bestv);
  if (has_grid && !grid_forced && rc == FLOQUET_OK) {
    rc = ensure_bar(op);
    HornerGridArgs<Real> ga = grid_args<Real>(op, pin, acc, tlo_of<Real>(op), 0, 11, nt, nt);
    if (rc == FLOQUET_OK) rc = build_phase_table<Real>(op, nullptr, nt, nt, st, &ga.ptab);
    float gbest = 3.0e38f;
    int gi = -1;
    for (int i = 0; i < (int)gs.size() && rc == FLOQUET_OK; ++i) {
      rc = gs[i].launch(ga, op->swap, false, st);
      cudaEventRecord(e0, st);
      if (rc == FLOQUET_OK) rc = gs[i].launch(ga, op->swap, false, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = FLOQUET_ECUDA;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (verbose)
        fprintf(stderr, "floquet tune: L=%d dtype=%d nvec=%d persistent kernel (NB=%d, RB=%d, "
                "C=%d): %.2f us per Horner step\n", op->L, t, nt, gs[i].NB, gs[i].RB, gs[i].C,
                1000.0 * ms / 10);
      if (rc == FLOQUET_OK && ms < gbest) {
        gbest = ms;
        gi = i;
      }
    }
    op->gshape[t] = (rc == FLOQUET_OK && (forced || gbest < best)) ? gi : -1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  destroy_graphs(op);
  if (rc == FLOQUET_OK && memo_ok) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_memo[key] = std::make_pair(op->variant[t], op->gshape[t]);
  }
  return rc;
}

template <typename Real>
int apply_u(floquet_op* op, const cplx<Real>* in, cplx<Real>* out, int nvec, int vec_per_prob,
            cudaStream_t st) {
  if (op->brick) {
    if constexpr (std::is_same<Real, double>::value) {
      return brick_apply(op->brick, in, out, nvec, st);
    } else {
      set_error("brickwork operator: complex128 sweeps only");
      return FLOQUET_EINVAL;
    }
  }
  FQ_TRY(tune<Real>(op, nvec, st));
  return u_passes<Real>(op, in, out, nvec, vec_per_prob, EPI_PHASE, nullptr, nullptr, 0, 0,
                        nullptr, st);
}
template int apply_u<float>(floquet_op*, const float2*, float2*, int, int, cudaStream_t);
template int apply_u<double>(floquet_op*, const double2*, double2*, int, int, cudaStream_t);
template int apply_u<dfloat>(floquet_op*, const float4*, float4*, int, int, cudaStream_t);

// ------------------------------------------------------------------ filter loops

static int ensure_workspace(floquet_op* op, size_t bytes) {
  if (op->work_bytes >= bytes) return FLOQUET_OK;
  destroy_graphs(op);  // graphs reference the old buffers
  cudaFree(op->work);
  cudaFree(op->acc);
  cudaFree(op->psi_in_copy);
  op->work = op->acc = op->psi_in_copy = nullptr;
  op->work_bytes = 0;
  if (cudaMalloc(&op->work, bytes) != cudaSuccess || cudaMalloc(&op->acc, bytes) != cudaSuccess ||
      cudaMalloc(&op->psi_in_copy, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("filter workspace: cudaMalloc of 3 x %zu bytes failed", bytes);
    return FLOQUET_ENOMEM;
  }
  op->work_bytes = bytes;
  return FLOQUET_OK;
}

// Grid-barrier words of the persistent filter kernel (allocated once per operator).
static int ensure_bar(floquet_op* op) {
  if (op->bar) return FLOQUET_OK;
  if (cudaMalloc(&op->bar, kBarWords * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    set_error("filter workspace: cudaMalloc of the barrier words failed");
    return FLOQUET_ENOMEM;
  }
  return FLOQUET_OK;
}

// The brickwork GEMM scratch, grown before a filter loop is captured; cached graphs hold the
// old buffer's address, so they are dropped when it grows.
static int brick_reserve_for_graphs(floquet_op* op, int nvec) {
  if (op->brick->tmp_elems < ((size_t)nvec << op->L)) destroy_graphs(op);
  return brick_reserve(op->brick, nvec);
}

static FilterGraph* find_graph(floquet_op* op, int64_t k, int nvec, int dtype, int form,
                               const void* coef, int vpp) {
  for (auto& g : op->graphs)
    if (g.k == k && g.nvec == nvec && g.dtype == dtype && g.form == form && g.key_coef == coef &&
        g.key_in == (const void*)(intptr_t)vpp)
      return &g;
  return nullptr;
}

// Runs `body(stream)` either directly on `st` or through a cached graph of it. Graphs are
// captured and replayed on the operator's own non-blocking stream, ordered after `st` and
// before any later work on `st` by events (the legacy default stream cannot be captured).
template <typename F>
static int run_loop(floquet_op* op, bool use_graph, int64_t k, int nvec, int dtype, int form,
                    const void* coef, int vpp, int64_t launches_per_body, cudaStream_t st,
                    F body) {
  const int kind = dtype == FLOQUET_C64 ? 1 : (dtype == FLOQUET_C128 ? 0 : 2);
  const double b = dtype == FLOQUET_C64 ? 8.0 : 16.0;
  const int64_t u_apps = (k - 1) * (int64_t)nvec;
  const double alg_bytes = (form == FLOQUET_FORM_ACC ? 4.0 : 3.0) * b * (double)op->d * u_apps;
  if (!use_graph) {
    cudaEvent_t a;
    const bool prof = profile_begin(st, &a);
    const int rc = body(st);
    if (prof) profile_end(st, a, kind, u_apps, alg_bytes);
    return rc;
  }
  if (!op->cap_stream) {
    FQ_CUDA(cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking));
    FQ_CUDA(cudaEventCreateWithFlags(&op->ev_in, cudaEventDisableTiming));
    FQ_CUDA(cudaEventCreateWithFlags(&op->ev_out, cudaEventDisableTiming));
  }
  cudaStream_t cs = op->cap_stream;
  FilterGraph* g = find_graph(op, k, nvec, dtype, form, coef, vpp);
  if (!g) {
    cudaGraph_t graph;
    FQ_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int rc = body(cs);
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc != FLOQUET_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) {
      set_error("graph capture failed: %s", cudaGetErrorString(e));
      return FLOQUET_ECUDA;
    }
    FilterGraph fg;
    fg.k = k;
    fg.nvec = nvec;
    fg.dtype = dtype;
    fg.form = form;
    fg.key_coef = coef;
    fg.key_in = (const void*)(intptr_t)vpp;
    fg.key_out = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&fg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      set_error("graph instantiate failed: %s", cudaGetErrorString(ei));
      return FLOQUET_ECUDA;
    }
    // the capture counted launches that did not run
    count_launch(-launches_per_body);
    op->graphs.push_back(fg);
    g = &op->graphs.back();
  }
  FQ_CUDA(cudaEventRecord(op->ev_in, st));
  FQ_CUDA(cudaStreamWaitEvent(cs, op->ev_in, 0));
  cudaEvent_t pa;
  const bool prof = profile_begin(cs, &pa);
  FQ_CUDA(cudaGraphLaunch(g->exec, cs));
  if (prof) profile_end(cs, pa, kind, u_apps, alg_bytes);
  FQ_CUDA(cudaEventRecord(op->ev_out, cs));
  FQ_CUDA(cudaStreamWaitEvent(st, op->ev_out, 0));
  count_launch(launches_per_body);
  return FLOQUET_OK;
}

template <typename Real, typename Rio>
int filter_coef(floquet_op* op, const cplx<Rio>* in, int64_t in_stride, cplx<Rio>* out,
                int64_t out_stride, const cplx<Real>* coef, int64_t k, int nvec,
                int vec_per_prob, bool use_graph, cudaStream_t st) {
  using C = cplx<Real>;
  const int64_t d = op->d;
  if (op->brick && !std::is_same<Real, double>::value) {
    set_error("brickwork operator: complex128 sweeps only");
    return FLOQUET_EINVAL;
  }
  if (!op->brick) FQ_TRY(tune<Real>(op, nvec, st));
  FQ_TRY(ensure_workspace(op, (size_t)nvec * d * sizeof(C)));
  C* work = reinterpret_cast<C*>(op->work);
  C* acc = reinterpret_cast<C*>(op->acc);
  if (op->brick) FQ_TRY(brick_reserve_for_graphs(op, nvec));  // before any capture
  FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, work, acc, coef, k, d, nvec, st)));
  const int np = op->brick ? 2 + nvec : (int)plan_of<Real>(op).passes.size();
  auto body = [&](cudaStream_t s) -> int {
    for (int64_t j = 1; j < k; ++j) {
      if constexpr (std::is_same<Real, double>::value) {
        if (op->brick) {
          FQ_TRY(brick_acc_step(op->brick, work, acc, coef, k, (int)j, nvec, s));
          continue;
        }
      }
      FQ_TRY(u_passes<Real>(op, work, work, nvec, vec_per_prob, EPI_PHASE_ACC, acc, coef, k,
                            (int)j, nullptr, s));
    }
    return FLOQUET_OK;
  };
  if (k > 1)
    FQ_TRY(run_loop(op, use_graph, k, nvec, sweep_dtype<Real>(),
                    FLOQUET_FORM_ACC, coef, vec_per_prob, (k - 1) * np, st, body));
  return launch_convert_strided<Real, Rio>(acc, out, out_stride, d, nvec, st);
}

// out[v * lo_n + j] = zs[v] * tab_lo[(v / vpp) * lo_n + j], the product formed in float64
template <typename Real>
__global__ void scale_lo_kernel(const cplx<Real>* __restrict__ tlo, int64_t lo_n, int vpp,
                                const cplx<Real>* __restrict__ zs, cplx<Real>* __restrict__ out,
                                int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / lo_n, j = i - v * lo_n;
    out[i] = from_d2<Real>(cmul(to_d2(zs[v]), to_d2(tlo[(v / vpp) * lo_n + j])));
  }
}

template <typename Real, typename Rio>
int filter_horner(floquet_op* op, const cplx<Rio>* in, int64_t in_stride, cplx<Rio>* out,
                  int64_t out_stride, const cplx<Real>* zs, int64_t k, int nvec,
                  int vec_per_prob, bool use_graph, cudaStream_t st) {
  using C = cplx<Real>;
  const int64_t d = op->d;
  if (op->brick) {
    if constexpr (std::is_same<Real, double>::value) {
      // brickwork: acc = psi_in + z U acc with U as two GEMMs, z as the second GEMM's alpha
      FQ_TRY(ensure_workspace(op, (size_t)nvec * d * sizeof(C)));
      FQ_TRY(brick_reserve_for_graphs(op, nvec));  // before any capture
      C* bpin = reinterpret_cast<C*>(op->psi_in_copy);
      C* bacc = reinterpret_cast<C*>(op->acc);
      FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, bpin, bacc, nullptr, 0, d, nvec, st)));
      auto bbody = [&](cudaStream_t s) -> int {
        for (int64_t j = 1; j < k; ++j)
          FQ_TRY(brick_horner_step(op->brick, bacc, bpin, zs, nvec, s));
        return FLOQUET_OK;
      };
      if (k > 1)
        FQ_TRY(run_loop(op, use_graph, k, nvec, sweep_dtype<Real>(), FLOQUET_FORM_HORNER, zs,
                        vec_per_prob, (k - 1) * (1 + nvec), st, bbody));
      return launch_convert_strided<Real, Rio>(bacc, out, out_stride, d, nvec, st);
    } else if constexpr (std::is_same<Real, dfloat>::value) {
      // brickwork in double-float: the split-K GEMMs of brickwork.cu, z folded into the
      // second product's epilogue
      FQ_TRY(ensure_workspace(op, (size_t)nvec * d * sizeof(C)));
      if (op->brick->tmp_elems < ((size_t)nvec << op->L)) destroy_graphs(op);
      const BrickOp before = *op->brick;
      FQ_TRY(brick_reserve_df(op->brick, nvec));  // before any capture
      if (op->brick->part != before.part || op->brick->tmp != before.tmp) destroy_graphs(op);
      C* bpin = reinterpret_cast<C*>(op->psi_in_copy);
      C* bacc = reinterpret_cast<C*>(op->acc);
      FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, bpin, bacc, nullptr, 0, d, nvec, st)));
      auto bbody = [&](cudaStream_t s) -> int {
        for (int64_t j = 1; j < k; ++j)
          FQ_TRY(brick_horner_step_df(op->brick, bacc, bpin, zs, nvec, s));
        return FLOQUET_OK;
      };
      if (k > 1)
        FQ_TRY(run_loop(op, use_graph, k, nvec, sweep_dtype<Real>(), FLOQUET_FORM_HORNER, zs,
                        vec_per_prob, (k - 1) * 4, st, bbody));
      return launch_convert_strided<Real, Rio>(bacc, out, out_stride, d, nvec, st);
    } else {
      set_error("brickwork operator: complex128 or double-float sweeps only");
      return FLOQUET_EINVAL;
    }
  }
  FQ_TRY(tune<Real>(op, nvec, st));
  FQ_TRY(ensure_workspace(op, (size_t)nvec * d * sizeof(C)));
  C* pin = reinterpret_cast<C*>(op->psi_in_copy);
  C* acc = reinterpret_cast<C*>(op->acc);
  // z folded into a per-vector copy of tab_lo, so the Horner epilogue is one complex
  // multiply-add; the buffer outlives the call because cached graphs hold its address
  const int64_t lo_n = op->tabs.lo_n;
  const size_t zbytes = (size_t)nvec * lo_n * sizeof(C);
  if (op->zlo_bytes < zbytes) {
    destroy_graphs(op);
    cudaFree(op->zlo);
    op->zlo = nullptr;
    op->zlo_bytes = 0;
    if (cudaMalloc(&op->zlo, zbytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("filter workspace: cudaMalloc of %zu bytes failed", zbytes);
      return FLOQUET_ENOMEM;
    }
    op->zlo_bytes = zbytes;
  }
  C* zlo = reinterpret_cast<C*>(op->zlo);
  scale_lo_kernel<Real><<<grid_for(nvec * lo_n, 256), 256, 0, st>>>(
      tlo_of<Real>(op), lo_n, vec_per_prob, zs, zlo, nvec * lo_n);
  count_launch();
  FQ_CHECK_LAUNCH();
  // persistent kernel: the whole loop in one cooperative launch (one grid barrier per U)
  const int gsi = op->gshape[sweep_dtype<Real>()];
  if (k > 1 && gsi >= 0) {
    const std::vector<HornerGridShape<Real>> gshapes = horner_grid_shapes<Real>(op->L);
    if (gsi < (int)gshapes.size()) {
      const HornerGridLaunch<Real> gl = gshapes[gsi].launch;
      FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, nullptr, pin, nullptr, 0, d, nvec,
                                            st)));
      FQ_TRY(ensure_bar(op));
      HornerGridArgs<Real> ga = grid_args<Real>(op, pin, acc, zlo, lo_n, k, nvec, vec_per_prob);
      // double-float: one table entry per amplitude (z D_s formed in float64) replaces the
      // double-float product of the two chunk tables in every step (arithmetic bound sweep)
      FQ_TRY(build_phase_table<Real>(op, zs, nvec, vec_per_prob, st, &ga.ptab));
      auto gbody = [&](cudaStream_t s) -> int { return gl(ga, op->swap, false, s); };
      FQ_TRY(run_loop(op, false, k, nvec, sweep_dtype<Real>(), FLOQUET_FORM_HORNER, zs,
                      vec_per_prob, 1, st, gbody));
      return launch_convert_strided<Real, Rio>(acc, out, out_stride, d, nvec, st);
    }
  }
  FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, pin, acc, nullptr, 0, d, nvec, st)));
  const int np = (int)plan_of<Real>(op).passes.size();
  // (the per-pass kernels form z D_s from the two chunk tables: a full per-amplitude table
  // read from L2 measured slower here, 30.9 against 29.4 us per vector-U at L = 20 with two
  // double-float vectors, than the arithmetic it saves)
  auto body = [&](cudaStream_t s) -> int {
    for (int64_t j = 1; j < k; ++j)
      FQ_TRY(u_passes<Real>(op, acc, acc, nvec, vec_per_prob, EPI_PHASE_HORNER, nullptr,
                            nullptr, 0, 0, pin, s, zlo));
    return FLOQUET_OK;
  };
  if (k > 1)
    FQ_TRY(run_loop(op, use_graph, k, nvec, sweep_dtype<Real>(),
                    FLOQUET_FORM_HORNER, zs, vec_per_prob, (k - 1) * np, st, body));
  return launch_convert_strided<Real, Rio>(acc, out, out_stride, d, nvec, st);
}

#define FQ_INST_FILTER(R, RIO)                                                            \
  template int filter_coef<R, RIO>(floquet_op*, const cplx<RIO>*, int64_t, cplx<RIO>*, int64_t, \
                                   const cplx<R>*, int64_t, int, int, bool, cudaStream_t);      \
  template int filter_horner<R, RIO>(floquet_op*, const cplx<RIO>*, int64_t, cplx<RIO>*,        \
                                     int64_t, const cplx<R>*, int64_t, int, int, bool,          \
                                     cudaStream_t);
FQ_INST_FILTER(float, float)
FQ_INST_FILTER(float, double)
FQ_INST_FILTER(double, double)
FQ_INST_FILTER(dfloat, double)

}  // namespace fq
