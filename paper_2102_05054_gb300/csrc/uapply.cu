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
#include <cstring>
#include <mutex>
#include <type_traits>

#include "floquet_internal.cuh"

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

// ------------------------------------------------------------------ double-float arithmetic

// Error-free transformations on the FP32 pipes (Dekker / Knuth two-sum and an FMA-based
// two-product). The _rn intrinsics keep the compiler from contracting or reassociating.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// x + t * y for double-float x, t, y
__device__ __forceinline__ float2 df_fma(float2 t, float2 y, float2 x) {
  const float p = __fmul_rn(t.x, y.x);
  const float pe = __fmaf_rn(t.x, y.x, -p);
  const float2 s = df_two_sum(x.x, p);
  const float lo = __fadd_rn(__fadd_rn(s.y, pe), __fmaf_rn(t.x, y.y, __fmaf_rn(t.y, y.x, x.y)));
  return df_quick_two_sum(s.x, lo);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)));
  return df_quick_two_sum(p, e);
}

// ------------------------------------------------------------------ per-precision arithmetic

// Butterfly x' = x - i tau y, y' = y - i tau x (one rounding per real output).
__device__ __forceinline__ void bfly(float2 x, float2 y, float tau, float2& xn, float2& yn) {
  xn = make_float2(fmaf(tau, y.y, x.x), fmaf(-tau, y.x, x.y));
  yn = make_float2(fmaf(tau, x.y, y.x), fmaf(-tau, x.x, y.y));
}
__device__ __forceinline__ void bfly(double2 x, double2 y, double tau, double2& xn,
                                     double2& yn) {
  xn = make_double2(fma(tau, y.y, x.x), fma(-tau, y.x, x.y));
  yn = make_double2(fma(tau, x.y, y.x), fma(-tau, x.x, y.y));
}
__device__ __forceinline__ void bfly(float4 x, float4 y, float2 tau, float4& xn, float4& yn) {
  // re(x') = re x + tau im y, im(x') = im x - tau re y
  const float2 nt = df_neg(tau);
  const float2 a = df_fma(tau, make_float2(y.z, y.w), make_float2(x.x, x.y));
  const float2 b = df_fma(nt, make_float2(y.x, y.y), make_float2(x.z, x.w));
  const float2 c = df_fma(tau, make_float2(x.z, x.w), make_float2(y.x, y.y));
  const float2 d = df_fma(nt, make_float2(x.x, x.y), make_float2(y.z, y.w));
  xn = make_float4(a.x, a.y, b.x, b.y);
  yn = make_float4(c.x, c.y, d.x, d.y);
}

// a * b (complex)
__device__ __forceinline__ float2 zmul(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float4 zmul(float4 a, float4 b) {
  const float2 ar = make_float2(a.x, a.y), ai = make_float2(a.z, a.w);
  const float2 br = make_float2(b.x, b.y), bi = make_float2(b.z, b.w);
  const float2 re = df_fma(ar, br, df_mul(df_neg(ai), bi));
  const float2 im = df_fma(ar, bi, df_mul(ai, br));
  return make_float4(re.x, re.y, im.x, im.y);
}
// acc + c * v (complex)
__device__ __forceinline__ float2 zfma(float2 c, float2 v, float2 acc) { return cfma(c, v, acc); }
__device__ __forceinline__ double2 zfma(double2 c, double2 v, double2 acc) {
  return cfma(c, v, acc);
}
__device__ __forceinline__ float4 zfma(float4 c, float4 v, float4 acc) {
  const float2 cr = make_float2(c.x, c.y), ci = make_float2(c.z, c.w);
  const float2 vr = make_float2(v.x, v.y), vi = make_float2(v.z, v.w);
  const float2 re = df_fma(cr, vr, df_fma(df_neg(ci), vi, make_float2(acc.x, acc.y)));
  const float2 im = df_fma(cr, vi, df_fma(ci, vr, make_float2(acc.z, acc.w)));
  return make_float4(re.x, re.y, im.x, im.y);
}

// ------------------------------------------------------------------ pass kernel

// Tile element e -> position in padded shared memory (one pad slot every 2^RB elements
// keeps the strided transposes free of bank conflicts).
template <int RB> __device__ __forceinline__ int smem_pos(int e) { return e + (e >> RB); }

// Element index of register r of thread t when the register bits are tile bits [g, g+RB).
template <int RB> __device__ __forceinline__ int tile_elem(int t, int r, int g) {
  return (t & ((1 << g) - 1)) | (r << g) | ((t >> g) << (g + RB));
}

template <typename Real, int RB, bool SWAP>
__device__ __forceinline__ void kick_registers(cplx<Real> (&v)[1 << RB], int g, int lo, int hi,
                                               scal<Real> tau) {
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    const int bit = g + b;
    if (bit >= lo && bit < hi) {
#pragma unroll
      for (int r = 0; r < (1 << RB); ++r) {
        if (r & (1 << b)) continue;
        cplx<Real> xn, yn;
        bfly(v[r], v[r | (1 << b)], tau, xn, yn);
        if (SWAP) {
          v[r] = yn;
          v[r | (1 << b)] = xn;
        } else {
          v[r] = xn;
          v[r | (1 << b)] = yn;
        }
      }
    }
  }
}

// NBT > 0: the tile size 2^NBT is a compile-time constant (the large tiles of the hot path),
// so every shared-memory index folds to a per-thread base plus a constant; NBT == 0: the
// tile size A.NB is read at run time (small states).
template <typename Real, int NBT, int RB, int EPI, bool SWAP>
__global__ void __launch_bounds__(256) pass_kernel(const PassArgs<Real> A) {
  using C = cplx<Real>;
  constexpr int R = 1 << RB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);

  const int NB = NBT > 0 ? NBT : A.NB;
  const int t = threadIdx.x;
  // flattened grid: blockIdx.x = vec * ntiles + tile (ntiles = 2^(L - NB))
  const int tilebits = A.L - NB;
  const int64_t vec = (int64_t)(blockIdx.x >> tilebits);
  const uint32_t cta = blockIdx.x & ((1u << tilebits) - 1u);
  const uint32_t mid = cta & ((1u << A.midbits) - 1u);
  const uint32_t top = cta >> A.midbits;
  const int c = A.c, start = A.start;
  const uint32_t cmask = (1u << c) - 1u;
  // global index of element e = t | (r << g_top): tbase + roff[r] (t and r bits are disjoint)
  const int g_top = NB - RB;
  const uint32_t tb = (uint32_t)t;
  const uint32_t tbase = ((mid << c) | (top << A.topshift)) + (tb & cmask) + ((tb >> c) << start);
  uint32_t roff[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t er = (uint32_t)r << g_top;
    roff[r] = (er & cmask) + ((er >> c) << start);
  }

  // Programmatic dependent launch: let the next pass be scheduled now (it waits for this
  // grid's completion before touching memory), then wait for the previous pass.
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const C* __restrict__ src = A.src + vec * A.d;
  C v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = src[tbase + roff[r]];
  // For complex64 (latency bound) the epilogue's other operand, the accumulator or Horner's
  // psi_in, is loaded together with the state so that its latency overlaps the kicks; the
  // wider types are arithmetic bound and keep their registers for the sweep instead.
  constexpr bool kPrefetch =
      (EPI == EPI_PHASE_ACC || EPI == EPI_PHASE_HORNER) && sizeof(C) == 8;
  const C* __restrict__ other = (EPI == EPI_PHASE_ACC ? A.acc : A.psi_in) + vec * A.d;
  C pre[kPrefetch ? R : 1];
  if (kPrefetch) {
#pragma unroll
    for (int r = 0; r < R; ++r) pre[r] = other[tbase + roff[r]];
  }

  // Round 0: register bits are the top RB tile bits.
  int hi = NB;
  int g = g_top;
  kick_registers<Real, RB, SWAP>(v, g, A.kick_from, hi, A.tau);
  hi = g;
  bool first_transpose = true;
  while (hi > A.kick_from) {
    const int gn = (hi - RB) > 0 ? (hi - RB) : 0;
    if (!first_transpose) __syncthreads();
    first_transpose = false;
#pragma unroll
    for (int r = 0; r < R; ++r) sm[smem_pos<RB>(tile_elem<RB>(t, r, g))] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sm[smem_pos<RB>(tile_elem<RB>(t, r, gn))];
    g = gn;
    kick_registers<Real, RB, SWAP>(v, g, A.kick_from, hi, A.tau);
    hi = g;
  }
  if (g != g_top) {  // back to the coalesced mapping
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) sm[smem_pos<RB>(tile_elem<RB>(t, r, g))] = v[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sm[smem_pos<RB>(tile_elem<RB>(t, r, g_top))];
  }

  C* __restrict__ dst = A.dst + vec * A.d;
  if (EPI == EPI_STORE) {
#pragma unroll
    for (int r = 0; r < R; ++r) dst[tbase + roff[r]] = v[r];
    return;
  }
  const int64_t prob = vec / A.vec_per_prob;
  const C* __restrict__ tlo = A.tab_lo + prob * A.tab_lo_stride;
  const C* __restrict__ thi = A.tab_hi + prob * A.tab_hi_stride;
  const uint32_t lomask = (1u << A.a) - 1u;
  const int am1 = A.a - 1;
  C cj;
  if (EPI == EPI_PHASE_ACC) cj = A.coef[vec * A.coef_stride + A.jstep];
  if (EPI == EPI_PHASE_HORNER) cj = A.coef[vec * A.coef_stride];
  C* __restrict__ acc = A.acc + vec * A.d;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t s = tbase + roff[r];
    const C p = zmul(__ldg(&tlo[s & lomask]), __ldg(&thi[((s >> am1) << 1) | (s & 1u)]));
    const C val = zmul(p, v[r]);
    if (EPI == EPI_PHASE) {
      dst[s] = val;
    } else {
      const C o = kPrefetch ? pre[kPrefetch ? r : 0] : other[s];
      if (EPI == EPI_PHASE_ACC) {
        dst[s] = val;
        acc[s] = zfma(cj, val, o);
      } else {  // Horner: dst (= acc) = psi_in + z * U acc
        dst[s] = zfma(cj, val, o);
      }
    }
  }
}

template <typename Real, int NBT, int RB, int EPI, bool SWAP>
static int launch_pass_t(const PassArgs<Real>& a, int nvec, cudaStream_t st) {
  const int threads = 1 << (a.NB - RB);
  // at most (2^12 + 2^8) * 8 or (2^11 + 2^8) * 16 bytes: below the 48 KiB default
  const size_t smem = (size_t)((1 << a.NB) + (1 << (a.NB - RB))) * sizeof(cplx<Real>);
  const int64_t ntiles = (int64_t)1 << (a.L - a.NB);
  if (ntiles * nvec > 0x7fffffffLL) {
    set_error("launch_pass: grid too large (nvec %d, tiles %lld)", nvec, (long long)ntiles);
    return FLOQUET_EINVAL;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ntiles * nvec));
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FQ_CUDA(cudaLaunchKernelEx(&cfg, pass_kernel<Real, NBT, RB, EPI, SWAP>, a));
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

template <typename Real, int NBT, int RB>
static int dispatch_epi(const PassArgs<Real>& a, int epi, bool swap, int nvec, cudaStream_t st) {
  switch (epi * 2 + (swap ? 1 : 0)) {
    case 0: return launch_pass_t<Real, NBT, RB, EPI_STORE, false>(a, nvec, st);
    case 1: return launch_pass_t<Real, NBT, RB, EPI_STORE, true>(a, nvec, st);
    case 2: return launch_pass_t<Real, NBT, RB, EPI_PHASE, false>(a, nvec, st);
    case 3: return launch_pass_t<Real, NBT, RB, EPI_PHASE, true>(a, nvec, st);
    case 4: return launch_pass_t<Real, NBT, RB, EPI_PHASE_ACC, false>(a, nvec, st);
    case 5: return launch_pass_t<Real, NBT, RB, EPI_PHASE_ACC, true>(a, nvec, st);
    case 6: return launch_pass_t<Real, NBT, RB, EPI_PHASE_HORNER, false>(a, nvec, st);
    case 7: return launch_pass_t<Real, NBT, RB, EPI_PHASE_HORNER, true>(a, nvec, st);
  }
  set_error("launch_pass: bad epilogue %d", epi);
  return FLOQUET_EINVAL;
}

// Largest tile (bits) per precision: 2^12 complex64 (34 KiB of shared memory with padding),
// 2^11 complex128 or double-float (36 KiB).
template <typename Real> static constexpr int max_tile_bits() { return 11; }
template <> constexpr int max_tile_bits<float>() { return 12; }

// Register bits per thread: 16 complex64 or 8 complex128 / double-float complex (32
// registers of data either way); a tile smaller than 2^4 complex64 uses 3.
template <typename Real>
int launch_pass(const PassArgs<Real>& a, int epi, bool swap, int nvec, cudaStream_t st) {
  constexpr int NBM = max_tile_bits<Real>();
  if constexpr (std::is_same<Real, float>::value) {
    if (a.NB == NBM) return dispatch_epi<Real, NBM, 4>(a, epi, swap, nvec, st);
    if (a.NB >= 4) return dispatch_epi<Real, 0, 4>(a, epi, swap, nvec, st);
    return dispatch_epi<Real, 0, 3>(a, epi, swap, nvec, st);
  } else {
    if (a.NB == NBM) return dispatch_epi<Real, NBM, 3>(a, epi, swap, nvec, st);
    return dispatch_epi<Real, 0, 3>(a, epi, swap, nvec, st);
  }
}
template int launch_pass<float>(const PassArgs<float>&, int, bool, int, cudaStream_t);
template int launch_pass<double>(const PassArgs<double>&, int, bool, int, cudaStream_t);
template int launch_pass<dfloat>(const PassArgs<dfloat>&, int, bool, int, cudaStream_t);

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
  op->plan32 = make_plan(L, max_tile_bits<float>(), 4);
  op->plan64 = make_plan(L, max_tile_bits<double>(), 3);
  return FLOQUET_OK;
}

static void destroy_graphs(floquet_op* op) {
  for (auto& g : op->graphs) cudaGraphExecDestroy(g.exec);
  op->graphs.clear();
}

void op_free(floquet_op* op) {
  destroy_graphs(op);
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
  cudaFree(op->coef);
}

template <typename Real> static int sweep_dtype();
template <> int sweep_dtype<float>() { return FLOQUET_C64; }
template <> int sweep_dtype<double>() { return FLOQUET_C128; }
template <> int sweep_dtype<dfloat>() { return FLOQUET_C128_DF; }

template <typename Real> static const Plan& plan_of(const floquet_op* op);
template <> const Plan& plan_of<float>(const floquet_op* op) { return op->plan32; }
template <> const Plan& plan_of<double>(const floquet_op* op) { return op->plan64; }
template <> const Plan& plan_of<dfloat>(const floquet_op* op) { return op->plan64; }
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
                    int64_t coef_stride, int jstep, const cplx<Real>* psi_in, cudaStream_t st) {
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
    }
    FQ_TRY(launch_pass<Real>(a, last ? epi : EPI_STORE, op->swap, nvec, st));
  }
  return FLOQUET_OK;
}

template <typename Real>
int apply_u(floquet_op* op, const cplx<Real>* in, cplx<Real>* out, int nvec, int vec_per_prob,
            cudaStream_t st) {
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
  FQ_TRY(ensure_workspace(op, (size_t)nvec * d * sizeof(C)));
  C* work = reinterpret_cast<C*>(op->work);
  C* acc = reinterpret_cast<C*>(op->acc);
  FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, work, acc, coef, k, d, nvec, st)));
  const int np = (int)plan_of<Real>(op).passes.size();
  auto body = [&](cudaStream_t s) -> int {
    for (int64_t j = 1; j < k; ++j)
      FQ_TRY(u_passes<Real>(op, work, work, nvec, vec_per_prob, EPI_PHASE_ACC, acc, coef, k,
                            (int)j, nullptr, s));
    return FLOQUET_OK;
  };
  if (k > 1)
    FQ_TRY(run_loop(op, use_graph, k, nvec, sweep_dtype<Real>(),
                    FLOQUET_FORM_ACC, coef, vec_per_prob, (k - 1) * np, st, body));
  return launch_convert_strided<Real, Rio>(acc, out, out_stride, d, nvec, st);
}

template <typename Real, typename Rio>
int filter_horner(floquet_op* op, const cplx<Rio>* in, int64_t in_stride, cplx<Rio>* out,
                  int64_t out_stride, const cplx<Real>* zs, int64_t k, int nvec,
                  int vec_per_prob, bool use_graph, cudaStream_t st) {
  using C = cplx<Real>;
  const int64_t d = op->d;
  FQ_TRY(ensure_workspace(op, (size_t)nvec * d * sizeof(C)));
  C* pin = reinterpret_cast<C*>(op->psi_in_copy);
  C* acc = reinterpret_cast<C*>(op->acc);
  FQ_TRY((launch_filter_init<Rio, Real>(in, in_stride, pin, acc, nullptr, 0, d, nvec, st)));
  const int np = (int)plan_of<Real>(op).passes.size();
  auto body = [&](cudaStream_t s) -> int {
    for (int64_t j = 1; j < k; ++j)
      FQ_TRY(u_passes<Real>(op, acc, acc, nvec, vec_per_prob, EPI_PHASE_HORNER, nullptr, zs, 1,
                            0, pin, s));
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
