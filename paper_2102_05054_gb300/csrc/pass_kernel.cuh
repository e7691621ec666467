// The U-application pass kernel (see uapply.cu for the method), shared by the per-precision
// translation units pass_f32.cu, pass_f64.cu and pass_df.cu.
#pragma once

#include <atomic>
#include <type_traits>

#include "floquet_internal.cuh"

namespace fq {

// The shared-memory opt-in above 48 KiB (cudaFuncSetAttribute) holds per device: remember,
// for one kernel instantiation, the devices on which it has been set (bit i = device i). The
// first launch on a device sets it, outside any stream capture (the autotuner launches every
// shape before a filter graph is captured).
template <typename K>
static int opt_in_smem(K kernel, size_t smem, std::atomic<uint64_t>& done) {
  int dev = 0;
  FQ_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load() & bit)) return FLOQUET_OK;
  FQ_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  done.fetch_or(bit);
  return FLOQUET_OK;
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
// x + t * y without the final renormalisation: the pair (hi, lo) is exact to ~2^-48 but lo
// may exceed half an ulp of hi; kick_registers renormalises once per register round.
__device__ __forceinline__ float2 df_fma_lazy(float2 t, float2 y, float2 x) {
  const float p = __fmul_rn(t.x, y.x);
  const float pe = __fmaf_rn(t.x, y.x, -p);
  const float2 s = df_two_sum(x.x, p);
  const float lo = __fadd_rn(__fadd_rn(s.y, pe), __fmaf_rn(t.x, y.y, __fmaf_rn(t.y, y.x, x.y)));
  return make_float2(s.x, lo);
}
__device__ __forceinline__ float4 df_renorm(float4 a) {
  const float2 r = df_quick_two_sum(a.x, a.y), i = df_quick_two_sum(a.z, a.w);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ void bfly(float4 x, float4 y, float2 tau, float4& xn, float4& yn) {
  // re(x') = re x + tau im y, im(x') = im x - tau re y
  const float2 nt = df_neg(tau);
  const float2 a = df_fma_lazy(tau, make_float2(y.z, y.w), make_float2(x.x, x.y));
  const float2 b = df_fma_lazy(nt, make_float2(y.x, y.y), make_float2(x.z, x.w));
  const float2 c = df_fma_lazy(tau, make_float2(x.z, x.w), make_float2(y.x, y.y));
  const float2 d = df_fma_lazy(nt, make_float2(x.x, x.y), make_float2(y.z, y.w));
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

// ------------------------------------------------------------------ last-pass epilogue

// Stores the R amplitudes v[r] that a thread holds at global indices tbase + roff[r] of
// vector vec: unchanged (EPI_STORE), or times the diagonal phase D_s (the product of the two
// table entries), followed by the accumulate update acc += coef_j D v or the Horner update
// dst = psi_in + (z D) v. other(r, s) returns the accumulator or psi_in value of register r.
template <typename Real, int R, int EPI, typename Other>
__device__ __forceinline__ void pass_epilogue(const PassArgs<Real>& A, int64_t vec,
                                              uint32_t tbase, const uint32_t (&roff)[R],
                                              const cplx<Real> (&v)[R], Other other) {
  using C = cplx<Real>;
  C* __restrict__ dst = A.dst + vec * A.d + tbase;
  if (EPI == EPI_STORE) {
#pragma unroll
    for (int r = 0; r < R; ++r) dst[roff[r]] = v[r];
    return;
  }
  const int64_t prob = vec / A.vec_per_prob;
  const C* __restrict__ tlo = A.tab_lo + (A.lo_by_vec ? vec : prob) * A.tab_lo_stride;
  const C* __restrict__ thi = A.tab_hi + prob * A.tab_hi_stride;
  const uint32_t lomask = (1u << A.a) - 1u;
  const int am1 = A.a - 1;
  C cj;
  if (EPI == EPI_PHASE_ACC) cj = A.coef[vec * A.coef_stride + A.jstep];
  const bool gen = EPI == EPI_PHASE_HORNER && A.hcoef != nullptr;
  C hc;
  if (gen) hc = A.hcoef[vec * A.hcoef_stride + A.jstep];
  C* __restrict__ acc = A.acc + vec * A.d + tbase;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t s = tbase + roff[r];
    const C p = zmul(__ldg(&tlo[s & lomask]), __ldg(&thi[((s >> am1) << 1) | (s & 1u)]));
    if (EPI == EPI_PHASE) {
      dst[roff[r]] = zmul(p, v[r]);
    } else if (EPI == EPI_PHASE_ACC) {
      const C val = zmul(p, v[r]);
      dst[roff[r]] = val;
      acc[roff[r]] = zfma(cj, val, other(r, s));
    } else {  // Horner: dst (= acc) = c_j psi_in + z U acc, z folded into the table
      const C o = other(r, s);
      dst[roff[r]] = zfma(p, v[r], gen ? zmul(hc, o) : o);
    }
  }
}

// ------------------------------------------------------------------ pass kernel

// Tile element e -> position in padded shared memory (one pad slot every 2^RB elements
// keeps the strided transposes free of bank conflicts).
template <int RB> __device__ __forceinline__ int smem_pos(int e) { return e + (e >> RB); }

// Element index of register r of thread t when the register bits are tile bits [g, g+RB).
template <int RB> __device__ __forceinline__ int tile_elem(int t, int r, int g) {
  return (t & ((1 << g) - 1)) | (r << g) | ((t >> g) << (g + RB));
}

template <typename Real, int RB, bool SWAP, bool RENORM = true>
__device__ __forceinline__ void kick_registers(cplx<Real> (&v)[1 << RB], int g, int lo, int hi,
                                               scal<Real> tau) {
  if constexpr (std::is_same<Real, dfloat>::value && RENORM) {
    // renormalise the double-float pairs left unnormalised by the previous round
#pragma unroll
    for (int r = 0; r < (1 << RB); ++r) v[r] = df_renorm(v[r]);
  }
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
template <int NBT, int RB> constexpr int pass_max_threads() {
  return NBT > 0 ? (1 << (NBT > RB ? NBT - RB : 0)) : 256;
}

template <typename Real, int NBT, int RB, int EPI, bool SWAP, int MINB>
__global__ void __launch_bounds__(pass_max_threads<NBT, RB>(), MINB)
    pass_kernel(const PassArgs<Real> A) {
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

  pass_epilogue<Real, R, EPI>(A, vec, tbase, roff, v, [&](int r, uint32_t s) -> C {
    if constexpr (kPrefetch) return pre[r];
    return other[s];
  });
}

template <typename Real, int NBT, int RB, int EPI, bool SWAP, int MINB>
static int launch_pass_t(const PassArgs<Real>& a, int nvec, cudaStream_t st) {
  const int threads = 1 << (a.NB - RB);
  const size_t smem = (size_t)((1 << a.NB) + (1 << (a.NB - RB))) * sizeof(cplx<Real>);
  if (smem > 48 * 1024) {
    // tiles above 48 KiB (2^12 complex128 / double-float) need the opt-in carve-out
    static std::atomic<uint64_t> opted{0};
    FQ_TRY(opt_in_smem(pass_kernel<Real, NBT, RB, EPI, SWAP, MINB>, smem, opted));
  }
  const int64_t ntiles = (int64_t)1 << (a.L - a.NB);
  if (ntiles * nvec > 0x7fffffffLL) {
    set_error("launch_pass: grid too large (nvec %d, tiles %lld)", nvec, (long long)ntiles);
    return FLOQUET_EINVAL;
  }
  pass_kernel<Real, NBT, RB, EPI, SWAP, MINB><<<dim3((unsigned)(ntiles * nvec)), threads, smem,
                                                st>>>(a);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

template <typename Real, int NBT, int RB, int MINB>
static int dispatch_epi(const PassArgs<Real>& a, int epi, bool swap, int nvec, cudaStream_t st) {
  switch (epi * 2 + (swap ? 1 : 0)) {
    case 0: return launch_pass_t<Real, NBT, RB, EPI_STORE, false, MINB>(a, nvec, st);
    case 1: return launch_pass_t<Real, NBT, RB, EPI_STORE, true, MINB>(a, nvec, st);
    case 2: return launch_pass_t<Real, NBT, RB, EPI_PHASE, false, MINB>(a, nvec, st);
    case 3: return launch_pass_t<Real, NBT, RB, EPI_PHASE, true, MINB>(a, nvec, st);
    case 4: return launch_pass_t<Real, NBT, RB, EPI_PHASE_ACC, false, MINB>(a, nvec, st);
    case 5: return launch_pass_t<Real, NBT, RB, EPI_PHASE_ACC, true, MINB>(a, nvec, st);
    case 6: return launch_pass_t<Real, NBT, RB, EPI_PHASE_HORNER, false, MINB>(a, nvec, st);
    case 7: return launch_pass_t<Real, NBT, RB, EPI_PHASE_HORNER, true, MINB>(a, nvec, st);
  }
  set_error("launch_pass: bad epilogue %d", epi);
  return FLOQUET_EINVAL;
}

}  // namespace fq
