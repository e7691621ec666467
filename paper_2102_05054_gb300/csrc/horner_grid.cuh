// Persistent Horner filter: the whole k-step loop acc <- c_j psi_in + z U acc of
// g_k(U) psi_in (Sec. 3, Eq. geo, evaluated by Horner's rule) in ONE cooperative launch,
// with one grid-wide barrier per U application instead of one kernel launch per pass.
//
// Half-step scheme. The state is tiled two ways: layout A, tiles of the NB lowest qubits
// (contiguous 2^NB amplitudes), and layout B, tiles of the L - NB highest qubits plus the
// C lowest bits as contiguous columns (L = 2 NB - C). The kick layer factorises over the
// qubits, K = K_A K_B with commuting factors, and D is diagonal, so consecutive U
// applications can share a layout:
//     step 0        : t = K_A psi_in                                (layout A)
//     step j (odd)  : t = K_B t  -> acc_j = c_j psi_in + z D t;  t = K_B acc_j   (layout B)
//     step j (even) : t = K_A t  -> acc_j = c_j psi_in + z D t;  t = K_A acc_j   (layout A)
// and the last step stores acc_{k-1} itself. Every step reads the state once, psi_in once
// and writes the state once: 3 d b bytes per U application, the Horner form's algorithmic
// traffic. Between steps all CTAs meet at a grid barrier (the next layout needs amplitudes
// written by other CTAs); the launch is cooperative, so every CTA is resident and the
// barrier cannot wait on a CTA that has not started. Each wait is bounded: after
// kSpinLimit polls the CTA raises the error word, fills its tile with NaN and leaves, so a
// failure ends the kernel with a visible result instead of a hang.
//
// Inside a tile the qubits are kicked as in the pass kernels (pass_kernel.cuh): 2^RB
// amplitudes per thread in registers, register rounds separated by padded shared-memory
// transposes, the round structure fixed at compile time.
#pragma once

#include <vector>

#include "pass_pipe.cuh"

namespace fq {

template <typename Real> struct HornerGridArgs {
  const cplx<Real>* psi_in;  // nvec states of d amplitudes
  cplx<Real>* t;             // nvec states: working state, acc_{k-1} on return
  int64_t d;
  int L, nvec, vec_per_prob, a;
  scal<Real> tau;
  const cplx<Real>* tab_lo;  // per vector (z folded in), stride lo_stride
  const cplx<Real>* tab_hi;  // per problem, stride hi_stride
  int64_t lo_stride, hi_stride;
  const cplx<Real>* coef;    // GEN: c_j of vector v at coef[v * coef_stride + j], j = 1..k-1
  int64_t coef_stride;
  int64_t nsteps;            // k: step 0 plus k - 1 Horner updates
  const cplx<Real>* ptab;    // nullable: the full phase table z D_s per vector (stride d),
                             // replacing the product of the two chunk tables
  int psi_smem;              // psi_in of the CTA's two tiles kept in shared memory (one tile
                             // per CTA and layout: grid == tiles per layout)
  unsigned* bar;             // kBarWords words: [0] arrivals, [kBarErr] error (zero at launch)
};

// Polls of a grid-barrier wait before the CTA gives up (with the 64 ns back-off, well over
// a second; a step takes microseconds to a few milliseconds).
constexpr unsigned kSpinLimit = 1u << 25;

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Words of the barrier block (kBarWords unsigned): the arrival counter and the error word sit
// on separate 128-byte lines, so the polls of one do not queue behind the other.
constexpr int kBarWords = 64;
constexpr int kBarErr = 32;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier: returns false if this CTA timed out or another CTA raised the error.
// After the CTA-wide sync, thread 0 arrives with a release reduction (orders the CTA's
// writes before the count, without waiting for a reply), polls the counter with acquire loads
// and a growing back-off, and the CTA-wide sync passes the acquired view to every thread.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(bar), "r"(1u) : "memory");
    int ok = 1;
    unsigned spins = 0, ns = 16;
    while (ld_acquire_u32(bar) < target) {
      if (ld_relaxed_u32(bar + kBarErr) != 0u || ++spins > kSpinLimit) {
        ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns *= 2;
    }
    if (!ok) atomicExch(bar + kBarErr, 1u);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ float2 ld_state(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ld_state(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ld_state(const float4* p) { return __ldcg(p); }

template <typename C> __device__ __forceinline__ C nan_value() {
  C r;
  r.x = __int_as_float(0x7fc00000);
  r.y = r.x;
  return r;
}
template <> __device__ __forceinline__ float4 nan_value<float4>() {
  const float n = __int_as_float(0x7fc00000);
  return make_float4(n, n, n, n);
}
template <> __device__ __forceinline__ double2 nan_value<double2>() {
  const double n = __longlong_as_double(0x7ff8000000000000LL);
  return make_double2(n, n);
}

// Register-bit position of round i of a layout's kicks (round 0: the top RB tile bits;
// round i > 0 sits where the i-th transpose of the pass kernels puts it).
__host__ __device__ constexpr int round_g(int NB, int RB, int i) {
  return i == 0 ? NB - RB : pipe_g(NB, RB, i - 1);
}

// Moves the tile from register mapping g_from to g_to through padded shared memory.
template <typename Real, int RB>
__device__ __forceinline__ void transpose_tile(cplx<Real> (&v)[1 << RB], cplx<Real>* sm, int t,
                                               int g_from, int g_to) {
  constexpr int R = 1 << RB;
  __syncthreads();  // earlier reads of sm are done
  const int pw = pipe_pos_t<RB>(t, g_from);
#pragma unroll
  for (int r = 0; r < R; ++r) sm[pw + pipe_pos_r<RB>(r, g_from)] = v[r];
  __syncthreads();
  const int pr = pipe_pos_t<RB>(t, g_to);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = sm[pr + pipe_pos_r<RB>(r, g_to)];
}

// All kicks of one layout (tile bits [KF, NB)) in rounds of RB register bits. Forward: from
// the top mapping round_g(0) down to the last round's mapping; reverse (REV): from the last
// round's mapping back up to the top one. Either way NT transposes and the same butterflies
// (the single-qubit factors commute).
// NORM0: the values entering the first round are normalised double-floats (they come from the
// epilogue), so that round skips the renormalisation.
template <typename Real, int NB, int RB, int KF, bool SWAP, bool REV, bool NORM0 = false>
__device__ __forceinline__ void kick_rounds(cplx<Real> (&v)[1 << RB], cplx<Real>* sm, int t,
                                            scal<Real> tau) {
  constexpr int NT = pipe_transposes(NB, RB, KF);
#pragma unroll
  for (int j = 0; j <= NT; ++j) {
    const int i = REV ? NT - j : j;
    const int g = round_g(NB, RB, i);
    const int hi = i == 0 ? NB : round_g(NB, RB, i - 1);
    if (j > 0) transpose_tile<Real, RB>(v, sm, t, REV ? round_g(NB, RB, i + 1)
                                                      : round_g(NB, RB, i - 1), g);
    if (NORM0 && j == 0)
      kick_registers<Real, RB, SWAP, false>(v, g, KF, hi, tau);
    else
      kick_registers<Real, RB, SWAP, true>(v, g, KF, hi, tau);
  }
}

// Global index (within a vector) of tile element e: layout A, (cta << NB) + e; layout B,
// (cta << C) + (e & (2^C - 1)) + ((e >> C) << NB). The map is additive over disjoint bits.
template <int NB, int C, bool LAYB> __device__ __forceinline__ uint32_t tile_to_global(uint32_t e) {
  return LAYB ? ((e & ((1u << C) - 1u)) + ((e >> C) << NB)) : e;
}

// One half-step on one tile of layout LAYB (false: A, true: B). The state arrives and
// leaves in the top register mapping (coalesced: lane bits are the tile's lowest, contiguous
// bits); the epilogue runs in the last kick round's mapping, where psi_in and the phase
// tables are read, and the second kick runs the rounds in reverse.
// The state values of one tile in the top register mapping (psi_in on the first step).
template <typename Real, int NB, int RB, int C, bool LAYB>
__device__ __forceinline__ void load_tile_state(const HornerGridArgs<Real>& A, uint32_t tile,
                                                bool first, cplx<Real> (&v)[1 << RB]) {
  using Cx = cplx<Real>;
  constexpr int g_top = NB - RB;
  const int tilebits = A.L - NB;
  const int64_t vec = (int64_t)(tile >> tilebits);
  const uint32_t cta = tile & ((1u << tilebits) - 1u);
  const uint32_t tile0 = LAYB ? (cta << C) : (cta << NB);
  const Cx* __restrict__ src = (first ? A.psi_in : (const Cx*)A.t) + vec * A.d + tile0 +
                               tile_to_global<NB, C, LAYB>((uint32_t)threadIdx.x);
#pragma unroll
  for (int r = 0; r < (1 << RB); ++r)
    v[r] = ld_state(src + tile_to_global<NB, C, LAYB>((uint32_t)r << g_top));
}

template <typename Real, int NB, int RB, int C, bool SWAP, bool GEN, bool LAYB>
__device__ __forceinline__ void horner_tile(const HornerGridArgs<Real>& A, cplx<Real>* sm,
                                            const cplx<Real>* psm, uint32_t tile, int64_t step,
                                            bool first, bool last, cplx<Real> (&v)[1 << RB]) {
  using Cx = cplx<Real>;
  constexpr int R = 1 << RB;
  constexpr int g_top = NB - RB;
  constexpr int KF = LAYB ? C : 0;
  constexpr int NT = pipe_transposes(NB, RB, KF);
  constexpr int g_last = round_g(NB, RB, NT);
  static_assert(g_top >= C, "register bits must lie above the column bits");
  const int t = threadIdx.x;
  const int tilebits = A.L - NB;
  const int64_t vec = (int64_t)(tile >> tilebits);
  const uint32_t cta = tile & ((1u << tilebits) - 1u);
  const uint32_t tile0 = LAYB ? (cta << C) : (cta << NB);
  const uint32_t ut = (uint32_t)t;
  // top mapping: element t | (r << g_top)
  const uint32_t tb_top = tile0 + tile_to_global<NB, C, LAYB>(ut);
  uint32_t ro_top[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ro_top[r] = tile_to_global<NB, C, LAYB>((uint32_t)r << g_top);

  if (!first) {
    // last-round mapping: element (t & (2^g_last - 1)) | (r << g_last) | ((t >> g_last) << (g_last + RB))
    const uint32_t tpart = (ut & ((1u << g_last) - 1u)) | ((ut >> g_last) << (g_last + RB));
    const uint32_t tb = tile0 + tile_to_global<NB, C, LAYB>(tpart);
    kick_rounds<Real, NB, RB, KF, SWAP, false>(v, sm, t, A.tau);
    // epilogue in chunks of at most four registers (psi_in from shared memory when it is
    // resident there, else through the read-only path), so that the loads in flight stay few
    const Cx* __restrict__ pp = A.psi_in + vec * A.d + tb;
    const int pb = pipe_pos_t<RB>(t, g_last);
    const int64_t prob = vec / A.vec_per_prob;
    const Cx* __restrict__ tlo = A.tab_lo + vec * A.lo_stride;
    const Cx* __restrict__ thi = A.tab_hi + prob * A.hi_stride;
    const uint32_t lomask = (1u << A.a) - 1u;
    const int am1 = A.a - 1;
    Cx cj;
    if (GEN) cj = __ldg(&A.coef[vec * A.coef_stride + step]);
    constexpr int CH = R < 4 ? R : 4;
#pragma unroll
    for (int r0 = 0; r0 < R; r0 += CH) {
      Cx pin[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int r = r0 + c;
        pin[c] = (A.psi_smem && psm)
                     ? psm[pb + pipe_pos_r<RB>(r, g_last)]
                     : __ldg(pp + tile_to_global<NB, C, LAYB>((uint32_t)r << g_last));
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int r = r0 + c;
        const uint32_t s = tb + tile_to_global<NB, C, LAYB>((uint32_t)r << g_last);
        const Cx p = A.ptab ? __ldg(&A.ptab[vec * A.d + s])
                            : zmul(__ldg(&tlo[s & lomask]), __ldg(&thi[((s >> am1) << 1) | (s & 1u)]));
        const Cx base = GEN ? zmul(cj, pin[c]) : pin[c];
        v[r] = zfma(p, v[r], base);
      }
      if (r0 + CH < R) asm volatile("" ::: "memory");
    }
    if (last) {
      // acc_{k-1}: store from the last-round mapping
      Cx* __restrict__ dst = A.t + vec * A.d + tb;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[tile_to_global<NB, C, LAYB>((uint32_t)r << g_last)] = v[r];
      return;
    }
    kick_rounds<Real, NB, RB, KF, SWAP, true, true>(v, sm, t, A.tau);
  } else {
    kick_rounds<Real, NB, RB, KF, SWAP, false>(v, sm, t, A.tau);
    if (NT > 0) transpose_tile<Real, RB>(v, sm, t, g_last, g_top);
  }
  Cx* __restrict__ dst = A.t + vec * A.d + tb_top;
#pragma unroll
  for (int r = 0; r < R; ++r) dst[ro_top[r]] = v[r];
}

// psi_in of this CTA's tile of one layout into shared memory (padded like the transposes).
template <typename Real, int NB, int RB, int C, bool LAYB>
__device__ __forceinline__ void load_psi_tile(const HornerGridArgs<Real>& A, cplx<Real>* psm,
                                              uint32_t tile) {
  constexpr int R = 1 << RB;
  constexpr int g_top = NB - RB;
  const int tilebits = A.L - NB;
  const int64_t vec = (int64_t)(tile >> tilebits);
  const uint32_t cta = tile & ((1u << tilebits) - 1u);
  const uint32_t tile0 = LAYB ? (cta << C) : (cta << NB);
  const int t = threadIdx.x;
  const cplx<Real>* src = A.psi_in + vec * A.d + tile0 + tile_to_global<NB, C, LAYB>((uint32_t)t);
  const int pb = pipe_pos_t<RB>(t, g_top);
#pragma unroll
  for (int r = 0; r < R; ++r)
    psm[pb + pipe_pos_r<RB>(r, g_top)] =
        __ldg(src + tile_to_global<NB, C, LAYB>((uint32_t)r << g_top));
}

// One step over this CTA's tiles of one layout. MULTI: a CTA has several tiles per step (for
// complex64 the next tile's state is loaded into registers while the current one is processed).
template <typename Real, int NB, int RB, int C, bool SWAP, bool GEN, bool MULTI, bool LAYB>
__device__ __forceinline__ void grid_step(const HornerGridArgs<Real>& A, cplx<Real>* sm,
                                          const cplx<Real>* psm, int64_t step, bool first,
                                          bool last, uint32_t total) {
  constexpr int R = 1 << RB;
  uint32_t tile = blockIdx.x;
  if (tile >= total) return;
  cplx<Real> v[R];
  load_tile_state<Real, NB, RB, C, LAYB>(A, tile, first, v);
  // complex64 prefetches the next tile; the wider types need the registers for the sweep
  // (their tile takes long enough to cover the load)
  constexpr bool kPrefetch = sizeof(cplx<Real>) == 8;
  if (!MULTI || !kPrefetch) {
    for (;;) {
      horner_tile<Real, NB, RB, C, SWAP, GEN, LAYB>(A, sm, psm, tile, step, first, last, v);
      if (!MULTI) return;
      tile += gridDim.x;
      if (tile >= total) return;
      load_tile_state<Real, NB, RB, C, LAYB>(A, tile, first, v);
    }
  }
  for (;;) {
    const uint32_t next = tile + gridDim.x;
    const bool more = next < total;
    cplx<Real> nv[R];
    if (more) load_tile_state<Real, NB, RB, C, LAYB>(A, next, first, nv);
    horner_tile<Real, NB, RB, C, SWAP, GEN, LAYB>(A, sm, psm, tile, step, first, last, v);
    if (!more) break;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = nv[r];
    tile = next;
  }
}

template <typename Real, int NB, int RB, int C, bool SWAP, bool GEN, bool MULTI, int MINB>
__global__ void __launch_bounds__(1 << (NB - RB), MINB)
    horner_grid_kernel(const HornerGridArgs<Real> A) {
  using Cx = cplx<Real>;
  constexpr int SLOT = (1 << NB) + (1 << (NB - RB));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx* sm = reinterpret_cast<Cx*>(smem_raw);
  Cx* psmA = sm + SLOT;       // psi_in of the CTA's layout-A tile (psi_smem only)
  Cx* psmB = sm + 2 * SLOT;   // and of its layout-B tile
  const uint32_t total = (uint32_t)A.nvec << (A.L - NB);  // tiles per layout
  if (!MULTI && A.psi_smem) {
    load_psi_tile<Real, NB, RB, C, false>(A, psmA, blockIdx.x);
    load_psi_tile<Real, NB, RB, C, true>(A, psmB, blockIdx.x);
    __syncthreads();
  }
  for (int64_t step = 0; step < A.nsteps; ++step) {
    const bool first = step == 0, last = step + 1 == A.nsteps;
    const bool layb = (step & 1) != 0;
    if (layb)
      grid_step<Real, NB, RB, C, SWAP, GEN, MULTI, true>(A, sm, psmB, step, first, last, total);
    else
      grid_step<Real, NB, RB, C, SWAP, GEN, MULTI, false>(A, sm, psmA, step, first, last, total);
    if (last) break;
    if (!grid_barrier(A.bar, (unsigned)(step + 1) * gridDim.x)) {
      // timed out (or another CTA did): poison this CTA's tiles of the next layout and leave
      const bool nb = !layb;
      constexpr int R = 1 << RB;
      for (uint32_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int tilebits = A.L - NB;
        const int64_t vec = (int64_t)(tile >> tilebits);
        const uint32_t cta = tile & ((1u << tilebits) - 1u);
        const uint32_t ut = threadIdx.x;
        const uint32_t tbase = nb ? ((cta << C) + (ut & ((1u << C) - 1u)) + ((ut >> C) << NB))
                                  : ((cta << NB) + ut);
        for (int r = 0; r < R; ++r) {
          const uint32_t ro = nb ? ((((uint32_t)r << (NB - RB)) >> C) << NB)
                                 : ((uint32_t)r << (NB - RB));
          A.t[vec * A.d + tbase + ro] = nan_value<Cx>();
        }
      }
      return;
    }
  }
}

// Shapes of the persistent Horner kernel per sweep precision: tile bits NB, register bits RB
// and column bits C, so that L = 2 NB - C. Returns the instantiation's launcher or nullptr.
template <typename Real>
using HornerGridLaunch = int (*)(const HornerGridArgs<Real>&, bool swap, bool gen,
                                 cudaStream_t st);

// Resident CTAs (and the opt-in) of one kernel instantiation at `smem` bytes, cached per
// instantiation.
template <typename K> static int grid_resident(K kernel, int threads, size_t smem, int* cache,
                                               std::atomic<uint64_t>& opted) {
  if (*cache >= 0) return *cache;
  *cache = 0;
  if (smem > 227 * 1024) return 0;
  if (smem > 48 * 1024 && opt_in_smem(kernel, smem, opted) != FLOQUET_OK) {
    cudaGetLastError();
    return 0;
  }
  *cache = pipe_resident_ctas(kernel, threads, smem);
  return *cache;
}

template <typename Real, int NB, int RB, int C, bool SWAP, bool GEN>
static int launch_horner_grid_t(const HornerGridArgs<Real>& a, cudaStream_t st) {
  constexpr int threads = 1 << (NB - RB);
  constexpr size_t smem = (size_t)((1 << NB) + (1 << (NB - RB))) * sizeof(cplx<Real>);
  constexpr int fit = (int)((227 * 1024) / (smem + 1024));
  // Resident threads per SM the launch bounds ask for. One tile per CTA: 1024 for complex64
  // with up to eight amplitudes per thread and for any type with four (latency bound), 512
  // otherwise (the registers hold the tile). Several tiles per CTA (next tile prefetched into registers): 512.
  constexpr int want1 = ((sizeof(cplx<Real>) == 8 && RB <= 3) || RB <= 2 ? 1024 : 512) / threads;
  constexpr int wantm = 512 / threads;
  constexpr int minb1 = want1 < 1 ? 1 : (want1 < fit ? want1 : fit);
  constexpr int minbm = wantm < 1 ? 1 : (wantm < fit ? wantm : fit);
  auto k1 = horner_grid_kernel<Real, NB, RB, C, SWAP, GEN, false, minb1>;
  auto km = horner_grid_kernel<Real, NB, RB, C, SWAP, GEN, true, minbm>;
  static int res1 = -1, res1_psi = -1, resm = -1;
  static std::atomic<uint64_t> op1{0}, op1_psi{0}, opm{0};
  const int64_t total = (int64_t)a.nvec << (a.L - NB);
  if (total > 0x7fffffffLL) {
    set_error("horner_grid: too many tiles (nvec %d)", a.nvec);
    return FLOQUET_EINVAL;
  }
  HornerGridArgs<Real> args = a;
  args.psi_smem = 0;
  const void* kernel;
  unsigned grid;
  size_t shmem;
  // psi_in stays in shared memory when every CTA owns exactly one tile per layout and two
  // more tile buffers fit next to the transpose buffer
  const int r1p = grid_resident(k1, threads, 3 * smem, &res1_psi, op1_psi);
  const int r1 = grid_resident(k1, threads, smem, &res1, op1);
  if (total <= r1p) {
    args.psi_smem = 1;
    kernel = (const void*)k1;
    grid = (unsigned)total;
    shmem = 3 * smem;
  } else if (total <= r1) {
    kernel = (const void*)k1;
    grid = (unsigned)total;
    shmem = smem;
  } else {
    const int rm = grid_resident(km, threads, smem, &resm, opm);
    if (rm < 1) {
      set_error("horner_grid: occupancy query failed");
      return FLOQUET_ECUDA;
    }
    kernel = (const void*)km;
    grid = (unsigned)rm;
    shmem = smem;
  }
  if (grid < 1) {
    set_error("horner_grid: occupancy query failed");
    return FLOQUET_ECUDA;
  }
  void* params[] = {(void*)&args};
  FQ_CUDA(cudaMemsetAsync(a.bar, 0, kBarWords * sizeof(unsigned), st));
  FQ_CUDA(cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(threads), params, shmem, st));
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

template <typename Real, int NB, int RB, int C>
static int launch_horner_grid_shape(const HornerGridArgs<Real>& a, bool swap, bool gen,
                                    cudaStream_t st) {
  if (a.L != 2 * NB - C) {
    set_error("horner_grid: shape (NB %d, C %d) does not fit L = %d", NB, C, a.L);
    return FLOQUET_EINVAL;
  }
  if (gen) {  // per-step coefficients: not compiled into the launchers (no caller uses them)
    set_error("horner_grid: general Horner coefficients are not compiled in");
    return FLOQUET_EINVAL;
  }
  return swap ? launch_horner_grid_t<Real, NB, RB, C, true, false>(a, st)
              : launch_horner_grid_t<Real, NB, RB, C, false, false>(a, st);
}

// Launchers of the persistent Horner kernel for chains of L qubits in sweep precision Real,
// fastest-first by expectation (the autotuner times them all); none: the per-pass kernels.
template <typename Real> struct HornerGridShape {
  HornerGridLaunch<Real> launch;
  int NB, RB, C;
};
template <typename Real> std::vector<HornerGridShape<Real>> horner_grid_shapes(int L);

}  // namespace fq
