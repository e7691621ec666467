// Persistent, software-pipelined form of the U-application pass kernel (pass_kernel.cuh has
// the method). Differences from the one-tile-per-CTA kernel:
//
//  * The grid holds as many CTAs as fit on the GPU at once; each CTA walks the tiles
//    blockIdx.x, blockIdx.x + gridDim.x, ... so no CTA waits for a launch wave.
//  * While a tile is being kicked, the amplitudes of the CTA's next tile are already on their
//    way into a second shared-memory buffer (cp.async, one 8- or 16-byte copy per amplitude
//    issued by the thread that will own it in the first register round), so the L2 latency
//    of the loads is hidden behind the arithmetic. The buffer a tile arrived in then serves
//    as that tile's transpose scratch.
//  * The pass's kicked bit range [KF, NB) is a template parameter, so the register rounds
//    unroll completely and every shared-memory offset is a per-thread base plus a constant.
//
// A tile is still one set of 2^NB amplitudes of one pass (tiles of a pass are disjoint), so
// in-place passes (src == dst) stay correct: a tile's elements are read before any of them is
// written, and no other tile touches them.
#pragma once

#include "pass_kernel.cuh"

namespace fq {

__device__ __forceinline__ void cp_async_elem(float2* smem, const float2* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* smem, const double2* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(float4* smem, const float4* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait until at most N of this thread's committed copy groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Number of shared-memory transposes of a pass that kicks tile bits [KF, NB) in rounds of RB
// bits from the top down (the first round needs none).
__host__ __device__ constexpr int pipe_transposes(int NB, int RB, int KF) {
  int hi = NB - RB, n = 0;
  while (hi > KF) {
    hi = hi - RB > 0 ? hi - RB : 0;
    ++n;
  }
  return n;
}
// register-bit position after transpose i (the first round, before any transpose, has its
// register bits at NB - RB)
__host__ __device__ constexpr int pipe_g(int NB, int RB, int i) {
  return NB - RB * (i + 2) > 0 ? NB - RB * (i + 2) : 0;
}

// Padded shared-memory position of tile element tile_elem(t, r, g), split into a per-thread
// part and a per-register constant: the two parts of the element index have disjoint bits, so
// e + (e >> RB) separates into the same expression on each part.
template <int RB> __device__ __forceinline__ int pipe_pos_t(int t, int g) {
  const int base = (t & ((1 << g) - 1)) | ((t >> g) << (g + RB));
  return base + (base >> RB);
}
template <int RB> __host__ __device__ constexpr int pipe_pos_r(int r, int g) {
  return (r << g) + ((r << g) >> RB);
}

template <typename Real, int NB, int RB, int KF, int EPI, bool SWAP, int MINB>
__global__ void __launch_bounds__(1 << (NB - RB), MINB)
    pass_pipe_kernel(const PassArgs<Real> A, const uint32_t total_tiles) {
  using C = cplx<Real>;
  constexpr int R = 1 << RB;
  constexpr int E = 1 << NB;
  constexpr int SLOT = E + (E >> RB);
  constexpr int g_top = NB - RB;
  constexpr int NT = pipe_transposes(NB, RB, KF);
  constexpr int g_last = NT > 0 ? pipe_g(NB, RB, NT - 1) : g_top;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const buf0 = reinterpret_cast<C*>(smem_raw);

  const int t = threadIdx.x;
  const int tilebits = A.L - NB;
  const uint32_t tilemask = (1u << tilebits) - 1u;
  const uint32_t midmask = (1u << A.midbits) - 1u;
  const int c = A.c, start = A.start;
  const uint32_t cmask = (1u << c) - 1u;
  const uint32_t tb = (uint32_t)t;
  const uint32_t t_part = (tb & cmask) + ((tb >> c) << start);
  uint32_t roff[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t er = (uint32_t)r << g_top;
    roff[r] = (er & cmask) + ((er >> c) << start);
  }
  // round-0 positions of this thread's registers (its own cp.async destinations)
  const int p_top = pipe_pos_t<RB>(t, g_top);

  auto tile_base = [&](uint32_t tile, int64_t& vec) -> uint32_t {
    vec = (int64_t)(tile >> tilebits);
    const uint32_t cta = tile & tilemask;
    return (((cta & midmask) << c) | ((cta >> A.midbits) << A.topshift)) + t_part;
  };
  auto prefetch = [&](uint32_t tile, C* buf) {
    int64_t vec;
    const uint32_t tbase = tile_base(tile, vec);
    const C* src = A.src + vec * A.d + tbase;
#pragma unroll
    for (int r = 0; r < R; ++r) cp_async_elem(buf + p_top + pipe_pos_r<RB>(r, g_top), src + roff[r]);
  };

  uint32_t tile = blockIdx.x;
  if (tile < total_tiles) prefetch(tile, buf0);
  cp_async_commit();
  for (int it = 0; tile < total_tiles; ++it, tile += gridDim.x) {
    C* const cur = buf0 + (it & 1) * SLOT;
    C* const nxt = buf0 + ((it & 1) ^ 1) * SLOT;
    // every thread has finished with nxt (the previous tile's transpose scratch)
    __syncthreads();
    const uint32_t ntile = tile + gridDim.x;
    if (ntile < total_tiles) prefetch(ntile, nxt);
    cp_async_commit();
    cp_async_wait<1>();  // this tile's copies (all but the group just committed) have landed

    int64_t vec;
    const uint32_t tbase = tile_base(tile, vec);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cur[p_top + pipe_pos_r<RB>(r, g_top)];
    // the epilogue's other operand (accumulator or Horner's psi_in) is loaded now so that its
    // latency overlaps the kicks
    constexpr bool kOther = (EPI == EPI_PHASE_ACC || EPI == EPI_PHASE_HORNER);
    C pre[kOther ? R : 1];
    if constexpr (kOther) {
      const C* __restrict__ other =
          (EPI == EPI_PHASE_ACC ? (const C*)A.acc : A.psi_in) + vec * A.d + tbase;
#pragma unroll
      for (int r = 0; r < R; ++r) pre[r] = other[roff[r]];
    }

    kick_registers<Real, RB, SWAP>(v, g_top, KF, NB, A.tau);
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int gp = i == 0 ? g_top : pipe_g(NB, RB, i - 1);
      const int gn = pipe_g(NB, RB, i);
      __syncthreads();  // all reads of the buffer (round-0 loads or the last transpose) done
      const int pw = pipe_pos_t<RB>(t, gp);
#pragma unroll
      for (int r = 0; r < R; ++r) cur[pw + pipe_pos_r<RB>(r, gp)] = v[r];
      __syncthreads();
      const int pr = pipe_pos_t<RB>(t, gn);
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = cur[pr + pipe_pos_r<RB>(r, gn)];
      kick_registers<Real, RB, SWAP>(v, gn, KF, gp, A.tau);
    }
    if (g_last != g_top) {  // back to the coalesced mapping
      __syncthreads();
      const int pw = pipe_pos_t<RB>(t, g_last);
#pragma unroll
      for (int r = 0; r < R; ++r) cur[pw + pipe_pos_r<RB>(r, g_last)] = v[r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = cur[p_top + pipe_pos_r<RB>(r, g_top)];
    }

    pass_epilogue<Real, R, EPI>(A, vec, tbase, roff, v,
                                [&](int r, uint32_t) -> C { return pre[kOther ? r : 0]; });
  }
  cp_async_wait<0>();
}

// CTAs of one pipelined kernel that fit on the device at once (the caller caches it per
// kernel instantiation).
template <typename K> static int pipe_resident_ctas(K kernel, int threads, size_t smem) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return nsm * per_sm;
}

// Resident CTAs per SM the launch bounds ask for: 768 threads per SM for the plain passes,
// 512 when the epilogue keeps a second register copy of the tile (accumulator or psi_in),
// 1024 for four amplitudes per thread; never more than the shared memory holds.
template <int EPI, int THREADS, int RB, size_t SMEM> constexpr int pipe_min_blocks() {
  constexpr int want = (RB <= 2 ? 1024
                        : (EPI == EPI_PHASE_ACC || EPI == EPI_PHASE_HORNER) ? 512 : 768) /
                       THREADS;
  constexpr int fit = (int)((227 * 1024) / (SMEM + 1024));
  return want < 1 ? 1 : (want < fit ? want : (fit < 1 ? 1 : fit));
}

template <typename Real, int NB, int RB, int KF, int EPI, bool SWAP>
static int launch_pipe_t(const PassArgs<Real>& a, int nvec, cudaStream_t st) {
  constexpr int threads = 1 << (NB - RB);
  constexpr size_t smem = 2 * (size_t)((1 << NB) + (1 << (NB - RB))) * sizeof(cplx<Real>);
  auto kernel = pass_pipe_kernel<Real, NB, RB, KF, EPI, SWAP, pipe_min_blocks<EPI, threads, RB, smem>()>;
  if (smem > 48 * 1024) {
    static std::atomic<uint64_t> opted{0};
    FQ_TRY(opt_in_smem(kernel, smem, opted));
  }

  const int64_t total = ((int64_t)1 << (a.L - NB)) * nvec;
  if (total > 0x7fffffffLL) {
    set_error("launch_pass: grid too large (nvec %d)", nvec);
    return FLOQUET_EINVAL;
  }
  static int resident = 0;  // one value per instantiation
  if (resident < 1) resident = pipe_resident_ctas(kernel, threads, smem);
  if (resident < 1) {
    set_error("launch_pass: occupancy query failed for the pipelined pass kernel");
    return FLOQUET_ECUDA;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(total, resident);
  kernel<<<grid, threads, smem, st>>>(a, (uint32_t)total);
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// Launch a pass of a pipelined shape: the first pass (kick_from = 0, store epilogue) or a
// later pass whose column bits equal KF. Returns false (nothing launched) for any other form,
// which the caller then runs with the one-tile-per-CTA kernel.
template <typename Real, int NB, int RB, int KF>
static bool pipe_launch_later(const PassArgs<Real>& a, int epi, bool swap, int nvec,
                              cudaStream_t st, int* rc) {
  if (a.kick_from != KF || a.c != KF) return false;
  switch (epi * 2 + (swap ? 1 : 0)) {
    case 0: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_STORE, false>(a, nvec, st); return true;
    case 1: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_STORE, true>(a, nvec, st); return true;
    case 2: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_PHASE, false>(a, nvec, st); return true;
    case 3: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_PHASE, true>(a, nvec, st); return true;
    case 4: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_PHASE_ACC, false>(a, nvec, st); return true;
    case 5: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_PHASE_ACC, true>(a, nvec, st); return true;
    case 6: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_PHASE_HORNER, false>(a, nvec, st); return true;
    case 7: *rc = launch_pipe_t<Real, NB, RB, KF, EPI_PHASE_HORNER, true>(a, nvec, st); return true;
  }
  return false;
}

template <typename Real, int NB, int RB>
static bool pipe_launch_first(const PassArgs<Real>& a, int epi, bool swap, int nvec,
                              cudaStream_t st, int* rc) {
  if (a.kick_from != 0 || a.c != NB || epi != EPI_STORE) return false;
  *rc = swap ? launch_pipe_t<Real, NB, RB, 0, EPI_STORE, true>(a, nvec, st)
             : launch_pipe_t<Real, NB, RB, 0, EPI_STORE, false>(a, nvec, st);
  return true;
}

}  // namespace fq
