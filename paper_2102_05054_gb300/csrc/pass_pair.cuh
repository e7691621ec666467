// Cluster-pair form of the pipelined pass kernel (pass_pipe.cuh): a tile of 2^(NBL+1)
// amplitudes is split between the two CTAs of a thread-block cluster, each holding the
// 2^NBL amplitudes whose top tile bit equals its cluster rank. The butterfly on that top bit
// pairs an amplitude with the one at the same local position in the partner CTA, read
// through distributed shared memory; every other kicked bit is local and runs exactly as in
// the pipelined kernel. With half-size CTAs a pass has twice as many work units (at L = 20:
// 1024 halves instead of 512 tiles on 152 SMs), so the last units of a pass are spread over
// more SMs, while a tile still covers NBL + 1 qubits (two passes per U at L = 20).
//
// Both CTAs of a cluster walk the same tiles (cluster index + i * clusters), so they meet at
// every cluster barrier the same number of times; the partner's buffer is read only between
// two cluster barriers, after which neither CTA touches the other's memory again.
#pragma once

#include <cooperative_groups.h>

#include "pass_pipe.cuh"

namespace fq {

template <typename Real, int NBL, int RB, int KF, int EPI, bool SWAP, int MINB>
__global__ void __launch_bounds__(1 << (NBL - RB), MINB)
    pass_pair_kernel(const PassArgs<Real> A, const uint32_t total_tiles) {
  namespace cg = cooperative_groups;
  using C = cplx<Real>;
  constexpr int R = 1 << RB;
  constexpr int E = 1 << NBL;
  constexpr int SLOT = E + (E >> RB);
  constexpr int g_top = NBL - RB;
  constexpr int NT = pipe_transposes(NBL, RB, KF);
  constexpr int g_last = NT > 0 ? pipe_g(NBL, RB, NT - 1) : g_top;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* const buf0 = reinterpret_cast<C*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t rank = cluster.block_rank();  // 0 or 1: the tile's top bit
  const uint32_t cid = blockIdx.x >> 1, nclusters = gridDim.x >> 1;

  const int t = threadIdx.x;
  // tiles are 2^(NBL+1) amplitudes (A.NB = NBL + 1); the global index of tile element e is
  // base(tile) + f(e), f(e) = (e & cmask) + ((e >> c) << start), linear over disjoint bits
  const int tilebits = A.L - (NBL + 1);
  const uint32_t tilemask = (1u << tilebits) - 1u;
  const uint32_t midmask = (1u << A.midbits) - 1u;
  const int c = A.c, start = A.start;
  const uint32_t cmask = (1u << c) - 1u;
  auto f = [&](uint32_t e) -> uint32_t { return (e & cmask) + ((e >> c) << start); };
  const uint32_t t_part = f((uint32_t)t) + f(rank << NBL);
  uint32_t roff[R];
#pragma unroll
  for (int r = 0; r < R; ++r) roff[r] = f((uint32_t)r << g_top);
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
    for (int r = 0; r < R; ++r)
      cp_async_elem(buf + p_top + pipe_pos_r<RB>(r, g_top), src + roff[r]);
  };

  uint32_t tile = cid;
  if (tile < total_tiles) prefetch(tile, buf0);
  cp_async_commit();
  for (int it = 0; tile < total_tiles; ++it, tile += nclusters) {
    C* const cur = buf0 + (it & 1) * SLOT;
    C* const nxt = buf0 + ((it & 1) ^ 1) * SLOT;
    __syncthreads();  // nxt (the previous tile's scratch) is no longer read in this CTA
    const uint32_t ntile = tile + nclusters;
    if (ntile < total_tiles) prefetch(ntile, nxt);
    cp_async_commit();
    cp_async_wait<1>();

    int64_t vec;
    const uint32_t tbase = tile_base(tile, vec);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cur[p_top + pipe_pos_r<RB>(r, g_top)];
    // the top tile bit: the partner holds the other amplitude of every pair at the same
    // local position of its buffer (both halves have landed once both CTAs arrive)
    cluster.sync();
    {
      const C* rem = cluster.map_shared_rank(cur, rank ^ 1u);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const C y = rem[p_top + pipe_pos_r<RB>(r, g_top)];
        C xn, yn;
        if (rank == 0) {
          bfly(v[r], y, A.tau, xn, yn);
          v[r] = SWAP ? yn : xn;
        } else {
          bfly(y, v[r], A.tau, xn, yn);
          v[r] = SWAP ? xn : yn;
        }
      }
    }
    cluster.sync();  // the partner has read this CTA's buffer before it is overwritten
    // the epilogue's other operand, loaded now so that its latency overlaps the kicks
    constexpr bool kOther = (EPI == EPI_PHASE_ACC || EPI == EPI_PHASE_HORNER);
    C pre[kOther ? R : 1];
    if constexpr (kOther) {
      const C* __restrict__ other =
          (EPI == EPI_PHASE_ACC ? (const C*)A.acc : A.psi_in) + vec * A.d + tbase;
#pragma unroll
      for (int r = 0; r < R; ++r) pre[r] = other[roff[r]];
    }

    kick_registers<Real, RB, SWAP>(v, g_top, KF, NBL, A.tau);
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int gp = i == 0 ? g_top : pipe_g(NBL, RB, i - 1);
      const int gn = pipe_g(NBL, RB, i);
      __syncthreads();
      const int pw = pipe_pos_t<RB>(t, gp);
#pragma unroll
      for (int r = 0; r < R; ++r) cur[pw + pipe_pos_r<RB>(r, gp)] = v[r];
      __syncthreads();
      const int pr = pipe_pos_t<RB>(t, gn);
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = cur[pr + pipe_pos_r<RB>(r, gn)];
      kick_registers<Real, RB, SWAP>(v, gn, KF, gp, A.tau);
    }
    if (g_last != g_top) {
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

template <typename Real, int NBL, int RB, int KF, int EPI, bool SWAP>
static int launch_pair_t(const PassArgs<Real>& a, int nvec, cudaStream_t st) {
  constexpr int threads = 1 << (NBL - RB);
  constexpr size_t smem = 2 * (size_t)((1 << NBL) + (1 << (NBL - RB))) * sizeof(cplx<Real>);
  auto kernel =
      pass_pair_kernel<Real, NBL, RB, KF, EPI, SWAP, pipe_min_blocks<EPI, threads, RB, smem>()>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  if (smem > 48 * 1024) {
    static std::atomic<uint64_t> opted{0};
    FQ_TRY(opt_in_smem(kernel, smem, opted));
  }

  const int64_t total = ((int64_t)1 << (a.L - (NBL + 1))) * nvec;
  if (total > 0x3fffffffLL) {
    set_error("launch_pass: grid too large (nvec %d)", nvec);
    return FLOQUET_EINVAL;
  }
  static int resident = 0;  // co-resident clusters, one value per instantiation
  if (resident < 1) {
    cfg.gridDim = dim3(2 * 152 * 8);
    if (cudaOccupancyMaxActiveClusters(&resident, kernel, &cfg) != cudaSuccess || resident < 1) {
      cudaGetLastError();
      set_error("launch_pass: cluster occupancy query failed for the paired pass kernel");
      resident = 0;
      return FLOQUET_ECUDA;
    }
  }
  cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(total, resident)));
  FQ_CUDA(cudaLaunchKernelEx(&cfg, kernel, a, (uint32_t)total));
  count_launch();
  FQ_CHECK_LAUNCH();
  return FLOQUET_OK;
}

// A pass of the paired shape (tile NBL + 1): the first pass or a later pass with KF column
// bits; false (nothing launched) for any other form.
template <typename Real, int NBL, int RB, int KF>
static bool pair_launch_later(const PassArgs<Real>& a, int epi, bool swap, int nvec,
                              cudaStream_t st, int* rc) {
  if (a.kick_from != KF || a.c != KF) return false;
  switch (epi * 2 + (swap ? 1 : 0)) {
    case 0: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_STORE, false>(a, nvec, st); return true;
    case 1: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_STORE, true>(a, nvec, st); return true;
    case 2: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_PHASE, false>(a, nvec, st); return true;
    case 3: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_PHASE, true>(a, nvec, st); return true;
    case 4: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_PHASE_ACC, false>(a, nvec, st); return true;
    case 5: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_PHASE_ACC, true>(a, nvec, st); return true;
    case 6: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_PHASE_HORNER, false>(a, nvec, st); return true;
    case 7: *rc = launch_pair_t<Real, NBL, RB, KF, EPI_PHASE_HORNER, true>(a, nvec, st); return true;
  }
  return false;
}

template <typename Real, int NBL, int RB>
static bool pair_launch_first(const PassArgs<Real>& a, int epi, bool swap, int nvec,
                              cudaStream_t st, int* rc) {
  if (a.kick_from != 0 || a.c != NBL + 1 || epi != EPI_STORE) return false;
  *rc = swap ? launch_pair_t<Real, NBL, RB, 0, EPI_STORE, true>(a, nvec, st)
             : launch_pair_t<Real, NBL, RB, 0, EPI_STORE, false>(a, nvec, st);
  return true;
}

}  // namespace fq
