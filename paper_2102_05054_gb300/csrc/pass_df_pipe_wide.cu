// Pipelined pass kernels for double-float sweeps with 512 threads per tile: 2^12 tiles with
// eight amplitudes per thread (one CTA per SM) and 2^11 tiles with four (two CTAs per SM).
#include <algorithm>

#include "pass_pipe.cuh"

namespace fq {

template <int NB, int RB>
static bool pipe_df(const PassArgs<dfloat>& a, int epi, bool swap, int nvec, cudaStream_t st,
                    int* rc) {
  return pipe_launch_first<dfloat, NB, RB>(a, epi, swap, nvec, st, rc) ||
         pipe_launch_later<dfloat, NB, RB, 2>(a, epi, swap, nvec, st, rc) ||
         pipe_launch_later<dfloat, NB, RB, 3>(a, epi, swap, nvec, st, rc) ||
         pipe_launch_later<dfloat, NB, RB, 4>(a, epi, swap, nvec, st, rc);
}

bool launch_pass_pipe_df_wide(int NB, int RB, const PassArgs<dfloat>& a, int epi, bool swap,
                              int nvec, cudaStream_t st, int* rc) {
  if (a.NB != NB) return false;
  if (NB == 12 && RB == 3) return pipe_df<12, 3>(a, epi, swap, nvec, st, rc);
  if (NB == 11 && RB == 2) return pipe_df<11, 2>(a, epi, swap, nvec, st, rc);
  return false;
}

}  // namespace fq
