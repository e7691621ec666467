// Pipelined (persistent, cp.async double-buffered) pass kernels for double-float sweeps: the
// first pass and the later passes with 2, 3 or 4 column bits of the 2^11 and 2^10 tiles, which
// cover the two-pass plans of L = 16..20.
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

bool launch_pass_pipe_df(int NB, int RB, const PassArgs<dfloat>& a, int epi, bool swap,
                         int nvec, cudaStream_t st, int* rc) {
  if (a.NB != NB) return false;
  if (NB == 11 && RB == 3) return pipe_df<11, 3>(a, epi, swap, nvec, st, rc);
  if (NB == 10 && RB == 3) return pipe_df<10, 3>(a, epi, swap, nvec, st, rc);
  return false;
}

}  // namespace fq
