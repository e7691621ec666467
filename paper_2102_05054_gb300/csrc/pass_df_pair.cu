// Cluster-pair pass kernels for double-float sweeps: 2^11 tiles split over two CTAs of
// 2^10 amplitudes (the first pass and later passes with 2, 3 or 4 column bits: L = 18..20
// in two passes).
#include <algorithm>

#include "pass_pair.cuh"

namespace fq {

bool launch_pass_pair_df(int NB, int RB, const PassArgs<dfloat>& a, int epi, bool swap,
                         int nvec, cudaStream_t st, int* rc) {
  if (a.NB != NB || NB != 11 || RB != 3) return false;
  return pair_launch_first<dfloat, 10, 3>(a, epi, swap, nvec, st, rc) ||
         pair_launch_later<dfloat, 10, 3, 2>(a, epi, swap, nvec, st, rc) ||
         pair_launch_later<dfloat, 10, 3, 3>(a, epi, swap, nvec, st, rc) ||
         pair_launch_later<dfloat, 10, 3, 4>(a, epi, swap, nvec, st, rc);
}

}  // namespace fq
