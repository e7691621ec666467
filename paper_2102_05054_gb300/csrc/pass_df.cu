// Pass-kernel instantiations for double-float complex sweeps and their launch shapes.
#include "pass_kernel.cuh"

namespace fq {

// {tile bits, register bits}: large tiles for large states, smaller tiles so that mid-size
// states (L = 12..18) still give every SM a few CTAs per pass.
// Shapes 4 and 5 keep two column bits in later passes (64-byte row segments), so that L = 20
// (2^11 tiles) and L = 18 (2^10 tiles) take two passes, and run them with the pipelined kernel.
// Shapes 6 and 7 give each tile 512 threads (2^12 tiles with eight amplitudes per thread,
// 2^11 tiles with four).
// Shape 8 splits each 2^11 tile over a two-CTA cluster (2^10 amplitudes per CTA, six CTAs
// per SM), so that a pass has twice as many work units.
static const PassVariant kVariants[] = {{11, 3}, {12, 4}, {10, 3}, {9, 3},
                                        {11, 3, 2, true}, {10, 3, 2, true},
                                        {12, 3, 4, true}, {11, 2, 2, true},
                                        {11, 3, 2, true, true}};

// pass_df_pipe.cu, pass_df_pipe_wide.cu: launch the pipelined kernel if it is compiled for
// this pass
bool launch_pass_pipe_df(int NB, int RB, const PassArgs<dfloat>& a, int epi, bool swap,
                         int nvec, cudaStream_t st, int* rc);
bool launch_pass_pipe_df_wide(int NB, int RB, const PassArgs<dfloat>& a, int epi, bool swap,
                              int nvec, cudaStream_t st, int* rc);
// pass_df_pair.cu: the cluster-pair kernel, if it is compiled for this pass
bool launch_pass_pair_df(int NB, int RB, const PassArgs<dfloat>& a, int epi, bool swap,
                         int nvec, cudaStream_t st, int* rc);

template <> int num_variants<dfloat>() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }
template <> PassVariant variant_info<dfloat>(int v) { return kVariants[v]; }

template <>
int launch_pass_variant<dfloat>(int v, const PassArgs<dfloat>& a, int epi, bool swap, int nvec,
                               cudaStream_t st) {
  // the shape's own tile uses its compile-time kernel (the pipelined one where compiled); a
  // smaller single-pass tile (L below the shape's tile bits) uses the generic one
  if (a.NB == kVariants[v].NB) {
    int rc = FLOQUET_OK;
    const PassVariant& pv = kVariants[v];
    if (pv.pair && launch_pass_pair_df(pv.NB, pv.RB, a, epi, swap, nvec, st, &rc)) return rc;
    if (pv.pipe && !pv.pair &&
        (launch_pass_pipe_df(pv.NB, pv.RB, a, epi, swap, nvec, st, &rc) ||
                    launch_pass_pipe_df_wide(pv.NB, pv.RB, a, epi, swap, nvec, st, &rc)))
      return rc;
    switch (v) {
      case 0: case 4: case 7: case 8: return dispatch_epi<dfloat, 11, 3, 3>(a, epi, swap, nvec, st);
      case 1: return dispatch_epi<dfloat, 12, 4, 2>(a, epi, swap, nvec, st);
      case 2: case 5: return dispatch_epi<dfloat, 10, 3, 3>(a, epi, swap, nvec, st);
      case 3: return dispatch_epi<dfloat, 9, 3, 3>(a, epi, swap, nvec, st);
      case 6: return dispatch_epi<dfloat, 12, 4, 2>(a, epi, swap, nvec, st);
    }
  }
  return dispatch_epi<dfloat, 0, 3, 1>(a, epi, swap, nvec, st);
}

}  // namespace fq
