// Pass-kernel instantiations for complex64 sweeps and their launch shapes.
#include "pass_kernel.cuh"

namespace fq {

// {tile bits, register bits}: large tiles for large states, smaller tiles so that mid-size
// states (L = 13..18) still give every SM a few CTAs per pass.
static const PassVariant kVariants[] = {{12, 4}, {12, 3}, {11, 4}, {10, 4}};

template <> int num_variants<float>() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }
template <> PassVariant variant_info<float>(int v) { return kVariants[v]; }

template <>
int launch_pass_variant<float>(int v, const PassArgs<float>& a, int epi, bool swap, int nvec,
                               cudaStream_t st) {
  if (a.NB == kVariants[v].NB) {
    switch (v) {
      case 0: return dispatch_epi<float, 12, 4, 2>(a, epi, swap, nvec, st);
      case 1: return dispatch_epi<float, 12, 3, 1>(a, epi, swap, nvec, st);
      case 2: return dispatch_epi<float, 11, 4, 2>(a, epi, swap, nvec, st);
      case 3: return dispatch_epi<float, 10, 4, 2>(a, epi, swap, nvec, st);
    }
  }
  if (a.NB >= 4) return dispatch_epi<float, 0, 4, 1>(a, epi, swap, nvec, st);
  return dispatch_epi<float, 0, 3, 1>(a, epi, swap, nvec, st);
}

}  // namespace fq
