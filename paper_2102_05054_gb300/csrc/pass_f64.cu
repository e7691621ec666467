// Pass-kernel instantiations for complex128 sweeps and their launch shapes.
#include "pass_kernel.cuh"

namespace fq {

// {tile bits, register bits}: large tiles for large states, smaller tiles so that mid-size
// states (L = 12..18) still give every SM a few CTAs per pass.
static const PassVariant kVariants[] = {{11, 3}, {12, 4}, {10, 3}, {9, 3}};

template <> int num_variants<double>() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }
template <> PassVariant variant_info<double>(int v) { return kVariants[v]; }

template <>
int launch_pass_variant<double>(int v, const PassArgs<double>& a, int epi, bool swap, int nvec,
                               cudaStream_t st) {
  if (a.NB == 11) return dispatch_epi<double, 11, 3, 3>(a, epi, swap, nvec, st);
  if (a.NB == 12) return dispatch_epi<double, 12, 4, 2>(a, epi, swap, nvec, st);
  if (a.NB == 10) return dispatch_epi<double, 10, 3, 3>(a, epi, swap, nvec, st);
  if (a.NB == 9) return dispatch_epi<double, 9, 3, 3>(a, epi, swap, nvec, st);
  return dispatch_epi<double, 0, 3, 1>(a, epi, swap, nvec, st);
}

}  // namespace fq
