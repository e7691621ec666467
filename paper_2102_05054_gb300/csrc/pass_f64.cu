// Pass-kernel instantiations for complex128 sweeps and their launch shapes.
#include "pass_kernel.cuh"

namespace fq {

// {tile bits, register bits}: large tiles for large states, smaller tiles so that mid-size
// states (L = 12..18) still give every SM a few CTAs per pass.
static const PassVariant kVariants[] = {{11, 3}, {12, 4}, {10, 3}, {9, 3}, {11, 3}};

template <> int num_variants<double>() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }
template <> PassVariant variant_info<double>(int v) { return kVariants[v]; }

template <>
int launch_pass_variant<double>(int v, const PassArgs<double>& a, int epi, bool swap, int nvec,
                               cudaStream_t st) {
  // the shape's own tile uses its compile-time kernel; a smaller single-pass tile (L below
  // the shape's tile bits) uses the generic one. Shape 4 is shape 0 limited to 64 registers
  // (four CTAs per SM: 512 tiles of an L = 20 pass then fit one wave).
  if (a.NB == kVariants[v].NB) {
    switch (v) {
      case 0: return dispatch_epi<double, 11, 3, 3>(a, epi, swap, nvec, st);
      case 1: return dispatch_epi<double, 12, 4, 2>(a, epi, swap, nvec, st);
      case 2: return dispatch_epi<double, 10, 3, 3>(a, epi, swap, nvec, st);
      case 3: return dispatch_epi<double, 9, 3, 3>(a, epi, swap, nvec, st);
      case 4: return dispatch_epi<double, 11, 3, 4>(a, epi, swap, nvec, st);
    }
  }
  return dispatch_epi<double, 0, 3, 1>(a, epi, swap, nvec, st);
}

}  // namespace fq
