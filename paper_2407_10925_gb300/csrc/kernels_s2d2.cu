// Instantiation of the sigma = d = 2 sweep that uses both the complement and
// the swap symmetry, over 64-bit and over offset-normalised 32-bit storage.
#include "sweep_s2d2.cuh"

namespace lcs {

const KernelSet* kernels_s2d2() {
  static const KernelSet k = make_s2d2_set();
  return &k;
}

const KernelSet* kernels_s2d2_narrow() {
  static const KernelSet k = make_s2d2_narrow_set();
  return &k;
}

}  // namespace lcs
