// Instantiation of the sigma = d = 2 sweep that uses both the complement and
// the swap symmetry.
#include "sweep_s2d2.cuh"

namespace lcs {

const KernelSet* kernels_s2d2() {
  static const KernelSet k = make_s2d2_set();
  return &k;
}

}  // namespace lcs
