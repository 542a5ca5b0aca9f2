// Instantiations of the generic sweep for sigma = 4 and 5 (d = 2).
#include "sweep_generic.cuh"

namespace lcs {

const KernelSet* kernels_sigma45(int sigma, int d, int f_mode) {
  if (f_mode != 0) return nullptr;
  static const KernelSet sets[] = {make_generic_set<4, 2, false>(), make_generic_set<5, 2, false>()};
  for (const auto& k : sets)
    if (k.sigma == sigma && k.d == d) return &k;
  return nullptr;
}

}  // namespace lcs
