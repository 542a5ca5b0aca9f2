// Instantiations of the generic sweep for sigma = 3.
#include "sweep_generic.cuh"

namespace lcs {

const KernelSet* kernels_sigma3(int d, int f_mode) {
  static const KernelSet sets[] = {make_generic_set<3, 2, false>(), make_generic_set<3, 3, false>(),
                                   make_generic_set<3, 2, false, true>()};
  for (const auto& k : sets)
    if (k.d == d && k.f_mode == f_mode) return &k;
  return nullptr;
}

}  // namespace lcs
