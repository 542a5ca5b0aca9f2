// Instantiations of the generic sweep for the binary alphabet (sigma = 2),
// with and without complement-symmetric storage.
#include "sweep_generic.cuh"

namespace lcs {

const KernelSet* kernels_sigma2(int d, int sym, int f_mode) {
  static const KernelSet sets[] = {
      make_generic_set<2, 2, false>(),       make_generic_set<2, 2, true>(),       make_generic_set<2, 3, false>(),
      make_generic_set<2, 3, true>(),        make_generic_set<2, 4, false>(),      make_generic_set<2, 4, true>(),
      make_generic_set<2, 5, false>(),       make_generic_set<2, 5, true>(),
      // every non-empty advance set (f_mode = 1)
      make_generic_set<2, 2, false, true>(), make_generic_set<2, 2, true, true>(), make_generic_set<2, 3, false, true>(),
      make_generic_set<2, 3, true, true>(),
  };
  for (const auto& k : sets)
    if (k.d == d && k.sym == sym && k.f_mode == f_mode) return &k;
  return nullptr;
}

}  // namespace lcs
