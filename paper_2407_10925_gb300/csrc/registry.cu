// Lookup of the kernels compiled for an alphabet size, string count and
// storage mode.
#include "lcs_common.h"

namespace lcs {

const KernelSet* kernels_sigma2(int d, int sym, int f_mode);
const KernelSet* kernels_sigma3(int d, int f_mode);
const KernelSet* kernels_sigma45(int sigma, int d, int f_mode);
const KernelSet* kernels_s2d2();
const KernelSet* kernels_d2s(int sigma);
const KernelSet* kernels_d3s(int f_mode);

const KernelSet* find_kernels(int sigma, int d, int sym, int f_mode) {
  if (sym == 2) return (sigma == 2 && d == 2 && f_mode == 0) ? kernels_s2d2() : nullptr;
  if (sym == 3) return (sigma >= 3 && d == 2 && f_mode == 0) ? kernels_d2s(sigma) : nullptr;
  if (sym == 4) return (sigma == 2 && d == 3 && (f_mode == 0 || f_mode == 1)) ? kernels_d3s(f_mode) : nullptr;
  if (sigma == 2) return kernels_sigma2(d, sym, f_mode);
  if (sym) return nullptr;
  if (sigma == 3) return kernels_sigma3(d, f_mode);
  if (sigma == 4 || sigma == 5) return kernels_sigma45(sigma, d, f_mode);
  return nullptr;
}

}  // namespace lcs
