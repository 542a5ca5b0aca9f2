// Instantiation of the general sweep and check for sigma = 9 .. 10 (any d up
// to kMaxD, full storage, f_mode 0).  The alphabet sizes are spread over
// several translation units so that they compile in parallel; kernels_rt.cu
// dispatches on sigma.
#include "sweep_rt.cuh"

namespace lcs {

const KernelSet* kernels_rt_s9_10(int sigma) {
  static const KernelSet k[] = {make_rt_set<9>(), make_rt_set<10>()};
  return sigma >= 9 && sigma <= 10 ? &k[sigma - 9] : nullptr;
}

bool rt_offsets_fill_s9_10(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s) {
  switch (sigma) {
    case 9:
      launch_rtb_offsets<9>(d, offs, start, s);
      return true;
    case 10:
      launch_rtb_offsets<10>(d, offs, start, s);
      return true;
    default:
      return false;
  }
}

}  // namespace lcs
