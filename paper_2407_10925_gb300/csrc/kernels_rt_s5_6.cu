// Instantiation of the general sweep and check for sigma = 5 .. 6 (any d up
// to kMaxD, full storage, f_mode 0).  The alphabet sizes are spread over
// several translation units so that they compile in parallel; kernels_rt.cu
// dispatches on sigma.
#include "sweep_rt.cuh"

namespace lcs {

const KernelSet* kernels_rt_s5_6(int sigma) {
  static const KernelSet k[] = {make_rt_set<5>(), make_rt_set<6>()};
  return sigma >= 5 && sigma <= 6 ? &k[sigma - 5] : nullptr;
}

bool rt_offsets_fill_s5_6(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s) {
  switch (sigma) {
    case 5:
      launch_rtb_offsets<5>(d, offs, start, s);
      return true;
    case 6:
      launch_rtb_offsets<6>(d, offs, start, s);
      return true;
    default:
      return false;
  }
}

}  // namespace lcs
