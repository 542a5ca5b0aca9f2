// Instantiation of the general sweep and check for sigma = 2 .. 4 (any d up
// to kMaxD, full storage, f_mode 0).  The alphabet sizes are spread over
// several translation units so that they compile in parallel; kernels_rt.cu
// dispatches on sigma.
#include "sweep_rt.cuh"

namespace lcs {

const KernelSet* kernels_rt_s2_4(int sigma) {
  static const KernelSet k[] = {make_rt_set<2>(), make_rt_set<3>(), make_rt_set<4>()};
  return sigma >= 2 && sigma <= 4 ? &k[sigma - 2] : nullptr;
}

bool rt_offsets_fill_s2_4(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s) {
  switch (sigma) {
    case 2:
      launch_rtb_offsets<2>(d, offs, start, s);
      return true;
    case 3:
      launch_rtb_offsets<3>(d, offs, start, s);
      return true;
    case 4:
      launch_rtb_offsets<4>(d, offs, start, s);
      return true;
    default:
      return false;
  }
}

}  // namespace lcs
