// Instantiation of the general sweep and check for sigma = 7 .. 8 (any d up
// to kMaxD, full storage, f_mode 0).  The alphabet sizes are spread over
// several translation units so that they compile in parallel; kernels_rt.cu
// dispatches on sigma.
#include "sweep_rt.cuh"

namespace lcs {

const KernelSet* kernels_rt_s7_8(int sigma) {
  static const KernelSet k[] = {make_rt_set<7>(), make_rt_set<8>()};
  return sigma >= 7 && sigma <= 8 ? &k[sigma - 7] : nullptr;
}

bool rt_offsets_fill_s7_8(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s) {
  switch (sigma) {
    case 7:
      launch_rtb_offsets<7>(d, offs, start, s);
      return true;
    case 8:
      launch_rtb_offsets<8>(d, offs, start, s);
      return true;
    default:
      return false;
  }
}

}  // namespace lcs
