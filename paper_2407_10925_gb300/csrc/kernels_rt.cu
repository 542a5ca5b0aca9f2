// Instantiation of the general sweep and check (any d up to kMaxD, full
// storage, f_mode 0) for sigma = 2 .. 10.
#include "sweep_rt.cuh"

namespace lcs {

const KernelSet* kernels_rt(int sigma) {
  static const KernelSet k[] = {make_rt_set<2>(), make_rt_set<3>(), make_rt_set<4>(), make_rt_set<5>(),
                                make_rt_set<6>(), make_rt_set<7>(), make_rt_set<8>(), make_rt_set<9>(),
                                make_rt_set<10>()};
  return sigma >= 2 && sigma <= 10 ? &k[sigma - 2] : nullptr;
}

// threads' worth of work of one general sweep or check, for sizing its grid:
// one CTA per tail tuple, one warp per tail tuple (small tables, many
// tuples), or one warp per state (sigma = 2, d >= kRtWarpD)
unsigned long long rt_work_items(int sigma, int d, unsigned long long n_states, unsigned long long n_tail) {
  if (sigma == 2 && d >= kRtWarpD) return n_states * 32;
  return rt_warp_tails(sigma, d, n_tail) ? n_tail * 32 : n_tail * kBlock;
}

}  // namespace lcs
