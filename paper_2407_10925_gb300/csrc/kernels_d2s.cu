// Instantiation of the d = 2, sigma >= 3 sweep and check that use the swap
// symmetry, and their host-side geometry.
#include "sweep_d2s.cuh"

namespace lcs {

const KernelSet* kernels_d2s(int sigma) {
  static const KernelSet k3 = make_d2s_set<3>();
  static const KernelSet k4 = make_d2s_set<4>();
  static const KernelSet k5 = make_d2s_set<5>();
  if (sigma == 3) return &k3;
  if (sigma == 4) return &k4;
  if (sigma == 5) return &k5;
  return nullptr;
}

// smallest h the tiles fit (L = h - 1 >= KA)
int d2s_min_h(int sigma) {
  if (sigma == 3) return D2sGeo<3>::KA + 1;
  if (sigma == 4) return D2sGeo<4>::KA + 1;
  if (sigma == 5) return D2sGeo<5>::KA + 1;
  return 1 << 30;
}

template <int SIG>
static unsigned long long slots_of(int h) {
  using G = D2sGeo<SIG>;
  return (d2s_live_tiles<SIG>(h - 1) + G::TPB - 1) / G::TPB;
}

// CTAs' worth of work in one sweep or check (one tile slot per CTA and step)
unsigned long long d2s_slots(int sigma, int h) {
  if (sigma == 3) return slots_of<3>(h);
  if (sigma == 4) return slots_of<4>(h);
  if (sigma == 5) return slots_of<5>(h);
  return 0;
}

void launch_swap_check_d2s(int sigma, const long long* v, unsigned long long n, int h, DevState* st, int grid,
                           cudaStream_t s) {
  if (sigma == 3) swap_check_d2s_kernel<3><<<grid, kBlock, 0, s>>>(v, n, h, st);
  if (sigma == 4) swap_check_d2s_kernel<4><<<grid, kBlock, 0, s>>>(v, n, h, st);
  if (sigma == 5) swap_check_d2s_kernel<5><<<grid, kBlock, 0, s>>>(v, n, h, st);
}

}  // namespace lcs
