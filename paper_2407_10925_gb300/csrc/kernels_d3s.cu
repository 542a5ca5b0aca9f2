// Instantiation of the sigma = 2, d = 3 sweep and check that use the string
// permutations and the complement, and their host-side geometry.
#include "sweep_d3s.cuh"

namespace lcs {

const KernelSet* kernels_d3s(int f_mode) {
  static const KernelSet k0 = make_d3s_set<false>();
  static const KernelSet k1 = make_d3s_set<true>();
  return f_mode ? &k1 : &k0;
}

// smallest h the 4 x 8 x 8 tiles fit (L = h - 1 >= 3)
int d3s_min_h() { return 4; }

// largest h the sweep's 32-bit indices cover
int d3s_max_h() { return kD3sMaxH; }

// tiles of one sweep or check (every CTA step takes one)
unsigned long long d3s_tiles(int h) { return 1ull << (3 * (h - 1) - 8); }

void launch_perm_check_d3s(const long long* v, unsigned long long n_stored, unsigned long long n_total, DevState* st,
                           int grid, cudaStream_t s) {
  perm_check_d3s_kernel<><<<grid, kBlock, 0, s>>>(v, n_stored, n_total, st);
}

}  // namespace lcs
