// The general sweep and check (any d up to kMaxD, full storage, f_mode 0)
// for sigma = 2 .. 10: dispatch over the translation units that instantiate
// them (kernels_rt_s*.cu), and the host-side helpers.
#include <vector>

#include "sweep_rt.cuh"

namespace lcs {

const KernelSet* kernels_rt_s2_4(int sigma);
const KernelSet* kernels_rt_s5_6(int sigma);
const KernelSet* kernels_rt_s7_8(int sigma);
const KernelSet* kernels_rt_s9_10(int sigma);
bool rt_offsets_fill_s2_4(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s);
bool rt_offsets_fill_s5_6(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s);
bool rt_offsets_fill_s7_8(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s);
bool rt_offsets_fill_s9_10(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s);

const KernelSet* kernels_rt(int sigma) {
  if (sigma >= 2 && sigma <= 4) return kernels_rt_s2_4(sigma);
  if (sigma >= 5 && sigma <= 6) return kernels_rt_s5_6(sigma);
  if (sigma >= 7 && sigma <= 8) return kernels_rt_s7_8(sigma);
  if (sigma >= 9 && sigma <= 10) return kernels_rt_s9_10(sigma);
  return nullptr;
}

// threads' worth of work of one general sweep or check, for sizing its grid:
// one CTA per tail tuple, one warp per tail tuple (small tables, many
// tuples), or one warp per state (sigma = 2, d >= kRtWarpD); in block form,
// one thread per state (the second phase; the first sizes its own grid)
unsigned long long rt_work_items(int sigma, int d, unsigned long long n_states, unsigned long long n_tail,
                                 bool blocks) {
  if (blocks) return n_states;
  if (sigma == 2 && d >= kRtWarpD) return n_states * 32;
  return rt_warp_tails(sigma, d, n_tail) ? n_tail * 32 : n_tail * kBlock;
}

bool rt_blocks_apply(int sigma, int d, int h) { return sigma <= 10 && rtb_applies(sigma, d, h); }

size_t rt_offsets_len(int sigma, int d) {
  size_t n = 1;
  for (int i = 0; i < d; ++i) n *= (size_t)(sigma + 1);
  return n;
}

void rt_offsets_fill(int sigma, int d, unsigned short* offs, unsigned* start, cudaStream_t s) {
  if (!rt_offsets_fill_s2_4(sigma, d, offs, start, s) && !rt_offsets_fill_s5_6(sigma, d, offs, start, s) &&
      !rt_offsets_fill_s7_8(sigma, d, offs, start, s))
    rt_offsets_fill_s9_10(sigma, d, offs, start, s);
}

// The first phase's tiles that hold a task, as (k << 48) | run index: a run
// of G blocks of v_k has one when some block's top digits carry one letter
// on at least d - k strings (every run for k = d).
std::vector<unsigned long long> rt_tile_list(int sigma, int d, int h) {
  std::vector<unsigned long long> out;
  unsigned long long sd = 1, n_tail = 1;
  for (int i = 0; i < d; ++i) sd *= (unsigned long long)sigma;
  for (int i = 0; i < d * (h - 1); ++i) n_tail *= (unsigned long long)sigma;
  const unsigned long long topw = n_tail / sd;
  const unsigned G = rtb_blocks_per_tile((unsigned)sd);
  // the most strings sharing one top letter, for each top group
  std::vector<unsigned char> most(sd);
  for (unsigned long long top = 0; top < sd; ++top) {
    int c[16] = {0};
    unsigned long long x = top;
    int m = 0;
    for (int j = 0; j < d; ++j) {
      m = std::max(m, ++c[x % (unsigned long long)sigma]);
      x /= (unsigned long long)sigma;
    }
    most[top] = (unsigned char)m;
  }
  const unsigned long long runs = (n_tail + G - 1) / G;
  std::vector<unsigned char> run_most(runs, 0);
  for (unsigned long long Y = 0; Y < n_tail; ++Y) {
    unsigned char& r = run_most[Y / G];
    r = std::max(r, most[Y / topw]);
  }
  for (int k = 1; k <= d; ++k)
    for (unsigned long long ty = 0; ty < runs; ++ty)
      if (k == d || run_most[ty] >= d - k) out.push_back(((unsigned long long)k << 48) | ty);
  return out;
}

}  // namespace lcs
