// The orbit form of a sigma = d = 2 vector under complement-symmetric storage
// that is also symmetric under exchanging the two strings.
//
// With the complement (section 3.3, Eq. impl:comp_eq) and the string swap, the
// stored states (heads 00 and 01) of a tail t = (a, b) fall into one orbit of
// eight with those of ~t = (~a, ~b), t' = (~b, ~a) and ~t' = (b, a), and the
// orbit holds at most four distinct values:
//   v(00, t)  = v(00, ~t')   (swap)
//   v(00, ~t) = v(00, t')    (swap)
//   v(01, t)  = v(01, t')    (complement, then swap: heads 01 -> 10 -> 01)
//   v(01, ~t) = v(01, ~t')
// The orbit form keeps those four values, in that order, for one
// representative per orbit: (s, a, beta) with a <= beta < 2^(h-2) (leading bit
// 0) and b = beta (s = 0) or b = 2^(h-1) - 1 - beta (s = 1), the
// representatives the sigma = d = 2 sweep walks.  The representative's place
// is s K (K + 1) / 2 + beta (beta + 1) / 2 + a with K = 2^(h-2), so the form
// holds 4 K (K + 1) = 4^(h-1) + 2^h values: about half the stored form.
//
// pack: stored form -> orbit form (the source must have the swap symmetry);
// unpack: orbit form -> stored form, writing all eight states of every orbit,
// and max |v| into the device state.  Both walk the sweep's 16 x 16 tiles of
// (a, beta) in the sweep's Morton order, so their stored-side accesses are
// those of the sweep (a warp covers 32 consecutive tails); the orbit side is
// read or written in runs of four representatives (128 B).
#include <climits>

#include "sweep_s2d2.cuh"

namespace lcs {

namespace {

// the orbit of thread tid of tile k and its place in the orbit form
__device__ __forceinline__ bool orbit_place(unsigned long long k, const S2D2Geo& g, unsigned tid, S2D2Orbit& o,
                                            unsigned long long& place) {
  if (!s2d2_orbit(k, g.tn, g.L, g.nt, g.maskE, tid, o)) return false;
  const unsigned long long per_s = (unsigned long long)g.tn * g.tn;
  const unsigned long long s = k / per_s, rem = k - s * per_s;
  const unsigned long long A = rem / g.tn, B = rem - A * g.tn;
  unsigned long long ia = 0, ib = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ib |= (unsigned long long)((tid >> (2 * i)) & 1u) << i;
    ia |= (unsigned long long)((tid >> (2 * i + 1)) & 1u) << i;
  }
  const unsigned long long a = A * kS2D2Tile + ia, beta = B * kS2D2Tile + ib;
  const unsigned long long K = (unsigned long long)g.tn * kS2D2Tile;
  place = s * (K * (K + 1) / 2) + beta * (beta + 1) / 2 + a;
  return true;
}

__global__ void __launch_bounds__(kBlock) orbit_unpack_kernel(const long long* __restrict__ orb,
                                                              long long* __restrict__ out, int h,
                                                              unsigned long long n_tail, DevState* st) {
  const S2D2Geo g = s2d2_geo(h, n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  const unsigned long long nt = g.nt;
  long long m = 0;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;  // below the diagonal: no representative
    S2D2Orbit o;
    unsigned long long q;
    if (!orbit_place(k, g, threadIdx.x, o, q)) continue;
    const longlong2 p0 = ld_pair<false>(orb, 4 * q), p1 = ld_pair<false>(orb, 4 * q + 2);
    out[o.t] = p0.x;
    out[o.sw] = p0.x;
    out[o.tc] = p0.y;
    out[o.tp] = p0.y;
    out[nt + o.t] = p1.x;
    out[nt + o.tp] = p1.x;
    out[nt + o.tc] = p1.y;
    out[nt + o.sw] = p1.y;
    const long long vals[4] = {p0.x, p0.y, p1.x, p1.y};
#pragma unroll
    for (int j = 0; j < 4; ++j) m = max(m, vals[j] == LLONG_MIN ? LLONG_MAX : (vals[j] < 0 ? -vals[j] : vals[j]));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&st->maxabs, m);
}

__global__ void __launch_bounds__(kBlock) orbit_pack_kernel(const long long* __restrict__ v,
                                                            long long* __restrict__ orb, int h,
                                                            unsigned long long n_tail) {
  const S2D2Geo g = s2d2_geo(h, n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  const unsigned long long nt = g.nt;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;
    S2D2Orbit o;
    unsigned long long q;
    if (!orbit_place(k, g, threadIdx.x, o, q)) continue;
    longlong2* dst = reinterpret_cast<longlong2*>(orb + 4 * q);
    dst[0] = make_longlong2(v[o.t], v[o.tc]);
    dst[1] = make_longlong2(v[nt + o.t], v[nt + o.tc]);
  }
}

}  // namespace

// values in the orbit form for this h (h >= 6)
unsigned long long orbit_len(int h) {
  const unsigned long long K = 1ull << (h - 2);
  return 4 * K * (K + 1);
}

static int orbit_grid(int h) {
  const unsigned long long tn = (1ull << (h - 2)) / kS2D2Tile;
  return (int)std::min<unsigned long long>(4096, 2 * tn * tn);
}

void launch_orbit_unpack(const long long* orb, long long* out, int h, unsigned long long n_tail, DevState* st,
                         cudaStream_t s) {
  orbit_unpack_kernel<<<orbit_grid(h), kBlock, 0, s>>>(orb, out, h, n_tail, st);
}

void launch_orbit_pack(const long long* v, long long* orb, int h, unsigned long long n_tail, cudaStream_t s) {
  orbit_pack_kernel<<<orbit_grid(h), kBlock, 0, s>>>(v, orb, h, n_tail);
}

}  // namespace lcs
