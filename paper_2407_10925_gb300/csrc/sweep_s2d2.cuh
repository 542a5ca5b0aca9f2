// sweep_s2d2.cuh -- the sweep and check for sigma = d = 2 using both exact
// symmetries of the binary two-string case (Heineman et al., arXiv 2407.10925):
//
//   complement (section 3.3, Eq. impl:comp_eq): v[(~a, ~b)] = v[(a, b)];
//   swap: v[(b, a)] = v[(a, b)] -- the LCS does not depend on the order of
//         its arguments, and F commutes with exchanging the two strings.
//
// In int64 fixed point both hold bit for bit at every iteration once the
// start vectors have them (the zero start does): sums are exact and the max
// over the two advance choices is symmetric.  Storage keeps the complement
// half (x < N/2: heads 00 and 01); the swap is used to read less.
//
// Write a tail tuple t = (a, b) (each an (h-1)-bit string) and its orbit
//   t = (a, b),  ~t = (~a, ~b),  t' = (~b, ~a),  ~t' = (b, a).
// Then, with Sb(x) the sum of v_{t-1} over the two states reached by
// advancing the second string of the heads-01 state of tail x (Algorithm 1,
// F_0 of the binary case):
//   * the heads-01 state of t has the two candidates Sb(t) (advance b) and,
//     because v_{t-1}[(a c, 1 b)] = v_{t-1}[(0 ~b, ~a ~c)], Sb(t') (advance a);
//     so v[01, t] = v[01, t'] = floor(max(Sb(t), Sb(t')) / 2), and likewise
//     v[01, ~t] = v[01, ~t'];
//   * the heads-00 states of all four tails read the same four values of
//     v_{t-2} (Eq. ineq1), so they share one value 1 + floor(sum / 4).
// One thread owns one orbit: 12 loads (four pairs of v_{t-1}, one block of
// four of v_{t-2}) produce its 8 stored values.  Per stored state that is
// 12 B read + 8 B written, against 24 + 8 without the swap.
//
// Orbit representatives: a has leading bit 0 and a <= beta, where the second
// string is b = beta (s = 0) or b = ~beta (s = 1) with beta's leading bit 0.
// Tiles of 16 x 16 (a, beta) pairs are walked by a persistent grid; tiles
// below the diagonal are skipped as a whole.  Inside a tile the thread index
// is the Morton code of (a, beta) low bits, so a warp covers 32 consecutive
// tail indices and every stream it touches is contiguous.
#pragma once

#include <climits>

#include "lcs_common.h"
#include "sweep_generic.cuh"

namespace lcs {

// insert a zero bit above every bit of x (x < 2^32)
__device__ __forceinline__ unsigned long long spread_bits(unsigned long long x) {
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

constexpr int kS2D2Tile = 16;  // (a, beta) tile side; 256 threads = one tile

struct S2D2Orbit {
  unsigned long long t, tc, tp, sw;  // t, ~t, t', ~t' as tail indices
  unsigned long long yb[4];          // first of the two adjacent v_{t-1} reads: Sb(t), Sb(~t), Sb(t'), Sb(~t')
};

// The orbit owned by thread `tid` of tile k; false if the thread has none.
__device__ __forceinline__ bool s2d2_orbit(unsigned long long k, unsigned tn, int L, unsigned long long nt,
                                           unsigned long long maskE, unsigned tid, S2D2Orbit& o) {
  const unsigned long long per_s = (unsigned long long)tn * tn;
  const unsigned s = (unsigned)(k / per_s);
  const unsigned long long rem = k - (unsigned long long)s * per_s;
  const unsigned A = (unsigned)(rem / tn), B = (unsigned)(rem - (unsigned long long)A * tn);
  // Morton order inside the tile: odd bits -> a, even bits -> beta
  unsigned ia = 0, ib = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ib |= ((tid >> (2 * i)) & 1u) << i;
    ia |= ((tid >> (2 * i + 1)) & 1u) << i;
  }
  const unsigned long long a = (unsigned long long)A * kS2D2Tile + ia;
  const unsigned long long beta = (unsigned long long)B * kS2D2Tile + ib;
  if (a > beta) return false;
  const unsigned long long b = s ? (((1ull << L) - 1) - beta) : beta;
  const unsigned long long Ea = spread_bits(a), Eb = spread_bits(b);
  o.t = (Ea << 1) | Eb;
  o.sw = (Eb << 1) | Ea;
  o.tc = nt - 1 - o.t;
  o.tp = nt - 1 - o.sw;
  const unsigned long long Eac = maskE - Ea, Ebc = maskE - Eb;
  o.yb[0] = (Ea << 1) | (Eb << 2);
  o.yb[1] = (Eac << 1) | (Ebc << 2);
  o.yb[2] = (Ebc << 1) | (Eac << 2);
  o.yb[3] = (Eb << 1) | (Ea << 2);
  return true;
}

template <bool CG>
__device__ __forceinline__ longlong2 ld_pair(const long long* v, unsigned long long y) {
  const longlong2* q = reinterpret_cast<const longlong2*>(v + y);  // y is even: 16-byte aligned
  if constexpr (CG)
    return __ldcg(q);
  else
    return __ldg(q);
}

template <bool CG = false>
__device__ __forceinline__ long long pair_sum(const long long* v, unsigned long long y) {
  const longlong2 q = ld_pair<CG>(v, y);
  return q.x + q.y;
}

template <bool CG = false>
__device__ __forceinline__ long long quad_sum(const long long* v, unsigned long long y) {
  const longlong2 q0 = ld_pair<CG>(v, y);
  const longlong2 q1 = ld_pair<CG>(v, y + 2);
  return q0.x + q0.y + q1.x + q1.y;
}

// geometry of the orbit tiles for one h
struct S2D2Geo {
  int L;                     // h - 1: length of a tail string
  unsigned tn;               // tiles per side: 2^(L-1) / 16
  unsigned long long nt;     // tail tuples: 4^L
  unsigned long long maskE;  // spread of L one-bits
};

__device__ __forceinline__ S2D2Geo s2d2_geo(int h, unsigned long long n_tail) {
  S2D2Geo g;
  g.L = h - 1;
  g.tn = (1u << (g.L - 1)) / kS2D2Tile;
  g.nt = n_tail;
  g.maskE = spread_bits((1ull << g.L) - 1);
  return g;
}

// One thread's orbit of tile k: the 8 stored outputs; INCR folds one
// increment candidate per class of equal values into (best_v, best_x).
template <bool INCR, bool CG = false>
__device__ __forceinline__ void s2d2_sweep_orbit(const SweepParams& p, const S2D2Geo& g, unsigned long long k,
                                                 long long& best_v, unsigned long long& best_x) {
  S2D2Orbit o;
  if (!s2d2_orbit(k, g.tn, g.L, g.nt, g.maskE, threadIdx.x, o)) return;
  const unsigned long long nt = g.nt;
  const long long* v1 = p.prev[0];
  const long long* v2 = p.prev[1];
  const long long s00 = quad_sum<CG>(v2, 4 * o.t);
  const long long sb_t = pair_sum<CG>(v1, o.yb[0]);
  const long long sb_tc = pair_sum<CG>(v1, o.yb[1]);
  const long long sb_tp = pair_sum<CG>(v1, o.yb[2]);
  const long long sb_sw = pair_sum<CG>(v1, o.yb[3]);
  const long long e00 = p.one + (s00 >> 2);
  const long long u_t = max(sb_t, sb_tp) >> 1;    // heads 01 at t and t'
  const long long u_tc = max(sb_tc, sb_sw) >> 1;  // heads 01 at ~t and ~t'
  long long* out = p.out;
  out[o.t] = e00;
  out[o.tc] = e00;
  out[o.tp] = e00;
  out[o.sw] = e00;
  out[nt + o.t] = u_t;
  out[nt + o.tp] = u_t;
  out[nt + o.tc] = u_tc;
  out[nt + o.sw] = u_tc;
  if constexpr (INCR) {
    // equal values have equal increments (v_{t-1} has the same symmetries):
    // one candidate per class, at the class's smallest index
    const unsigned long long m00 = min(min(o.t, o.tc), min(o.tp, o.sw));
    const long long i00 = e00 - ld_vec<CG>(v1 + o.t);
    const long long i01 = u_t - ld_vec<CG>(v1 + nt + o.t);
    const long long i01c = u_tc - ld_vec<CG>(v1 + nt + o.tc);
    if (red_better(i00, m00, best_v, best_x, p.r_mode)) best_v = i00, best_x = m00;
    if (red_better(i01, nt + min(o.t, o.tp), best_v, best_x, p.r_mode)) best_v = i01, best_x = nt + min(o.t, o.tp);
    if (red_better(i01c, nt + min(o.tc, o.sw), best_v, best_x, p.r_mode)) best_v = i01c, best_x = nt + min(o.tc, o.sw);
  }
}

// W = u + 2R - F(u + R, u) at the 8 stored states of one orbit (3 distinct).
template <bool CG = false>
__device__ __forceinline__ void s2d2_check_orbit(const CheckParams& p, const S2D2Geo& g, long long R,
                                                 unsigned long long k, long long& best) {
  S2D2Orbit o;
  if (!s2d2_orbit(k, g.tn, g.L, g.nt, g.maskE, threadIdx.x, o)) return;
  const unsigned long long nt = g.nt;
  const long long* u = p.u;
  const long long s00 = quad_sum<CG>(u, 4 * o.t);
  const long long sb_t = pair_sum<CG>(u, o.yb[0]);
  const long long sb_tc = pair_sum<CG>(u, o.yb[1]);
  const long long sb_tp = pair_sum<CG>(u, o.yb[2]);
  const long long sb_sw = pair_sum<CG>(u, o.yb[3]);
  // equal heads: only the all-advance candidate, shifted by (d - d) R = 0;
  // heads 01: both candidates advance one string, shifted by (d - 1) R = R
  const long long w00 = ld_vec<CG>(u + o.t) + 2 * R - (p.one + (s00 >> 2));
  const long long w01 = ld_vec<CG>(u + nt + o.t) + 2 * R - ((max(sb_t, sb_tp) >> 1) + R);
  const long long w01c = ld_vec<CG>(u + nt + o.tc) + 2 * R - ((max(sb_tc, sb_sw) >> 1) + R);
  best = max(best, max(w00, max(w01, w01c)));
}

// the upper-triangle tile index q (A <= B) of one s-half as (A, B)
__device__ __forceinline__ void tri_decode(unsigned long long q, unsigned& A, unsigned& B) {
  unsigned long long b = (unsigned long long)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  while (b * (b + 1) / 2 > q) --b;
  while ((b + 1) * (b + 2) / 2 <= q) ++b;
  B = (unsigned)b;
  A = (unsigned)(q - b * (b + 1) / 2);
}

template <bool INCR>
__global__ void __launch_bounds__(kBlock) sweep_s2d2_kernel(SweepParams p) {
  const S2D2Geo g = s2d2_geo(p.h, p.n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;  // tile below the diagonal: the whole CTA skips it
    s2d2_sweep_orbit<INCR>(p, g, k, best_v, best_x);
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

template <int UNUSED = 0>
__global__ void __launch_bounds__(kBlock) check_s2d2_kernel(CheckParams p) {
  const S2D2Geo g = s2d2_geo(p.h, p.n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  const long long R = p.R_from_state ? p.state->R : p.R;
  long long best = LLONG_MIN;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;
    s2d2_check_orbit(p, g, R, k, best);
  }
  block_reduce_max(best, p.partials);
}

inline void launch_sweep_s2d2(const SweepParams& p, int grid, cudaStream_t s) {
  if (p.incr)
    sweep_s2d2_kernel<true><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_s2d2_kernel<false><<<grid, kBlock, 0, s>>>(p);
}

inline void launch_check_s2d2(const CheckParams& p, int grid, cudaStream_t s) {
  check_s2d2_kernel<0><<<grid, kBlock, 0, s>>>(p);
}

inline KernelSet make_s2d2_set() {
  KernelSet k{};
  k.sigma = 2;
  k.d = 2;
  k.sym = 2;
  k.sweep = &launch_sweep_s2d2;
  k.check = &launch_check_s2d2;
  k.sweep_fn = (const void*)&sweep_s2d2_kernel<true>;
  k.check_fn = (const void*)&check_s2d2_kernel<0>;
  k.tails_per_thread = 4;
  k.sweep_algo_bytes = 20;  // 8 B of v_{t-1} + 4 B of v_{t-2} (its distinct half) + 8 B written
  k.check_algo_bytes = 8;
  return k;
}

}  // namespace lcs
