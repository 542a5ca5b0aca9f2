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
//
// Storage.  The element type T of the iterate vectors is long long (the
// fixed-point value itself) or int: offset-normalised storage, where a stored
// w stands for v = w + c with one int64 offset c per vector (SweepParams).
// Lemma 1's translation invariance makes this exact: each mean of one vector
// is the mean of its w plus c, because c is added to every term of the sum
// and floor((S + m c) / m) = floor(S / m) + c.  The sums, the max and the
// increment are formed in int64 from v; only the stored output is narrowed,
// v - c_out, and one that leaves 32 bits is flagged.  The check needs no
// offset at all: W = u + dR - F(u + (d-1)R, .., u) is unchanged when the same
// c is added to u everywhere.
#pragma once

#include <climits>

#include "../../include/lcs_bound.h"
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

// the same loads for either storage type (the int ones: 8- and 16-byte vectors)
template <bool CG, class T>
__device__ __forceinline__ long long pair_sum_t(const T* v, unsigned long long y) {
  if constexpr (sizeof(T) == 8) {
    return pair_sum<CG>(reinterpret_cast<const long long*>(v), y);
  } else {
    const int2* q = reinterpret_cast<const int2*>(v + y);  // y even: 8-byte aligned
    const int2 r = CG ? __ldcg(q) : __ldg(q);
    return (long long)r.x + r.y;
  }
}

template <bool CG, class T>
__device__ __forceinline__ long long quad_sum_t(const T* v, unsigned long long y) {
  if constexpr (sizeof(T) == 8) {
    return quad_sum<CG>(reinterpret_cast<const long long*>(v), y);
  } else {
    const int4* q = reinterpret_cast<const int4*>(v + y);  // y a multiple of 4: 16-byte aligned
    const int4 r = CG ? __ldcg(q) : __ldg(q);
    return (long long)r.x + r.y + r.z + r.w;
  }
}

template <bool CG, class T>
__device__ __forceinline__ long long ld_one_t(const T* v, unsigned long long y) {
  if constexpr (sizeof(T) == 8)
    return ld_vec<CG>(reinterpret_cast<const long long*>(v) + y);
  else
    return CG ? __ldcg(v + y) : __ldg(v + y);
}

// the offsets of one narrow sweep: inputs c1 (newest), c2, and the output's
struct NarrowOffs {
  long long c1, c2, cout;
};

// The output's offset is anchored to an actual value: the newest input's
// value at state 0 plus the last increment R (0 before the first one), so
// w_out = v_out - c_out stays within the spread of one iterate plus one
// step's increments, however many sweeps run.  One thread per CTA reads the
// anchor (it may sit in host memory) and shares it.
template <class T>
__device__ __forceinline__ NarrowOffs narrow_offsets(const SweepParams& p) {
  NarrowOffs o{0, 0, 0};
  if constexpr (sizeof(T) == 4) {
    __shared__ long long s_anchor;
    if (threadIdx.x == 0) s_anchor = (long long)__ldcg(reinterpret_cast<const int*>(p.prev[0]));
    __syncthreads();
    o.c1 = __ldcg(p.offs + p.slot_in0);
    o.c2 = __ldcg(p.offs + p.slot_in1);
    o.cout = o.c1 + s_anchor + (__ldcg(&p.state->R_iter) ? __ldcg(&p.state->R) : p.step);
  }
  return o;
}

// store v at out[x] (narrow storage: v - cout, flagging a value outside 32 bits)
template <class T>
__device__ __forceinline__ void store_t(T* out, unsigned long long x, long long v, long long cout, bool& bad) {
  if constexpr (sizeof(T) == 8) {
    out[x] = v;
  } else {
    const long long w = v - cout;
    bad |= w < INT_MIN || w > INT_MAX;
    out[x] = (int)w;
  }
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
template <bool INCR, bool CG = false, class T = long long>
__device__ __forceinline__ void s2d2_sweep_orbit(const SweepParams& p, const S2D2Geo& g, unsigned long long k,
                                                 long long& best_v, unsigned long long& best_x,
                                                 const NarrowOffs& c = NarrowOffs{0, 0, 0}) {
  S2D2Orbit o;
  if (!s2d2_orbit(k, g.tn, g.L, g.nt, g.maskE, threadIdx.x, o)) return;
  const unsigned long long nt = g.nt;
  const T* v1 = reinterpret_cast<const T*>(p.prev[0]);
  const T* v2 = reinterpret_cast<const T*>(p.prev[1]);
  const long long s00 = quad_sum_t<CG>(v2, 4 * o.t);
  const long long sb_t = pair_sum_t<CG>(v1, o.yb[0]);
  const long long sb_tc = pair_sum_t<CG>(v1, o.yb[1]);
  const long long sb_tp = pair_sum_t<CG>(v1, o.yb[2]);
  const long long sb_sw = pair_sum_t<CG>(v1, o.yb[3]);
  // narrow storage: a mean of one vector is the mean of its w plus its offset
  const long long e00 = p.one + (s00 >> 2) + c.c2;
  const long long u_t = (max(sb_t, sb_tp) >> 1) + c.c1;    // heads 01 at t and t'
  const long long u_tc = (max(sb_tc, sb_sw) >> 1) + c.c1;  // heads 01 at ~t and ~t'
  T* out = reinterpret_cast<T*>(p.out);
  bool bad = false;
  store_t(out, o.t, e00, c.cout, bad);
  store_t(out, o.tc, e00, c.cout, bad);
  store_t(out, o.tp, e00, c.cout, bad);
  store_t(out, o.sw, e00, c.cout, bad);
  store_t(out, nt + o.t, u_t, c.cout, bad);
  store_t(out, nt + o.tp, u_t, c.cout, bad);
  store_t(out, nt + o.tc, u_tc, c.cout, bad);
  store_t(out, nt + o.sw, u_tc, c.cout, bad);
  if (sizeof(T) == 4 && bad) atomicExch((unsigned long long*)&p.state->status, (unsigned long long)LCS_EOVERFLOW);
  if constexpr (INCR) {
    // equal values have equal increments (v_{t-1} has the same symmetries):
    // one candidate per class, at the class's smallest index
    const unsigned long long m00 = min(min(o.t, o.tc), min(o.tp, o.sw));
    const long long i00 = e00 - (ld_one_t<CG>(v1, o.t) + c.c1);
    const long long i01 = u_t - (ld_one_t<CG>(v1, nt + o.t) + c.c1);
    const long long i01c = u_tc - (ld_one_t<CG>(v1, nt + o.tc) + c.c1);
    if (red_better(i00, m00, best_v, best_x, p.r_mode)) best_v = i00, best_x = m00;
    if (red_better(i01, nt + min(o.t, o.tp), best_v, best_x, p.r_mode)) best_v = i01, best_x = nt + min(o.t, o.tp);
    if (red_better(i01c, nt + min(o.tc, o.sw), best_v, best_x, p.r_mode)) best_v = i01c, best_x = nt + min(o.tc, o.sw);
  }
}

// The sweep of one orbit fused with the check of its newest input u =
// v_{t-1} (Algorithm 2's check of the previous iteration, R = that
// iteration's increment): W = u + 2R - F(u + R, u) at the orbit's states
// needs the four pairs of u the sweep already reads, the values of u at the
// orbit's three classes (the increment reads them too) and one quad of u --
// 4 more bytes per stored state instead of a 12-byte pass of its own.  With
// narrow storage W is formed from the stored w of u: the offset cancels.
template <bool INCR, class T = long long>
__device__ __forceinline__ void s2d2_sweep_check_orbit(const SweepParams& p, const S2D2Geo& g, unsigned long long k,
                                                       long long& best_v, unsigned long long& best_x, long long& best_w,
                                                       long long R, const NarrowOffs& c) {
  S2D2Orbit o;
  if (!s2d2_orbit(k, g.tn, g.L, g.nt, g.maskE, threadIdx.x, o)) return;
  const unsigned long long nt = g.nt;
  const T* v1 = reinterpret_cast<const T*>(p.prev[0]);
  const T* v2 = reinterpret_cast<const T*>(p.prev[1]);
  const long long s00 = quad_sum_t<false>(v2, 4 * o.t);
  const long long q00 = quad_sum_t<false>(v1, 4 * o.t);  // the check's all-advance block of u
  const long long sb_t = pair_sum_t<false>(v1, o.yb[0]);
  const long long sb_tc = pair_sum_t<false>(v1, o.yb[1]);
  const long long sb_tp = pair_sum_t<false>(v1, o.yb[2]);
  const long long sb_sw = pair_sum_t<false>(v1, o.yb[3]);
  const long long u00 = ld_one_t<false>(v1, o.t);
  const long long u01 = ld_one_t<false>(v1, nt + o.t);
  const long long u01c = ld_one_t<false>(v1, nt + o.tc);
  const long long m01 = max(sb_t, sb_tp) >> 1, m01c = max(sb_tc, sb_sw) >> 1;
  const long long e00 = p.one + (s00 >> 2) + c.c2;
  const long long u_t = m01 + c.c1;
  const long long u_tc = m01c + c.c1;
  T* out = reinterpret_cast<T*>(p.out);
  bool bad = false;
  store_t(out, o.t, e00, c.cout, bad);
  store_t(out, o.tc, e00, c.cout, bad);
  store_t(out, o.tp, e00, c.cout, bad);
  store_t(out, o.sw, e00, c.cout, bad);
  store_t(out, nt + o.t, u_t, c.cout, bad);
  store_t(out, nt + o.tp, u_t, c.cout, bad);
  store_t(out, nt + o.tc, u_tc, c.cout, bad);
  store_t(out, nt + o.sw, u_tc, c.cout, bad);
  if (sizeof(T) == 4 && bad) atomicExch((unsigned long long*)&p.state->status, (unsigned long long)LCS_EOVERFLOW);
  // the check of u (as s2d2_check_orbit)
  const long long w00 = u00 + 2 * R - (p.one + (q00 >> 2));
  const long long w01 = u01 + 2 * R - (m01 + R);
  const long long w01c = u01c + 2 * R - (m01c + R);
  best_w = max(best_w, max(w00, max(w01, w01c)));
  if constexpr (INCR) {
    const unsigned long long m00 = min(min(o.t, o.tc), min(o.tp, o.sw));
    const long long i00 = e00 - (u00 + c.c1);
    const long long i01 = u_t - (u01 + c.c1);
    const long long i01c = u_tc - (u01c + c.c1);
    if (red_better(i00, m00, best_v, best_x, p.r_mode)) best_v = i00, best_x = m00;
    if (red_better(i01, nt + min(o.t, o.tp), best_v, best_x, p.r_mode)) best_v = i01, best_x = nt + min(o.t, o.tp);
    if (red_better(i01c, nt + min(o.tc, o.sw), best_v, best_x, p.r_mode)) best_v = i01c, best_x = nt + min(o.tc, o.sw);
  }
}

// W = u + 2R - F(u + R, u) at the 8 stored states of one orbit (3 distinct).
// With narrow storage the stored w serve as u: the offset cancels.
template <bool CG = false, class T = long long>
__device__ __forceinline__ void s2d2_check_orbit(const CheckParams& p, const S2D2Geo& g, long long R,
                                                 unsigned long long k, long long& best) {
  S2D2Orbit o;
  if (!s2d2_orbit(k, g.tn, g.L, g.nt, g.maskE, threadIdx.x, o)) return;
  const unsigned long long nt = g.nt;
  const T* u = reinterpret_cast<const T*>(p.u);
  const long long s00 = quad_sum_t<CG>(u, 4 * o.t);
  const long long sb_t = pair_sum_t<CG>(u, o.yb[0]);
  const long long sb_tc = pair_sum_t<CG>(u, o.yb[1]);
  const long long sb_tp = pair_sum_t<CG>(u, o.yb[2]);
  const long long sb_sw = pair_sum_t<CG>(u, o.yb[3]);
  // equal heads: only the all-advance candidate, shifted by (d - d) R = 0;
  // heads 01: both candidates advance one string, shifted by (d - 1) R = R
  const long long w00 = ld_one_t<CG>(u, o.t) + 2 * R - (p.one + (s00 >> 2));
  const long long w01 = ld_one_t<CG>(u, nt + o.t) + 2 * R - ((max(sb_t, sb_tp) >> 1) + R);
  const long long w01c = ld_one_t<CG>(u, nt + o.tc) + 2 * R - ((max(sb_tc, sb_sw) >> 1) + R);
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

template <bool INCR, class T = long long>
__global__ void __launch_bounds__(kBlock) sweep_s2d2_kernel(SweepParams p) {
  const S2D2Geo g = s2d2_geo(p.h, p.n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  const NarrowOffs c = narrow_offsets<T>(p);
  if (sizeof(T) == 4 && blockIdx.x == 0 && threadIdx.x == 0) p.offs[p.slot_out] = c.cout;
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;  // tile below the diagonal: the whole CTA skips it
    s2d2_sweep_orbit<INCR, false, T>(p, g, k, best_v, best_x, c);
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

// The sweep with the check of its newest input fused in: per-CTA increment
// partials (INCR) into p.partials, per-CTA max W into p.check_partials.
template <bool INCR, class T = long long>
__global__ void __launch_bounds__(kBlock) sweep_check_s2d2_kernel(SweepParams p) {
  const S2D2Geo g = s2d2_geo(p.h, p.n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  const NarrowOffs c = narrow_offsets<T>(p);
  if (sizeof(T) == 4 && blockIdx.x == 0 && threadIdx.x == 0) p.offs[p.slot_out] = c.cout;
  const long long R = __ldcg(&p.state->R);
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  long long best_w = LLONG_MIN;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;
    s2d2_sweep_check_orbit<INCR, T>(p, g, k, best_v, best_x, best_w, R, c);
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
  block_reduce_max(best_w, p.check_partials);
}

template <class T = long long>
__global__ void __launch_bounds__(kBlock) check_s2d2_kernel(CheckParams p) {
  const S2D2Geo g = s2d2_geo(p.h, p.n_tail);
  const unsigned long long n_tiles = 2ull * g.tn * g.tn;
  const long long R = p.R_from_state ? p.state->R : p.R;
  long long best = LLONG_MIN;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    const unsigned long long rem = k % ((unsigned long long)g.tn * g.tn);
    if (rem / g.tn > rem % g.tn) continue;
    s2d2_check_orbit<false, T>(p, g, R, k, best);
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
  check_s2d2_kernel<long long><<<grid, kBlock, 0, s>>>(p);
}

template <class T>
inline void launch_sweep_check_s2d2(const SweepParams& p, int grid, cudaStream_t s) {
  if (p.incr)
    sweep_check_s2d2_kernel<true, T><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_check_s2d2_kernel<false, T><<<grid, kBlock, 0, s>>>(p);
}

inline void launch_sweep_s2d2_narrow(const SweepParams& p, int grid, cudaStream_t s) {
  if (p.incr)
    sweep_s2d2_kernel<true, int><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_s2d2_kernel<false, int><<<grid, kBlock, 0, s>>>(p);
}

inline void launch_check_s2d2_narrow(const CheckParams& p, int grid, cudaStream_t s) {
  check_s2d2_kernel<int><<<grid, kBlock, 0, s>>>(p);
}

inline KernelSet make_s2d2_set() {
  KernelSet k{};
  k.sigma = 2;
  k.d = 2;
  k.sym = 2;
  k.sweep = &launch_sweep_s2d2;
  k.check = &launch_check_s2d2;
  k.sweep_fn = (const void*)&sweep_s2d2_kernel<true>;
  k.check_fn = (const void*)&check_s2d2_kernel<long long>;
  k.tails_per_thread = 4;
  k.sweep_algo_bytes = 20;  // 8 B of v_{t-1} + 4 B of v_{t-2} (its distinct half) + 8 B written
  k.check_algo_bytes = 8;
  k.sweep_check = &launch_sweep_check_s2d2<long long>;
  k.sweep_check_fn = (const void*)&sweep_check_s2d2_kernel<true, long long>;
  return k;
}

// the same sweep over offset-normalised 32-bit storage: half the bytes
inline KernelSet make_s2d2_narrow_set() {
  KernelSet k = make_s2d2_set();
  k.sweep = &launch_sweep_s2d2_narrow;
  k.check = &launch_check_s2d2_narrow;
  k.sweep_fn = (const void*)&sweep_s2d2_kernel<true, int>;
  k.check_fn = (const void*)&check_s2d2_kernel<int>;
  k.sweep_algo_bytes = 10;  // 4 B of v_{t-1} + 2 B of v_{t-2} + 4 B written
  k.check_algo_bytes = 4;
  k.sweep_check = &launch_sweep_check_s2d2<int>;
  k.sweep_check_fn = (const void*)&sweep_check_s2d2_kernel<true, int>;
  return k;
}

}  // namespace lcs
