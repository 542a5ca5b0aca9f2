// sweep_d3s.cuh -- the sweep and check for sigma = 2, d = 3 that use the
// permutations of the three strings and the complement, under
// complement-symmetric storage (states x < N/2, the first letter of string 0
// is 0).  Both symmetries hold bit for bit in fixed point once the start
// vectors have them (the zero start does): the LCS does not depend on the
// order of its arguments, and F commutes with permuting the strings and with
// complementing every letter (section 3.3).
//
// A tail tuple is tau = (T0, T1, T2), three strings of L = h - 1 bits.  One
// thread owns the orbit of tau under the 6 permutations together with the
// orbit of its complement ~tau (never the same orbit): up to 12 tails, 96
// states, 48 of them stored.  With binary heads a state whose heads are not
// all equal has a majority letter m (two strings) and a minority string j,
// and Eq. ineq3 has two candidates (Algorithm 1):
//   z = m: advance j alone, the others keep head m   -> v_{t-1}, 2 values
//   z = 1 - m: advance the two majority strings     -> v_{t-2}, 4 values
// By the permutation symmetry the first sum depends only on which component
// of the tail string j carries and on m; by the complement, m = 1 is the
// m = 0 sum of the complemented tail.  So the thread forms
//   A1(X, k) = sum over c of v_{t-1}[(0 U0, 0 U1, U2 c)],     U2 = X_k,
//   A2(X, k) = sum over c1, c2 of v_{t-2}[(0 U0, U1 c1, U2 c2)], U0 = X_k,
// ({U0, U1} resp. {U1, U2} the other two components) for X in {tau, ~tau}
// and k in {0, 1, 2}, all in the stored half, plus the all-advance block of
// v_{t-3} once (permuting or complementing the tail only permutes it): 44
// reads for 48 stored outputs, against roughly 40 B read per stored state by
// the generic gather.  Tails with equal components reuse the equal sums.
//
// Orbit representatives: T0 <= T1 <= T2 and (T0, T1, T2) <= (~T2, ~T1, ~T0)
// lexicographically, i.e. T0 + T2 < 2^L - 1, or T0 + T2 = 2^L - 1 and
// T1 < 2^(L-1).  Tiles of 4 x 8 x 8 (T0, T1, T2) values, one per CTA; tiles
// with no representative are skipped whole.
#pragma once

#include <climits>

#include "lcs_common.h"
#include "sweep_generic.cuh"

namespace lcs {

// bit i of x (i < 21) moved to bit 3i
__device__ __forceinline__ unsigned long long spread3(unsigned long long x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// The sweep's indices in 32 bits: for h <= 11 every state of the stored half
// is below 2^(3h - 1) <= 2^32, and a tail string has L = h - 1 <= 10 bits.
// (h = 12 would hold 4 x 256 GiB.)
constexpr int kD3sMaxH = 11;

// bit i of x (i < 10) moved to bit 3i
__device__ __forceinline__ unsigned spread3_32(unsigned x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// the index of the tail tuple (a, b, c) from the spread strings; a string
// followed by one more letter c is (its spread << 3) | c
__device__ __forceinline__ unsigned d3s_tail32(unsigned sa, unsigned sb, unsigned sc) {
  return (sa << 2) | (sb << 1) | sc;
}

// two adjacent values at an even index (16-byte aligned)
template <bool CG>
__device__ __forceinline__ longlong2 d3s_ld2(const long long* v, unsigned long long y) {
  const longlong2* q = reinterpret_cast<const longlong2*>(v + y);
  if constexpr (CG)
    return __ldcg(q);
  else
    return __ldg(q);
}

__device__ __forceinline__ unsigned long long d3s_tail(unsigned long long a, unsigned long long b,
                                                       unsigned long long c) {
  return (spread3(a) << 2) | (spread3(b) << 1) | spread3(c);
}

struct D3sOrbit {
  unsigned long long T[3];  // the representative tau
  unsigned long long C[3];  // its complement ~tau
};

// tiles of 4 x 8 x 8 representatives; tile k = (I0 n1 + I1) n2 + I2
__device__ __forceinline__ void d3s_tile(unsigned long long k, int L, unsigned long long& I0, unsigned long long& I1,
                                         unsigned long long& I2) {
  const unsigned long long n12 = 1ull << (L - 3);
  I2 = k & (n12 - 1);
  I1 = (k >> (L - 3)) & (n12 - 1);
  I0 = k >> (2 * (L - 3));
}

// does tile (I0, I1, I2) hold a representative?
__device__ __forceinline__ bool d3s_tile_live(unsigned long long I0, unsigned long long I1, unsigned long long I2,
                                              unsigned long long M) {
  return 4 * I0 <= 8 * I1 + 7 && 8 * I1 <= 8 * I2 + 7 && 4 * I0 + 8 * I2 <= M;
}

// the representative of thread tid in tile (I0, I1, I2); false if none.  The
// thread's bits are T1_0, T0_0, T2_0, T1_1, T0_1, T2_1, T1_2, T2_2 (low
// first): the digit order of the addresses of A1(tau, 2).
__device__ __forceinline__ bool d3s_rep(unsigned long long I0, unsigned long long I1, unsigned long long I2,
                                        unsigned long long M, int L, unsigned tid, D3sOrbit& o) {
  const unsigned t0 = ((tid >> 1) & 1u) | (((tid >> 4) & 1u) << 1);
  const unsigned t1 = (tid & 1u) | (((tid >> 3) & 1u) << 1) | (((tid >> 6) & 1u) << 2);
  const unsigned t2 = ((tid >> 2) & 1u) | (((tid >> 5) & 1u) << 1) | (((tid >> 7) & 1u) << 2);
  const unsigned long long T0 = 4 * I0 + t0, T1 = 8 * I1 + t1, T2 = 8 * I2 + t2;
  if (T0 > T1 || T1 > T2) return false;
  if (T0 + T2 > M) return false;
  if (T0 + T2 == M && T1 >= (1ull << (L - 1))) return false;
  o.T[0] = T0, o.T[1] = T1, o.T[2] = T2;
  o.C[0] = M - T0, o.C[1] = M - T1, o.C[2] = M - T2;
  return true;
}

// the six sums of one tail X (A1 from v1, A2 from v2)
template <bool CG>
__device__ __forceinline__ void d3s_sums(const long long* v1, const long long* v2, const unsigned long long (&X)[3],
                                         long long (&A1)[3], long long (&A2)[3]) {
  const bool e01 = X[0] == X[1], e12 = X[1] == X[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const bool reuse = (k == 1 && e01) || (k == 2 && e12);
    if (reuse) {
      A1[k] = A1[k - 1];
      A2[k] = A2[k - 1];
      continue;
    }
    const unsigned long long o0 = X[k == 0 ? 1 : 0], o1 = X[k == 2 ? 1 : 2];
    // A1: strings 0 and 1 hold the other components with head 0, string 2 = X_k c
    const unsigned long long a1 = d3s_tail(o0, o1, X[k] << 1);
    const longlong2 p = d3s_ld2<CG>(v1, a1);
    A1[k] = p.x + p.y;
    // A2: string 0 = 0 X_k, strings 1 and 2 hold the others, each followed by a letter
    const unsigned long long a2 = d3s_tail(X[k], o0 << 1, o1 << 1);
    const longlong2 q0 = d3s_ld2<CG>(v2, a2), q1 = d3s_ld2<CG>(v2, a2 + 2);
    A2[k] = q0.x + q0.y + q1.x + q1.y;
  }
}

template <bool CG>
__device__ __forceinline__ long long d3s_block(const long long* v3, unsigned long long t) {
  const unsigned long long b = 8 * t;
  long long s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const longlong2 q = d3s_ld2<CG>(v3, b + 2 * i);
    s += q.x + q.y;
  }
  return s;
}

// f_mode 1 also advances one string while the other two keep different
// heads: B1(X, k, o) = sum over c of v_{t-1}[(0 X_o, 1 X_r, X_k c)], r the
// third index (string 0 keeps head 0, string 1 head 1).  For ~X the same sum
// is B1(X, k, r): complement every letter, then exchange strings 0 and 1.
template <bool CG>
__device__ __forceinline__ void d3s_b1(const long long* v1, const unsigned long long (&X)[3], int L,
                                       long long (&B1)[3][3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      if (o == k) {
        B1[k][o] = 0;
        continue;
      }
      const int r = 3 - k - o;
      const longlong2 q = d3s_ld2<CG>(v1, d3s_tail(X[o], (1ull << L) | X[r], X[k] << 1));
      B1[k][o] = q.x + q.y;
    }
}

// the six permutations of three components
__device__ __forceinline__ int d3s_perm(int p, int j) {
  // (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0)
  constexpr unsigned char P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  return P[p][j];
}

// the six sums of one side of an orbit pair from the spreads S of its tail
// X; e01 / e12: X_0 = X_1 / X_1 = X_2 (the equal sums are reused)
__device__ __forceinline__ void d3s_sums32(const long long* v1, const long long* v2, const unsigned (&S)[3], bool e01,
                                           bool e12, long long (&A1)[3], long long (&A2)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const bool reuse = (k == 1 && e01) || (k == 2 && e12);
    if (reuse) {
      A1[k] = A1[k - 1];
      A2[k] = A2[k - 1];
      continue;
    }
    const unsigned s0 = S[k == 0 ? 1 : 0], s1 = S[k == 2 ? 1 : 2];
    // A1: strings 0 and 1 hold the other components with head 0, string 2 = X_k c
    const longlong2 p = d3s_ld2<false>(v1, d3s_tail32(s0, s1, S[k] << 3));
    A1[k] = p.x + p.y;
    // A2: string 0 = 0 X_k, strings 1 and 2 hold the others, each followed by a letter
    const unsigned a2 = d3s_tail32(S[k], s0 << 3, s1 << 3);
    const longlong2 q0 = d3s_ld2<false>(v2, a2), q1 = d3s_ld2<false>(v2, a2 + 2);
    A2[k] = q0.x + q0.y + q1.x + q1.y;
  }
}

// which of the six permutations repeat an earlier one, for a tail whose
// components are ordered (X_0 <= X_1 <= X_2, or >= for the complement)
__device__ __forceinline__ unsigned d3s_dup_mask(bool e01, bool e12) {
  // X_0 = X_1: (1,0,2) (1,2,0) (2,1,0) repeat (0,1,2) (0,2,1) (2,0,1);
  // X_1 = X_2: (0,2,1) (2,0,1) (2,1,0) repeat (0,1,2) (1,0,2) (1,2,0)
  return e01 && e12 ? 0x3eu : e01 ? 0x2cu : e12 ? 0x32u : 0u;
}

// the stored outputs of one side of an orbit pair: the distinct permutations
// of its tail (spreads S) at the 4 stored heads.  A1s/A2s are this side's
// sums, A1o/A2o the complement side's; b1(k, o) is this side's B1 (f_mode 1).
template <bool INCR, bool FALL, class B1F>
__device__ __forceinline__ void d3s_emit_side(const SweepParams& p, unsigned nt, const unsigned (&S)[3], unsigned dup,
                                              const long long (&A1s)[3], const long long (&A2s)[3],
                                              const long long (&A1o)[3], const long long (&A2o)[3], B1F&& b1,
                                              long long B, long long& best_v, unsigned long long& best_x) {
  const long long e000 = p.one + (B >> 3);
  // f_mode 0: heads 001 and 010 (majority 0, minority string 2 resp. 1) take
  // m0 of the minority's component, heads 011 (majority 1, minority string 0) m1
  long long m0[3], m1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m0[k] = max(4 * A1s[k], 2 * A2o[k]) >> 3;
    m1[k] = max(4 * A1o[k], 2 * A2s[k]) >> 3;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if ((dup >> q) & 1u) continue;
    const int p0 = d3s_perm(q, 0), p1 = d3s_perm(q, 1), p2 = d3s_perm(q, 2);
    const unsigned x0 = d3s_tail32(S[p0], S[p1], S[p2]), x1 = nt + x0, x2 = 2 * nt + x0, x3 = 3 * nt + x0;
    long long v000, v001, v010, v011;
    if constexpr (!FALL) {
      v000 = e000;
      v001 = m0[p2];
      v010 = m0[p1];
      v011 = m1[p0];
    } else {
      // every non-empty advance set at the common denominator 8: one string
      // (4 x its pair sum), two strings (2 x the quad sum), all three (the
      // block, + 8 one when the heads agree)
      v000 = max(max(4 * max(max(A1s[0], A1s[1]), A1s[2]), 2 * max(max(A2s[0], A2s[1]), A2s[2])),
                 B + 8 * p.one) >> 3;
      v001 = max(max(4 * max(max(b1(p0, p1), b1(p1, p0)), A1s[p2]),
                     2 * max(max(A2s[p0], A2s[p1]), A2o[p2])), B) >> 3;
      v010 = max(max(4 * max(max(b1(p0, p2), b1(p2, p0)), A1s[p1]),
                     2 * max(max(A2s[p0], A2s[p2]), A2o[p1])), B) >> 3;
      v011 = max(max(4 * max(max(A1o[p0], b1(p1, p0)), b1(p2, p0)),
                     2 * max(max(A2s[p0], A2o[p1]), A2o[p2])), B) >> 3;
    }
    p.out[x0] = v000;
    p.out[x1] = v001;
    p.out[x2] = v010;
    p.out[x3] = v011;
    if constexpr (INCR) {
      const long long i0 = v000 - ld_vec<false>(p.prev[0] + x0);
      const long long i1 = v001 - ld_vec<false>(p.prev[0] + x1);
      const long long i2 = v010 - ld_vec<false>(p.prev[0] + x2);
      const long long i3 = v011 - ld_vec<false>(p.prev[0] + x3);
      if (red_better(i0, x0, best_v, best_x, p.r_mode)) best_v = i0, best_x = x0;
      if (red_better(i1, x1, best_v, best_x, p.r_mode)) best_v = i1, best_x = x1;
      if (red_better(i2, x2, best_v, best_x, p.r_mode)) best_v = i2, best_x = x2;
      if (red_better(i3, x3, best_v, best_x, p.r_mode)) best_v = i3, best_x = x3;
    }
  }
}

// W = u + 3R - F(u + 2R, u + R, u) at the 8 heads of tau: every class of
// equal values of the orbit pair has a member with tail tau.  (f_mode 1: at
// the 4 stored heads of tau and of ~tau, the same classes.)
template <bool FALL, bool CG>
__device__ __forceinline__ void d3s_check_orbit(const CheckParams& p, const D3sOrbit& o, int L, long long R,
                                                long long& best) {
  const unsigned long long nt = p.n_tail;
  const unsigned long long n_total = 8 * nt;
  long long A1t[3], A2t[3], A1c[3], A2c[3];
  d3s_sums<CG>(p.u, p.u, o.T, A1t, A2t);
  d3s_sums<CG>(p.u, p.u, o.C, A1c, A2c);
  const unsigned long long ty = d3s_tail(o.T[0], o.T[1], o.T[2]);
  const long long Bs = d3s_block<CG>(p.u, ty);
  if constexpr (FALL) {
    // one string advances: mean of u + 2R; two: mean of u + R; three: mean of u
    long long B1t[3][3];
    d3s_b1<CG>(p.u, o.T, L, B1t);
    const long long K3 = Bs >> 3;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const long long* A1s = side == 0 ? A1t : A1c;
      const long long* A2s = side == 0 ? A2t : A2c;
      const long long* A1o = side == 0 ? A1c : A1t;
      const long long* A2o = side == 0 ? A2c : A2t;
      auto b1 = [&](int k, int oo) { return side == 0 ? B1t[k][oo] : B1t[k][3 - k - oo]; };
      const unsigned long long t = side == 0 ? ty : d3s_tail(o.C[0], o.C[1], o.C[2]);
      const long long F[4] = {
          max(max((max(max(A1s[0], A1s[1]), A1s[2]) >> 1) + 2 * R, (max(max(A2s[0], A2s[1]), A2s[2]) >> 2) + R),
              K3 + p.one),
          max(max((max(max(b1(0, 1), b1(1, 0)), A1s[2]) >> 1) + 2 * R, (max(max(A2s[0], A2s[1]), A2o[2]) >> 2) + R),
              K3),
          max(max((max(max(b1(0, 2), b1(2, 0)), A1s[1]) >> 1) + 2 * R, (max(max(A2s[0], A2s[2]), A2o[1]) >> 2) + R),
              K3),
          max(max((max(max(A1o[0], b1(1, 0)), b1(2, 0)) >> 1) + 2 * R, (max(max(A2s[0], A2o[1]), A2o[2]) >> 2) + R),
              K3)};
#pragma unroll
      for (int H = 0; H < 4; ++H) best = max(best, ld_vec<CG>(p.u + (unsigned long long)H * nt + t) + 3 * R - F[H]);
    }
    return;
  }
  const long long eq = p.one + (Bs >> 3);  // all three advance: shift 0
#pragma unroll
  for (int H = 0; H < 8; ++H) {
    const int h0 = H >> 2, h1 = (H >> 1) & 1, h2 = H & 1;
    long long F;
    if (H == 0 || H == 7) {
      F = eq;
    } else {
      const int m = (h0 + h1 + h2) >= 2 ? 1 : 0;
      const int j = h0 != m ? 0 : (h1 != m ? 1 : 2);
      // one string advances: mean of u + 2R; two advance: mean of u + R
      const long long k1 = m == 0 ? A1t[j] : A1c[j];
      const long long k2 = m == 0 ? A2c[j] : A2t[j];
      F = max((k1 >> 1) + 2 * R, (k2 >> 2) + R);
    }
    const unsigned long long x = (unsigned long long)H * nt + ty;
    const long long u = ld_vec<CG>(p.u + (x < n_total / 2 ? x : n_total - 1 - x));
    best = max(best, u + 3 * R - F);
  }
}

// The sweep runs two threads per orbit pair: lanes 2i and 2i + 1 load the sums
// of tau and of ~tau (and half of the block, and of the f_mode 1 sums each),
// exchange them with one shuffle each, and write the outputs of their own
// side: half the dependent loads per thread and twice the threads of the
// one-thread form, which at (2, 3, 8) is about one wave of long threads.
// Tiles of 4 x 4 x 8 representatives (128 per CTA); the thread bits above
// the side bit are T1_0, T0_0, T2_0, T1_1, T0_1, T2_1, T2_2.  Indices are
// 32-bit (h <= 11); the complement's spreads are the representative's XOR
// the spread of 2^L - 1.
// Tile (I0, I1, I2) holds a representative iff I0 <= I1, I1 / 2 <= I2 and
// 4 I0 + 8 I2 <= 2^L - 1 (T0 <= T1, T1 <= T2, T0 + T2 <= 2^L - 1 at its
// smallest corner).  The sweep walks the box J0 < 2^max(L-3, 1), J1 < 2^(L-2),
// J2 < 2^(L-3) (J2 fastest) with I0 = J0, I1 = J0 + J1, I2 = I1 / 2 + J2: the
// first two conditions hold by construction, so about one tile in six is live
// instead of one in twelve.  Within each row (J0, J1) the offset J2 is rotated
// by 37 x the row index: a row's live tiles stay one contiguous run (one wrap
// at most), but no longer all sit at the row's start, where the same few of
// the grid's stride classes would take them (at h = 11 the busiest CTA then
// has 1.39 x the mean number of live tiles; rotated, 1.01 x).
__device__ __forceinline__ bool d3s2_tile(unsigned k, int L, unsigned M, unsigned& I0, unsigned& I1, unsigned& I2) {
  const unsigned row = k >> (L - 3);
  I0 = k >> (2 * L - 5);
  I1 = I0 + (row & ((1u << (L - 2)) - 1));
  I2 = (I1 >> 1) + ((k + 37u * row) & ((1u << (L - 3)) - 1));
  return I1 < (1u << (L - 2)) && 4 * I0 + 8 * I2 <= M;
}

__device__ __forceinline__ bool d3s2_rep(unsigned I0, unsigned I1, unsigned I2, unsigned M, int L, unsigned r,
                                         unsigned (&T)[3]) {
  const unsigned t1 = (r & 1u) | (((r >> 3) & 1u) << 1);
  const unsigned t0 = ((r >> 1) & 1u) | (((r >> 4) & 1u) << 1);
  const unsigned t2 = ((r >> 2) & 1u) | (((r >> 5) & 1u) << 1) | (((r >> 6) & 1u) << 2);
  T[0] = 4 * I0 + t0, T[1] = 4 * I1 + t1, T[2] = 8 * I2 + t2;
  if (T[0] > T[1] || T[1] > T[2]) return false;
  if (T[0] + T[2] > M) return false;
  if (T[0] + T[2] == M && T[1] >= (1u << (L - 1))) return false;
  return true;
}

template <bool INCR, bool FALL>
__global__ void __launch_bounds__(kBlock) sweep_d3s_kernel(SweepParams p) {
  const int L = p.h - 1;
  const unsigned M = (1u << L) - 1;
  const unsigned SM = spread3_32(M);
  const unsigned nt = 1u << (3 * L);
  const unsigned n_tiles = 1u << (max(L - 3, 1) + 2 * L - 5);
  const int side = threadIdx.x & 1;
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  for (unsigned k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    unsigned I0, I1, I2;
    if (!d3s2_tile(k, L, M, I0, I1, I2)) continue;  // the whole CTA skips it
    unsigned T[3];
    const bool ok = d3s2_rep(I0, I1, I2, M, L, threadIdx.x >> 1, T);  // the same for both lanes of a pair
    const unsigned ST[3] = {spread3_32(T[0]), spread3_32(T[1]), spread3_32(T[2])};
    const unsigned flip = side ? SM : 0u;
    const unsigned S[3] = {ST[0] ^ flip, ST[1] ^ flip, ST[2] ^ flip};  // this lane's side: tau or ~tau
    const bool e01 = T[0] == T[1], e12 = T[1] == T[2];
    long long A1m[3] = {0, 0, 0}, A2m[3] = {0, 0, 0}, Bm[3] = {0, 0, 0}, Bs = 0;
    if (ok) {
      d3s_sums32(p.prev[0], p.prev[1], S, e01, e12, A1m, A2m);
      if constexpr (FALL) {
        // B1(T, k, o) at tail(T_o, 1 T_r, T_k c): lane 0 takes (k, o) = (0, 1),
        // (0, 2), (1, 0); lane 1 (1, 2), (2, 0), (2, 1)
        const unsigned top = 1u << (3 * L + 1);
        const unsigned a0 = side ? d3s_tail32(ST[2], ST[0], ST[1] << 3) : d3s_tail32(ST[1], ST[2], ST[0] << 3);
        const unsigned a1 = side ? d3s_tail32(ST[0], ST[1], ST[2] << 3) : d3s_tail32(ST[2], ST[1], ST[0] << 3);
        const unsigned a2 = side ? d3s_tail32(ST[1], ST[0], ST[2] << 3) : d3s_tail32(ST[0], ST[2], ST[1] << 3);
        const longlong2 q0 = d3s_ld2<false>(p.prev[0], a0 | top), q1 = d3s_ld2<false>(p.prev[0], a1 | top),
                        q2 = d3s_ld2<false>(p.prev[0], a2 | top);
        Bm[0] = q0.x + q0.y, Bm[1] = q1.x + q1.y, Bm[2] = q2.x + q2.y;
      }
      const unsigned b = (d3s_tail32(ST[0], ST[1], ST[2]) << 3) + 4 * side;
      const longlong2 q0 = d3s_ld2<false>(p.prev[2], b), q1 = d3s_ld2<false>(p.prev[2], b + 2);
      Bs = q0.x + q0.y + q1.x + q1.y;
    }
    long long A1x[3], A2x[3], Bx[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      A1x[i] = __shfl_xor_sync(0xffffffffu, A1m[i], 1);
      A2x[i] = __shfl_xor_sync(0xffffffffu, A2m[i], 1);
      Bx[i] = FALL ? __shfl_xor_sync(0xffffffffu, Bm[i], 1) : 0;
    }
    const long long B = Bs + __shfl_xor_sync(0xffffffffu, Bs, 1);
    if (ok) {
      long long B1t[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      if constexpr (FALL) {
        // lane 0's three sums and lane 1's, whichever lane this is
        const long long l00 = side ? Bx[0] : Bm[0], l01 = side ? Bx[1] : Bm[1], l02 = side ? Bx[2] : Bm[2];
        const long long l10 = side ? Bm[0] : Bx[0], l11 = side ? Bm[1] : Bx[1], l12 = side ? Bm[2] : Bx[2];
        B1t[0][1] = l00, B1t[0][2] = l01, B1t[1][0] = l02;
        B1t[1][2] = l10, B1t[2][0] = l11, B1t[2][1] = l12;
      }
      d3s_emit_side<INCR, FALL>(
          p, nt, S, d3s_dup_mask(e01, e12), A1m, A2m, A1x, A2x,
          [&](int kk, int oo) { return side ? B1t[kk][3 - kk - oo] : B1t[kk][oo]; }, B, best_v, best_x);
    }
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

template <bool FALL>
__global__ void __launch_bounds__(kBlock) check_d3s_kernel(CheckParams p) {
  const int L = p.h - 1;
  const unsigned long long M = (1ull << L) - 1;
  const unsigned long long n_tiles = 1ull << (3 * L - 8);
  const long long R = p.R_from_state ? p.state->R : p.R;
  long long best = LLONG_MIN;
  for (unsigned long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
    unsigned long long I0, I1, I2;
    d3s_tile(k, L, I0, I1, I2);
    if (!d3s_tile_live(I0, I1, I2, M)) continue;
    D3sOrbit o;
    if (d3s_rep(I0, I1, I2, M, L, threadIdx.x, o)) d3s_check_orbit<FALL, false>(p, o, L, R, best);
  }
  block_reduce_max(best, p.partials);
}

// are the stored values invariant under the string permutations?  (the
// complement holds by construction of the storage; two transpositions
// generate the permutations)
template <int UNUSED = 0>
__global__ void perm_check_d3s_kernel(const long long* __restrict__ v, unsigned long long n_stored,
                                      unsigned long long n_total, DevState* st) {
  constexpr unsigned long long S0 = 0x4924924924924924ull;  // bits of string 0 (positions 3i + 2)
  constexpr unsigned long long S1 = S0 >> 1, S2 = S0 >> 2;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_stored;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    // exchange strings 0 and 1, and strings 1 and 2
    unsigned long long y = (x & S2) | ((x & S0) >> 1) | ((x & S1) << 1);
    unsigned long long z = (x & S0) | ((x & S1) >> 1) | ((x & S2) << 1);
    if (y >= n_stored) y = n_total - 1 - y;
    if (z >= n_stored) z = n_total - 1 - z;
    if (v[y] != v[x] || v[z] != v[x]) atomicExch((unsigned long long*)&st->swap_bad, 1ull);
  }
}

template <bool FALL>
void launch_sweep_d3s(const SweepParams& p, int grid, cudaStream_t s) {
  if (p.incr)
    sweep_d3s_kernel<true, FALL><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_d3s_kernel<false, FALL><<<grid, kBlock, 0, s>>>(p);
}

template <bool FALL>
void launch_check_d3s(const CheckParams& p, int grid, cudaStream_t s) {
  check_d3s_kernel<FALL><<<grid, kBlock, 0, s>>>(p);
}

template <bool FALL>
KernelSet make_d3s_set() {
  KernelSet k{};
  k.sigma = 2;
  k.d = 3;
  k.f_mode = FALL ? 1 : 0;
  k.sym = 4;
  k.sweep = &launch_sweep_d3s<FALL>;
  k.check = &launch_check_d3s<FALL>;
  k.sweep_fn = (const void*)&sweep_d3s_kernel<false, FALL>;  // the plain sweep sizes the grid
  k.check_fn = (const void*)&check_d3s_kernel<FALL>;
  k.tails_per_thread = 12;
  // per orbit pair (12 tails, 48 stored states): 12 + 24 + 8 values read (f_mode 1:
  // 12 more), 48 written: 15.3 B (17.3 B) per stored state, counted as 15 (17)
  k.sweep_algo_bytes = FALL ? 17 : 15;
  k.check_algo_bytes = 8;
  return k;
}

}  // namespace lcs
