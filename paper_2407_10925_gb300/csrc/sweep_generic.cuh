// sweep_generic.cuh -- the feasible-triplet sweep and check for a compile-time
// alphabet size SIG and number of strings D (Heineman et al., arXiv
// 2407.10925, section 2.1).
//
// State index (paper section 3.2, generalised to base SIG): the digit of string
// j at position p (0 = head) has weight SIG^(D (h-1-p) + (D-1-j)).  Writing the
// index as x = H * n_tail + t splits it into the head tuple H (the D head
// digits, string 0 most significant) and the tail tuple t (every other digit).
//
// One thread owns one tail tuple t and computes every head tuple H that shares
// it.  All states with tail t read the same values:
//   * advancing every string (Eq. ineq1, and Eq. ineq2 when some letter is no
//     string's head) reads the SIG^D contiguous values t*SIG^D + c of v_D;
//   * advancing the set N of strings whose head differs from z (Algorithm 1)
//     reads SIG^|N| values of v_|N| that depend on (N, z) and t only.
// So each thread loads the all-advance block once and one partial sum per
// (N, z), then fans them out to the SIG^D head tuples in registers.  Sums are
// exact in int64; each candidate is scaled to the common denominator SIG^D so
// the max (Eq. ineq3) compares integers and one floor division per state
// produces the mean rounded down.
//
// Complement symmetry (paper section 3.3, Eq. impl:comp_eq; SIG = 2 only):
// complementing every string maps index x to N-1-x and leaves v unchanged.
// With SYM the buffers hold only x < N/2 (first string starts with 0); a thread
// owns the tail pair (t, n_tail-1-t) with t < n_tail/2 and computes the heads
// with H_0 = 0 for both; loads that fall in the upper half are reflected.  In
// exact integer arithmetic the result equals the full computation bit for bit.
#pragma once

#include <climits>
#include <utility>

#include "lcs_common.h"

namespace lcs {

__host__ __device__ constexpr unsigned long long cpow(int b, int e) {
  return e == 0 ? 1ull : (unsigned long long)b * cpow(b, e - 1);
}
__host__ __device__ constexpr int cpopc(unsigned m) { return m == 0 ? 0 : (int)(m & 1u) + cpopc(m >> 1); }
__host__ __device__ constexpr int cctz(unsigned long long v) { return (v & 1ull) ? 0 : 1 + cctz(v >> 1); }

template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// floor(a / C) for a compile-time C > 0
template <unsigned long long C>
__device__ __forceinline__ long long floor_div(long long a) {
  if constexpr ((C & (C - 1)) == 0) {
    return a >> cctz(C);  // arithmetic shift rounds toward -infinity
  } else {
    long long q = a / (long long)C;
    return q - ((a - q * (long long)C) < 0);
  }
}

// Loads of iterate vectors.  Standalone launches read vectors that no thread
// of the launch writes: the read-only path.  A persistent launch that runs
// several iterations reads what other CTAs wrote earlier in the same launch:
// L2-coherent loads that bypass L1 (CG = true).
template <bool CG = false>
__device__ __forceinline__ long long ld_vec(const long long* p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return __ldg(p);
}
__device__ __forceinline__ long long ld_stream(const long long* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Reductions.  The increment reduction keeps (value, index): the minimum (or
// maximum with r_mode = 1) value, ties broken by the smallest index.  The check
// reduction keeps the maximum value.

__device__ __forceinline__ bool red_better(long long v, unsigned long long x, long long bv, unsigned long long bx,
                                           int r_mode) {
  if (v != bv) return r_mode ? (v > bv) : (v < bv);
  return x < bx;
}

__device__ __forceinline__ void block_reduce_arg_to(long long& v, unsigned long long& x, int r_mode, RedPartial* slot) {
  __shared__ long long sv[kBlock / 32];
  __shared__ unsigned long long sx[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    unsigned long long ox = __shfl_xor_sync(0xffffffffu, x, o);
    if (red_better(ov, ox, v, x, r_mode)) v = ov, x = ox;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sv[w] = v, sx[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = l < nw ? sv[l] : sv[0];
    x = l < nw ? sx[l] : sx[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long ov = __shfl_xor_sync(0xffffffffu, v, o);
      unsigned long long ox = __shfl_xor_sync(0xffffffffu, x, o);
      if (red_better(ov, ox, v, x, r_mode)) v = ov, x = ox;
    }
    if (l == 0) *slot = RedPartial{v, x};
  }
  __syncthreads();  // the shared scratch may be reused by a following reduction
}

__device__ __forceinline__ void block_reduce_arg(long long& v, unsigned long long& x, int r_mode, RedPartial* out) {
  block_reduce_arg_to(v, x, r_mode, out + blockIdx.x);
}

__device__ __forceinline__ void block_reduce_max_to(long long v, RedPartial* slot) {
  __shared__ long long sv[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sv[w] = v;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = l < nw ? sv[l] : sv[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) *slot = RedPartial{v, 0ull};
  }
  __syncthreads();
}

__device__ __forceinline__ void block_reduce_max(long long v, RedPartial* out) { block_reduce_max_to(v, out + blockIdx.x); }

// ---------------------------------------------------------------------------
// Index algebra for compile-time (SIG, D).

template <int SIG, int D>
struct Geo {
  static constexpr unsigned long long SD = cpow(SIG, D);        // head tuples
  static constexpr unsigned FULL = (1u << D) - 1;               // every string advanced
  static constexpr int NSETS = (int)FULL - 1;                   // proper non-empty advance sets
  static constexpr int NP = NSETS * SIG;                        // partial sums (N, z)
  static constexpr int HW = (int)cpow(SIG, D - 1);              // f_mode 1: head slots per advance set
  static constexpr int NPA = (NSETS > 0 ? NSETS : 1) * HW;      // f_mode 1: partial sums (N, heads outside N)
  static constexpr bool POW2 = (SIG & (SIG - 1)) == 0;
  static constexpr int BITS = POW2 ? cctz(SIG) : 0;

  // weight of string j's digit at the last position: SIG^(D-1-j)
  __host__ __device__ static constexpr unsigned long long wlast(int j) { return cpow(SIG, D - 1 - j); }

  // head digit of string j in head tuple H
  __host__ __device__ static constexpr int head(int H, int j) { return (int)((H / cpow(SIG, D - 1 - j)) % SIG); }

  // N_z of head tuple H as a bit mask (bit j set: string j's head differs from z)
  __host__ __device__ static constexpr unsigned nz(int H, int z) {
    unsigned m = 0;
    for (int j = 0; j < D; ++j)
      if (head(H, j) != z) m |= 1u << j;
    return m;
  }

  __host__ __device__ static constexpr bool all_equal(int H) {
    for (int j = 1; j < D; ++j)
      if (head(H, j) != head(H, 0)) return false;
    return true;
  }

  // offset of the cc-th appended tuple for the advance set N: the digits of cc
  // (first string of N most significant) go to the last position of the
  // strings in N
  __host__ __device__ static constexpr unsigned long long coff(unsigned N, int cc) {
    unsigned long long off = 0;
    for (int j = D - 1; j >= 0; --j)
      if (N >> j & 1u) {
        off += (unsigned long long)(cc % SIG) * wlast(j);
        cc /= SIG;
      }
    return off;
  }

  // the heads of the strings outside N in head tuple H, first such string most
  // significant (f_mode 1)
  __host__ __device__ static constexpr int heads_outside(int H, unsigned N) {
    int hc = 0;
    for (int j = 0; j < D; ++j)
      if (!(N >> j & 1u)) hc = hc * SIG + head(H, j);
    return hc;
  }

  // pattern of string j's digits inside a tail index (power-of-two SIG)
  __host__ __device__ static constexpr unsigned long long pattern(int j) {
    unsigned long long m = 0;
    for (int q = 0; (q + 1) * D * BITS <= 64; ++q)
      m |= ((1ull << BITS) - 1) << ((unsigned long long)(q * D + (D - 1 - j)) * BITS);
    return m;
  }
};

// S[j] = the digits of string j inside tail index t, kept in place.
template <int SIG, int D>
__device__ __forceinline__ void tail_fields(unsigned long long t, int h, unsigned long long (&S)[D]) {
  using G = Geo<SIG, D>;
  if constexpr (G::POW2) {
#pragma unroll
    for (int j = 0; j < D; ++j) S[j] = t & G::pattern(j);
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) S[j] = 0;
    unsigned long long rem = t, w = 1;
    for (int q = 0; q + 1 < h; ++q) {
      const unsigned long long dq = rem % G::SD;
      rem /= G::SD;
#pragma unroll
      for (int j = 0; j < D; ++j) S[j] += ((dq / G::wlast(j)) % SIG) * G::wlast(j) * w;
      w *= G::SD;
    }
  }
}

// Sum of v_|N| over the SIG^|N| states reached from tail fields S by advancing
// the strings of N (appending every tuple of letters) while the others keep
// head Z.  REFLECT: the addresses lie in the upper half and are read through
// the complement symmetry (only with SYM).
template <int SIG, int D, unsigned N, int Z, bool REFLECT, bool CG = false>
__device__ __forceinline__ long long partial_sum(const long long* const* prev, const unsigned long long (&S)[D],
                                                 unsigned long long n_tail, unsigned long long n_total) {
  using G = Geo<SIG, D>;
  constexpr int K = cpopc(N);
  const long long* v = prev[K - 1];
  unsigned long long base = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (N >> j & 1u)
      base += S[j] * G::SD;
    else
      base += S[j] + (unsigned long long)Z * n_tail * G::wlast(j);
  }
  long long acc = 0;
  static_for<0, (int)cpow(SIG, K)>([&](auto cc) {
    constexpr unsigned long long off = G::coff(N, decltype(cc)::value);
    const unsigned long long y = base + off;
    acc += ld_vec<CG>(v + (REFLECT ? (n_total - 1 - y) : y));
  });
  return acc;
}

// As partial_sum, but the strings outside N keep arbitrary heads: HC lists
// them (the head digit of the k-th string outside N, string order, as a
// base-SIG number with the first such string most significant).
template <int SIG, int D, unsigned N, int HC, bool REFLECT, bool CG>
__device__ __forceinline__ long long partial_sum_heads(const long long* const* prev, const unsigned long long (&S)[D],
                                                       unsigned long long n_tail, unsigned long long n_total) {
  using G = Geo<SIG, D>;
  constexpr int K = cpopc(N);
  const long long* v = prev[K - 1];
  unsigned long long base = 0;
  int hc = HC;
#pragma unroll
  for (int j = D - 1; j >= 0; --j) {
    if (N >> j & 1u) {
      base += S[j] * G::SD;
    } else {
      base += S[j] + (unsigned long long)(hc % SIG) * n_tail * G::wlast(j);
      hc /= SIG;
    }
  }
  long long acc = 0;
  static_for<0, (int)cpow(SIG, K)>([&](auto cc) {
    constexpr unsigned long long off = G::coff(N, decltype(cc)::value);
    const unsigned long long y = base + off;
    acc += ld_vec<CG>(v + (REFLECT ? (n_total - 1 - y) : y));
  });
  return acc;
}

// f_mode = 1: one partial sum per (proper non-empty N, heads outside N);
// index (N - 1) * SIG^(D-1) + HC.  With SYM only heads with H_0 = 0 are
// computed, so sets without string 0 need HC with string 0's head 0.
template <int SIG, int D, bool SYM, bool UPPER, bool CG>
__device__ __forceinline__ void all_partials_fall(const long long* const* prev, const unsigned long long (&S)[D],
                                                  unsigned long long n_tail, unsigned long long n_total,
                                                  long long (&P)[Geo<SIG, D>::NPA]) {
  using G = Geo<SIG, D>;
  constexpr int W = G::HW;
  static_for<0, G::NSETS * W>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr unsigned N = (unsigned)(i / W) + 1;
    constexpr int HC = i % W;
    constexpr int K = cpopc(N);
    if constexpr (HC >= (int)cpow(SIG, D - K)) {
      P[i] = 0;  // fewer strings outside N than the slot allows
    } else {
      constexpr bool has0 = (N & 1u) != 0;
      // string 0 outside N: its head is HC's leading digit
      constexpr int head0 = has0 ? 0 : (int)(HC / cpow(SIG, D - K - 1));
      if constexpr (SYM && !has0 && head0 != 0) {
        P[i] = 0;  // only heads with H_0 = 0 are stored
      } else {
        P[i] = partial_sum_heads<SIG, D, N, HC, SYM && UPPER && has0, CG>(prev, S, n_tail, n_total);
      }
    }
  });
}

// f_mode = 1 value of head tuple H: the max over every non-empty advance set;
// the full set carries the +1 when all heads agree
template <int SIG, int D, int H>
__device__ __forceinline__ long long state_value_fall(
    long long s_all, const long long (&P)[Geo<SIG, D>::NPA],
    long long one) {
  using G = Geo<SIG, D>;
  constexpr int W = G::HW;
  long long key = G::all_equal(H) ? s_all + (long long)G::SD * one : s_all;
  static_for<1, (int)G::FULL>([&](auto Nc) {
    constexpr unsigned N = (unsigned)decltype(Nc)::value;
    constexpr int i = (int)(N - 1) * W + G::heads_outside(H, N);
    key = max(key, P[i] * (long long)cpow(SIG, D - cpopc(N)));
  });
  return floor_div<G::SD>(key);
}

template <int SIG, int D, int H>
__device__ __forceinline__ long long state_w_fall(
    long long u, long long s_all,
    const long long (&P)[Geo<SIG, D>::NPA], long long one,
    long long R) {
  using G = Geo<SIG, D>;
  constexpr int W = G::HW;
  long long best = floor_div<G::SD>(s_all) + (G::all_equal(H) ? one : 0);
  static_for<1, (int)G::FULL>([&](auto Nc) {
    constexpr unsigned N = (unsigned)decltype(Nc)::value;
    constexpr int K = cpopc(N);
    constexpr int i = (int)(N - 1) * W + G::heads_outside(H, N);
    best = max(best, floor_div<cpow(SIG, K)>(P[i]) + (long long)(D - K) * R);
  });
  return u + (long long)D * R - best;
}

// Every partial sum a head tuple of the thread may need.  With SYM only heads
// with H_0 = 0 are computed: then z = 0 goes with sets N without string 0 and
// z = 1 with sets containing it; UPPER marks the reflected tail of the pair.
template <int SIG, int D, bool SYM, bool UPPER, bool CG = false>
__device__ __forceinline__ void all_partials(const long long* const* prev, const unsigned long long (&S)[D],
                                             unsigned long long n_tail, unsigned long long n_total,
                                             long long (&P)[Geo<SIG, D>::NP > 0 ? Geo<SIG, D>::NP : 1]) {
  using G = Geo<SIG, D>;
  static_for<0, G::NP>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr unsigned N = (unsigned)(i / SIG) + 1;
    constexpr int Z = i % SIG;
    if constexpr (!SYM) {
      P[i] = partial_sum<SIG, D, N, Z, false, CG>(prev, S, n_tail, n_total);
    } else {
      constexpr bool has0 = (N & 1u) != 0;
      if constexpr ((Z == 0 && !has0) || (Z == 1 && has0)) {
        // sets without string 0 keep its head z = 0 (lower half); sets with it
        // take string 0's second digit, which is 1 exactly for the upper tail
        P[i] = partial_sum<SIG, D, N, Z, UPPER && has0, CG>(prev, S, n_tail, n_total);
      } else {
        P[i] = 0;
      }
    }
  });
}

// The new value of head tuple H (fixed point), from the all-advance sum and the
// partial sums (Eq. ineq3 with Algorithm 1's F_z; means rounded down).
template <int SIG, int D, int H>
__device__ __forceinline__ long long state_value(long long s_all, const long long (&P)[Geo<SIG, D>::NP > 0 ? Geo<SIG, D>::NP : 1],
                                                 long long one) {
  using G = Geo<SIG, D>;
  if constexpr (G::all_equal(H)) {
    return one + floor_div<G::SD>(s_all);
  } else {
    long long key = LLONG_MIN;
    static_for<0, SIG>([&](auto zc) {
      constexpr int z = decltype(zc)::value;
      constexpr unsigned N = G::nz(H, z);
      if constexpr (N == G::FULL) {
        key = max(key, s_all);
      } else {
        constexpr int i = (int)(N - 1) * SIG + z;
        constexpr unsigned long long scale = cpow(SIG, D - cpopc(N));
        key = max(key, P[i] * (long long)scale);
      }
    });
    return floor_div<G::SD>(key);
  }
}

// The check's W at head tuple H: u + dR - F(u + (d-1)R, .., u).  Each candidate
// is its own mean rounded down plus (d - |N|) R (translation invariance of F,
// exact in fixed point).
template <int SIG, int D, int H>
__device__ __forceinline__ long long state_w(long long u, long long s_all,
                                             const long long (&P)[Geo<SIG, D>::NP > 0 ? Geo<SIG, D>::NP : 1],
                                             long long one, long long R) {
  using G = Geo<SIG, D>;
  long long F;
  if constexpr (G::all_equal(H)) {
    F = one + floor_div<G::SD>(s_all);
  } else {
    long long best = LLONG_MIN;
    static_for<0, SIG>([&](auto zc) {
      constexpr int z = decltype(zc)::value;
      constexpr unsigned N = G::nz(H, z);
      long long cand;
      if constexpr (N == G::FULL) {
        cand = floor_div<G::SD>(s_all);
      } else {
        constexpr int i = (int)(N - 1) * SIG + z;
        constexpr int K = cpopc(N);
        cand = floor_div<cpow(SIG, K)>(P[i]) + (long long)(D - K) * R;
      }
      best = max(best, cand);
    });
    F = best;
  }
  return u + (long long)D * R - F;
}

// ---------------------------------------------------------------------------
// Kernels.

// f_mode = 1 bodies (every non-empty advance set; an extension the paper does
// not use, see the oracle's reading R9)
template <int SIG, int D, bool SYM, bool INCR, bool CG>
__device__ __forceinline__ void generic_sweep_thread_fall(const SweepParams& p, unsigned long long t, long long& best_v,
                                                          unsigned long long& best_x) {
  using G = Geo<SIG, D>;
  constexpr int NPA = G::NPA;
  const unsigned long long nt = p.n_tail;
  const unsigned long long n_total = nt * G::SD;
  unsigned long long S[D];
  tail_fields<SIG, D>(t, p.h, S);
  long long s_all = 0;
  {
    const long long* vd = p.prev[D - 1];
    const unsigned long long b = t * G::SD;
    static_for<0, (int)G::SD>([&](auto c) { s_all += ld_vec<CG>(vd + b + decltype(c)::value); });
  }
  long long P[NPA];
  all_partials_fall<SIG, D, SYM, false, CG>(p.prev, S, nt, n_total, P);
  auto emit = [&](auto Hc, unsigned long long tt, const auto& PP) {
    constexpr int H = decltype(Hc)::value;
    const long long val = state_value_fall<SIG, D, H>(s_all, PP, p.one);
    const unsigned long long x = (unsigned long long)H * nt + tt;
    if constexpr (INCR) {
      const long long inc = val - ld_vec<CG>(p.prev[0] + x);
      if (red_better(inc, x, best_v, best_x, p.r_mode)) best_v = inc, best_x = x;
    }
    p.out[x] = val;
  };
  constexpr int NH = SYM ? (int)(G::SD / SIG) : (int)G::SD;
  static_for<0, NH>([&](auto Hc) { emit(Hc, t, P); });
  if constexpr (SYM) {
    const unsigned long long tu = nt - 1 - t;
    unsigned long long SU[D];
    tail_fields<SIG, D>(tu, p.h, SU);
    long long PU[NPA];
    all_partials_fall<SIG, D, true, true, CG>(p.prev, SU, nt, n_total, PU);
    static_for<0, NH>([&](auto Hc) { emit(Hc, tu, PU); });
  }
}

template <int SIG, int D, bool SYM, bool CG>
__device__ __forceinline__ void generic_check_thread_fall(const CheckParams& p, long long R, unsigned long long t,
                                                          long long& best) {
  using G = Geo<SIG, D>;
  constexpr int NPA = G::NPA;
  const unsigned long long nt = p.n_tail;
  const unsigned long long n_total = nt * G::SD;
  const long long* prev[kMaxD];
#pragma unroll
  for (int k = 0; k < D; ++k) prev[k] = p.u;
  unsigned long long S[D];
  tail_fields<SIG, D>(t, p.h, S);
  long long s_all = 0;
  {
    const unsigned long long b = t * G::SD;
    static_for<0, (int)G::SD>([&](auto c) { s_all += ld_vec<CG>(p.u + b + decltype(c)::value); });
  }
  long long P[NPA];
  all_partials_fall<SIG, D, SYM, false, CG>(prev, S, nt, n_total, P);
  constexpr int NH = SYM ? (int)(G::SD / SIG) : (int)G::SD;
  static_for<0, NH>([&](auto Hc) {
    constexpr int H = decltype(Hc)::value;
    const unsigned long long x = (unsigned long long)H * nt + t;
    best = max(best, state_w_fall<SIG, D, H>(ld_vec<CG>(p.u + x), s_all, P, p.one, R));
  });
  if constexpr (SYM) {
    const unsigned long long tu = nt - 1 - t;
    unsigned long long SU[D];
    tail_fields<SIG, D>(tu, p.h, SU);
    long long PU[NPA];
    all_partials_fall<SIG, D, true, true, CG>(prev, SU, nt, n_total, PU);
    static_for<0, NH>([&](auto Hc) {
      constexpr int H = decltype(Hc)::value;
      const unsigned long long x = (unsigned long long)H * nt + tu;
      best = max(best, state_w_fall<SIG, D, H>(ld_vec<CG>(p.u + x), s_all, PU, p.one, R));
    });
  }
}

// One thread's share of a sweep: tail tuple t (with SYM also its complement)
// and every head tuple stored for it.  INCR folds the increment of each state
// into (best_v, best_x).
template <int SIG, int D, bool SYM, bool INCR, bool CG = false, bool FALL = false>
__device__ __forceinline__ void generic_sweep_thread(const SweepParams& p, unsigned long long t, long long& best_v,
                                                     unsigned long long& best_x) {
  if constexpr (FALL) {
    generic_sweep_thread_fall<SIG, D, SYM, INCR, CG>(p, t, best_v, best_x);
    return;
  }
  using G = Geo<SIG, D>;
  const unsigned long long nt = p.n_tail;
  const unsigned long long n_total = nt * G::SD;
  unsigned long long S[D];
  tail_fields<SIG, D>(t, p.h, S);
  long long s_all = 0;
  {
    const long long* vd = p.prev[D - 1];
    const unsigned long long b = t * G::SD;
    static_for<0, (int)G::SD>([&](auto c) { s_all += ld_vec<CG>(vd + b + decltype(c)::value); });
  }
  long long P[G::NP > 0 ? G::NP : 1];
  all_partials<SIG, D, SYM, false, CG>(p.prev, S, nt, n_total, P);

  auto emit = [&](auto Hc, unsigned long long tt, const long long(&PP)[G::NP > 0 ? G::NP : 1]) {
    constexpr int H = decltype(Hc)::value;
    const long long val = state_value<SIG, D, H>(s_all, PP, p.one);
    const unsigned long long x = (unsigned long long)H * nt + tt;
    if constexpr (INCR) {
      const long long inc = val - ld_vec<CG>(p.prev[0] + x);
      if (red_better(inc, x, best_v, best_x, p.r_mode)) best_v = inc, best_x = x;
    }
    p.out[x] = val;
  };
  constexpr int NH = SYM ? (int)(G::SD / SIG) : (int)G::SD;  // SYM: heads with H_0 = 0
  static_for<0, NH>([&](auto Hc) { emit(Hc, t, P); });
  if constexpr (SYM) {
    const unsigned long long tu = nt - 1 - t;  // the complementary tail
    unsigned long long SU[D];
    tail_fields<SIG, D>(tu, p.h, SU);
    long long PU[G::NP > 0 ? G::NP : 1];
    all_partials<SIG, D, true, true, CG>(p.prev, SU, nt, n_total, PU);
    // equal heads of the upper tail read the reflection of t's block: same sum
    static_for<0, NH>([&](auto Hc) { emit(Hc, tu, PU); });
  }
}

// One thread's share of a check: max of W over the states it owns.
template <int SIG, int D, bool SYM, bool CG = false, bool FALL = false>
__device__ __forceinline__ void generic_check_thread(const CheckParams& p, long long R, unsigned long long t,
                                                     long long& best) {
  if constexpr (FALL) {
    generic_check_thread_fall<SIG, D, SYM, CG>(p, R, t, best);
    return;
  }
  using G = Geo<SIG, D>;
  const unsigned long long nt = p.n_tail;
  const unsigned long long n_total = nt * G::SD;
  const long long* prev[kMaxD];
#pragma unroll
  for (int k = 0; k < D; ++k) prev[k] = p.u;
  unsigned long long S[D];
  tail_fields<SIG, D>(t, p.h, S);
  long long s_all = 0;
  {
    const unsigned long long b = t * G::SD;
    static_for<0, (int)G::SD>([&](auto c) { s_all += ld_vec<CG>(p.u + b + decltype(c)::value); });
  }
  long long P[G::NP > 0 ? G::NP : 1];
  all_partials<SIG, D, SYM, false, CG>(prev, S, nt, n_total, P);
  constexpr int NH = SYM ? (int)(G::SD / SIG) : (int)G::SD;
  static_for<0, NH>([&](auto Hc) {
    constexpr int H = decltype(Hc)::value;
    const unsigned long long x = (unsigned long long)H * nt + t;
    best = max(best, state_w<SIG, D, H>(ld_vec<CG>(p.u + x), s_all, P, p.one, R));
  });
  if constexpr (SYM) {
    const unsigned long long tu = nt - 1 - t;
    unsigned long long SU[D];
    tail_fields<SIG, D>(tu, p.h, SU);
    long long PU[G::NP > 0 ? G::NP : 1];
    all_partials<SIG, D, true, true, CG>(prev, SU, nt, n_total, PU);
    static_for<0, NH>([&](auto Hc) {
      constexpr int H = decltype(Hc)::value;
      const unsigned long long x = (unsigned long long)H * nt + tu;
      best = max(best, state_w<SIG, D, H>(ld_vec<CG>(p.u + x), s_all, PU, p.one, R));
    });
  }
}

// threads a sweep or check of this kind runs: one per tail tuple (SYM: per pair)
template <int SIG, int D, bool SYM>
__host__ __device__ inline unsigned long long generic_threads(unsigned long long n_tail) {
  return SYM ? n_tail / 2 : n_tail;
}

template <int SIG, int D, bool SYM, bool INCR, bool FALL = false>
__global__ void __launch_bounds__(kBlock) sweep_generic_kernel(SweepParams p) {
  const unsigned long long n_threads = generic_threads<SIG, D, SYM>(p.n_tail);
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_threads;
       t += (unsigned long long)gridDim.x * blockDim.x)
    generic_sweep_thread<SIG, D, SYM, INCR, false, FALL>(p, t, best_v, best_x);
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

template <int SIG, int D, bool SYM, bool FALL = false>
__global__ void __launch_bounds__(kBlock) check_generic_kernel(CheckParams p) {
  const unsigned long long n_threads = generic_threads<SIG, D, SYM>(p.n_tail);
  const long long R = p.R_from_state ? p.state->R : p.R;
  long long best = LLONG_MIN;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_threads;
       t += (unsigned long long)gridDim.x * blockDim.x)
    generic_check_thread<SIG, D, SYM, false, FALL>(p, R, t, best);
  block_reduce_max(best, p.partials);
}

template <int SIG, int D, bool SYM, bool FALL = false>
void launch_sweep_generic(const SweepParams& p, int grid, cudaStream_t s) {
  if (p.incr)
    sweep_generic_kernel<SIG, D, SYM, true, FALL><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_generic_kernel<SIG, D, SYM, false, FALL><<<grid, kBlock, 0, s>>>(p);
}

template <int SIG, int D, bool SYM, bool FALL = false>
void launch_check_generic(const CheckParams& p, int grid, cudaStream_t s) {
  check_generic_kernel<SIG, D, SYM, FALL><<<grid, kBlock, 0, s>>>(p);
}

template <int SIG, int D, bool SYM, bool FALL = false>
KernelSet make_generic_set() {
  KernelSet k{};
  k.sigma = SIG;
  k.d = D;
  k.sym = SYM ? 1 : 0;
  k.f_mode = FALL ? 1 : 0;
  k.sweep = &launch_sweep_generic<SIG, D, SYM, FALL>;
  k.check = &launch_check_generic<SIG, D, SYM, FALL>;
  // the plain sweep sizes the grid: the fused-increment variant (one launch in
  // check_every) needs more registers, and its extra CTAs simply queue
  k.sweep_fn = (const void*)&sweep_generic_kernel<SIG, D, SYM, false, FALL>;
  k.check_fn = (const void*)&check_generic_kernel<SIG, D, SYM, FALL>;
  k.tails_per_thread = SYM ? 2 : 1;
  k.sweep_algo_bytes = 8 * (D + 1);
  k.check_algo_bytes = 8;
  return k;
}

}  // namespace lcs
