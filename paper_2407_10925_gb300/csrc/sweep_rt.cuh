// sweep_rt.cuh -- the sweep and check for every shape without a specialised
// kernel: d only known at run time (2 .. kMaxD), sigma a template parameter,
// full storage, the paper's F (f_mode 0).
//
// Algorithm 1 and Eq. ineq3 for a state with heads H and tail tuple t (the
// h - 1 non-head positions of the d strings): for every letter z whose set
// N_z = {j : H_j != z} of strings to advance is not empty, the candidate is
//   M(z, S) / sigma^|N|,   S = {j : H_j = z},  N = the other strings,
//   M(z, S) = sum over c in Sigma^|N| of v_{t-|N|}[state with string j = z t_j
//             for j in S and string j = t_j c_j for j in N],
// and v = [all heads equal] + max of the candidates, every mean rounded down.
// M depends on the heads only through (z, S), and M(z, {}) (every string
// advances) not on z.  One CTA takes one tail tuple at a time: it forms the
// table of every M(z, S) in shared memory, then its threads take the sigma^d
// head combinations and read their sigma candidates from the table.  An
// entry serves the (sigma - 1)^|N| head combinations with heads z on S and
// other letters on N.  Where the table would not fit (sigma = 2 with d >= 12,
// where no entry serves two states anyway) each thread forms its own
// candidates.  For sigma = 2 from d = kRtWarpD on, one warp takes one state
// instead (grid-stride over all states): its lanes split each candidate's
// 2^|N| terms, lane bits filling the five lowest offset bits and each lane
// walking the remaining ones as submasks, so a state's cost (2^#ones +
// 2^#zeros terms, from 2 2^(d/2) to 2^d) no longer decides a thread's, and an
// h = 1 sweep (one tail tuple) spreads over the whole GPU.
//
// Index arithmetic (the STATE INDEX of the interface): the tail tuple t is the
// low d (h-1) base-sigma digits of a state's index and the heads the top d, so
// state (H, t) is Hidx n_tail + t with Hidx = sum_j H_j sigma^(d-1-j).  With
// tp_j the digits of string j in t (at their weights in t), string j = z t_j
// contributes z n_tail sigma^(d-1-j) + tp_j, and string j = t_j c contributes
// sigma^d tp_j + c sigma^(d-1-j): advancing shifts its digits up one position.
#pragma once

#include <climits>

#include "lcs_common.h"
#include "sweep_generic.cuh"
#include "sweep_rtb.cuh"

namespace lcs {

constexpr int kRtTable = 6000;  // entries of the shared table (47 KiB; the static limit is 48 KiB)
constexpr int kRtWarpD = 9;     // sigma = 2: one warp per state from this d on
// one warp per tail tuple, each with a table of its own, when a table holds
// at most this many entries and there are enough tuples to fill the GPU
constexpr int kRtWarpTable = kRtTable / (kBlock / 32);
constexpr unsigned long long kRtWarpTails = 1ull << 13;

// one warp per tail tuple (host side: the same rule as the launch)
inline bool rt_warp_tails(int sigma, int d, unsigned long long n_tail) {
  return ((unsigned long long)sigma << d) <= (unsigned long long)kRtWarpTable && n_tail >= kRtWarpTails;
}

template <int SIG>
struct RtGeo {
  int d;
  unsigned full;                  // the set of all d strings
  unsigned long long sd;          // sigma^d head combinations
  unsigned long long n_tail;
  unsigned long long pw[kMaxD + 1];  // sigma^k
  bool table;                     // the table fits in shared memory
};

template <int SIG>
__device__ __forceinline__ RtGeo<SIG> rt_geo(unsigned long long n_stored, int h, unsigned long long n_tail) {
  RtGeo<SIG> g;
  int dh = 0;
  for (unsigned long long m = n_stored; m > 1; m /= SIG) ++dh;
  g.d = dh / h;
  g.full = (1u << g.d) - 1;
  g.pw[0] = 1;
  for (int k = 1; k <= kMaxD; ++k) g.pw[k] = g.pw[k - 1] * (k <= g.d ? SIG : 1);
  g.sd = g.pw[g.d];
  g.n_tail = n_tail;
  g.table = (unsigned long long)SIG << g.d <= (unsigned long long)kRtTable;
  return g;
}

// floor(a / m) for m > 0
__device__ __forceinline__ long long rt_floor_div(long long a, unsigned long long m) {
  const long long mm = (long long)m;
  long long q = a / mm;
  return q - ((a - q * mm) < 0);
}

// tp[j]: the digits of string j in tail tuple t
template <int SIG>
__device__ __forceinline__ void rt_tail_parts(const RtGeo<SIG>& g, int h, unsigned long long t,
                                              unsigned long long (&tp)[kMaxD]) {
  for (int j = 0; j < g.d; ++j) tp[j] = 0;
  unsigned long long w = 1;
  for (int q = 0; q < g.d * (h - 1); ++q) {
    tp[g.d - 1 - q % g.d] += (t % SIG) * w;
    t /= SIG;
    w *= SIG;
  }
}

// the terms m0 .. m1-1 of M(z, S) from vector v: strings in S keep head z and
// their tail, the others advance and take every letter c; term m is the c
// whose base-sigma digits, least significant first, are the letters of the
// advanced strings from the last one back.  The addresses do not depend on
// the loaded values, so the walk forms four of them before it loads: four
// loads in flight per thread instead of one.
template <int SIG>
__device__ __forceinline__ long long rt_sum_range(const RtGeo<SIG>& g, const unsigned long long (&tp)[kMaxD], int z,
                                                  unsigned S, const long long* __restrict__ v, unsigned long long m0,
                                                  unsigned long long m1) {
  unsigned long long base = 0;
  unsigned long long w[kMaxD];
  int n = 0;
  for (int j = g.d - 1; j >= 0; --j) {
    if ((S >> j) & 1u) {
      base += (unsigned long long)z * g.n_tail * g.pw[g.d - 1 - j] + tp[j];
    } else {
      base += g.sd * tp[j];
      w[n++] = g.pw[g.d - 1 - j];
    }
  }
  // the counter's digits at term m0
  int c[kMaxD];
  unsigned long long off = 0, m = m0;
  for (int i = 0; i < n; ++i) {
    c[i] = (int)(m % SIG);
    m /= SIG;
    off += (unsigned long long)c[i] * w[i];
  }
  const long long* vb = v + base;
  if (n >= 2 && SIG <= 8 && m0 % SIG == 0 && m1 % SIG == 0) {
    // whole runs of the lowest digit: SIG loads at off + c0 w[0] per step of
    // the higher digits, two steps at a time -- 2 SIG loads in flight
    auto step_hi = [&]() {
      for (int i = 1; i < n; ++i) {
        if (++c[i] < SIG) {
          off += w[i];
          return;
        }
        c[i] = 0;
        off -= (unsigned long long)(SIG - 1) * w[i];
      }
    };
    const unsigned long long w0 = w[0];
    long long acc[SIG];
#pragma unroll
    for (int j = 0; j < SIG; ++j) acc[j] = 0;
    unsigned long long t = m0;
    for (; t + 2 * SIG <= m1; t += 2 * SIG) {
      const unsigned long long oa = off;
      step_hi();
      const unsigned long long ob = off;
      step_hi();
      long long la[SIG], lb[SIG];
#pragma unroll
      for (int j = 0; j < SIG; ++j) la[j] = ld_vec<false>(vb + oa + j * w0);
#pragma unroll
      for (int j = 0; j < SIG; ++j) lb[j] = ld_vec<false>(vb + ob + j * w0);
#pragma unroll
      for (int j = 0; j < SIG; ++j) acc[j] += la[j] + lb[j];
    }
    if (t < m1) {
#pragma unroll
      for (int j = 0; j < SIG; ++j) acc[j] += ld_vec<false>(vb + off + j * w0);
    }
    long long sum = 0;
#pragma unroll
    for (int j = 0; j < SIG; ++j) sum += acc[j];
    return sum;
  }
  auto step = [&]() {
    for (int i = 0; i < n; ++i) {
      if (++c[i] < SIG) {
        off += w[i];
        return;
      }
      c[i] = 0;
      off -= (unsigned long long)(SIG - 1) * w[i];
    }
  };
  long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  unsigned long long t = m0;
  for (; t + 4 <= m1; t += 4) {
    const unsigned long long o0 = off;
    step();
    const unsigned long long o1 = off;
    step();
    const unsigned long long o2 = off;
    step();
    const unsigned long long o3 = off;
    step();
    s0 += ld_vec<false>(vb + o0);
    s1 += ld_vec<false>(vb + o1);
    s2 += ld_vec<false>(vb + o2);
    s3 += ld_vec<false>(vb + o3);
  }
  for (; t < m1; ++t) {
    s0 += ld_vec<false>(vb + off);
    step();
  }
  return (s0 + s1) + (s2 + s3);
}

// every term of M(z, S)
template <int SIG>
__device__ __forceinline__ long long rt_sum(const RtGeo<SIG>& g, const unsigned long long (&tp)[kMaxD], int z,
                                            unsigned S, const long long* __restrict__ v) {
  return rt_sum_range<SIG>(g, tp, z, S, v, 0, g.pw[g.d - __popc(S)]);
}

// the table entry of (z, S): S = {} is shared by every z
__device__ __forceinline__ int rt_entry(int z, unsigned S, int d) { return S ? (z << d) | (int)S : 0; }

// the terms one of `parts` threads or lanes sums: for sigma <= 8 a whole
// number of runs of the lowest digit (terms = sigma^k is a multiple of sigma)
template <int SIG>
__device__ __forceinline__ unsigned long long rt_chunk(unsigned long long terms, unsigned parts) {
  const unsigned long long per = (terms + parts - 1) / parts;
  return SIG <= 8 ? (per + SIG - 1) / SIG * SIG : per;  // rt_sum_range unrolls the runs up to sigma = 8
}

constexpr unsigned long long kRtWarpTerms = 32;  // entries with this many terms or more: one warp each
constexpr unsigned long long kRtCtaTerms = 2048;  // entries with this many terms or more: the whole CTA

// The table of one tail tuple.  An entry's terms are loads that mostly miss
// the caches; the entry where every string advances has sigma^d of them.  So
// the work is split by size: entries of fewer than 32 terms go to single
// threads, those up to 2048 to one warp each (lanes sum contiguous blocks),
// and the largest to the whole CTA (every thread a contiguous block, the sums
// meeting in the table through shared-memory atomics).  The CTA-wide entries
// are enumerated directly (every S of d - k strings kept, by Gosper's
// next-combination step), so no thread walks the whole table for them.  The
// caller synchronises before and after.
template <int SIG>
__device__ __forceinline__ void rt_fill_table(const RtGeo<SIG>& g, const unsigned long long (&tp)[kMaxD],
                                              const long long* const* vs, long long* table) {
  const int entries = SIG << g.d;
  auto used = [&](int e) {
    const unsigned S = (unsigned)e & g.full;
    return !(S == g.full || (S == 0 && (e >> g.d) > 0));  // no candidate / shared entry
  };
  const bool cta_entries = g.sd >= kRtCtaTerms;  // uniform: the largest entry has sigma^d terms
  if (cta_entries) {  // the CTA-wide entries start at zero
    for (int e = threadIdx.x; e < entries; e += blockDim.x)
      if (used(e) && g.pw[g.d - __popc((unsigned)e & g.full)] >= kRtCtaTerms) table[e] = 0;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < entries; e += blockDim.x) {
    if (!used(e)) continue;
    const int z = e >> g.d;
    const unsigned S = (unsigned)e & g.full;
    const int k = g.d - __popc(S);
    if (g.pw[k] < kRtWarpTerms) table[e] = rt_sum<SIG>(g, tp, z, S, vs[k - 1]);
  }
  const int lane = threadIdx.x & 31;
  for (int e = threadIdx.x >> 5; e < entries; e += blockDim.x >> 5) {  // uniform over the warp
    if (!used(e)) continue;
    const int z = e >> g.d;
    const unsigned S = (unsigned)e & g.full;
    const int k = g.d - __popc(S);
    const unsigned long long terms = g.pw[k];
    if (terms < kRtWarpTerms || terms >= kRtCtaTerms) continue;
    const unsigned long long per = rt_chunk<SIG>(terms, 32);
    const unsigned long long m0 = min(terms, (unsigned long long)lane * per), m1 = min(terms, m0 + per);
    long long sum = rt_sum_range<SIG>(g, tp, z, S, vs[k - 1], m0, m1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) table[e] = sum;
  }
  // uniform over the CTA: k advanced strings, from every string down
  for (int k = g.d; cta_entries && k >= 1 && g.pw[k] >= kRtCtaTerms; --k) {
    const unsigned long long terms = g.pw[k];
    const unsigned long long per = rt_chunk<SIG>(terms, blockDim.x);
    const unsigned long long m0 = min(terms, (unsigned long long)threadIdx.x * per), m1 = min(terms, m0 + per);
    unsigned S = (1u << (g.d - k)) - 1;  // the smallest set of d - k kept strings
    while (S < g.full) {
      for (int z = 0; z < (S ? SIG : 1); ++z) {  // S = {}: one entry for every z
        long long sum = rt_sum_range<SIG>(g, tp, z, S, vs[k - 1], m0, m1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(table + rt_entry(z, S, g.d)), (unsigned long long)sum);
      }
      if (S == 0) break;
      const unsigned c = S & (0u - S), r = S + c;
      S = (((r ^ S) >> 2) / c) | r;  // the next set of the same size
    }
  }
}

// The table of one tail tuple filled by one warp (the warp-per-tuple form):
// entries below 32 terms by single lanes, the others by the whole warp.  The
// caller synchronises the warp before and after.
template <int SIG>
__device__ __forceinline__ void rt_fill_table_warp(const RtGeo<SIG>& g, const unsigned long long (&tp)[kMaxD],
                                                   const long long* const* vs, long long* table) {
  const int entries = SIG << g.d;
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < entries; e += 32) {
    const int z = e >> g.d;
    const unsigned S = (unsigned)e & g.full;
    if (S == g.full || (S == 0 && z > 0)) continue;
    const int k = g.d - __popc(S);
    if (g.pw[k] < kRtWarpTerms) table[e] = rt_sum<SIG>(g, tp, z, S, vs[k - 1]);
  }
  for (int e = 0; e < entries; ++e) {  // uniform over the warp
    const int z = e >> g.d;
    const unsigned S = (unsigned)e & g.full;
    if (S == g.full || (S == 0 && z > 0)) continue;
    const int k = g.d - __popc(S);
    const unsigned long long terms = g.pw[k];
    if (terms < kRtWarpTerms) continue;
    const unsigned long long per = rt_chunk<SIG>(terms, 32);
    const unsigned long long m0 = min(terms, (unsigned long long)lane * per), m1 = min(terms, m0 + per);
    long long sum = rt_sum_range<SIG>(g, tp, z, S, vs[k - 1], m0, m1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) table[e] = sum;
  }
}

// the heads of combination Hidx as the sets S_z = {j : H_j = z}
template <int SIG>
__device__ __forceinline__ void rt_head_sets(const RtGeo<SIG>& g, unsigned long long Hidx, unsigned (&sets)[SIG]) {
#pragma unroll
  for (int z = 0; z < SIG; ++z) sets[z] = 0;
  for (int j = g.d - 1; j >= 0; --j) {
    const int hz = (int)(Hidx % SIG);
    Hidx /= SIG;
#pragma unroll
    for (int z = 0; z < SIG; ++z)
      if (hz == z) sets[z] |= 1u << j;
  }
}

// the value of head combination Hidx of tail tuple t from its table (or, for
// tables too large for shared memory, from the sums themselves)
template <int SIG>
__device__ __forceinline__ long long rt_state_value(const RtGeo<SIG>& g, const unsigned long long (&tp)[kMaxD],
                                                    unsigned long long Hidx, const long long* table,
                                                    const long long* const* vs, long long one, long long R_shift) {
  unsigned sets[SIG];
  rt_head_sets<SIG>(g, Hidx, sets);
  bool equal = false;
  long long best = LLONG_MIN;
#pragma unroll
  for (int z = 0; z < SIG; ++z) {
    if (sets[z] == g.full) {
      equal = true;
      continue;
    }
    const int k = g.d - __popc(sets[z]);
    const long long M = g.table ? table[rt_entry(z, sets[z], g.d)] : rt_sum<SIG>(g, tp, z, sets[z], vs[k - 1]);
    best = max(best, rt_floor_div(M, g.pw[k]) + (long long)(g.d - k) * R_shift);
  }
  return best + (equal ? one : 0);
}

// WARP: one warp per tail tuple with a table of its own (small tables, many
// tuples), else one CTA per tail tuple
template <int SIG, bool INCR, bool WARP>
__global__ void __launch_bounds__(kBlock, 4) sweep_rt_kernel(SweepParams p) {
  __shared__ long long table_all[kRtTable];
  const RtGeo<SIG> g = rt_geo<SIG>(p.n_stored, p.h, p.n_tail);
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  constexpr unsigned kUnits = WARP ? kBlock / 32 : 1;
  const unsigned unit = WARP ? threadIdx.x >> 5 : 0;
  const unsigned lane = WARP ? threadIdx.x & 31 : threadIdx.x;
  constexpr unsigned kStride = WARP ? 32 : kBlock;
  long long* table = table_all + (WARP ? unit * kRtWarpTable : 0);
  for (unsigned long long t = (unsigned long long)blockIdx.x * kUnits + unit; t < g.n_tail;
       t += (unsigned long long)gridDim.x * kUnits) {
    unsigned long long tp[kMaxD];
    rt_tail_parts<SIG>(g, p.h, t, tp);
    if constexpr (WARP) {
      rt_fill_table_warp<SIG>(g, tp, p.prev, table);
      __syncwarp();
    } else {
      if (g.table) rt_fill_table<SIG>(g, tp, p.prev, table);
      __syncthreads();
    }
    for (unsigned long long Hidx = lane; Hidx < g.sd; Hidx += kStride) {
      const long long v = rt_state_value<SIG>(g, tp, Hidx, table, p.prev, p.one, 0);
      const unsigned long long x = Hidx * g.n_tail + t;
      p.out[x] = v;
      if constexpr (INCR) {
        const long long inc = v - ld_vec<false>(p.prev[0] + x);
        if (red_better(inc, x, best_v, best_x, p.r_mode)) best_v = inc, best_x = x;
      }
    }
    if constexpr (WARP)
      __syncwarp();
    else
      __syncthreads();  // the table is rewritten for the next tuple
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

// W = u + dR - F(u + (d-1)R, .., u): a candidate advancing k strings reads
// argument k = u + (d - k)R, whose mean is the mean of u plus (d - k)R
template <int SIG, bool WARP>
__global__ void __launch_bounds__(kBlock, 4) check_rt_kernel(CheckParams q) {
  __shared__ long long table_all[kRtTable];
  const RtGeo<SIG> g = rt_geo<SIG>(q.n_stored, q.h, q.n_tail);
  const long long R = q.R_from_state ? q.state->R : q.R;
  const long long* us[kMaxD];
  for (int k = 0; k < kMaxD; ++k) us[k] = q.u;
  long long best_w = LLONG_MIN;
  constexpr unsigned kUnits = WARP ? kBlock / 32 : 1;
  const unsigned unit = WARP ? threadIdx.x >> 5 : 0;
  const unsigned lane = WARP ? threadIdx.x & 31 : threadIdx.x;
  constexpr unsigned kStride = WARP ? 32 : kBlock;
  long long* table = table_all + (WARP ? unit * kRtWarpTable : 0);
  for (unsigned long long t = (unsigned long long)blockIdx.x * kUnits + unit; t < g.n_tail;
       t += (unsigned long long)gridDim.x * kUnits) {
    unsigned long long tp[kMaxD];
    rt_tail_parts<SIG>(g, q.h, t, tp);
    if constexpr (WARP) {
      rt_fill_table_warp<SIG>(g, tp, us, table);
      __syncwarp();
    } else {
      if (g.table) rt_fill_table<SIG>(g, tp, us, table);
      __syncthreads();
    }
    for (unsigned long long Hidx = lane; Hidx < g.sd; Hidx += kStride) {
      const unsigned long long x = Hidx * g.n_tail + t;
      const long long F = rt_state_value<SIG>(g, tp, Hidx, table, us, q.one, R);
      best_w = max(best_w, ld_vec<false>(q.u + x) + (long long)g.d * R - F);
    }
    if constexpr (WARP)
      __syncwarp();
    else
      __syncthreads();
  }
  block_reduce_max(best_w, q.partials);
}

// ---------------------------------------------------------------------------
// sigma = 2, d >= kRtWarpD: one warp per state

// the offsets of the terms of a candidate: bit d-1-j for every advanced string j
__device__ __forceinline__ unsigned rt2_offset_bits(unsigned N, int d) {
  return __brev(N) >> (32 - d);
}

// the deposit of the low bits of v into the set bits of mask
__device__ __forceinline__ unsigned rt2_deposit(unsigned v, unsigned mask) {
  unsigned out = 0;
  for (int i = 0; mask; ++i) {
    const unsigned b = mask & (0u - mask);
    if ((v >> i) & 1u) out |= b;
    mask ^= b;
  }
  return out;
}

// M(z, S) summed by the whole warp; every lane returns it
__device__ __forceinline__ long long rt2_warp_sum(const RtGeo<2>& g, const unsigned long long (&tp)[kMaxD], int z,
                                                  unsigned S, const long long* __restrict__ v, int lane) {
  unsigned long long base = 0;
  for (int j = 0; j < g.d; ++j)
    base += ((S >> j) & 1u) ? (unsigned long long)z * g.n_tail * g.pw[g.d - 1 - j] + tp[j] : g.sd * tp[j];
  const unsigned bits = rt2_offset_bits(g.full ^ S, g.d);
  unsigned low = 0, rest = bits;
  for (int i = 0; i < 5 && rest; ++i) {
    const unsigned b = rest & (0u - rest);
    low |= b;
    rest ^= b;
  }
  long long s = 0;
  if (lane < (1 << __popc(low))) {
    const unsigned long long lo = rt2_deposit((unsigned)lane, low);
    unsigned sub = 0;
    do {
      s += ld_vec<false>(v + base + sub + lo);
      sub = (sub - rest) & rest;
    } while (sub);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <bool INCR>
__global__ void __launch_bounds__(kBlock) sweep_rt2_kernel(SweepParams p) {
  const RtGeo<2> g = rt_geo<2>(p.n_stored, p.h, p.n_tail);
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  for (unsigned long long x = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < p.n_stored;
       x += warps) {
    const unsigned long long t = x % g.n_tail, Hidx = x / g.n_tail;
    unsigned long long tp[kMaxD];
    rt_tail_parts<2>(g, p.h, t, tp);
    const unsigned ones = __brev((unsigned)Hidx) >> (32 - g.d);  // bit j: string j's head is 1
    bool equal = false;
    long long best = LLONG_MIN;
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      const unsigned S = z ? ones : (g.full ^ ones);
      if (S == g.full) {
        equal = true;
        continue;
      }
      const int k = g.d - __popc(S);
      best = max(best, rt2_warp_sum(g, tp, z, S, p.prev[k - 1], lane) >> k);  // floor of the mean
    }
    const long long v = best + (equal ? p.one : 0);
    if (lane == 0) {
      p.out[x] = v;
      if constexpr (INCR) {
        const long long inc = v - ld_vec<false>(p.prev[0] + x);
        if (red_better(inc, x, best_v, best_x, p.r_mode)) best_v = inc, best_x = x;
      }
    }
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

// (a template, so that the translation units that include this header share
// one definition)
template <int SIG2 = 2>
__global__ void __launch_bounds__(kBlock) check_rt2_kernel(CheckParams q) {
  const RtGeo<2> g = rt_geo<2>(q.n_stored, q.h, q.n_tail);
  const long long R = q.R_from_state ? q.state->R : q.R;
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  long long best_w = LLONG_MIN;
  for (unsigned long long x = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < q.n_stored;
       x += warps) {
    const unsigned long long t = x % g.n_tail, Hidx = x / g.n_tail;
    unsigned long long tp[kMaxD];
    rt_tail_parts<2>(g, q.h, t, tp);
    const unsigned ones = __brev((unsigned)Hidx) >> (32 - g.d);
    bool equal = false;
    long long best = LLONG_MIN;
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      const unsigned S = z ? ones : (g.full ^ ones);
      if (S == g.full) {
        equal = true;
        continue;
      }
      const int k = g.d - __popc(S);
      best = max(best, (rt2_warp_sum(g, tp, z, S, q.u, lane) >> k) + (long long)(g.d - k) * R);
    }
    const long long F = best + (equal ? q.one : 0);
    if (lane == 0) best_w = max(best_w, ld_vec<false>(q.u + x) + (long long)g.d * R - F);
  }
  block_reduce_max(best_w, q.partials);
}

// d of a general-kernel launch: sigma^(d h) states are stored
template <int SIG>
inline int rt_d_of(unsigned long long n_stored, int h) {
  int dh = 0;
  for (unsigned long long m = n_stored; m > 1; m /= SIG) ++dh;
  return dh / h;
}

template <int SIG>
void launch_sweep_rt(const SweepParams& p, int grid, cudaStream_t s) {
  const int d = rt_d_of<SIG>(p.n_stored, p.h);
  if (p.rt_means && rtb_applies(SIG, d, p.h)) {
    launch_sweep_rtb<SIG>(p, d, grid, s);
    return;
  }
  if (SIG == 2 && d >= kRtWarpD) {
    if (p.incr)
      sweep_rt2_kernel<true><<<grid, kBlock, 0, s>>>(p);
    else
      sweep_rt2_kernel<false><<<grid, kBlock, 0, s>>>(p);
    return;
  }
  if (rt_warp_tails(SIG, d, p.n_tail)) {
    if (p.incr)
      sweep_rt_kernel<SIG, true, true><<<grid, kBlock, 0, s>>>(p);
    else
      sweep_rt_kernel<SIG, false, true><<<grid, kBlock, 0, s>>>(p);
    return;
  }
  if (p.incr)
    sweep_rt_kernel<SIG, true, false><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_rt_kernel<SIG, false, false><<<grid, kBlock, 0, s>>>(p);
}

template <int SIG>
void launch_check_rt(const CheckParams& q, int grid, cudaStream_t s) {
  const int d = rt_d_of<SIG>(q.n_stored, q.h);
  if (q.rt_means && rtb_applies(SIG, d, q.h)) {
    launch_check_rtb<SIG>(q, d, grid, s);
    return;
  }
  if (SIG == 2 && d >= kRtWarpD) {
    check_rt2_kernel<2><<<grid, kBlock, 0, s>>>(q);
    return;
  }
  if (rt_warp_tails(SIG, d, q.n_tail))
    check_rt_kernel<SIG, true><<<grid, kBlock, 0, s>>>(q);
  else
    check_rt_kernel<SIG, false><<<grid, kBlock, 0, s>>>(q);
}

// tails_per_thread = 0 marks a set that takes one tail tuple per CTA
template <int SIG>
KernelSet make_rt_set() {
  KernelSet k{};
  k.sigma = SIG;
  k.d = 0;  // any d
  k.f_mode = 0;
  k.sym = 0;
  k.sweep = &launch_sweep_rt<SIG>;
  k.check = &launch_check_rt<SIG>;
  k.sweep_fn = (const void*)&sweep_rt_kernel<SIG, true, false>;
  k.check_fn = (const void*)&check_rt_kernel<SIG, false>;
  k.tails_per_thread = 0;
  k.sweep_algo_bytes = 0;  // set per handle: 8 (d + 1)
  k.check_algo_bytes = 8;
  return k;
}

}  // namespace lcs
