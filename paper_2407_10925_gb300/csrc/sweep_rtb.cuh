// sweep_rtb.cuh -- the general sweep and check in block form (h >= 2, sigma^d
// at most kRtbMaxBlock), for every shape without a specialised kernel.
//
// Algorithm 1 and Eq. ineq3: state (H, t) -- heads H, tail tuple t -- takes,
// over the letters z whose set N_z = {j : H_j != z} is not empty, the max of
// the floored means M(z, S_z, t) / sigma^|N_z| (S_z = the other strings), plus
// 1 when all heads agree, where
//   M(z, S, t) = sum over c in Sigma^|N| of v_{|N|}[string j = z t_j on S,
//                string j = t_j c_j on N].
// All sigma^|N| terms of one M differ only in the last letters of the strings
// in N, and every string's last letter sits in the lowest d base-sigma digits
// of the state index.  So the terms lie in one BLOCK of sigma^d consecutive
// values of v_{|N|}: block Y, whose higher digits are t_j's letters for j in
// N and z followed by t_j without its last letter for j in S.  Conversely a
// block Y of v_k holds every term of the M with |N| = k, N = the complement of
// S, for each S whose strings all carry one letter z in Y's top digit group;
// such a (Y, N) -- a TASK -- yields sigma^|S| of them, one for each choice of
// the last letters on S (the block's digits there), each the sum of the
// block's values over the digits on N.  Every M needed by some state arises
// from exactly one task.
//
// Phase 1 (rtb_means_kernel): a persistent CTA walks the tiles that hold a
// task (listed once per handle), stages each -- consecutive blocks of one
// vector -- in shared memory with one bulk copy (TMA) completed on an
// mbarrier, lists the tile's tasks, and sums each M over shared memory,
// reading the offsets of its terms from a table built once
// (rtb_offsets_kernel): per output, split over the threads on the lowest
// advanced digits (sigma >= 3), or per task by a warp whose lanes are the
// block's five lowest digits (sigma = 2).  It stores the floored mean (plus
// (d - k) R for the check, whose k-th argument is u + (d - k) R) at
// means[e(z, S) n_tail + t], e(z, S) = the entry index of sweep_rt.cuh.
// Phase 2 (rtb_state_kernel): for one head combination and a span of tail
// tuples, the candidate rows e(z, S_z) are formed once; each thread reads
// them at its columns t -- consecutive states, consecutive t -- and writes v
// with the fused increment reduction, or reduces the check's max W.
//
// Reads: each block of each argument once per sweep (algorithmic), plus the
// means table (sigma 2^d values per tail tuple, against sigma^d states).
//
// Index arithmetic: the interface's state index is Hidx n_tail + t with Hidx =
// sum_j H_j sigma^(d-1-j); the digit of letter position p (0 = head) of string
// j has weight sigma^((h-1-p) d + d-1-j).  Block Y covers states Y sigma^d ..
// Y sigma^d + sigma^d - 1; digit i of Y (i < (h-1) d) belongs to string
// d-1-(i mod d), and its top group (i >= (h-2) d) is the head letters.  The
// tail tuple of a task's M is then: Y's digits on N at their own weights, plus
// sigma^d times Y's digits on S below the top group, plus the block digits on
// S (the last letters, at weight sigma^(d-1-j)).
#pragma once

#include <climits>

#include "../../include/lcs_bound.h"
#include "lcs_common.h"
#include "sweep_generic.cuh"

namespace lcs {

constexpr unsigned kRtbMaxBlock = 16384;  // sigma^d values of one block at most (128 KiB of shared memory)
constexpr unsigned kRtbTileVals = 8192;   // blocks below 2048 values are staged several to a tile of up to this many
constexpr unsigned kRtbMaxG = 64;         // blocks of one tile at most
constexpr unsigned kRtbTasks = kBlock;    // tasks listed at once: one per thread

// the block form serves (sigma, d, h)
inline bool rtb_applies(int sigma, int d, int h) {
  if (h < 2 || d < 2 || d > kMaxD || sigma < 2) return false;
  unsigned long long sd = 1;
  for (int i = 0; i < d; ++i) {
    sd *= (unsigned long long)sigma;
    if (sd > kRtbMaxBlock) return false;
  }
  return true;
}

__host__ __device__ inline unsigned rtb_blocks_per_tile(unsigned sd) {
  const unsigned g = sd >= 2048 ? 1u : kRtbTileVals / sd;
  return g < kRtbMaxG ? g : kRtbMaxG;
}

constexpr unsigned kRtbAcc = kBlock / 2;  // outputs split over several threads in one pass at most

// one staging buffer: a tile plus one element of slack (the bulk copy starts
// at an even element), a multiple of 16 bytes
__host__ __device__ inline unsigned rtb_stage_bytes(unsigned sd) {
  return (rtb_blocks_per_tile(sd) * sd * 8 + 8 + 15) / 16 * 16;
}

// shared memory of a phase-1 CTA: the stages, then the task list (N, block
// offset, entry, tail base), the per-block task counts, the parts' sums, two
// mbarriers and a flag
__host__ __device__ inline size_t rtb_smem_bytes(unsigned sd, int nstage) {
  return (size_t)nstage * rtb_stage_bytes(sd) + (size_t)kRtbTasks * (4 + 4 + 4 + 8) + (kRtbMaxG + 2) * 4 +
         kRtbAcc * 8 + 2 * 8 + 16;
}

// two stages when three CTAs with two stages each still fit an SM (the
// kernel is bound by its summation more than by its staging, so occupancy
// comes first), else one
__host__ __device__ inline int rtb_stages(unsigned sd) { return rtb_smem_bytes(sd, 2) <= 74u * 1024 ? 2 : 1; }

// arguments of phase 1
struct RtbArgs {
  const long long* v[kMaxD];  // v[k-1]: the argument of the candidates advancing k strings
  long long* means;           // sigma 2^d rows of n_tail values
  const unsigned short* offs; // offs[start[N] + m]: the offset in a block of term m of an N-sum
  const unsigned* start;
  unsigned long long n_tail;
  unsigned sd;                // sigma^d
  int d, h;
  const DevState* state;      // check: R from state->R when R_from_state, else R
  int R_from_state;
  long long R;
  DevState* state_out;        // status: LCS_ETIMEOUT if a staging wait gives up
  const unsigned long long* tiles;  // sweep: the tiles with a task, (k << 48) | run index
  unsigned long long n_tiles;
  int nstage;
};

// arguments of phase 2
struct RtbStateArgs {
  const long long* means;
  long long* out;             // sweep: the new iterate
  const long long* prev0;     // sweep: v_{t-1} (increment reduction)
  const long long* u;         // check: the vector checked
  unsigned long long n_tail, n_stored;
  unsigned sd;
  int d;
  long long one;
  int r_mode;
  RedPartial* partials;
  const DevState* state;
  int R_from_state;
  long long R;
};

__device__ __forceinline__ unsigned rtb_binom(unsigned n, unsigned s) {
  if (s > n) return 0;
  unsigned c = 1;
  for (unsigned i = 0; i < s; ++i) c = c * (n - i) / (i + 1);  // exact at every step
  return c;
}

// the sets {j : the top-group letter of string j in block Y is z}
template <int SIG>
__device__ __forceinline__ void rtb_top_sets(unsigned long long Y, unsigned long long topw, int d,
                                             unsigned (&Z)[SIG]) {
#pragma unroll
  for (int z = 0; z < SIG; ++z) Z[z] = 0;
  unsigned top = (unsigned)(Y / topw);
  for (int j = d - 1; j >= 0; --j) {
    const unsigned c = top % SIG;
    top /= SIG;
#pragma unroll
    for (int z = 0; z < SIG; ++z)
      if (c == (unsigned)z) Z[z] |= 1u << j;
  }
}

// tasks of block Y advancing k = d - s strings
template <int SIG>
__device__ __forceinline__ unsigned rtb_count(unsigned long long Y, unsigned long long topw, int d, int s) {
  if (s == 0) return 1;
  unsigned Z[SIG];
  rtb_top_sets<SIG>(Y, topw, d, Z);
  unsigned c = 0;
#pragma unroll
  for (int z = 0; z < SIG; ++z) c += rtb_binom(__popc(Z[z]), s);
  return c;
}

// task r of block Y (its sets S of s strings: for each z in turn, the
// s-subsets of Z[z] in colex order), as N, entry and tail base
template <int SIG>
__device__ __forceinline__ void rtb_task(unsigned long long Y, unsigned long long topw, int d, int h, int s,
                                         unsigned r, unsigned& N, unsigned& e, unsigned long long& tbase) {
  const unsigned full = (1u << d) - 1;
  unsigned S = 0;
  int zsel = 0;
  if (s > 0) {
    unsigned Z[SIG];
    rtb_top_sets<SIG>(Y, topw, d, Z);
    unsigned mask = 0;
    bool found = false;
#pragma unroll
    for (int z = 0; z < SIG; ++z) {
      const unsigned c = rtb_binom(__popc(Z[z]), s);
      if (!found) {
        if (r < c) {
          found = true;
          zsel = z;
          mask = Z[z];
        } else {
          r -= c;
        }
      }
    }
    // unrank r among the s-subsets of the n = popc(mask) members of mask
    const int n = __popc(mask);
    unsigned local = 0;
    int left = s;
    for (int i = n - 1; i >= 0 && left > 0; --i) {
      const unsigned c = rtb_binom((unsigned)i, (unsigned)left);
      if (c <= r) {
        local |= 1u << i;
        r -= c;
        --left;
      }
    }
    // member i of mask (in increasing bit order) joins S when bit i of local is set
    for (int i = 0; mask; ++i) {
      const unsigned b = mask & (0u - mask);
      if ((local >> i) & 1u) S |= b;
      mask ^= b;
    }
  }
  N = full ^ S;
  e = S ? ((unsigned)zsel << d) | S : 0u;
  // the tail tuple's digits other than the block's: Y's digits on N at their
  // weights, sigma^d times Y's digits on S below the top group
  unsigned long long tN = 0, tS = 0, w = 1, y = Y;
  const int low_groups = (h - 2) * d;
  for (int i = 0; i < (h - 1) * d; ++i) {
    const unsigned long long c = y % SIG;
    y /= SIG;
    const int j = d - 1 - i % d;
    if ((N >> j) & 1u)
      tN += c * w;
    else if (i < low_groups)
      tS += c * w;
    w *= SIG;
  }
  unsigned long long sd = 1;
  for (int i = 0; i < d; ++i) sd *= SIG;
  tbase = tN + sd * tS;
}

// the offset in the block of output lowS of a task with kept strings S: the
// digits of lowS, least significant first, on the strings of S from the last
// one back
template <int SIG>
__device__ __forceinline__ unsigned rtb_s_offset(unsigned S, int d, unsigned lowS) {
  unsigned off = 0, w = 1;
  for (int j = d - 1; j >= 0; --j) {
    if ((S >> j) & 1u) {
      off += (lowS % SIG) * w;
      lowS /= SIG;
    }
    w *= SIG;
  }
  return off;
}

template <int SIG>
__device__ __forceinline__ long long rtb_floor_mean(long long sum, unsigned T, int k) {
  if constexpr ((SIG & (SIG - 1)) == 0) {
    return sum >> (k * __ffs(SIG) - k);  // sigma = 2^b: T = 2^(b k); arithmetic shift floors
  } else {
    const long long m = (long long)T;
    long long q = sum / m;
    return q - ((sum - q * m) < 0);
  }
}

// ---------------------------------------------------------------------------
// staging: bulk copies (TMA) into shared memory, completed on an mbarrier

__device__ __forceinline__ uint32_t rtb_smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void rtb_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// bounded wait on an mbarrier phase; false when the budget (in clock cycles) runs out
__device__ __forceinline__ bool rtb_wait(uint32_t bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

constexpr long long kRtbWaitBudget = 1ll << 31;  // clock cycles (about a second)

// One tile: nb blocks of sigma^d values from element e0 of vector v.  A bulk
// copy wants 16-byte aligned ends, so it covers [e0 rounded down to an even
// element, end rounded up to one) and the tile starts `shift` elements in; it
// is used only when that range lies inside the vector (else plain loads).
struct RtbTile {
  const long long* v;
  unsigned long long e0;
  unsigned vals;      // nb sigma^d
  unsigned shift;     // 0 or 1
  unsigned bytes;     // of the copy
  bool bulk;
};

__device__ __forceinline__ RtbTile rtb_tile(const long long* v, unsigned long long n_stored, unsigned long long e0,
                                            unsigned vals) {
  RtbTile t;
  t.v = v;
  t.e0 = e0;
  t.vals = vals;
  t.shift = (unsigned)(e0 & 1);
  const unsigned long long a0 = e0 - t.shift, a1 = (e0 + vals + 1) & ~1ull;
  t.bytes = (unsigned)((a1 - a0) * 8);
  t.bulk = ((reinterpret_cast<uintptr_t>(v) & 15) == 0) && a1 <= n_stored;
  return t;
}

// The inner digits of a part's sum: the U lowest-weight strings of N left
// after the part's own digits are walked in registers, so one lookup in the
// offset table serves sigma^U loads.
template <int SIG>
struct RtbInner {
  static constexpr int U = SIG == 2 ? 3 : SIG == 3 ? 2 : 1;
  static constexpr int IN = SIG == 2 ? 8 : SIG == 3 ? 9 : SIG;
};

// Part `part` (of sigma^a) of one output: the terms whose a lowest N digits
// are part's digits.  bb points at the output's block position (its S digits
// included).  offs/start: the term-offset table.
template <int SIG>
__device__ __forceinline__ long long rtb_part_sum(const long long* bb, unsigned N, int d, int k, int a, unsigned part,
                                                  const unsigned short* __restrict__ offs,
                                                  const unsigned* __restrict__ start) {
  constexpr int U = RtbInner<SIG>::U, IN = RtbInner<SIG>::IN;
  unsigned low = 0, rest = N, partset = 0, w = 1, w0 = 0, w1 = 0, w2 = 0;
  int i = 0;
  for (int j = d - 1; j >= 0; --j, w *= SIG) {
    if (!((N >> j) & 1u)) continue;
    if (i < a) {
      low += (part % SIG) * w;
      part /= SIG;
      rest &= ~(1u << j);
      partset |= 1u << j;
    } else if (i < a + U) {
      if (i == a) w0 = w;
      else if (i == a + 1) w1 = w;
      else w2 = w;
      rest &= ~(1u << j);
    }
    ++i;
  }
  const long long* b = bb + low;
  long long acc[IN];
#pragma unroll
  for (int c = 0; c < IN; ++c) acc[c] = 0;
  if (k - a >= U) {
    // inner offsets: the U digits, least significant first
    unsigned in[IN];
#pragma unroll
    for (int c = 0; c < IN; ++c) {
      unsigned q = c, o = 0;
      o += (q % SIG) * w0;
      q /= SIG;
      if (U > 1) {
        o += (q % SIG) * w1;
        q /= SIG;
      }
      if (U > 2) o += (q % SIG) * w2;
      in[c] = o;
    }
    unsigned J = 1;
    for (int q = a + U; q < k; ++q) J *= SIG;
    const unsigned short* on = offs + start[rest];
    for (unsigned jj = 0; jj < J; ++jj) {
      const long long* bj = b + __ldg(on + jj);
#pragma unroll
      for (int c = 0; c < IN; ++c) acc[c] += bj[in[c]];
    }
  } else {
    // fewer than U digits left: one lookup per term, over every N string but the part's
    unsigned J = 1;
    for (int q = a; q < k; ++q) J *= SIG;
    const unsigned short* on = offs + start[N & ~partset];
    for (unsigned jj = 0; jj < J; ++jj) acc[0] += b[__ldg(on + jj)];
  }
  long long sum = 0;
#pragma unroll
  for (int c = 0; c < IN; ++c) sum += acc[c];
  return sum;
}

// Lane-digit form of the sums (used for sigma = 2): a warp takes whole tasks, its
// lanes are the block's A lowest base-sigma digits (the last letters of the
// strings d-1 .. d-A), so every shared-memory read of the warp is L <= 32
// consecutive values.  A lane sums, for each combination of the kept strings
// above the lane digits (the outer loop), its values over every combination
// of the advanced strings above them (the inner loop, offsets from the
// table); shuffles then sum over the advanced strings among the lane digits,
// and the lanes whose digits there are 0 file the outputs.
template <int SIG>
struct RtbLanes {
  static constexpr int A = SIG == 2 ? 5 : SIG == 3 ? 3 : 2;
  static constexpr unsigned L = SIG == 2 ? 32 : SIG == 3 ? 27 : SIG == 4 ? 16 : 25;
};

// The inner sum of a lane: over every combination of the advanced strings
// above the lane digits (offsets from the table, the same for every lane,
// so each lookup is one broadcast); lookups j0, j0 + step, .. are this call's.
template <int SIG>
__device__ __forceinline__ long long rtb_lane_inner(const long long* base, const unsigned short* __restrict__ on,
                                                    unsigned J, unsigned j0, unsigned step) {
  long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  unsigned n = j0;
  for (; n + 3 * step < J; n += 4 * step) {
    const unsigned o0 = __ldg(on + n), o1 = __ldg(on + n + step), o2 = __ldg(on + n + 2 * step),
                   o3 = __ldg(on + n + 3 * step);
    s0 += base[o0];
    s1 += base[o1];
    s2 += base[o2];
    s3 += base[o3];
  }
  for (; n < J; n += step) s0 += base[__ldg(on + n)];
  return (s0 + s1) + (s2 + s3);
}

// sum acc over the lanes that differ only in the lane digits at the
// positions of nlo (warp-uniform); every lane of the warp takes part
template <int SIG>
__device__ __forceinline__ long long rtb_lane_reduce(long long acc, unsigned nlo, unsigned lane) {
  unsigned w = 1;
#pragma unroll
  for (int p = 0; p < RtbLanes<SIG>::A; ++p, w *= SIG) {
    if (!((nlo >> p) & 1u)) continue;
    if constexpr (SIG == 2) {
      acc += __shfl_xor_sync(0xffffffffu, acc, (int)w);
    } else {
      const unsigned b0 = lane - ((lane / w) % SIG) * w;  // the lane with digit p = 0
      long long tot = 0;
#pragma unroll
      for (int c = 0; c < SIG; ++c) tot += __shfl_sync(0xffffffffu, acc, (int)((b0 + c * w) & 31u));
      acc = tot;
    }
  }
  return acc;
}

// One batch of tasks (listed in t_*), all advancing k strings, by warps.
// With a single task that advances every string (one output), every warp
// sums a share and the shares meet in acc[0] (zeroed by the caller).
template <int SIG, bool CHECK>
__device__ __forceinline__ void rtb_lane_batch(const RtbArgs& a, const long long* blk, const unsigned* t_N,
                                               const unsigned* t_boff, const unsigned* t_e,
                                               const unsigned long long* t_base, long long* acc, unsigned nbatch,
                                               int d, int k, unsigned T, long long R, unsigned long long n_tail) {
  constexpr int A = RtbLanes<SIG>::A;
  constexpr unsigned L = RtbLanes<SIG>::L;
  const unsigned warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const unsigned full = (1u << d) - 1;
  const unsigned hi = (1u << (d - A)) - 1;  // strings whose last letter lies above the lane digits
  const bool live = lane < L;
  auto file = [&](unsigned task, unsigned offS, long long sum) {
    long long mean = rtb_floor_mean<SIG>(sum, T, k);
    if (CHECK) mean += (long long)(d - k) * R;
    a.means[(unsigned long long)t_e[task] * n_tail + t_base[task] + offS] = mean;
  };
  if (nbatch == 1 && k == d) {
    unsigned J = 1;
    for (int q = 0; q < d - A; ++q) J *= SIG;
    long long sum = live ? rtb_lane_inner<SIG>(blk + t_boff[0] + lane, a.offs + a.start[full & hi], J, warp, nwarps)
                         : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)sum);
    __syncthreads();
    if (threadIdx.x == 0) file(0, 0, acc[0]);
    return;
  }
  // a task is split over `pp` warps on its outer loop when the batch is small
  const unsigned pp = nbatch >= nwarps ? 1u : nwarps / nbatch;
  for (unsigned u = warp; u < nbatch * pp; u += nwarps) {
    const unsigned task = u / pp, piece = u - task * pp;
    const unsigned N = t_N[task], S = full ^ N;
    unsigned nlo = 0;  // lane digits of advanced strings (position p = string d-1-p)
#pragma unroll
    for (int p = 0; p < A; ++p)
      if ((N >> (d - 1 - p)) & 1u) nlo |= 1u << p;
    bool writer = live;  // the lane's digits at nlo are all 0
    {
      unsigned l = lane;
#pragma unroll
      for (int p = 0; p < A; ++p) {
        if (((nlo >> p) & 1u) && (l % SIG) != 0) writer = false;
        l /= SIG;
      }
    }
    unsigned J = 1, Q = 1;
    for (int q = 0; q < __popc(N & hi); ++q) J *= SIG;
    for (int q = 0; q < __popc(S & hi); ++q) Q *= SIG;
    const unsigned short* __restrict__ on = a.offs + a.start[N & hi];
    const unsigned short* __restrict__ os = a.offs + a.start[S & hi];
    const long long* bb = blk + t_boff[task] + lane;
    for (unsigned q = piece; q < Q; q += pp) {
      const unsigned offSh = __ldg(os + q);
      long long sum = live ? rtb_lane_inner<SIG>(bb + offSh, on, J, 0, 1) : 0;
      sum = rtb_lane_reduce<SIG>(sum, nlo, lane);
      if (writer) file(task, offSh + lane, sum);
    }
  }
}

// Phase 1.  Tiles: the listed (k, run of G blocks) for the sweep (v_k's
// blocks; runs without a task are not listed), every run of G blocks for the
// check (u's, all k from one staging).  Two stages when they fit: the copy of
// the tile after next is issued as soon as a tile is done.
template <int SIG, bool CHECK>
__global__ void __launch_bounds__(kBlock, 4) rtb_means_kernel(RtbArgs a) {
  extern __shared__ __align__(16) unsigned char rtb_smem[];
  const unsigned sd = a.sd;
  const int d = a.d;
  const unsigned G = rtb_blocks_per_tile(sd);
  const unsigned stage_bytes = rtb_stage_bytes(sd);
  const int nstage = a.nstage;
  unsigned char* stage0 = rtb_smem;
  unsigned* t_N = reinterpret_cast<unsigned*>(rtb_smem + (size_t)nstage * stage_bytes);
  unsigned* t_boff = t_N + kRtbTasks;
  unsigned* t_e = t_boff + kRtbTasks;
  unsigned long long* t_base = reinterpret_cast<unsigned long long*>(t_e + kRtbTasks);
  unsigned* cnt = reinterpret_cast<unsigned*>(t_base + kRtbTasks);
  long long* acc = reinterpret_cast<long long*>(cnt + kRtbMaxG + 2);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(acc + kRtbAcc);
  int* flag = reinterpret_cast<int*>(bars + 2);

  const unsigned long long n_tail = a.n_tail;
  const unsigned long long topw = n_tail / sd;  // sigma^((h-2) d): weight of Y's top group
  const unsigned long long n_ty = (n_tail + G - 1) / G;
  const unsigned long long n_stored = n_tail * sd;
  const unsigned full = (1u << d) - 1;
  const long long R = CHECK ? (a.R_from_state ? a.state->R : a.R) : 0;
  const unsigned long long n_tiles = CHECK ? n_ty : a.n_tiles;
  const int tid = threadIdx.x, lane = tid & 31;

  // tile i of this CTA: its first k and run of blocks
  auto tile_of = [&](unsigned long long it, int& k, unsigned long long& Y0, unsigned& nb) {
    unsigned long long ty;
    if (CHECK) {
      k = 1;
      ty = it;
    } else {
      const unsigned long long e = a.tiles[it];
      k = (int)(e >> 48);
      ty = e & ((1ull << 48) - 1);
    }
    Y0 = ty * G;
    nb = (unsigned)min((unsigned long long)G, n_tail - Y0);
  };
  auto tile_desc = [&](unsigned long long it) {
    int k;
    unsigned long long Y0;
    unsigned nb;
    tile_of(it, k, Y0, nb);
    return rtb_tile(a.v[k - 1], n_stored, Y0 * sd, nb * sd);
  };
  auto issue = [&](unsigned long long it, int st) {  // one thread
    const RtbTile t = tile_desc(it);
    if (!t.bulk) return;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    rtb_bulk_load(rtb_smem_addr(stage0 + (size_t)st * stage_bytes), t.v + (t.e0 - t.shift), t.bytes,
                  rtb_smem_addr(bars + st));
  };

  if (tid == 0) {
    for (int st = 0; st < nstage; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(rtb_smem_addr(bars + st)), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int st = 0; st < nstage; ++st) {
      const unsigned long long it = blockIdx.x + (unsigned long long)st * gridDim.x;
      if (it < n_tiles) issue(it, st);
    }
  }
  __syncthreads();
  unsigned phase = 0;  // bit st: the parity the next bulk copy into stage st completes
  unsigned long long i = 0;
  for (unsigned long long it = blockIdx.x; it < n_tiles; it += gridDim.x, ++i) {
    const int st = nstage == 2 ? (int)(i & 1) : 0;
    int k_first;
    unsigned long long Y0;
    unsigned nb;
    tile_of(it, k_first, Y0, nb);
    const RtbTile tile = rtb_tile(a.v[k_first - 1], n_stored, Y0 * sd, nb * sd);
    long long* blk = reinterpret_cast<long long*>(stage0 + (size_t)st * stage_bytes) + tile.shift;
    if (tile.bulk) {
      if (tid == 0) {
        const bool ok = rtb_wait(rtb_smem_addr(bars + st), (phase >> st) & 1u, kRtbWaitBudget);
        *flag = ok ? 1 : 0;
        if (!ok) {
          atomicExch(reinterpret_cast<unsigned long long*>(&a.state_out->status), (unsigned long long)LCS_ETIMEOUT);
          // copies may still be in flight into this stage and the other one:
          // wait for each again (bounded) before the CTA leaves
          rtb_wait(rtb_smem_addr(bars + st), (phase >> st) & 1u, kRtbWaitBudget);
          const unsigned long long nxt = it + gridDim.x;
          if (nstage == 2 && nxt < n_tiles && tile_desc(nxt).bulk)
            rtb_wait(rtb_smem_addr(bars + (st ^ 1)), (phase >> (st ^ 1)) & 1u, kRtbWaitBudget);
        }
      }
      __syncthreads();
      if (!*flag) return;  // uniform
      phase ^= 1u << st;
    } else {
      for (unsigned q = tid; q < tile.vals; q += kBlock) blk[q] = __ldcs(tile.v + tile.e0 + q);
      __syncthreads();
    }
    const int k_last = CHECK ? d : k_first;
    for (int k = k_first; k <= k_last; ++k) {
      const int s = d - k;
      unsigned total;
      if (nb == 1) {  // one block: every thread counts its tasks, no barrier
        total = rtb_count<SIG>(Y0, topw, d, s);
      } else {
        if (tid < (int)nb) cnt[tid + 1] = rtb_count<SIG>(Y0 + tid, topw, d, s);
        if (tid == 0) cnt[0] = 0;
        __syncthreads();
        if (tid == 0)
          for (unsigned b = 1; b <= nb; ++b) cnt[b] += cnt[b - 1];
        __syncthreads();
        total = cnt[nb];
      }
      unsigned T = 1, O = 1;  // terms per output (sigma^k), outputs per task (sigma^s)
      for (int q = 0; q < k; ++q) T *= SIG;
      for (int q = 0; q < s; ++q) O *= SIG;
      for (unsigned i0 = 0; i0 < total; i0 += kRtbTasks) {
        const unsigned nbatch = min(kRtbTasks, total - i0);
        if (tid < (int)nbatch) {
          const unsigned ti = i0 + tid;
          unsigned b = 0, first = 0;
          if (nb > 1) {
            while (cnt[b + 1] <= ti) ++b;
            first = cnt[b];
          }
          unsigned N, e;
          unsigned long long tb;
          rtb_task<SIG>(Y0 + b, topw, d, a.h, s, ti - first, N, e, tb);
          t_N[tid] = N;
          t_boff[tid] = b * sd;
          t_e[tid] = e;
          t_base[tid] = tb;
        }
        if constexpr (SIG == 2) {  // measured: faster for sigma = 2 only ((2,12,2) 4.1 ms against 7.1)
          if (d >= RtbLanes<SIG>::A) {  // uniform
            if (tid == 0) acc[0] = 0;
            __syncthreads();  // the task list is ready
            rtb_lane_batch<SIG, CHECK>(a, blk, t_N, t_boff, t_e, t_base, acc, nbatch, d, k, T, R, n_tail);
            __syncthreads();  // the task list and acc are rewritten by the next batch
            continue;
          }
        }
        // outputs: nbatch * O, each the sum of T terms split over P = sigma^a
        // threads (the part is the a lowest N digits); parts meet in acc
        const unsigned nOut = nbatch * O;
        int a_lo = 0;
        unsigned P = 1;
        while (a_lo < k - RtbInner<SIG>::U && nOut * P * SIG <= (unsigned)kBlock) {
          P *= SIG;
          ++a_lo;
        }
        const unsigned slots = nOut * P;
        if (P > 1 && tid < (int)nOut) acc[tid] = 0;
        __syncthreads();  // the task list (and acc) are ready
        for (unsigned base = 0; base < slots; base += kBlock) {  // uniform trip count
          const unsigned slot = base + tid;
          const bool act = slot < slots;
          const unsigned o = slot / P, part = slot - o * P;
          long long sum = 0;
          unsigned task = 0, offS = 0;
          if (act) {
            task = o / O;
            const unsigned N = t_N[task];
            offS = rtb_s_offset<SIG>(full ^ N, d, o - task * O);
            sum = rtb_part_sum<SIG>(blk + t_boff[task] + offS, N, d, k, a_lo, part, a.offs, a.start);
          }
          if (P > 1) {
            // segmented sum over the lanes of one output within this warp
#pragma unroll
            for (unsigned w = 1; w < 32; w <<= 1) {
              const long long up = __shfl_down_sync(0xffffffffu, sum, w);
              if (lane + w < 32 && part + w < P) sum += up;
            }
            if (act && (part == 0 || lane == 0))
              atomicAdd(reinterpret_cast<unsigned long long*>(acc + o), (unsigned long long)sum);
          } else if (act) {
            long long mean = rtb_floor_mean<SIG>(sum, T, k);
            if (CHECK) mean += (long long)(d - k) * R;
            a.means[(unsigned long long)t_e[task] * n_tail + t_base[task] + offS] = mean;
          }
        }
        if (P > 1) {
          __syncthreads();
          if (tid < (int)nOut) {
            const unsigned task = tid / O;
            const unsigned offS = rtb_s_offset<SIG>(full ^ t_N[task], d, tid - task * O);
            long long mean = rtb_floor_mean<SIG>(acc[tid], T, k);
            if (CHECK) mean += (long long)(d - k) * R;
            a.means[(unsigned long long)t_e[task] * n_tail + t_base[task] + offS] = mean;
          }
        }
        __syncthreads();  // the task list and acc are rewritten by the next batch
      }
      __syncthreads();  // cnt is rewritten by the next k
    }
    // every thread is done with this stage: refill it with the tile after next
    if (tid == 0) {
      const unsigned long long nxt = it + (unsigned long long)nstage * gridDim.x;
      if (nxt < n_tiles) issue(nxt, st);
    }
  }
}

// Phase 2: v (sweep) or W (check) of every state from the means table.  A
// unit is one head combination and a span of kRtbSpan consecutive tail
// tuples (chunk-major: the CTAs in flight share the table's columns); its
// candidate rows are formed once, then each thread takes kRtbPer states,
// issuing all their loads before it uses one.
constexpr int kRtbPer = 8;
constexpr unsigned kRtbSpan = kRtbPer * kBlock;

template <int SIG, bool INCR, bool CHECK>
__global__ void __launch_bounds__(kBlock) rtb_state_kernel(RtbStateArgs a) {
  const unsigned long long n_tail = a.n_tail;
  const int d = a.d;
  const unsigned full = (1u << d) - 1;
  const unsigned long long chunks = (n_tail + kRtbSpan - 1) / kRtbSpan;
  const unsigned long long units = chunks * a.sd;
  const long long R = CHECK ? (a.R_from_state ? a.state->R : a.R) : 0;
  long long best_v = a.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  long long best_w = LLONG_MIN;
  for (unsigned long long u = blockIdx.x; u < units; u += gridDim.x) {
    const unsigned long long c = u / a.sd;
    const unsigned Hidx = (unsigned)(u - c * a.sd);
    unsigned sets[SIG];
#pragma unroll
    for (int z = 0; z < SIG; ++z) sets[z] = 0;
    unsigned hh = Hidx;
    for (int j = d - 1; j >= 0; --j) {
      const unsigned cz = hh % SIG;
      hh /= SIG;
#pragma unroll
      for (int z = 0; z < SIG; ++z)
        if (cz == (unsigned)z) sets[z] |= 1u << j;
    }
    // candidate rows: one per letter on some but not all heads, and row 0
    // (every string advances) for the first letter on no head
    unsigned long long rows[SIG];
    bool use[SIG];
    bool equal = false, absent = false;
#pragma unroll
    for (int z = 0; z < SIG; ++z) {
      use[z] = sets[z] != full && (sets[z] != 0 || !absent);
      rows[z] = sets[z] ? (unsigned long long)(((unsigned)z << d) | sets[z]) * n_tail : 0ull;
      equal |= sets[z] == full;
      absent |= sets[z] == 0;
    }
    const long long bonus = equal ? a.one : 0;
    // the rows used, packed: at most min(sigma, d + 1) of them, and d + 1 <= 5
    // for sigma >= 7 (sigma^d <= 16384)
    constexpr int CM = SIG <= 6 ? SIG : 5;
    unsigned long long crow[CM];
    int ncr = 0;
#pragma unroll
    for (int j = 0; j < CM; ++j) crow[j] = 0;
#pragma unroll
    for (int z = 0; z < SIG; ++z) {
      if (!use[z]) continue;
#pragma unroll
      for (int j = 0; j < CM; ++j)
        if (j == ncr) crow[j] = rows[z];
      ++ncr;
    }
    const unsigned long long x0 = (unsigned long long)Hidx * n_tail;
    const unsigned long long t0 = c * kRtbSpan + threadIdx.x;
    long long best[kRtbPer], other[kRtbPer];
#pragma unroll
    for (int q = 0; q < kRtbPer; ++q) {
      const unsigned long long t = t0 + (unsigned)(q * kBlock);
      best[q] = LLONG_MIN;
      other[q] = 0;
      if (t < n_tail) {
#pragma unroll
        for (int j = 0; j < CM; ++j)
          if (j < ncr) best[q] = max(best[q], __ldg(a.means + crow[j] + t));
        if (CHECK) other[q] = __ldcs(a.u + x0 + t);
        else if (INCR) other[q] = __ldcs(a.prev0 + x0 + t);
      }
    }
#pragma unroll
    for (int q = 0; q < kRtbPer; ++q) {
      const unsigned long long t = t0 + (unsigned)(q * kBlock);
      if (t >= n_tail) continue;
      const long long v = best[q] + bonus;
      const unsigned long long x = x0 + t;
      if constexpr (CHECK) {
        best_w = max(best_w, other[q] + (long long)d * R - v);
      } else {
        __stcs(a.out + x, v);
        if constexpr (INCR) {
          const long long inc = v - other[q];
          if (red_better(inc, x, best_v, best_x, a.r_mode)) best_v = inc, best_x = x;
        }
      }
    }
  }
  if constexpr (CHECK)
    block_reduce_max(best_w, a.partials);
  else if constexpr (INCR)
    block_reduce_arg(best_v, best_x, a.r_mode, a.partials);
}

// The term offsets of every advance set N: offs[start[N] + m] is the offset
// in a block of term m of an N-sum (the digits of m, least significant first,
// on the strings of N from the last one back).  start[N] = the terms of every
// set below N: sum over the members b of N of sigma^(members of N above b)
// (1 + sigma)^b.  One CTA per set.
template <int SIG>
__global__ void __launch_bounds__(kBlock) rtb_offsets_kernel(unsigned short* offs, unsigned* start, int d) {
  const unsigned N = blockIdx.x;
  unsigned long long st = 0, p1 = 1;
  for (int b = 0; b < d; ++b) {
    if ((N >> b) & 1u) {
      unsigned long long sp = 1;
      for (int i = 0; i < __popc(N >> (b + 1)); ++i) sp *= SIG;
      st += sp * p1;
    }
    p1 *= SIG + 1;
  }
  if (threadIdx.x == 0) start[N] = (unsigned)st;
  unsigned T = 1;
  for (int i = 0; i < __popc(N); ++i) T *= SIG;
  for (unsigned m = threadIdx.x; m < T; m += blockDim.x) {
    unsigned off = 0, w = 1, mm = m;
    for (int j = d - 1; j >= 0; --j) {
      if ((N >> j) & 1u) {
        off += (mm % SIG) * w;
        mm /= SIG;
      }
      w *= SIG;
    }
    offs[st + m] = (unsigned short)off;
  }
}

// ---------------------------------------------------------------------------
// launchers

template <int SIG, bool CHECK>
inline int rtb_means_grid(size_t smem, unsigned long long tiles) {
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rtb_means_kernel<SIG, CHECK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rtb_means_kernel<SIG, CHECK>, kBlock, smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (int)min((unsigned long long)sms * per_sm, tiles > 0 ? tiles : 1ull);
}

template <int SIG>
void launch_sweep_rtb(const SweepParams& p, int d, int grid, cudaStream_t s) {
  RtbArgs a{};
  for (int k = 0; k < d; ++k) a.v[k] = p.prev[k];
  a.means = p.rt_means;
  a.offs = p.rt_offs;
  a.start = p.rt_start;
  a.n_tail = p.n_tail;
  a.sd = (unsigned)(p.n_stored / p.n_tail);
  a.d = d;
  a.h = p.h;
  a.state_out = p.state;
  a.tiles = p.rt_tiles;
  a.n_tiles = p.rt_n_tiles;
  a.nstage = rtb_stages(a.sd);
  const size_t smem = rtb_smem_bytes(a.sd, a.nstage);
  if (a.n_tiles > 0)
    rtb_means_kernel<SIG, false><<<rtb_means_grid<SIG, false>(smem, a.n_tiles), kBlock, smem, s>>>(a);
  RtbStateArgs b{};
  b.means = p.rt_means;
  b.out = p.out;
  b.prev0 = p.prev[0];
  b.n_tail = p.n_tail;
  b.n_stored = p.n_stored;
  b.sd = a.sd;
  b.d = d;
  b.one = p.one;
  b.r_mode = p.r_mode;
  b.partials = p.partials;
  if (p.incr)
    rtb_state_kernel<SIG, true, false><<<grid, kBlock, 0, s>>>(b);
  else
    rtb_state_kernel<SIG, false, false><<<grid, kBlock, 0, s>>>(b);
}

template <int SIG>
void launch_check_rtb(const CheckParams& q, int d, int grid, cudaStream_t s) {
  RtbArgs a{};
  for (int k = 0; k < d; ++k) a.v[k] = q.u;
  a.means = q.rt_means;
  a.offs = q.rt_offs;
  a.start = q.rt_start;
  a.n_tail = q.n_tail;
  a.sd = (unsigned)(q.n_stored / q.n_tail);
  a.d = d;
  a.h = q.h;
  a.state = q.state;
  a.R_from_state = q.R_from_state;
  a.R = q.R;
  a.state_out = const_cast<DevState*>(q.state);  // the handle's state: its status is writable
  a.nstage = rtb_stages(a.sd);
  const size_t smem = rtb_smem_bytes(a.sd, a.nstage);
  const unsigned G = rtb_blocks_per_tile(a.sd);
  const unsigned long long tiles = (q.n_tail + G - 1) / G;
  rtb_means_kernel<SIG, true><<<rtb_means_grid<SIG, true>(smem, tiles), kBlock, smem, s>>>(a);
  RtbStateArgs b{};
  b.means = q.rt_means;
  b.u = q.u;
  b.n_tail = q.n_tail;
  b.n_stored = q.n_stored;
  b.sd = a.sd;
  b.d = d;
  b.one = q.one;
  b.partials = q.partials;
  b.state = q.state;
  b.R_from_state = q.R_from_state;
  b.R = q.R;
  rtb_state_kernel<SIG, false, true><<<grid, kBlock, 0, s>>>(b);
}

template <int SIG>
void launch_rtb_offsets(int d, unsigned short* offs, unsigned* start, cudaStream_t s) {
  rtb_offsets_kernel<SIG><<<1u << d, kBlock, 0, s>>>(offs, start, d);
}

}  // namespace lcs
