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
// Phase 1 (rtb_means_kernel): a CTA stages a tile of consecutive blocks of one
// vector in shared memory with one contiguous read, lists the valid tasks,
// and sums each M over shared memory, reading the offsets of its terms from a
// table built once (rtb_offsets_kernel).  It stores the floored mean (plus
// (d - k) R for the check, whose k-th argument is u + (d - k) R) at
// means[e(z, S) n_tail + t], e(z, S) = the entry index of sweep_rt.cuh.
// Phase 2 (rtb_state_kernel): one thread per state reads its candidates from
// rows e(z, S_z) at column t -- consecutive states, consecutive t -- and
// writes v with the fused increment reduction, or reduces the check's max W.
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

#include "lcs_common.h"
#include "sweep_generic.cuh"

namespace lcs {

constexpr unsigned kRtbMaxBlock = 16384;  // sigma^d values of one block at most (128 KiB of shared memory)
constexpr unsigned kRtbTileVals = 2048;   // smaller blocks are staged several to a tile
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
  const unsigned g = sd >= kRtbTileVals ? 1u : kRtbTileVals / sd;
  return g < kRtbMaxG ? g : kRtbMaxG;
}

// shared memory of a phase-1 CTA: the tile, then the task list (N, block
// offset, entry, tail base), the per-block task counts, the cross-warp sums
__host__ __device__ inline size_t rtb_smem_bytes(unsigned sd) {
  return (size_t)rtb_blocks_per_tile(sd) * sd * 8 + (size_t)kRtbTasks * (4 + 4 + 4 + 8) + (kRtbMaxG + 2) * 4 + 8 * 8;
}

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

// Phase 1.  Tiles: (k, run of G blocks) for the sweep (v_k's blocks), runs of
// G blocks for the check (u's, every k from one staging).
template <int SIG, bool CHECK>
__global__ void __launch_bounds__(kBlock) rtb_means_kernel(RtbArgs a) {
  extern __shared__ __align__(16) unsigned char rtb_smem[];
  const unsigned sd = a.sd;
  const int d = a.d;
  const unsigned G = rtb_blocks_per_tile(sd);
  long long* blk = reinterpret_cast<long long*>(rtb_smem);
  unsigned* t_N = reinterpret_cast<unsigned*>(rtb_smem + (size_t)G * sd * 8);
  unsigned* t_boff = t_N + kRtbTasks;
  unsigned* t_e = t_boff + kRtbTasks;
  unsigned long long* t_base = reinterpret_cast<unsigned long long*>(t_e + kRtbTasks);
  unsigned* cnt = reinterpret_cast<unsigned*>(t_base + kRtbTasks);
  long long* acc = reinterpret_cast<long long*>(cnt + kRtbMaxG + 2);

  const unsigned long long n_tail = a.n_tail;
  const unsigned long long topw = n_tail / sd;  // sigma^((h-2) d): weight of Y's top group
  const unsigned long long n_ty = (n_tail + G - 1) / G;
  const unsigned full = (1u << d) - 1;
  const long long R = CHECK ? (a.R_from_state ? a.state->R : a.R) : 0;
  const unsigned long long n_tiles = (CHECK ? 1ull : (unsigned long long)d) * n_ty;
  const int tid = threadIdx.x;

  for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int k_first = CHECK ? 1 : (int)(tile / n_ty) + 1;
    const int k_last = CHECK ? d : k_first;
    const unsigned long long Y0 = (tile % n_ty) * G;
    const unsigned nb = (unsigned)min((unsigned long long)G, n_tail - Y0);
    const long long* __restrict__ src = a.v[k_first - 1] + Y0 * sd;
    bool staged = false;
    for (int k = k_first; k <= k_last; ++k) {
      const int s = d - k;
      __syncthreads();  // the previous pass is done with cnt and the task list
      if (tid < (int)nb) cnt[tid + 1] = rtb_count<SIG>(Y0 + tid, topw, d, s);
      if (tid == 0) cnt[0] = 0;
      __syncthreads();
      if (tid == 0)
        for (unsigned b = 1; b <= nb; ++b) cnt[b] += cnt[b - 1];
      __syncthreads();
      const unsigned total = cnt[nb];
      if (total == 0) continue;  // uniform
      if (!staged) {
        // one contiguous read of nb sigma^d values, four loads in flight per thread
        const unsigned vals = nb * sd;
        for (unsigned i = tid; i < vals; i += 4 * kBlock) {
          long long x[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const unsigned ii = i + q * kBlock;
            x[q] = ii < vals ? __ldcs(src + ii) : 0;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const unsigned ii = i + q * kBlock;
            if (ii < vals) blk[ii] = x[q];
          }
        }
        staged = true;
      }
      unsigned T = 1, O = 1;  // terms per output (sigma^k), outputs per task (sigma^s)
      for (int i = 0; i < k; ++i) T *= SIG;
      for (int i = 0; i < s; ++i) O *= SIG;
      for (unsigned i0 = 0; i0 < total; i0 += kRtbTasks) {
        const unsigned nbatch = min(kRtbTasks, total - i0);
        if (tid < (int)nbatch) {
          const unsigned i = i0 + tid;
          unsigned b = 0;
          while (cnt[b + 1] <= i) ++b;
          unsigned N, e;
          unsigned long long tb;
          rtb_task<SIG>(Y0 + b, topw, d, a.h, s, i - cnt[b], N, e, tb);
          t_N[tid] = N;
          t_boff[tid] = b * sd;
          t_e[tid] = e;
          t_base[tid] = tb;
        }
        __syncthreads();  // also: the staged tile is visible
        // outputs: nbatch * O, each the sum of T terms split over P threads
        const unsigned nOut = nbatch * O;
        unsigned P = 1;
        if (nOut < (unsigned)kBlock) {
          while (P * 2 * nOut <= (unsigned)kBlock && P * 2 <= T) P *= 2;
        }
        const int lgP = __ffs(P) - 1;
        const unsigned slots = nOut << lgP;
        if (P > 32) {
          if (tid < (int)nOut) acc[tid] = 0;
          __syncthreads();
        }
        for (unsigned base = 0; base < slots; base += kBlock) {  // uniform trip count
          const unsigned slot = base + tid;
          const bool act = slot < slots;
          const unsigned o = slot >> lgP, part = slot & (P - 1);
          long long sum = 0;
          unsigned task = 0, offS = 0;
          if (act) {
            task = o / O;
            const unsigned N = t_N[task];
            offS = rtb_s_offset<SIG>(full ^ N, d, o - task * O);
            const unsigned short* __restrict__ on = a.offs + a.start[N];
            const long long* bb = blk + t_boff[task] + offS;
            long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            unsigned m = part;
            for (; m + 3 * P < T; m += 4 * P) {
              const unsigned o0 = __ldg(on + m), o1 = __ldg(on + m + P), o2 = __ldg(on + m + 2 * P),
                             o3 = __ldg(on + m + 3 * P);
              s0 += bb[o0];
              s1 += bb[o1];
              s2 += bb[o2];
              s3 += bb[o3];
            }
            for (; m < T; m += P) s0 += bb[__ldg(on + m)];
            sum = (s0 + s1) + (s2 + s3);
          }
          if (P > 1) {
            const unsigned width = P < 32 ? P : 32;
            for (unsigned w = width >> 1; w; w >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, w);
          }
          if (P > 32) {
            if (act && (tid & 31) == 0)
              atomicAdd(reinterpret_cast<unsigned long long*>(acc + o), (unsigned long long)sum);
          } else if (act && part == 0) {
            long long mean = rtb_floor_mean<SIG>(sum, T, k);
            if (CHECK) mean += (long long)(d - k) * R;
            a.means[(unsigned long long)t_e[task] * n_tail + t_base[task] + offS] = mean;
          }
        }
        if (P > 32) {
          __syncthreads();
          if (tid < (int)nOut) {
            const unsigned task = tid / O;
            const unsigned offS = rtb_s_offset<SIG>(full ^ t_N[task], d, tid - task * O);
            long long mean = rtb_floor_mean<SIG>(acc[tid], T, k);
            if (CHECK) mean += (long long)(d - k) * R;
            a.means[(unsigned long long)t_e[task] * n_tail + t_base[task] + offS] = mean;
          }
        }
        __syncthreads();  // the task list is rewritten by the next batch
      }
    }
  }
}

// Phase 2: v (sweep) or W (check) of every state from the means table
template <int SIG, bool INCR, bool CHECK>
__global__ void __launch_bounds__(kBlock) rtb_state_kernel(RtbStateArgs a) {
  const unsigned long long n_tail = a.n_tail;
  const int d = a.d;
  const unsigned full = (1u << d) - 1;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long sq = stride / n_tail, sr = stride % n_tail;
  unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long Hidx = x / n_tail, t = x % n_tail;
  const long long R = CHECK ? (a.R_from_state ? a.state->R : a.R) : 0;
  long long best_v = a.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  long long best_w = LLONG_MIN;
  for (; x < a.n_stored; x += stride) {
    unsigned sets[SIG];
#pragma unroll
    for (int z = 0; z < SIG; ++z) sets[z] = 0;
    unsigned hh = (unsigned)Hidx;
    for (int j = d - 1; j >= 0; --j) {
      const unsigned c = hh % SIG;
      hh /= SIG;
#pragma unroll
      for (int z = 0; z < SIG; ++z)
        if (c == (unsigned)z) sets[z] |= 1u << j;
    }
    bool equal = false, absent = false;
    long long best = LLONG_MIN;
#pragma unroll
    for (int z = 0; z < SIG; ++z) {
      if (sets[z] == full) {
        equal = true;
      } else if (sets[z] == 0) {
        absent = true;  // every string advances: the shared entry 0
      } else {
        best = max(best, __ldg(a.means + ((unsigned long long)(((unsigned)z << d) | sets[z])) * n_tail + t));
      }
    }
    if (absent) best = max(best, __ldg(a.means + t));
    const long long v = best + (equal ? a.one : 0);
    if constexpr (CHECK) {
      best_w = max(best_w, __ldcs(a.u + x) + (long long)d * R - v);
    } else {
      __stcs(a.out + x, v);
      if constexpr (INCR) {
        const long long inc = v - __ldcs(a.prev0 + x);
        if (red_better(inc, x, best_v, best_x, a.r_mode)) best_v = inc, best_x = x;
      }
    }
    t += sr;
    Hidx += sq;
    if (t >= n_tail) {
      t -= n_tail;
      ++Hidx;
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
    cudaFuncSetAttribute(rtb_means_kernel<SIG, CHECK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rtb_smem_bytes(kRtbMaxBlock));
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
  return (int)min((unsigned long long)sms * per_sm, tiles);
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
  const size_t smem = rtb_smem_bytes(a.sd);
  const unsigned G = rtb_blocks_per_tile(a.sd);
  const unsigned long long tiles = (unsigned long long)d * ((p.n_tail + G - 1) / G);
  rtb_means_kernel<SIG, false><<<rtb_means_grid<SIG, false>(smem, tiles), kBlock, smem, s>>>(a);
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
  const size_t smem = rtb_smem_bytes(a.sd);
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
