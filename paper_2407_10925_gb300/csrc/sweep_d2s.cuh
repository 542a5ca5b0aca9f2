// sweep_d2s.cuh -- the sweep and check for d = 2 and sigma >= 3 that use the
// swap symmetry v[(p, q)] = v[(q, p)] (the LCS does not depend on the order of
// its arguments, and F commutes with exchanging the two strings; in fixed
// point it holds bit for bit once the start vectors have it, as the zero start
// does).  Storage is full (there is no complement symmetry for sigma >= 3).
//
// Write a tail tuple t = (a, b) (two strings of L = h - 1 letters, as base-
// sigma integers A and B) and its swap ts = (b, a).  For a string-0 head g let
//   P(t, g) = sum over c of v_{t-1}[(g a, b c)]
// (Algorithm 1's F_z for z = g, which advances string 1 of a state whose
// string-0 head is g).  The other single advance reads, by the symmetry,
//   sum over c of v_{t-1}[(a c, g b)] = sum over c of v_{t-1}[(g b, a c)] = P(ts, g).
// So the thread that owns the pair {t, ts} forms P(t, g) and P(ts, g) for every
// g and needs no other read of v_{t-1}: each value of v_{t-1} is read once
// (the value at (g a, b c) belongs to exactly one pair).  The all-advance
// block of v_{t-2} (sigma^2 values at sigma^2 t) serves both tails, because
// the block of ts holds the same values.  Per state: 8 B of v_{t-1}, 4 B of
// v_{t-2}, 8 B written, against 32 B for the generic kernel.
//
// Heads (g0, g1), Eq. ineq3 at the common denominator sigma^2:
//   g0 == g1: v = 1 + floor(S / sigma^2),   S = the all-advance block sum;
//   g0 != g1: v = floor(max(sigma P(t, g0), sigma P(ts, g1), S) / sigma^2)
// (z = g0 advances string 1, z = g1 string 0, any other z both).  For ts the
// roles of P(t, .) and P(ts, .) exchange, so v[(g0 g1), ts] = v[(g1 g0), t].
//
// Tiles.  A tile covers sigma^KA values of A by sigma^KB values of B
// (KA = KB or KB + 1), one pair per thread; inside a tile the thread index
// interleaves the digits A0, B0, A1, B1, ..., which is the digit order of the
// addresses of P(t, g): a warp's reads of v_{t-1} are contiguous.  Tile
// (TA, TB) holds a pair (some A <= B) iff TB >= RHO TA with RHO =
// sigma^(KA - KB), so row TA holds nTB - RHO TA live tiles; the kernels walk
// the live tiles only, numbered row by row, and CTAs take every grid-th one:
// the work splits evenly over the CTAs and the tiles in flight are
// neighbours.  Threads with A > B have no pair.
#pragma once

#include <climits>

#include "lcs_common.h"
#include "sweep_generic.cuh"

namespace lcs {

template <int SIG>
struct D2sGeo {
  static constexpr int KA = SIG == 3 ? 3 : 2;
  static constexpr int KB = SIG == 5 ? 1 : 2;
  static constexpr int T = (int)cpow(SIG, KA + KB);  // threads of one tile
  static constexpr int TPB = kBlock / T;             // tiles per CTA
  static constexpr unsigned long long RHO = cpow(SIG, KA - KB);
  static constexpr unsigned long long S2 = (unsigned long long)SIG * SIG;
  static_assert(TPB >= 1, "a tile must fit a CTA");
};

// sigma^e for a run-time e
template <int SIG>
__host__ __device__ inline unsigned long long d2s_pow(int e) {
  unsigned long long r = 1;
  for (int i = 0; i < e; ++i) r *= (unsigned long long)SIG;
  return r;
}

// the base-sigma digits of x (L of them) moved to base sigma^2 positions
template <int SIG>
__device__ __forceinline__ unsigned long long d2s_spread(unsigned long long x, int L) {
  unsigned long long r = 0, m = 1;
  for (int i = 0; i < L; ++i) {
    r += (x % SIG) * m;
    x /= SIG;
    m *= D2sGeo<SIG>::S2;
  }
  return r;
}

// live tiles before row TA: P(TA) = TA nTB - RHO TA (TA - 1) / 2
template <int SIG>
__host__ __device__ inline unsigned long long d2s_live_before(unsigned long long TA, unsigned long long nTB) {
  return TA * nTB - D2sGeo<SIG>::RHO * (TA * (TA - 1) / 2);
}

// live tiles of one sweep (every row TA < nTA holds at least RHO of them)
template <int SIG>
__host__ __device__ inline unsigned long long d2s_live_tiles(int L) {
  using G = D2sGeo<SIG>;
  return d2s_live_before<SIG>(d2s_pow<SIG>(L - G::KA), d2s_pow<SIG>(L - G::KB));
}

// live tile j -> (TA, TB): TA is the row with P(TA) <= j < P(TA + 1), the
// root of the quadratic P(TA) = j estimated in float and corrected exactly
template <int SIG>
__device__ __forceinline__ void d2s_live_tile(unsigned long long j, unsigned long long nTB, unsigned long long& TA,
                                              unsigned long long& TB) {
  constexpr float rho = (float)D2sGeo<SIG>::RHO;
  const float b = (float)nTB + 0.5f * rho;
  const float disc = fmaxf(b * b - 2.0f * rho * (float)j, 0.0f);
  long long t = (long long)((b - sqrtf(disc)) / rho);
  if (t < 0) t = 0;
  while (t > 0 && d2s_live_before<SIG>((unsigned long long)t, nTB) > j) --t;
  while (d2s_live_before<SIG>((unsigned long long)t + 1, nTB) <= j) ++t;
  TA = (unsigned long long)t;
  TB = D2sGeo<SIG>::RHO * TA + (j - d2s_live_before<SIG>(TA, nTB));
}

struct D2sPair {
  unsigned long long t, ts;  // tail indices of (a, b) and (b, a)
  unsigned long long eA, eB;  // spread digits of A and B
};

// The pair owned by thread r of live tile j; false if it has none.
template <int SIG>
__device__ __forceinline__ bool d2s_pair(unsigned long long j, int L, unsigned r, D2sPair& o) {
  using G = D2sGeo<SIG>;
  const unsigned long long nTB = d2s_pow<SIG>(L - G::KB);
  unsigned long long TA, TB;
  d2s_live_tile<SIG>(j, nTB, TA, TB);
  // digits of r: A0, B0, A1, B1, ... (A first); A has KA digits, B has KB
  unsigned long long ia = 0, ib = 0, wa = 1, wb = 1;
  unsigned rr = r;
#pragma unroll
  for (int i = 0; i < G::KA + G::KB; ++i) {
    const unsigned dgt = rr % SIG;
    rr /= SIG;
    if ((i & 1) == 0 || i / 2 >= G::KB) {
      ia += dgt * wa;
      wa *= SIG;
    } else {
      ib += dgt * wb;
      wb *= SIG;
    }
  }
  const unsigned long long A = TA * cpow(SIG, G::KA) + ia;
  const unsigned long long B = TB * cpow(SIG, G::KB) + ib;
  if (A > B) return false;
  o.eA = d2s_spread<SIG>(A, L);
  o.eB = d2s_spread<SIG>(B, L);
  o.t = o.eA * SIG + o.eB;
  o.ts = o.eB * SIG + o.eA;
  return true;
}

// P(t, g) for every g: sum over c of v[g sigma^(2L+1) + sigma eA + sigma^2 eB + c]
template <int SIG, bool CG>
__device__ __forceinline__ void d2s_partials(const long long* v, unsigned long long gstride, unsigned long long eA,
                                             unsigned long long eB, long long (&P)[SIG]) {
  const unsigned long long base = eA * SIG + eB * D2sGeo<SIG>::S2;
#pragma unroll
  for (int g = 0; g < SIG; ++g) {
    long long s = 0;
#pragma unroll
    for (int c = 0; c < SIG; ++c) s += ld_vec<CG>(v + g * gstride + base + c);
    P[g] = s;
  }
}

template <int SIG, bool CG>
__device__ __forceinline__ long long d2s_block(const long long* v, unsigned long long t) {
  constexpr unsigned long long S2 = D2sGeo<SIG>::S2;
  long long s = 0;
#pragma unroll
  for (int c = 0; c < (int)S2; ++c) s += ld_vec<CG>(v + t * S2 + c);
  return s;
}

// one thread's pair: the 2 sigma^2 new values (sigma^2 if t = ts)
template <int SIG, bool INCR, bool CG>
__device__ __forceinline__ void d2s_sweep_pair(const SweepParams& p, const D2sPair& o, int L, long long& best_v,
                                               unsigned long long& best_x) {
  constexpr unsigned long long S2 = D2sGeo<SIG>::S2;
  const unsigned long long nt = p.n_tail;  // sigma^(2L)
  const unsigned long long gstride = nt * SIG;
  const bool diag = o.t == o.ts;  // a = b: the pair is one tail
  long long Pt[SIG], Ps[SIG];
  d2s_partials<SIG, CG>(p.prev[0], gstride, o.eA, o.eB, Pt);
  if (diag) {
#pragma unroll
    for (int g = 0; g < SIG; ++g) Ps[g] = Pt[g];
  } else {
    d2s_partials<SIG, CG>(p.prev[0], gstride, o.eB, o.eA, Ps);
  }
  const long long S = d2s_block<SIG, CG>(p.prev[1], o.t);
  const long long eq = p.one + floor_div<S2>(S);
#pragma unroll
  for (int g0 = 0; g0 < SIG; ++g0) {
#pragma unroll
    for (int g1 = 0; g1 < SIG; ++g1) {
      long long vt, vs;  // the states (g0 g1, t) and (g0 g1, ts)
      if (g0 == g1) {
        vt = vs = eq;
      } else {
        vt = floor_div<S2>(max(max(Pt[g0], Ps[g1]) * (long long)SIG, S));
        vs = floor_div<S2>(max(max(Ps[g0], Pt[g1]) * (long long)SIG, S));
      }
      const unsigned long long H = (unsigned long long)(g0 * SIG + g1);
      const unsigned long long xt = H * nt + o.t, xs = H * nt + o.ts;
      p.out[xt] = vt;
      if (!diag) p.out[xs] = vs;
      if constexpr (INCR) {
        // (g0 g1, t) and (g1 g0, ts) hold equal values in v_t and v_{t-1}:
        // one candidate per class, at the class's smallest index
        if (g0 <= g1) {
          const unsigned long long xm = min(xt, (unsigned long long)(g1 * SIG + g0) * nt + o.ts);
          const long long inc = vt - ld_vec<CG>(p.prev[0] + xt);
          if (red_better(inc, xm, best_v, best_x, p.r_mode)) best_v = inc, best_x = xm;
          if (g0 != g1 && !diag) {
            // the class of (g1 g0, t) and (g0 g1, ts)
            const unsigned long long yt = (unsigned long long)(g1 * SIG + g0) * nt + o.t;
            const unsigned long long ym = min(yt, xs);
            const long long inc2 = vs - ld_vec<CG>(p.prev[0] + xs);
            if (red_better(inc2, ym, best_v, best_x, p.r_mode)) best_v = inc2, best_x = ym;
          }
        }
      }
    }
  }
}

// W = u + 2R - F(u + R, u) at the states (g0 g1, t): with u swap-symmetric,
// W at (g0 g1, ts) equals W at (g1 g0, t), so these cover every class
template <int SIG, bool CG>
__device__ __forceinline__ void d2s_check_pair(const CheckParams& p, const D2sPair& o, long long R, long long& best) {
  constexpr unsigned long long S2 = D2sGeo<SIG>::S2;
  const unsigned long long nt = p.n_tail;
  const unsigned long long gstride = nt * SIG;
  long long Pt[SIG], Ps[SIG];
  d2s_partials<SIG, CG>(p.u, gstride, o.eA, o.eB, Pt);
  if (o.t == o.ts) {
#pragma unroll
    for (int g = 0; g < SIG; ++g) Ps[g] = Pt[g];
  } else {
    d2s_partials<SIG, CG>(p.u, gstride, o.eB, o.eA, Ps);
  }
  const long long S = d2s_block<SIG, CG>(p.u, o.t);
  const long long all = floor_div<S2>(S);  // both strings advance: shift (d - 2) R = 0
#pragma unroll
  for (int g0 = 0; g0 < SIG; ++g0) {
#pragma unroll
    for (int g1 = 0; g1 < SIG; ++g1) {
      const unsigned long long H = (unsigned long long)(g0 * SIG + g1);
      long long F;
      if (g0 == g1) {
        F = p.one + all;
      } else {
        // one string advances: its mean of u + R is floor(P / sigma) + R
        F = max(max(floor_div<SIG>(Pt[g0]), floor_div<SIG>(Ps[g1])) + R, all);
      }
      best = max(best, ld_vec<CG>(p.u + H * nt + o.t) + 2 * R - F);
    }
  }
}

template <int SIG, bool INCR>
__global__ void __launch_bounds__(kBlock) sweep_d2s_kernel(SweepParams p) {
  using G = D2sGeo<SIG>;
  const int L = p.h - 1;
  const unsigned long long n_tiles = d2s_live_tiles<SIG>(L);
  const unsigned long long n_slots = (n_tiles + G::TPB - 1) / G::TPB;
  const unsigned sub = threadIdx.x / G::T, r = threadIdx.x % G::T;
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  if (sub < (unsigned)G::TPB) {
    for (unsigned long long s = blockIdx.x; s < n_slots; s += gridDim.x) {
      const unsigned long long k = s * G::TPB + sub;
      D2sPair o;
      if (k < n_tiles && d2s_pair<SIG>(k, L, r, o)) d2s_sweep_pair<SIG, INCR, false>(p, o, L, best_v, best_x);
    }
  }
  if constexpr (INCR) block_reduce_arg(best_v, best_x, p.r_mode, p.partials);
}

template <int SIG>
__global__ void __launch_bounds__(kBlock) check_d2s_kernel(CheckParams p) {
  using G = D2sGeo<SIG>;
  const int L = p.h - 1;
  const unsigned long long n_tiles = d2s_live_tiles<SIG>(L);
  const unsigned long long n_slots = (n_tiles + G::TPB - 1) / G::TPB;
  const unsigned sub = threadIdx.x / G::T, r = threadIdx.x % G::T;
  const long long R = p.R_from_state ? p.state->R : p.R;
  long long best = LLONG_MIN;
  if (sub < (unsigned)G::TPB) {
    for (unsigned long long s = blockIdx.x; s < n_slots; s += gridDim.x) {
      const unsigned long long k = s * G::TPB + sub;
      D2sPair o;
      if (k < n_tiles && d2s_pair<SIG>(k, L, r, o)) d2s_check_pair<SIG, false>(p, o, R, best);
    }
  }
  block_reduce_max(best, p.partials);
}

// is v invariant under exchanging the two strings?  (full storage, d = 2)
template <int SIG>
__global__ void swap_check_d2s_kernel(const long long* __restrict__ v, unsigned long long n, int h, DevState* st) {
  constexpr unsigned long long S2 = D2sGeo<SIG>::S2;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long y = 0, m = 1, r = x;
    for (int i = 0; i < h; ++i) {
      const unsigned long long pd = r % S2;
      r /= S2;
      y += ((pd % SIG) * SIG + pd / SIG) * m;
      m *= S2;
    }
    if (v[y] != v[x]) atomicExch((unsigned long long*)&st->swap_bad, 1ull);
  }
}

template <int SIG>
void launch_sweep_d2s(const SweepParams& p, int grid, cudaStream_t s) {
  if (p.incr)
    sweep_d2s_kernel<SIG, true><<<grid, kBlock, 0, s>>>(p);
  else
    sweep_d2s_kernel<SIG, false><<<grid, kBlock, 0, s>>>(p);
}

template <int SIG>
void launch_check_d2s(const CheckParams& p, int grid, cudaStream_t s) {
  check_d2s_kernel<SIG><<<grid, kBlock, 0, s>>>(p);
}

template <int SIG>
KernelSet make_d2s_set() {
  KernelSet k{};
  k.sigma = SIG;
  k.d = 2;
  k.f_mode = 0;
  k.sym = 3;
  k.sweep = &launch_sweep_d2s<SIG>;
  k.check = &launch_check_d2s<SIG>;
  k.sweep_fn = (const void*)&sweep_d2s_kernel<SIG, false>;  // the plain sweep sizes the grid
  k.check_fn = (const void*)&check_d2s_kernel<SIG>;
  k.tails_per_thread = 2;
  k.sweep_algo_bytes = 20;  // 8 B of v_{t-1} + 4 B of v_{t-2} (the block serves both tails) + 8 B written
  k.check_algo_bytes = 8;
  return k;
}

}  // namespace lcs
