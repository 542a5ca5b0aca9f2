/*
 * lcs_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * feasible-triplet method of Heineman et al., "Improved Lower Bounds on the
 * Expected Length of Longest Common Subsequences" (arXiv 2407.10925).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header,
 * table or constant with the CUDA library and the library never calls it.
 *
 * What it computes (paper section 2.1):
 *   - states are d-tuples A = (a_1..a_d) of length-h strings over an alphabet
 *     of sigma letters; an iterate is a vector over all sigma^(d h) states;
 *   - F_z(v_1..v_d, A) (Algorithm 1): N = strings whose head differs from z;
 *     the mean, over all appended characters c in Sigma^|N|, of v_|N| at the
 *     tuple where each string in N loses its head and gains c_j at its end;
 *   - F(v_1..v_d)[A] = b(A) + max_z F_z (Eq. ineq3), b(A) = 1 iff all heads
 *     agree;
 *   - FeasibleTriplet (Algorithm 2): v_t = F(v_{t-1},..,v_{t-d}) from a zero
 *     start; R from the increment v_t - v_{t-1}; W = v_t + dR -
 *     F(v_t + (d-1)R, .., v_t); E = max(0, max W); keep (v_t, R, E) when
 *     R - E >= r - eps; the bound is d (r - eps) (Eq. lwrbound).
 *
 * Index of a state (paper section 3.2, generalised from bits to base-sigma
 * digits): digits are written head first, and within one position string
 * a_1 first, so for sigma = d = 2 the index interleaves the bits of a and b
 * starting with a.  The digit of string j (0-based) at position p (0 = head)
 * has weight sigma^(d (h-1-p) + (d-1-j)).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   R1  w_n is indexed by the total number of random characters; advancing k
 *       strings reads the iterate k steps back (F_z reads v_|N|).
 *   R2  F_z with N empty (all heads equal z) is not a candidate of the max.
 *       Letters z with the same N_z give the same F_z; each N is evaluated once.
 *   R3  b is added once, outside the max.
 *   R4  R is the minimum increment by default: the text defines r as the
 *       largest value that every entry of the increment reaches.  r_mode = 1
 *       takes the maximum, the reading of Algorithm 2 as printed.  Both give
 *       feasible triplets because E is evaluated for whichever R is taken.
 *   R5  Summation order (f64 arithmetic): one flat left-to-right accumulation
 *       over c in lexicographic order, c of the first advanced string most
 *       significant, exactly as the loop of Algorithm 1 is written; then one
 *       IEEE division by sigma^|N|.
 *   R6  Arithmetic.  "f64": IEEE double, round to nearest, for the iterates;
 *       the feasibility check is evaluated in directed rounding (F rounded
 *       down, W rounded up) so the bound is rigorous.  "fx": every value is an
 *       integer multiple of 2^-K held in an int64; sums are exact and each mean
 *       is rounded down (floor), so the same F serves the iteration and the
 *       check, and the check is exact except for floors that only lower F.
 *   R7  argmin of the increment: the smallest index among minimisers.
 *   R8  The triplet test uses ">=", so a later iteration wins ties.
 *   R9  f_mode = 1 (an extension the paper does not use): the max runs over
 *       every non-empty set of advanced strings; for equal heads the full set
 *       carries the +1 of the match.  The paper prints no value for it;
 *       it is pinned by brute force instead (every candidate drops heads,
 *       which can only lower the LCS, so F <= F_all <= W_n) and by values
 *       worked out by hand at single states, one for each kind of winning
 *       set: a singleton of a majority string, a pair with the minority
 *       string, the full set without a match, a proper subset beating the
 *       match on the exact W tables, the full set with its +1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 16
#define ORC_MAXH 64
#define ORC_MAXSIGMA 64
#define ORC_MAXSETS 64 /* sigma sets (f_mode 0) or 2^d - 1 (f_mode 1, d <= 6) */

/* ORC_MUTANT selects a deliberately wrong variant for the mutation test of the
 * pins (tests only; 0 = the oracle as described above). */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EOVERFLOW 3

typedef struct {
  int sigma, d, h;
  uint64_t n; /* number of states sigma^(d h) */
} shape_t;

static int make_shape(int sigma, int d, int h, shape_t* s) {
  if (sigma < 2 || d < 2 || h < 1 || sigma > ORC_MAXSIGMA || d > ORC_MAXD || h > ORC_MAXH) return ORC_EINVAL;
  uint64_t n = 1;
  for (int i = 0; i < d * h; ++i) {
    if (n > UINT64_MAX / (uint64_t)sigma) return ORC_EINVAL;
    n *= (uint64_t)sigma;
  }
  s->sigma = sigma;
  s->d = d;
  s->h = h;
  s->n = n;
  return ORC_OK;
}

static uint64_t upow(uint64_t b, int e) {
  uint64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

/* digits X[p*d + j]: string j, position p (0 = head) */
static void decode(const shape_t* s, uint64_t x, int* X) {
  for (int p = s->h - 1; p >= 0; --p)
    for (int j = s->d - 1; j >= 0; --j) {
      X[p * s->d + j] = (int)(x % (uint64_t)s->sigma);
      x /= (uint64_t)s->sigma;
    }
}

static uint64_t encode(const shape_t* s, const int* X) {
  uint64_t x = 0;
  for (int p = 0; p < s->h; ++p)
    for (int j = 0; j < s->d; ++j) {
#if ORC_MUTANT == 8
      x = x * (uint64_t)s->sigma + (uint64_t)X[p * s->d + (s->d - 1 - j)];
#else
      x = x * (uint64_t)s->sigma + (uint64_t)X[p * s->d + j];
#endif
    }
  return x;
}

/* Y = X with every string listed in adv[0..k) shifted by one character (its
 * head dropped) and character c[m] appended to string adv[m]. */
static void advance(const shape_t* s, const int* X, const int* adv, int k, const int* c, int* Y) {
  memcpy(Y, X, sizeof(int) * (size_t)(s->d * s->h));
  for (int m = 0; m < k; ++m) {
    int j = adv[m];
#if ORC_MUTANT == 1
    for (int p = s->h - 1; p > 0; --p) Y[p * s->d + j] = X[(p - 1) * s->d + j];
    Y[j] = c[m];
#else
    for (int p = 0; p + 1 < s->h; ++p) Y[p * s->d + j] = X[(p + 1) * s->d + j];
    Y[(s->h - 1) * s->d + j] = c[m];
#endif
  }
}

/* c = the cc-th tuple of Sigma^k in lexicographic order (c[0] most significant) */
static void tuple_of(int sigma, int k, uint64_t cc, int* c) {
  for (int m = k - 1; m >= 0; --m) {
    c[m] = (int)(cc % (uint64_t)sigma);
    cc /= (uint64_t)sigma;
  }
}

static int heads_equal(const shape_t* s, const int* X) {
  for (int j = 1; j < s->d; ++j)
    if (X[j] != X[0]) return 0;
  return 1;
}

/* The candidate advance-sets of state X.  f_mode 0: one set per letter z,
 * N_z = strings whose head differs from z, empty sets dropped (R2).  f_mode 1:
 * every non-empty subset.  Sets are written as sorted index lists into
 * sets[i][0..sizes[i]); the return value is the number of sets. */
static int candidate_sets(const shape_t* s, const int* X, int f_mode, int sets[][ORC_MAXD], int* sizes) {
  int m = 0;
  if (f_mode == 0) {
    for (int z = 0; z < s->sigma; ++z) {
      int k = 0;
      for (int j = 0; j < s->d; ++j)
        if (X[j] != z) sets[m][k++] = j;
      if (k == 0) continue;
      /* F_z depends on z only through N_z: a set already listed adds nothing to the max */
      int dup = 0;
      for (int i = 0; i < m && !dup; ++i)
        dup = sizes[i] == k && memcmp(sets[i], sets[m], sizeof(int) * (size_t)k) == 0;
      if (!dup) sizes[m++] = k;
    }
  } else {
#if ORC_MUTANT == 13
    for (uint64_t mask = 1; mask < ((uint64_t)1 << s->d) - 1; ++mask) {
#else
    for (uint64_t mask = 1; mask < ((uint64_t)1 << s->d); ++mask) {
#endif
#if ORC_MUTANT == 12
      /* only the sets N_z of f_mode 0 and the full set */
      int is_nz = mask == ((uint64_t)1 << s->d) - 1;
      for (int z = 0; z < s->sigma && !is_nz; ++z) {
        uint64_t nz = 0;
        for (int j = 0; j < s->d; ++j)
          if (X[j] != z) nz |= (uint64_t)1 << j;
        is_nz = nz == mask;
      }
      if (!is_nz) continue;
#endif
      int k = 0;
      for (int j = 0; j < s->d; ++j)
        if (mask >> j & 1) sets[m][k++] = j;
      sizes[m++] = k;
    }
  }
  return m;
}

static int f_mode_ok(const shape_t* s, int f_mode) { return f_mode == 0 || (f_mode == 1 && s->d <= 6); }

/* ------------------------------------------------------------------------ */
/* f64 arithmetic with directed rounding.  Each helper returns the exact
 * result rounded in the stated direction, using error-free transformations:
 * Knuth's TwoSum for addition, the fma-computed residual for products and for
 * the remainder of a division (the remainder a - q b of q = RN(a/b) is exactly
 * representable).  Round-to-nearest results are plain IEEE operations. */

enum { RN = 0, RD = 1, RU = 2 };

static double add_dir(double a, double b, int mode) {
  double s = a + b;
  if (mode == RN || !isfinite(s)) return s;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb); /* exact: a + b = s + err */
  if (mode == RD && err < 0) return nextafter(s, -INFINITY);
  if (mode == RU && err > 0) return nextafter(s, INFINITY);
  return s;
}

static double mul_dir(double a, double b, int mode) {
  double p = a * b;
  if (mode == RN || !isfinite(p)) return p;
  double err = fma(a, b, -p); /* exact: a b = p + err */
  if (mode == RD && err < 0) return nextafter(p, -INFINITY);
  if (mode == RU && err > 0) return nextafter(p, INFINITY);
  return p;
}

/* a / m for m > 0 */
static double div_dir(double a, double m, int mode) {
  double q = a / m;
  if (mode == RN || !isfinite(q)) return q;
  double rem = fma(-q, m, a); /* exact: a = q m + rem */
  if (mode == RD && rem < 0) return nextafter(q, -INFINITY);
  if (mode == RU && rem > 0) return nextafter(q, INFINITY);
  return q;
}

/* exported for tests of the helpers */
double orc_add_dir(double a, double b, int mode) { return add_dir(a, b, mode); }
double orc_mul_dir(double a, double b, int mode) { return mul_dir(a, b, mode); }
double orc_div_dir(double a, double m, int mode) { return div_dir(a, m, mode); }

/* F at one state, f64.  v[k-1] is the k-th argument of F (v_k).  With mode RN
 * this is the iteration; with mode RD every operation rounds down, which makes
 * the result a lower bound of the exact F of the same inputs. */
static double F_state_f64(const shape_t* s, const double* const* v, uint64_t x, int f_mode, int mode, int* X, int* Y) {
  int sets[ORC_MAXSETS][ORC_MAXD];
  int sizes[ORC_MAXSETS];
  int c[ORC_MAXD];
  decode(s, x, X);
  int b = heads_equal(s, X);
  int m = candidate_sets(s, X, f_mode, sets, sizes);
  double best = -INFINITY;
  for (int i = 0; i < m; ++i) {
    int k = sizes[i];
    uint64_t terms = upow((uint64_t)s->sigma, k);
    double acc = 0.0;
    for (uint64_t cc = 0; cc < terms; ++cc) { /* Algorithm 1's loop */
      tuple_of(s->sigma, k, cc, c);
      advance(s, X, sets[i], k, c, Y);
#if ORC_MUTANT == 2
      acc = add_dir(acc, v[s->d - k][encode(s, Y)], mode);
#else
      acc = add_dir(acc, v[k - 1][encode(s, Y)], mode);
#endif
    }
#if ORC_MUTANT == 3
    double mean = div_dir(acc, (double)upow((uint64_t)s->sigma, s->d), mode);
#else
    double mean = div_dir(acc, (double)terms, mode);
#endif
#if ORC_MUTANT == 14
#elif ORC_MUTANT == 15
    if (f_mode == 1 && b) mean = add_dir(1.0, mean, mode);
#else
    if (f_mode == 1 && b && k == s->d) mean = add_dir(1.0, mean, mode); /* R9 */
#endif
#if ORC_MUTANT == 4
    if (best == -INFINITY || mean < best) best = mean;
#else
    if (mean > best) best = mean;
#endif
  }
  if (f_mode == 1) return best;
#if ORC_MUTANT == 5
  return best;
#else
  return add_dir((double)b, best, mode);
#endif
}

/* ------------------------------------------------------------------------ */
/* fx arithmetic: int64 multiples of 2^-K, exact sums, floor means. */

static int64_t floor_div128(__int128 a, int64_t m) { /* m > 0 */
  __int128 q = a / m;
  if (a % m != 0 && a < 0) q -= 1;
  return (int64_t)q;
}

static int fits64(__int128 a) { return a >= (__int128)INT64_MIN && a <= (__int128)INT64_MAX; }

static int F_state_fx(const shape_t* s, const int64_t* const* v, uint64_t x, int f_mode, int frac_bits, int* X, int* Y, int64_t* out) {
  int sets[ORC_MAXSETS][ORC_MAXD];
  int sizes[ORC_MAXSETS];
  int c[ORC_MAXD];
  const int64_t one = (int64_t)1 << frac_bits;
  decode(s, x, X);
  int b = heads_equal(s, X);
  int m = candidate_sets(s, X, f_mode, sets, sizes);
  __int128 best = 0;
  int have = 0;
  for (int i = 0; i < m; ++i) {
    int k = sizes[i];
    uint64_t terms = upow((uint64_t)s->sigma, k);
    __int128 acc = 0;
    for (uint64_t cc = 0; cc < terms; ++cc) {
      tuple_of(s->sigma, k, cc, c);
      advance(s, X, sets[i], k, c, Y);
#if ORC_MUTANT == 2
      acc += v[s->d - k][encode(s, Y)];
#else
      acc += v[k - 1][encode(s, Y)];
#endif
    }
#if ORC_MUTANT == 3
    __int128 mean = floor_div128(acc, (int64_t)upow((uint64_t)s->sigma, s->d));
#else
    __int128 mean = floor_div128(acc, (int64_t)terms);
#endif
#if ORC_MUTANT == 14
#elif ORC_MUTANT == 15
    if (f_mode == 1 && b) mean += one;
#else
    if (f_mode == 1 && b && k == s->d) mean += one; /* R9 */
#endif
#if ORC_MUTANT == 4
    if (!have || mean < best) best = mean, have = 1;
#else
    if (!have || mean > best) best = mean, have = 1;
#endif
  }
#if ORC_MUTANT != 5
  if (f_mode == 0 && b) best += one;
#endif
  if (!fits64(best)) return ORC_EOVERFLOW;
  *out = (int64_t)best;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Exported F over a range of states [x0, x1): out[x - x0]. */

int orc_F_f64(int sigma, int d, int h, int f_mode, int mode, const double* const* v, uint64_t x0, uint64_t x1, double* out) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (x1 > s.n || x0 > x1 || !f_mode_ok(&s, f_mode) || mode < RN || mode > RU) return ORC_EINVAL;
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  for (uint64_t x = x0; x < x1; ++x) out[x - x0] = F_state_f64(&s, v, x, f_mode, mode, X, Y);
  return ORC_OK;
}

int orc_F_fx(int sigma, int d, int h, int f_mode, int frac_bits, const int64_t* const* v, uint64_t x0, uint64_t x1, int64_t* out) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (x1 > s.n || x0 > x1 || !f_mode_ok(&s, f_mode) || frac_bits < 0 || frac_bits > 60) return ORC_EINVAL;
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  for (uint64_t x = x0; x < x1; ++x) {
    st = F_state_fx(&s, v, x, f_mode, frac_bits, X, Y, &out[x - x0]);
    if (st) return st;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Synthetic inputs defined by a counter-based generator, so that F can be
 * evaluated at sampled states of shapes whose vectors would not fit in host
 * memory.  gen_k[y] = base_k + (g(seed_k, y) mod spread) where g(seed, i) is
 * the i-th output of SplitMix64 started at seed (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the state
 * advances by 0x9e3779b97f4a7c15 per output and each output is the state
 * after its increment passed through the published 64-bit finaliser. */

static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ull;
#if ORC_MUTANT == 11
  z = (z ^ (z >> 29)) * 0xbf58476d1ce4e5b9ull;
#else
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
#endif
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

uint64_t orc_splitmix64_at(uint64_t seed, uint64_t i) { return splitmix64_at(seed, i); }

/* canonical index of y for generated inputs: symmetric = 0: y; 1: the smaller
 * of y and its complement N-1-y; 2 (sigma = d = 2): the smallest of y, its
 * complement, its swap (the two strings exchanged) and the swapped complement;
 * 3 (sigma = 2, d = 3): the smallest of the images of y under the six
 * orders of the three strings, each with and without the complement */
static uint64_t canonical_index(const shape_t* s, uint64_t y, int symmetric) {
  if (symmetric == 0) return y;
  uint64_t c = s->n - 1 - y, best = y < c ? y : c;
  if (symmetric == 2) {
    uint64_t w = ((y >> 1) & 0x5555555555555555ull) | ((y & 0x5555555555555555ull) << 1);
    uint64_t wc = s->n - 1 - w;
    if (w < best) best = w;
#if ORC_MUTANT != 10
    if (wc < best) best = wc;
#endif
  }
  if (symmetric == 3) {
    /* string j's letter at position p sits at bit 3 (h-1-p) + 2 - j */
    static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int q = 0; q < 6; ++q) {
      uint64_t w = 0;
      for (int j = 0; j < 3; ++j)      /* the new string j is the old string order[q][j] */
        for (int i = 0; i < s->h; ++i) /* bit i of string order[q][j] */
          w |= ((y >> (3 * i + 2 - order[q][j])) & 1ull) << (3 * i + 2 - j);
      uint64_t wc = s->n - 1 - w;
      if (w < best) best = w;
#if ORC_MUTANT != 9
      if (wc < best) best = wc;
#endif
    }
  }
  return best;
}

/* F (fx) at the states xs[0..m) with argument k (1-based) given by
 * base[k-1] + (splitmix64_at(seed[k-1], canonical_index(y)) mod spread), so
 * that symmetric = 1 gives inputs invariant under the complement map of
 * sigma = 2, symmetric = 2 inputs also invariant under exchanging the two
 * strings (sigma = d = 2) and symmetric = 3 inputs under every order of the
 * three strings (sigma = 2, d = 3).  Each state is evaluated exactly as F_state_fx
 * does, reading through the generator. */
int orc_F_fx_generated(int sigma, int d, int h, int frac_bits, const uint64_t* seed, const int64_t* base, uint64_t spread,
                       int symmetric, const uint64_t* xs, uint64_t m, int64_t* out) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (frac_bits < 0 || frac_bits > 60 || spread == 0 || symmetric < 0 || symmetric > 3) return ORC_EINVAL;
  if (symmetric && sigma != 2) return ORC_EINVAL;
  if (symmetric == 2 && d != 2) return ORC_EINVAL;
  if (symmetric == 3 && d != 3) return ORC_EINVAL;
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  int sets[ORC_MAXSETS][ORC_MAXD];
  int sizes[ORC_MAXSETS];
  int c[ORC_MAXD];
  const int64_t one = (int64_t)1 << frac_bits;
  for (uint64_t i = 0; i < m; ++i) {
    if (xs[i] >= s.n) return ORC_EINVAL;
    decode(&s, xs[i], X);
    int b = heads_equal(&s, X);
    int nsets = candidate_sets(&s, X, 0, sets, sizes);
    __int128 best = 0;
    int have = 0;
    for (int q = 0; q < nsets; ++q) {
      int k = sizes[q];
      uint64_t terms = upow((uint64_t)s.sigma, k);
      __int128 acc = 0;
      for (uint64_t cc = 0; cc < terms; ++cc) {
        tuple_of(s.sigma, k, cc, c);
        advance(&s, X, sets[q], k, c, Y);
        uint64_t y = canonical_index(&s, encode(&s, Y), symmetric);
        acc += base[k - 1] + (int64_t)(splitmix64_at(seed[k - 1], y) % spread);
      }
      __int128 mean = floor_div128(acc, (int64_t)terms);
      if (!have || mean > best) best = mean, have = 1;
    }
    if (b) best += one;
    if (!fits64(best)) return ORC_EOVERFLOW;
    out[i] = (int64_t)best;
  }
  return ORC_OK;
}

uint64_t orc_encode(int sigma, int d, int h, const int* X) {
  shape_t s;
  if (make_shape(sigma, d, h, &s)) return UINT64_MAX;
  return encode(&s, X);
}

int orc_decode(int sigma, int d, int h, uint64_t x, int* X) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (x >= s.n) return ORC_EINVAL;
  decode(&s, x, X);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Feasibility check (Algorithm 2's W and E; Lemma 1's third condition):
 * W = u + dR - F(u + (d-1)R, .., u + 0R), E = max(0, max W).  work holds
 * (d+1) * n values of scratch; W_out (n values) is optional. */

int orc_check_f64(int sigma, int d, int h, int f_mode, const double* u, double R, double* work, double* W_out, double* E_out) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (!f_mode_ok(&s, f_mode)) return ORC_EINVAL;
  const uint64_t n = s.n;
  const double* args[ORC_MAXD];
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  /* the k-th argument u + (d-k) R, rounded down */
  for (int k = 1; k <= d; ++k) {
    double* w = work + (uint64_t)(k - 1) * n;
#if ORC_MUTANT == 7
    double shift = 0.0;
#else
    double shift = mul_dir((double)(d - k), R, RD);
#endif
    for (uint64_t x = 0; x < n; ++x) w[x] = add_dir(u[x], shift, RD);
    args[k - 1] = w;
  }
  double* Fd = work + (uint64_t)d * n;
  for (uint64_t x = 0; x < n; ++x) Fd[x] = F_state_f64(&s, args, x, f_mode, RD, X, Y);
  double dR_up = mul_dir((double)d, R, RU);
  double E = 0.0;
  for (uint64_t x = 0; x < n; ++x) {
    double W = add_dir(add_dir(u[x], dR_up, RU), -Fd[x], RU); /* rounded up */
    if (W_out) W_out[x] = W;
    if (W > E) E = W;
  }
  *E_out = E;
  return ORC_OK;
}

int orc_check_fx(int sigma, int d, int h, int f_mode, int frac_bits, const int64_t* u, int64_t R, int64_t* work, int64_t* W_out,
                 int64_t* E_out) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (!f_mode_ok(&s, f_mode) || frac_bits < 0 || frac_bits > 60) return ORC_EINVAL;
  const uint64_t n = s.n;
  const int64_t* args[ORC_MAXD];
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  for (int k = 1; k <= d; ++k) {
    int64_t* w = work + (uint64_t)(k - 1) * n;
#if ORC_MUTANT == 7
    __int128 shift = 0;
#else
    __int128 shift = (__int128)(d - k) * R;
#endif
    for (uint64_t x = 0; x < n; ++x) {
      __int128 a = (__int128)u[x] + shift;
      if (!fits64(a)) return ORC_EOVERFLOW;
      w[x] = (int64_t)a;
    }
    args[k - 1] = w;
  }
  int64_t* Fd = work + (uint64_t)d * n;
  for (uint64_t x = 0; x < n; ++x) {
    st = F_state_fx(&s, args, x, f_mode, frac_bits, X, Y, &Fd[x]);
    if (st) return st;
  }
  __int128 E = 0;
  for (uint64_t x = 0; x < n; ++x) {
    __int128 W = (__int128)u[x] + (__int128)d * R - Fd[x];
    if (!fits64(W)) return ORC_EOVERFLOW;
    if (W_out) W_out[x] = (int64_t)W;
    if (W > E) E = W;
  }
  *E_out = (int64_t)E;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2.  The caller owns every buffer.
 *   hist: (d+1) * n values; on entry row k (k = 0..d-1) holds the start v_k.
 *         On return row res->newest_row holds the newest iterate and row
 *         (newest_row - k) mod (d+1) the k-th older one (k < d).
 *   work: (d+1) * n values of scratch for the feasibility check.
 *   u_out: optional, n values; receives the kept u (v_0 if no iterate is kept).
 * One iteration is one evaluation of F followed by the increment; iteration
 * `it` is checked when check_every > 0 and it % check_every == 0, and the
 * last iteration is always checked (check_every = 1 is Algorithm 2 as
 * printed).  n_iters iterations correspond to Algorithm 2's loop bound
 * n = d + n_iters - 1. */
typedef struct {
  int64_t iters_done;
  int64_t newest_row;
  int64_t have_check; /* at least one feasibility check was run */
  int64_t kept_iter;  /* iteration whose (v_t, R, E) is kept; -1 = the initial (v_0, 0, 0) */
  uint64_t argmin;    /* state index of the last iteration's R (smallest among ties) */
  /* last iteration */
  double R_f64, E_f64;
  int64_t R_fx, E_fx;
  /* kept triplet */
  double r_f64, eps_f64;
  int64_t r_fx, eps_fx;
  double bound_rd; /* d (r - eps), rounded down */
} orc_result;

/* round-down conversion of an int64 multiple of 2^-K to double */
static double fx_to_double_rd(int64_t a, int frac_bits) {
  double x = (double)a; /* round to nearest */
  if (x >= 9223372036854775808.0) x = nextafter(x, -INFINITY);
  else if ((__int128)(int64_t)x > (__int128)a) x = nextafter(x, -INFINITY);
  return ldexp(x, -frac_bits);
}

double orc_fx_to_double_rd(int64_t a, int frac_bits) { return fx_to_double_rd(a, frac_bits); }

int orc_run_f64(int sigma, int d, int h, int64_t n_iters, int check_every, int r_mode, int f_mode, double* hist, double* work,
                double* u_out, orc_result* res) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (n_iters < 0 || check_every < 0 || (r_mode != 0 && r_mode != 1) || !f_mode_ok(&s, f_mode)) return ORC_EINVAL;
  const uint64_t n = s.n;
  const int rows = d + 1;
  memset(res, 0, sizeof(*res));
  res->kept_iter = -1;
  if (u_out) memcpy(u_out, hist, (size_t)n * sizeof(double)); /* the initial triplet (v_0, 0, 0) */
  double r = 0.0, eps = 0.0;
  int newest = d - 1; /* row holding v_{t-1} */
  const double* args[ORC_MAXD];
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  for (int64_t it = 1; it <= n_iters; ++it) {
    int out_row = (newest + 1) % rows;
    double* vt = hist + (uint64_t)out_row * n;
    for (int k = 1; k <= d; ++k) args[k - 1] = hist + (uint64_t)((newest - (k - 1) + rows) % rows) * n;
    for (uint64_t x = 0; x < n; ++x) vt[x] = F_state_f64(&s, args, x, f_mode, RN, X, Y);
    const double* vprev = args[0];
    double R = 0.0;
    uint64_t arg = 0;
    for (uint64_t x = 0; x < n; ++x) {
#if ORC_MUTANT == 6
      double inc = vprev[x] - vt[x];
#else
      double inc = vt[x] - vprev[x];
#endif
      if (x == 0 || (r_mode == 0 ? inc < R : inc > R)) R = inc, arg = x;
    }
    newest = out_row;
    res->R_f64 = R;
    res->argmin = arg;
    if ((check_every > 0 && it % check_every == 0) || it == n_iters) {
      double E;
      st = orc_check_f64(sigma, d, h, f_mode, vt, R, work, NULL, &E);
      if (st) return st;
      res->E_f64 = E;
      res->have_check = 1;
      if (R - E >= r - eps) {
        r = R;
        eps = E;
        res->kept_iter = it;
        if (u_out) memcpy(u_out, vt, (size_t)n * sizeof(double));
      }
    }
    res->iters_done = it;
  }
  res->newest_row = newest;
  res->r_f64 = r;
  res->eps_f64 = eps;
  res->bound_rd = mul_dir((double)d, add_dir(r, -eps, RD), RD);
  return ORC_OK;
}

int orc_run_fx(int sigma, int d, int h, int64_t n_iters, int check_every, int r_mode, int f_mode, int frac_bits, int64_t* hist,
               int64_t* work, int64_t* u_out, orc_result* res) {
  shape_t s;
  int st = make_shape(sigma, d, h, &s);
  if (st) return st;
  if (n_iters < 0 || check_every < 0 || (r_mode != 0 && r_mode != 1) || !f_mode_ok(&s, f_mode) || frac_bits < 0 || frac_bits > 60)
    return ORC_EINVAL;
  const uint64_t n = s.n;
  const int rows = d + 1;
  memset(res, 0, sizeof(*res));
  res->kept_iter = -1;
  if (u_out) memcpy(u_out, hist, (size_t)n * sizeof(int64_t));
  int64_t r = 0, eps = 0;
  int newest = d - 1;
  const int64_t* args[ORC_MAXD];
  int X[ORC_MAXD * ORC_MAXH], Y[ORC_MAXD * ORC_MAXH];
  for (int64_t it = 1; it <= n_iters; ++it) {
    int out_row = (newest + 1) % rows;
    int64_t* vt = hist + (uint64_t)out_row * n;
    for (int k = 1; k <= d; ++k) args[k - 1] = hist + (uint64_t)((newest - (k - 1) + rows) % rows) * n;
    for (uint64_t x = 0; x < n; ++x) {
      st = F_state_fx(&s, args, x, f_mode, frac_bits, X, Y, &vt[x]);
      if (st) return st;
    }
    const int64_t* vprev = args[0];
    int64_t R = 0;
    uint64_t arg = 0;
    for (uint64_t x = 0; x < n; ++x) {
#if ORC_MUTANT == 6
      __int128 inc128 = (__int128)vprev[x] - vt[x];
#else
      __int128 inc128 = (__int128)vt[x] - vprev[x];
#endif
      if (!fits64(inc128)) return ORC_EOVERFLOW;
      int64_t inc = (int64_t)inc128;
      if (x == 0 || (r_mode == 0 ? inc < R : inc > R)) R = inc, arg = x;
    }
    newest = out_row;
    res->R_fx = R;
    res->argmin = arg;
    if ((check_every > 0 && it % check_every == 0) || it == n_iters) {
      int64_t E;
      st = orc_check_fx(sigma, d, h, f_mode, frac_bits, vt, R, work, NULL, &E);
      if (st) return st;
      res->E_fx = E;
      res->have_check = 1;
      if ((__int128)R - E >= (__int128)r - eps) {
        r = R;
        eps = E;
        res->kept_iter = it;
        if (u_out) memcpy(u_out, vt, (size_t)n * sizeof(int64_t));
      }
    }
    res->iters_done = it;
  }
  res->newest_row = newest;
  res->r_fx = r;
  res->eps_fx = eps;
  __int128 B = (__int128)d * ((__int128)r - eps);
  if (!fits64(B)) return ORC_EOVERFLOW;
  res->bound_rd = fx_to_double_rd((int64_t)B, frac_bits);
  return ORC_OK;
}

/* size of orc_result, so the Python side can check its mirror of the struct */
int orc_result_size(void) { return (int)sizeof(orc_result); }
