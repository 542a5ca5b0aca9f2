/*
 * lcs_bound.h -- C ABI of the GB300 feasible-triplet library.
 *
 * The library computes rigorous lower bounds on the Chvatal-Sankoff constants
 * gamma_{sigma,d} with the feasible-triplet method of Heineman, Miller,
 * Reichman, Salls, Sarkozy and Soiffer, "Improved Lower Bounds on the Expected
 * Length of Longest Common Subsequences" (arXiv 2407.10925), section 2.1:
 *
 *   iterate   v_t = F(v_{t-1}, .., v_{t-d})        (Algorithm 2; F is Eq. ineq3
 *                                                   built from Algorithm 1's F_z)
 *   increment R_t = min_x (v_t - v_{t-1})[x]        (Algorithm 2; the text before it)
 *   check     E_t = max(0, max_x W[x]),
 *             W = v_t + dR - F(v_t + (d-1)R, .., v_t)    (Algorithm 2; Lemma 1)
 *   keep      (u, r, eps) <- (v_t, R_t, E_t) when R_t - E_t >= r - eps
 *   bound     gamma_{sigma,d} >= d (r - eps)         (Eq. lwrbound)
 *
 * STATE INDEX.  A state is a d-tuple of length-h strings over {0..sigma-1}.
 * Its index is the paper's interleaved index (section 3.2) generalised to base
 * sigma: the digit of string j (0-based) at position p (0 = head) has weight
 * sigma^(d (h-1-p) + (d-1-j)).  For sigma = d = 2 the bits of a and b are
 * interleaved starting with a: a = 1011, b = 0010 has index 142.  Every vector
 * that crosses this interface uses that order, and the device buffers use it
 * too.
 *
 * ARITHMETIC.  Iterates are stored as int64 fixed-point numbers: a stored
 * integer q means q * 2^-K (K = frac_bits, default 44).  Sums are exact; each
 * mean over sigma^k terms is rounded down (floor).  Because floor only lowers
 * F, the same F serves the iteration and the check, and E computed this way
 * is an upper bound of the exact E for the stored u and R: the reported
 * bound d (r - eps) is rigorous.  Doubles crossing the interface are
 * converted: inputs to fixed point rounding down, outputs to double rounding
 * to nearest, except the bound, which is rounded down.
 *
 * STREAMS AND ERRORS.  All device work is enqueued on the handle's stream.
 * Calls marked "asynchronous" return before the work ends; errors of the
 * enqueued work surface at the next synchronising call.  Every call returns a
 * status; lcs_bound_errstr() gives its text and lcs_bound_last_error() the
 * message of the most recent failure on the calling thread.  Handles are not
 * thread-safe: use one handle from one host thread at a time.
 *
 * OWNERSHIP.  The library owns every buffer it allocates (through the
 * allocator in lcs_bound_opts if one is given) and frees them in
 * lcs_bound_destroy().  Pointers passed in are borrowed for the duration of
 * the call (for device pointers: until the enqueued work has read them).
 */
#ifndef LCS_BOUND_H
#define LCS_BOUND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lcs_bound lcs_bound_t; /* opaque; library-owned */

typedef enum {
  LCS_OK = 0,
  LCS_EINVAL = 1,       /* bad argument (shape, mode, pointer, size) */
  LCS_ENOMEM = 2,       /* device or host allocation failed */
  LCS_ECUDA = 3,        /* a CUDA call failed; see lcs_bound_last_error() */
  LCS_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
  LCS_ENOBOUND = 5,     /* no feasibility check has run yet */
  LCS_EOVERFLOW = 6,    /* fixed-point headroom would be exceeded */
  LCS_EUNSUPPORTED = 7, /* (sigma, d, f_mode) has no kernel in the library */
  LCS_EIO = 8           /* a checkpoint file could not be written or read */
} lcs_status;

typedef struct {
  /* 0: check only at the last iteration of each lcs_bound_iterate() call;
   * k > 0: check every k-th iteration (counted from creation) and at the last
   * iteration of each call.  1 is Algorithm 2 as printed. */
  int check_every;
  /* 0: R = minimum increment (default).  1: R = maximum increment (Algorithm
   * 2 as printed).  E is evaluated for whichever R is taken. */
  int r_mode;
  /* 0: F as in the paper (max over z of F_z).  1: the max runs over every
   * non-empty set of advanced strings, and for equal heads the full set carries
   * the +1 of the match -- an extension the paper does not use (also a valid
   * lower bound: dropping heads never increases an LCS); kernels for sigma = 2,
   * d = 2, 3 and sigma = 3, d = 2, else LCS_EUNSUPPORTED. */
  int f_mode;
  /* K, the number of fractional bits of the fixed-point iterates; 0 -> 44.
   * Valid range 8..56. */
  int frac_bits;
  /* 1: keep a device copy of the kept u (one more vector of memory, and a
   * copy at each check that keeps).  0: u is not retained. */
  int keep_u;
  /* 1 (default): for sigma = 2, store and compute only the states whose first
   * string starts with 0, using the complement symmetry of the paper's
   * section 3.3 (v[N-1-x] = v[x]).  The start vectors must then be symmetric.
   * 0: store every state.  Ignored for sigma != 2. */
  int symmetry;
  /* 1: record CUDA events around each sweep and check launch; read them with
   * lcs_bound_stats().  0 (default): no events. */
  int timing;
  /* Device allocator.  NULL alloc -> cudaMalloc / cudaFree.  alloc returns a
   * device pointer aligned to at least 256 bytes, or NULL on failure. */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
  /* cudaStream_t to enqueue on; NULL -> the library creates its own stream. */
  void* stream;
  /* 0 (default): iterates stored as int64 fixed point.  1: offset-normalised
   * 32-bit storage -- each vector holds w = v - c in int32 with one int64
   * offset c per vector, kept on the device; half the bytes of every sweep.
   * F is computed exactly as with int64 storage (Lemma 1's translation
   * invariance: a mean of w + c is the mean of w plus c), so the iterates,
   * R, E and the bound are bit for bit those of int64 storage at the same
   * frac_bits, as long as every stored w fits in 32 bits; an output that does
   * not sets LCS_EOVERFLOW (sticky, reported by the next read).  The offset of
   * a new iterate is the previous iterate's value at state 0 plus the last
   * reduced R, so every w stays within the spread of one iterate plus one
   * step (2^(31 - frac_bits) units must hold it).  Needs sigma = d = 2,
   * h >= 6, complement-symmetric storage, f_mode 0, keep_u 0 and
   * frac_bits <= 30 (LCS_EUNSUPPORTED / LCS_EINVAL otherwise).  Starts and
   * exports take and give int64 values: lcs_bound_set_start_stored_fx,
   * lcs_bound_set_start_lift_fx, lcs_bound_export_fx, lcs_bound_export_stored_fx,
   * lcs_bound_export; the other start forms, the orbit form, save/restore and
   * check_vector return LCS_EUNSUPPORTED.  The start must be swap-symmetric. */
  int storage;
  /* 0 (default) or 1: the number of the d + 1 iterate vectors placed in
   * pinned, mapped host memory (an anonymous mapping advised for huge pages,
   * then registered) instead of device memory --
   * the sweeps read and write that vector over the host link, so a shape
   * whose vectors do not all fit in HBM runs out of core.  The host vector
   * does not come from `alloc`.  Results are bit for bit those of an all-HBM
   * handle. */
  int host_slots;
} lcs_bound_opts;

/* Fill *opts with the defaults listed above. */
lcs_status lcs_bound_default_opts(lcs_bound_opts* opts);

/* Create a handle for the shape (sigma, d, h): sigma >= 2, 2 <= d <= 16,
 * h >= 1, sigma^(d h) < 2^40 states (LCS_EINVAL otherwise).  Allocates d+1
 * iterate vectors (d+2 with keep_u) on the current device and sets v_0 = .. =
 * v_{d-1} = 0 (Algorithm 2's zero start).  opts may be NULL (defaults).  On
 * failure *out is NULL.  Synchronous.
 * Kernels: specialised ones for sigma = 2 (d = 2..5), sigma = 3 (d = 2, 3)
 * and sigma = 4, 5 (d = 2); every other shape with sigma <= 10 runs the
 * general kernels (f_mode 0 only, full storage whatever opts.symmetry says).
 * For h >= 2 and sigma^d <= 16384 they run in block form (Algorithm 1's sums
 * formed once per tail tuple from blocks of sigma^d consecutive values, then
 * one pass over the states); the handle then also allocates a table of
 * sigma 2^d means per tail tuple (8 sigma 2^d sigma^(d (h-1)) bytes), the
 * term offsets ((1 + sigma)^d 16-bit values) and a list of the blocks that
 * hold sums, all through `alloc` when given.  Larger sigma, or f_mode 1
 * without a specialised kernel: LCS_EUNSUPPORTED.  Sums of sigma^d values
 * must stay inside int64: large sigma^d needs fewer fractional bits
 * (LCS_EOVERFLOW otherwise). */
lcs_status lcs_bound_create(int sigma, int d, int h, const lcs_bound_opts* opts, lcs_bound_t** out);

/* Number of states sigma^(d h) of the handle's shape, and the number the
 * device stores (half of it under complement symmetry). */
lcs_status lcs_bound_size(const lcs_bound_t* hnd, uint64_t* n_states, uint64_t* n_stored);

/* The shape (sigma, d, h) a single-instance handle was created with; any
 * output pointer may be NULL.  LCS_EINVAL for a batch handle (its instances
 * have their own shapes).  Lets a caller size the d vectors that
 * set_start and export take without keeping the shape itself. */
lcs_status lcs_bound_shape(const lcs_bound_t* hnd, int* sigma, int* d, int* h);

/* Run n_iters >= 0 iterations of Algorithm 2: n_iters evaluations of F, the
 * increment of each iteration that is checked, and the checks selected by
 * check_every (always including the last of this call when n_iters > 0).
 * Asynchronous.  LCS_EOVERFLOW if the iterates could leave the fixed-point
 * range during the call (values grow by at most 1 per iteration). */
lcs_status lcs_bound_iterate(lcs_bound_t* hnd, int64_t n_iters);

/* The kept triplet and the bound.  Synchronises the stream.
 *   bound_rd:     d (r - eps) rounded down to a double (rigorous)
 *   argmin_state: index of a state attaining the increment R of the
 *                 iteration last checked (smallest index among ties)
 *   r, eps:       the kept R and E as doubles (rounded to nearest)
 *   at_iter:      iteration count (since creation) of the kept u; -1 if no
 *                 check has kept an iterate (the initial triplet (v_0, 0, 0))
 * Any output pointer may be NULL.  LCS_ENOBOUND if no check has run. */
lcs_status lcs_bound_read(lcs_bound_t* hnd, double* bound_rd, uint64_t* argmin_state, double* r, double* eps,
                          int64_t* at_iter);

/* Exact fixed-point form of the last results (all values in units of 2^-K). */
typedef struct {
  int64_t iters_done;  /* iterations run since creation (or since set_start) */
  int64_t R;           /* increment of the last checked iteration */
  uint64_t argmin;     /* state attaining R (smallest index among ties) */
  int64_t E;           /* E of the last check */
  int64_t r, eps;      /* kept triplet */
  int64_t kept_iter;   /* -1: the initial triplet (v_0, 0, 0) */
  int64_t have_check;  /* 1 once a check has run */
  int frac_bits;       /* K */
  int status;          /* sticky device-side error status (lcs_status) */
} lcs_bound_report;

/* Synchronises the stream. */
lcs_status lcs_bound_read_report(lcs_bound_t* hnd, lcs_bound_report* out);

/* Replace the d most recent iterates: v[k] (k = 0..d-1) becomes the iterate
 * k steps older than the newest (v[0] newest), each a vector of
 * sigma^(d h) doubles in state-index order, converted to fixed point rounding
 * down.  on_device = 1: the pointers are device pointers; 0: host pointers
 * (copied through a staging buffer).  Resets the iteration count and the kept
 * triplet to the initial (v_oldest, 0, 0).  Under complement symmetry the
 * vectors must satisfy v[N-1-x] = v[x] after conversion, else LCS_EINVAL.
 * Synchronous for host pointers; asynchronous for device pointers. */
lcs_status lcs_bound_set_start(lcs_bound_t* hnd, const double* const* v, int on_device);

/* As lcs_bound_set_start with fixed-point values (units of 2^-K), exact. */
lcs_status lcs_bound_set_start_fx(lcs_bound_t* hnd, const int64_t* const* v, int on_device);

/* The check history: one record per check since creation (or since the last
 * set_start / restore), the newest 4096 kept.  Fixed-point values in units
 * of 2^-K.  No counterpart in the paper beyond Algorithm 2's own quantities. */
typedef struct {
  int64_t iter;        /* iteration count of the checked iterate */
  int64_t R;           /* its increment */
  uint64_t argmin;     /* a state attaining R (smallest index among ties) */
  int64_t E;           /* the check's E */
  int64_t kept;        /* 1 if this check replaced the kept triplet */
  int64_t r, eps;      /* the kept triplet after the check */
  int64_t kept_iter;
} lcs_bound_check_record;
/* Copy the newest min(count, 4096, max_records) records, oldest first, into
 * out (host); *n_checks (may be NULL) receives the number of checks recorded.
 * Synchronises the stream.  LCS_EINVAL for batch handles. */
lcs_status lcs_bound_history(lcs_bound_t* hnd, lcs_bound_check_record* out, int64_t max_records, int64_t* n_checks);

/* The STORED FORM of an iterate: the n_stored values the handle keeps
 * (lcs_bound_size).  Under complement-symmetric storage (sigma = 2 and
 * opts.symmetry) that is the states x < N/2, the rest following from
 * v[N-1-x] = v[x] (section 3.3, Eq. impl:comp_eq); otherwise all N states.
 * These calls move iterates in that form -- half the bytes of the full
 * vectors under symmetry, with no conversion or symmetry check on the way.
 * set_start_stored_fx: as lcs_bound_set_start_fx (v[0] newest, same resets,
 * synchronous), each v[k] holding n_stored fixed-point values.
 * export_stored_fx: as lcs_bound_export_fx for k = -1..d-1, n_stored values;
 * synchronous for a host dst, asynchronous for a device dst.  The paper has
 * no counterpart of either call beyond the symmetry itself. */
lcs_status lcs_bound_set_start_stored_fx(lcs_bound_t* hnd, const int64_t* const* v, int on_device);

/* A start lifted from a shorter shape (sigma = d = 2, complement-symmetric
 * storage; the paper's prefix truncation as a warm start): src is the stored
 * form (4^h_from / 2 fixed-point values, states x < 4^h_from / 2) of an
 * iterate of (2, 2, h_from), 2 <= h_from <= h, on the host (read through the
 * staging pipeline) or the device.  The newest iterate of this handle becomes
 * v[x] = src[x >> 2 (h - h_from)] -- each string cut to its first h_from
 * letters -- and the older one v - r_hat (units of 2^-K).  The lift keeps the
 * complement and swap symmetries of src.  Resets as lcs_bound_set_start_fx.
 * Lemma 1 makes any start legitimate: the bound comes from the check.
 * Synchronous.  No counterpart in the paper beyond the truncation itself. */
lcs_status lcs_bound_set_start_lift_fx(lcs_bound_t* hnd, int h_from, const int64_t* src, int on_device, int64_t r_hat);
lcs_status lcs_bound_export_stored_fx(lcs_bound_t* hnd, int k, int64_t* dst, int on_device);

/* The ORBIT FORM (sigma = d = 2, complement-symmetric storage, h >= 6; other
 * handles get LCS_EUNSUPPORTED).  When an iterate is also symmetric under
 * exchanging the two strings, as every iterate from the zero start is, the
 * stored states of a tail t = (a, b) form one orbit of eight with those of
 * ~t = (~a, ~b), t' = (~b, ~a) and ~t' = (b, a) (each with heads 00 and 01),
 * holding at most four distinct values:
 *   v(00, t) = v(00, ~t'),  v(00, ~t) = v(00, t'),
 *   v(01, t) = v(01, t'),   v(01, ~t) = v(01, ~t').
 * The orbit form keeps those four values, in this order, for one
 * representative per orbit: (s, a, beta) with 0 <= a <= beta < K = 2^(h-2),
 * b = beta (s = 0) or 2^(h-1) - 1 - beta (s = 1).  Strings are (h-1)-bit
 * integers, most significant letter first; the representative's four values
 * sit at 4 q .. 4 q + 3 with q = s K (K + 1) / 2 + beta (beta + 1) / 2 + a.
 * v(g0 g1, (a, b)) is the value of the state whose strings are g0 a and g1 b
 * (heads g0, g1; STATE INDEX above).  *n_orbit = 4 K (K + 1) = 4^(h-1) + 2^h
 * values: about half of the stored form, a quarter of N.
 * set_start_orbit_fx: as lcs_bound_set_start_stored_fx, each v[k] holding
 * n_orbit values; the handle writes all eight states of every orbit, so the
 * start has both symmetries by construction (where an orbit has fewer than
 * eight distinct states its values must agree, as they do in any exported
 * orbit form).  Device vectors must be 16-byte aligned (LCS_EINVAL).
 * export_orbit_fx: as lcs_bound_export_stored_fx, n_orbit values; LCS_EINVAL
 * if the handle's start was not swap-symmetric.  A device dst must be
 * 16-byte aligned.  The paper has no counterpart of these calls beyond the
 * two symmetries. */
lcs_status lcs_bound_orbit_size(const lcs_bound_t* hnd, uint64_t* n_orbit);
lcs_status lcs_bound_set_start_orbit_fx(lcs_bound_t* hnd, const int64_t* const* v, int on_device);
lcs_status lcs_bound_export_orbit_fx(lcs_bound_t* hnd, int k, int64_t* dst, int on_device);

/* Checkpoint and resume (no counterpart in the paper).  lcs_bound_save writes
 * the whole state of a single-instance handle to a file: shape and options,
 * the d most recent iterates in stored form (newest first), the retained u
 * (keep_u), the device results (R, argmin, E, the kept r, eps and iteration,
 * the sticky status) and the iteration count.  lcs_bound_restore reads such a
 * file into a handle created with the same shape and options (LCS_EINVAL
 * otherwise); iterate then continues exactly -- bit for bit -- as the saved
 * handle would have (the check history restarts empty).  Binary,
 * little-endian, for this library version.
 * LCS_EIO when the file cannot be opened, written or is truncated.
 * Synchronous. */
lcs_status lcs_bound_save(lcs_bound_t* hnd, const char* path);
lcs_status lcs_bound_restore(lcs_bound_t* hnd, const char* path);

/* Copy the iterate k steps older than the newest (k = 0..d-1), or with
 * k = -1 the kept u (needs keep_u), into dst: sigma^(d h) values in
 * state-index order.  on_device selects the kind of dst.  Synchronises the
 * stream when dst is a host pointer; with a device pointer the copy is
 * asynchronous on the handle's stream (see lcs_bound_synchronize).
 * Device pointers given to any call are read on the handle's stream: the
 * caller must make sure their contents are complete (for example by
 * synchronising the stream that produced them). */
lcs_status lcs_bound_export(lcs_bound_t* hnd, int k, double* dst, int on_device);
lcs_status lcs_bound_export_fx(lcs_bound_t* hnd, int k, int64_t* dst, int on_device);

/* Evaluate the check of Algorithm 2 (Lemma 1) for an arbitrary vector u
 * (sigma^(d h) fixed-point values, device pointer, state-index order; under
 * complement symmetry only the stored half, the first n_stored values, is
 * read and u must be symmetric) and increment R: writes
 * E = max(0, max_x W[x]) to *E_out (host).  Does not touch the kept triplet.
 * Synchronises the stream. */
lcs_status lcs_bound_check_vector(lcs_bound_t* hnd, const int64_t* u_dev, int64_t R, int64_t* E_out);

/* Timing of the enqueued sweep and check kernels and of the host transfers
 * (needs opts.timing = 1).  Synchronises the stream.  Counts and milliseconds
 * since creation or the last reset. */
typedef struct {
  int64_t sweep_launches;
  double sweep_ms;
  int64_t check_launches;
  double check_ms;
  int64_t kernel_launches; /* every kernel this handle enqueued */
  uint64_t sweep_bytes;    /* algorithmic bytes of all sweeps: 8 (d+1) per stored state */
  uint64_t check_bytes;    /* algorithmic bytes of all checks: 8 per stored state */
  /* host transfers of set_start / export: the copies' device time and bytes in
   * each direction, and the time of the kernels that convert, unpack or pack
   * the transferred values (summed per operation; copies and kernels overlap) */
  double h2d_ms;
  uint64_t h2d_bytes;
  double d2h_ms;
  uint64_t d2h_bytes;
  double xfer_kernel_ms;
} lcs_bound_stats_t;
lcs_status lcs_bound_stats(lcs_bound_t* hnd, lcs_bound_stats_t* out, int reset);

/* Wait until every piece of work enqueued on the handle's stream has ended
 * (for example before reading a device vector filled by lcs_bound_export with
 * on_device = 1 from another stream).  Synchronous. */
lcs_status lcs_bound_synchronize(lcs_bound_t* hnd);

/* Free everything the handle owns (after the stream's pending work ends).
 * NULL is ignored. */
void lcs_bound_destroy(lcs_bound_t* hnd);

/* Host buffers for transfers (no counterpart in the paper): bytes of host
 * memory, pinned and mapped for the device, from an anonymous mapping aligned
 * to 512 MiB and advised for transparent huge pages.  Any call that takes a
 * host vector accepts them.  On this GB300's host link they keep the link's
 * rate from their first use, where parts of ordinary pinned buffers were
 * read at a fraction of it in processes that followed heavy use of the
 * machine.  The memory is not initialised.  lcs_host_free releases a buffer
 * of lcs_host_alloc (LCS_EINVAL for any other pointer; NULL is ignored).
 * Synchronous. */
lcs_status lcs_host_alloc(size_t bytes, void** out);
lcs_status lcs_host_free(void* ptr);

/* Static text of a status code. */
const char* lcs_bound_errstr(lcs_status st);

/* Message of the most recent failure on the calling thread ("" if none). */
const char* lcs_bound_last_error(void);

/* ------------------------------------------------------------------------ */
/* Batches: many small instances of uneven size in one persistent launch.
 *
 * lcs_bound_batch_create makes a handle for n instances (1 <= n <= 16),
 * shapes[i] = {sigma, d, h} (each below 2^36 states; kernels exist for
 * (2,2,h), (2,3,h), (2,4,h) with complement symmetry, (3,2,h), (4,2,h)).
 * Every instance runs Algorithm 2 from the zero start; lcs_bound_iterate(hnd,
 * n) advances all of them by n iterations in lockstep, in ONE cooperative
 * persistent kernel launch that walks a work list of (instance, item) pairs
 * and meets at a grid barrier between phases (sweep; on checked iterations
 * the increment reduction, the check and the keep test).  The launch of each
 * distinct n is captured once in a CUDA graph and replayed.  opts as for
 * lcs_bound_create (keep_u unsupported).  At creation an autotuner times a few
 * iterations for each candidate grid size and item size, and the concurrent
 * mode (lcs_bound_batch_set_mode), keeps the fastest, then returns every
 * vector to the zero start.
 *
 * The grid barrier waits with a clock budget (about 2 s by default); if it
 * runs out the launch ends and the status LCS_ETIMEOUT is reported by the
 * next read, instead of a hang.  lcs_bound_destroy and lcs_bound_synchronize
 * apply; lcs_bound_read/export/set_start/check_vector return LCS_EINVAL on a
 * batch handle: use the calls below, which take the instance index i. */
lcs_status lcs_bound_batch_create(int n, const int (*shapes)[3], const lcs_bound_opts* opts, lcs_bound_t** out);
lcs_status lcs_bound_batch_read(lcs_bound_t* hnd, int i, double* bound_rd, uint64_t* argmin_state, double* r,
                                double* eps, int64_t* at_iter);
lcs_status lcs_bound_batch_report(lcs_bound_t* hnd, int i, lcs_bound_report* out);
/* the newest iterate (k = 0) or an older one (k < d) of instance i, every state, fixed point */
lcs_status lcs_bound_batch_export_fx(lcs_bound_t* hnd, int i, int k, int64_t* dst, int on_device);

typedef struct {
  int n_instances;
  int grid;               /* CTAs of the persistent launch chosen by the autotuner */
  int units_per_item;     /* tiles per work item chosen by the autotuner */
  int graph;              /* 1: launches replay a captured CUDA graph */
  double tuned_ms_per_iter;
  int64_t launches;       /* persistent launches or graph replays so far (kernel launches in mode 1) */
  int mode;               /* 0: one persistent launch; 1: concurrent single-instance kernels; 2: 1 uncaptured */
  double persistent_ms_per_iter;  /* the autotuner's timings of both modes */
  double concurrent_ms_per_iter;
  int graph_captured;     /* 1 once a call was captured in a CUDA graph and instantiated (either mode) */
  int min_ctas_per_sm;    /* the persistent kernel's register budget the autotuner chose: 2 (128
                           * registers a thread) or 4 (64, the heaviest bodies spill) CTAs per SM */
  int64_t graph_replays;  /* iterate calls that replayed a captured graph */
} lcs_bound_batch_info_t;
lcs_status lcs_bound_batch_info(lcs_bound_t* hnd, lcs_bound_batch_info_t* out);
/* Force the execution mode of a batch before its first iteration (LCS_EINVAL
 * afterwards): 0 = the persistent launch with the autotuner's shape, 1 = each
 * instance's single-instance kernels on a stream of its own, forked from and
 * joined to the handle's stream, so the instances run concurrently; a call
 * whose schedule (length, check phase, every instance's ring slot) comes a
 * second time is captured in a CUDA graph and replayed from then on (the
 * iteration numbers the kernels record come from a device count, so a
 * replay records the right ones); 2 = mode 1 never captured.  All modes
 * compute the same iterates and bounds bit for bit; the autotuner times 0
 * and 1 at creation and keeps the faster. */
lcs_status lcs_bound_batch_set_mode(lcs_bound_t* hnd, int mode);

/* Set the grid barrier's clock budget in cycles (testing the timeout path);
 * also clears a previous LCS_ETIMEOUT status. */
lcs_status lcs_bound_batch_set_spin_budget(lcs_bound_t* hnd, int64_t cycles);

/* ------------------------------------------------------------------------ */
/* Learned warm start (sigma = d = 2).  Not part of the paper's method, whose
 * iteration starts from the zero vector; Lemma 1 makes any start legitimate
 * because the bound comes only from a triplet whose feasibility the check
 * verifies, so a warm start changes the work, never the rigor.
 *
 * A 3-layer MLP (49 -> 256 -> 256 -> 1, GELU, FP32 weights on the device)
 * predicts the relative value v[x] - v[0] of a converged iterate.  Inputs: a
 * one-hot of the letters at the first 12 positions of each string (zero
 * beyond h) and h / 16, computed from the smallest index of the state's orbit
 * under complement and string swap (so predictions are symmetric).  Parameters
 * are a flat float array of lcs_mlp_param_count() values: W1 (256 x 49), b1,
 * W2 (256 x 256, out x in), b2, w3, b3.  Handles are not thread-safe. */
typedef struct lcs_mlp lcs_mlp_t;
int64_t lcs_mlp_param_count(void);
/* random initialisation (uniform +-1/sqrt(fan-in), SplitMix64 stream `seed`) */
lcs_status lcs_mlp_create(uint64_t seed, lcs_mlp_t** out);
/* The same with a device allocator for every buffer of the network (as in
 * lcs_bound_opts: alloc returns a device pointer aligned to 256 bytes or NULL;
 * NULL alloc -> cudaMalloc / cudaFree).  A failed allocation gives LCS_ENOMEM:
 * at creation with *out = NULL and everything already allocated freed; later
 * (the training buffers, the inference table) with the handle still valid. */
lcs_status lcs_mlp_create_with_allocator(uint64_t seed, void* (*alloc)(size_t bytes, void* ctx),
                                         void (*free)(void* ptr, void* ctx), void* alloc_ctx, lcs_mlp_t** out);
lcs_status lcs_mlp_get_params(lcs_mlp_t* m, float* host_out);
lcs_status lcs_mlp_set_params(lcs_mlp_t* m, const float* host_in);
/* mean squared error over n host rows (states, their h, targets) and its
 * gradient (host, lcs_mlp_param_count() floats) -- the forward and backward
 * kernels the training uses, for checking them.  Synchronous. */
lcs_status lcs_mlp_gradient(lcs_mlp_t* m, int n, const int64_t* states, const int* hs, const float* targets,
                            float* loss_out, float* grad_out);
/* Adam steps on batches drawn from converged iterates: vectors[i] is a
 * full-length fixed-point device vector (units of 2^-frac_bits) of the shape
 * (2, 2, hs[i]); targets are v[x] - v[0] in units.  Synchronous. */
lcs_status lcs_mlp_train(lcs_mlp_t* m, int n_sets, const int64_t* const* vectors, const int* hs, int64_t steps,
                         int batch, float lr, uint64_t seed, int frac_bits, float* last_loss);
/* predictions (units) for n device states of length h into out_dev (device) */
lcs_status lcs_mlp_predict(lcs_mlp_t* m, int h, int64_t n, const int64_t* states_dev, float* out_dev);
/* the same predictions with BF16 inference for the consecutive states
 * base .. base+n-1 (base + n <= 4^h).  A state enters the network only
 * through the first min(h, 12) positions of its canonical form, so one fused
 * tensor-core kernel (tcgen05: layer 1 and GELU on the CUDA cores, the
 * 256 x 256 layer with bf16 operands and fp32 accumulators in tensor memory,
 * bias, GELU and head in the epilogue) evaluates a table over those prefixes
 * (2^(2 min(h,12) - 1) rows) and a gather reads it for each state.
 * Synchronous.  LCS_ETIMEOUT if a bounded wait on the tensor core ran out. */
lcs_status lcs_mlp_predict_bf16(lcs_mlp_t* m, int h, uint64_t base, int64_t n, float* out_dev);
/* a start for lcs_bound_set_start (device doubles, 4^h values each, h <= 16),
 * from the same BF16 table: older = u_hat, newest = u_hat + r_hat.
 * Synchronous. */
lcs_status lcs_mlp_start_vectors(lcs_mlp_t* m, int h, double r_hat, double* newest_dev, double* older_dev);
/* The same start for lcs_bound_set_start_stored_fx of a complement-symmetric
 * sigma = d = 2 handle: 4^h / 2 fixed-point values each (states x < 4^h / 2),
 * converted as lcs_bound_set_start converts the doubles (rounded down, K =
 * frac_bits, 0 = 44): a quarter of the bytes.  Device pointers; synchronous. */
lcs_status lcs_mlp_start_vectors_stored_fx(lcs_mlp_t* m, int h, double r_hat, int frac_bits, int64_t* newest_dev,
                                           int64_t* older_dev);
void lcs_mlp_destroy(lcs_mlp_t* m);

/* The non-learned control for the warm start (sigma = d = 2): a start for
 * shape h_to built from a full-length fixed-point vector of shape h_from by
 * cutting each tuple to its first h_from letters (the state index shifted
 * right by 2 (h_to - h_from) bits): older[x] = (src[x >> s] - src[0]) * 2^-K,
 * newest = older + r_hat.  Device pointers; uses the legacy default stream;
 * synchronous. */
lcs_status lcs_lift_prefix(int h_from, int h_to, const int64_t* src_dev, int frac_bits, double r_hat,
                           double* newest_dev, double* older_dev);

/* ------------------------------------------------------------------------ */
/* Experiment: float32 storage.  Runs n_iters iterations of Algorithm 2 from
 * the zero start with iterates stored as float32 w_t = v_t - t rho (offset
 * normalisation through F's translation invariance) and float32 arithmetic,
 * then writes the newest iterate v = w + t rho as doubles to newest_dev
 * (device, sigma^(d h) values).  (sigma, d) in {(2,2), (2,3), (3,2)}, full
 * storage.  *ms_per_sweep receives the mean sweep time.  No bound is derived:
 * the rounding is not directed; the point is the error against the exact
 * fixed-point iterates at half the bytes.  Legacy default stream; synchronous. */
lcs_status lcs_fp32_experiment(int sigma, int d, int h, int64_t n_iters, double rho, double* newest_dev,
                               double* ms_per_sweep);

/* ------------------------------------------------------------------------ */
/* Stateless entry point.
 *
 * One evaluation of F (Eq. ineq3; Algorithm 2's first line in the loop):
 * v_out = F(v_prev[0], .., v_prev[d-1]) where v_prev[k-1] is the iterate k
 * steps older than the one being computed (the k-th argument v_k of F).
 * All vectors are device pointers of sigma^(d h) fixed-point int64 values in
 * state-index order (no symmetry).  v_out must not share a byte with any
 * input (LCS_EINVAL).
 * f_mode and frac_bits as in lcs_bound_opts.  Shapes as lcs_bound_create
 * (the general kernels serve those without a specialised one).  stream:
 * cudaStream_t or NULL (legacy default stream).  Asynchronous; no allocation. */
lcs_status lcs_sweep_fx(int sigma, int d, int h, int f_mode, int frac_bits, const int64_t* const* v_prev, int64_t* v_out,
                        void* stream);

/* ------------------------------------------------------------------------ */
/* Entry point that allocates nothing.  The paper has no counterpart: it is an
 * interface for callers that cannot allocate device memory -- code running
 * inside a memory pool it does not own, a plugin whose host forbids device
 * allocations, or a process that has already committed all free HBM.
 *
 * One evaluation of F fused with the increment reduction, as one checked
 * iteration of lcs_bound_iterate performs it: v_out = F(v_prev[0], ..,
 * v_prev[d-1]) (v_prev[k-1] = the iterate k steps older than the one being
 * computed; sigma^(d h) fixed-point int64 values each, device pointers, state
 * order, no symmetry), then *R_out = min_x (v_out - v_prev[0])[x] (max with
 * r_mode = 1) and *argmin_out = the smallest state index attaining it.
 * R_out and argmin_out are device pointers owned by the caller.  frac_bits as
 * in lcs_bound_opts (0 -> 44).  stream: cudaStream_t or NULL.  Asynchronous.
 * The shapes with a specialised kernel only (see lcs_bound_create); others
 * return LCS_EUNSUPPORTED.
 *
 * v_out must not share a byte with any v_prev[k]; R_out and argmin_out (8
 * bytes each) must not share a byte with any vector or with each other
 * (LCS_EINVAL).  The inputs may share bytes with each other.
 *
 * Scratch: the per-CTA partials of the reduction live in a fixed 64 KiB
 * array inside the library (4096 partials), reserved on every device that
 * loads the library until the process exits.  Every call looks up that
 * array's device address (cudaGetSymbolAddress, which allocates nothing) with
 * the calling thread's current device, so the address stays right after the
 * device is reset.  The first call on each device also loads the library's
 * device code there: make that first call before any stream capture.  A call
 * whose launch would need more than 4096 partials returns LCS_EINVAL.  The
 * function calls no allocator (no cudaMalloc, cudaFree or allocating library
 * routine).  All calls share the one array and each call overwrites every
 * slot it later reads, so no state carries over -- but calls that overlap on
 * the GPU (different streams, or different host threads without ordering)
 * race on it: order them.  Errors: LCS_EINVAL, LCS_EUNSUPPORTED, LCS_ECUDA;
 * lcs_bound_last_error() gives the message. */
lcs_status lcs_sweep_incr_fx_noalloc(int sigma, int d, int h, int frac_bits, int r_mode, const int64_t* const* v_prev,
                                     int64_t* v_out, int64_t* R_out, uint64_t* argmin_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LCS_BOUND_H */
