// lcs_common.h -- types shared by the host driver and the kernels of the GB300
// feasible-triplet library (Heineman et al., arXiv 2407.10925, section 2.1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lcs {

constexpr int kMaxD = 16;         // largest d (the general kernel takes any d up to it)
constexpr int kBlock = 256;       // threads per CTA of the sweep and check kernels
constexpr int kFinalBlock = 1024; // threads of the single-CTA finalize kernels

// One CTA's partial of the increment reduction (value, state index) or of the
// check's max W (value only).
struct RedPartial {
  long long v;
  unsigned long long x;
};

// Device-resident results of Algorithm 2, updated by the finalize kernels so
// that a block of iterations needs no host synchronisation.  All values are
// fixed-point (units of 2^-K).
struct DevState {
  long long R;              // increment of the last reduced iteration
  unsigned long long argmin;
  long long R_iter;         // iteration count at which R was taken
  long long E;              // last check
  long long E_iter;
  long long r, eps;         // kept triplet
  long long kept_iter;      // -1: the initial triplet (v_0, 0, 0)
  long long have_check;
  long long kept_flag;      // 1 if the last check kept its iterate
  long long maxabs;         // scratch of the max-|v| reduction
  long long status;         // sticky error status (lcs_status values)
  long long swap_bad;       // set by the swap-symmetry check of start vectors
  long long pad[3];
};

// Arguments of one sweep launch: v_out = F(prev[0], .., prev[d-1]).
struct SweepParams {
  const long long* prev[kMaxD];  // prev[k-1]: the iterate k steps back (F's k-th argument)
  long long* out;
  unsigned long long n_tail;     // sigma^(d (h-1)): tail tuples; also the stride between head tuples
  unsigned long long n_stored;   // states held in each buffer
  int h;
  int incr;                      // 1: fused increment reduction against prev[0]
  int r_mode;                    // 0: min, 1: max
  long long one;                 // 2^K
  RedPartial* partials;          // one per CTA when incr
  // Offset-normalised 32-bit storage (sigma = d = 2 only): a stored w stands
  // for v = w + offs[slot] of its vector.  The output's offset is the first
  // input's value at state 0 plus the last increment R (state->R once one
  // has been reduced, else step); the sweep records it and flags an output
  // outside 32 bits in state->status.  Unused (null) with 64-bit storage.
  long long* offs;
  int slot_in0, slot_in1, slot_out;
  long long step;
  DevState* state;
  // a sweep fused with the check of its newest input (KernelSet::sweep_check):
  // one max-W partial per CTA; R is read from state
  RedPartial* check_partials;
  // general kernels in block form (sweep_rtb.cuh): the means table and the
  // term offsets; null: the one-pass general kernels run instead
  long long* rt_means;
  const unsigned short* rt_offs;
  const unsigned* rt_start;
  const unsigned long long* rt_tiles;  // the first phase's tiles with a task: (k << 48) | run index
  unsigned long long rt_n_tiles;
};

// Arguments of one check launch: W = u + dR - F(u + (d-1)R, .., u).
struct CheckParams {
  const long long* u;
  unsigned long long n_tail;
  unsigned long long n_stored;
  int h;
  long long one;
  const DevState* state;         // R is read from state->R when R_from_state
  int R_from_state;
  long long R;                   // used when !R_from_state
  RedPartial* partials;          // one per CTA
  long long* rt_means;           // as in SweepParams
  const unsigned short* rt_offs;
  const unsigned* rt_start;
};

// Host-visible description of the kernels compiled for one (sigma, d).
struct KernelSet {
  int sigma, d;
  int f_mode;                    // 0: the paper's F; 1: every non-empty advance set
  int sym;                       // 0: full storage; 1: complement-symmetric storage (sigma = 2);
                                 // 2: complement storage + swap-aware reads (sigma = d = 2);
                                 // 3: full storage + swap-aware reads (d = 2, sigma >= 3);
                                 // 4: complement storage + permutation-aware reads (sigma = 2, d = 3)
  void (*sweep)(const SweepParams&, int grid, cudaStream_t);
  void (*check)(const CheckParams&, int grid, cudaStream_t);
  const void* sweep_fn;          // kernel symbols, for occupancy queries
  const void* check_fn;
  int tails_per_thread;          // tail tuples one thread handles per loop step
  // algorithmic bytes per stored state: every output written once and every
  // distinct input value the kernel's storage scheme needs read once
  int sweep_algo_bytes;
  int check_algo_bytes;
  // optional: the sweep fused with the check of its newest input (null if none)
  void (*sweep_check)(const SweepParams&, int grid, cudaStream_t);
  const void* sweep_check_fn;
};

// Registry filled by the per-alphabet translation units.
const KernelSet* find_kernels(int sigma, int d, int sym, int f_mode = 0);

}  // namespace lcs
