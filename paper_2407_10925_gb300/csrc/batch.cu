// batch.cu -- many small (sigma, d, h) instances of uneven size in one
// persistent launch (Heineman et al., arXiv 2407.10925: Algorithm 2 for each
// instance, all instances advancing in lockstep).
//
// One cooperative kernel runs a block of iterations.  Each iteration walks a
// work list of (instance, item) pairs -- an item is a few tiles of one
// instance's sweep -- then meets at a grid barrier.  On a checked iteration
// the kernel also reduces each instance's increment (one CTA per instance),
// runs the check over the same work list and applies Algorithm 2's keep test,
// with a barrier between the phases.  Ring slots and the iteration count live
// on the device, so the same launch can be captured once in a CUDA graph and
// replayed.  Loads use the L2-coherent path: a buffer written in iteration t
// by one CTA is read in iteration t+1 by others inside the same launch.
//
// The grid barrier spins with a clock budget.  When the budget runs out the
// CTA records LCS_ETIMEOUT; every CTA checks that status at each barrier and
// leaves, so a lost participant ends the launch with an error, not a hang.
// Cooperative launch guarantees that all CTAs are resident together.
//
// Concurrent mode.  The persistent kernel carries every instance kind's body,
// so its register count (and occupancy) is set by the heaviest kind.  The
// alternative mode runs each instance's own single-instance kernels (the
// ones lcs_bound_iterate uses) on a stream of its own, forked from and joined
// to the handle's stream; the GPU overlaps the instances, and each kernel
// keeps its own occupancy.  Both modes share the buffers, the device states
// and the check schedule, so they give the same iterates and bounds bit for
// bit; the autotuner times both and keeps the faster.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/lcs_bound.h"
#include "batch.h"
#include "sweep_generic.cuh"
#include "sweep_s2d2.cuh"

namespace lcs {

void record_error(const char* msg);

static lcs_status bfail(lcs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  record_error(buf);
  return st;
}

#define B_CUDA(call)                                                                                      \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return bfail(LCS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                        __FILE__, __LINE__);                                              \
  } while (0)

// kinds of instance the batch kernel carries a body for
enum BatchKind : int { BK_S2D2 = 0, BK_G22S, BK_G23S, BK_G24S, BK_G32, BK_G42, BK_G22, BK_G23, BK_COUNT };

struct BatchInst {
  int kind, d, h, rows;
  unsigned long long n_tail, n_stored;
  unsigned long long units;        // tiles (s2d2: orbit tiles; generic: 256 thread slots) per sweep
  unsigned long long items;        // work items per sweep: ceil(units / units_per_item)
  unsigned long long item_begin;   // first item in the batch's work list
  unsigned long long units_per_item;
  unsigned long long n_threads;    // generic: thread slots per sweep
  unsigned tn;                     // s2d2: tiles per side
  unsigned long long tri;          // s2d2: upper-triangle tiles per half
  double cost;                     // host only: estimated loads per unit (orders the work list)
  long long* ring[kMaxD + 1];
  RedPartial* partials;            // one per item
  DevState* state;
};

struct BatchCtl {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned long long ticket;  // items handed out so far in this launch
  long long status;
  long long iter_done;
  long long call_end;
  long long spin_budget;
  int newest[kMaxBatch];
};

// ---------------------------------------------------------------------------
// device side

__device__ __forceinline__ bool grid_barrier(BatchCtl* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = &ctl->bar_gen;
    volatile long long* status = &ctl->status;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      const long long budget = ctl->spin_budget;
      while (*gen == g) {
        if (*status != 0) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > budget) {
          atomicCAS((unsigned long long*)&ctl->status, 0ull, (unsigned long long)LCS_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (*status != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int SIG, int D, bool SYM>
__device__ __forceinline__ void generic_item(const BatchInst& in, const SweepParams& p, unsigned long long q,
                                             bool incr, RedPartial* slot) {
  long long best_v = p.r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long best_x = ULLONG_MAX;
  const unsigned long long u0 = q * in.units_per_item, u1 = min(u0 + in.units_per_item, in.units);
  for (unsigned long long u = u0; u < u1; ++u) {
    const unsigned long long t = u * kBlock + threadIdx.x;
    if (t < in.n_threads) {
      if (incr)
        generic_sweep_thread<SIG, D, SYM, true, true>(p, t, best_v, best_x);
      else
        generic_sweep_thread<SIG, D, SYM, false, true>(p, t, best_v, best_x);
    }
  }
  if (incr) block_reduce_arg_to(best_v, best_x, p.r_mode, slot);
}

template <int SIG, int D, bool SYM>
__device__ __forceinline__ void generic_check_item(const BatchInst& in, const CheckParams& c, long long R,
                                                   unsigned long long q, RedPartial* slot) {
  long long best = LLONG_MIN;
  const unsigned long long u0 = q * in.units_per_item, u1 = min(u0 + in.units_per_item, in.units);
  for (unsigned long long u = u0; u < u1; ++u) {
    const unsigned long long t = u * kBlock + threadIdx.x;
    if (t < in.n_threads) generic_check_thread<SIG, D, SYM, true>(c, R, t, best);
  }
  block_reduce_max_to(best, slot);
}

__device__ __forceinline__ unsigned long long s2d2_tile_of(const BatchInst& in, unsigned long long u) {
  const unsigned long long s = u / in.tri, q = u - s * in.tri;
  unsigned A, B;
  tri_decode(q, A, B);
  return s * (unsigned long long)in.tn * in.tn + (unsigned long long)A * in.tn + B;
}

__device__ void batch_sweep_item(const BatchInst& in, int newest, unsigned long long q, bool incr, int r_mode,
                                 long long one) {
  SweepParams p;
  for (int k = 1; k <= in.d; ++k) p.prev[k - 1] = in.ring[(newest - (k - 1) + in.rows) % in.rows];
  p.out = in.ring[(newest + 1) % in.rows];
  p.n_tail = in.n_tail;
  p.n_stored = in.n_stored;
  p.h = in.h;
  p.incr = incr;
  p.r_mode = r_mode;
  p.one = one;
  p.partials = nullptr;
  RedPartial* slot = in.partials + q;
  switch (in.kind) {
    case BK_S2D2: {
      const S2D2Geo g = s2d2_geo(in.h, in.n_tail);
      long long best_v = r_mode ? LLONG_MIN : LLONG_MAX;
      unsigned long long best_x = ULLONG_MAX;
      const unsigned long long u0 = q * in.units_per_item, u1 = min(u0 + in.units_per_item, in.units);
      for (unsigned long long u = u0; u < u1; ++u) {
        if (incr)
          s2d2_sweep_orbit<true, true>(p, g, s2d2_tile_of(in, u), best_v, best_x);
        else
          s2d2_sweep_orbit<false, true>(p, g, s2d2_tile_of(in, u), best_v, best_x);
      }
      if (incr) block_reduce_arg_to(best_v, best_x, r_mode, slot);
      break;
    }
    case BK_G22S: generic_item<2, 2, true>(in, p, q, incr, slot); break;
    case BK_G23S: generic_item<2, 3, true>(in, p, q, incr, slot); break;
    case BK_G24S: generic_item<2, 4, true>(in, p, q, incr, slot); break;
    case BK_G32: generic_item<3, 2, false>(in, p, q, incr, slot); break;
    case BK_G42: generic_item<4, 2, false>(in, p, q, incr, slot); break;
    case BK_G22: generic_item<2, 2, false>(in, p, q, incr, slot); break;
    case BK_G23: generic_item<2, 3, false>(in, p, q, incr, slot); break;
  }
}

__device__ void batch_check_item(const BatchInst& in, int newest, unsigned long long q, long long one) {
  CheckParams c;
  c.u = in.ring[newest];
  c.n_tail = in.n_tail;
  c.n_stored = in.n_stored;
  c.h = in.h;
  c.one = one;
  c.state = in.state;
  c.R_from_state = 1;
  c.R = 0;
  c.partials = nullptr;
  const long long R = __ldcg(&in.state->R);
  RedPartial* slot = in.partials + q;
  switch (in.kind) {
    case BK_S2D2: {
      const S2D2Geo g = s2d2_geo(in.h, in.n_tail);
      long long best = LLONG_MIN;
      const unsigned long long u0 = q * in.units_per_item, u1 = min(u0 + in.units_per_item, in.units);
      for (unsigned long long u = u0; u < u1; ++u) s2d2_check_orbit<true>(c, g, R, s2d2_tile_of(in, u), best);
      block_reduce_max_to(best, slot);
      break;
    }
    case BK_G22S: generic_check_item<2, 2, true>(in, c, R, q, slot); break;
    case BK_G23S: generic_check_item<2, 3, true>(in, c, R, q, slot); break;
    case BK_G24S: generic_check_item<2, 4, true>(in, c, R, q, slot); break;
    case BK_G32: generic_check_item<3, 2, false>(in, c, R, q, slot); break;
    case BK_G42: generic_check_item<4, 2, false>(in, c, R, q, slot); break;
    case BK_G22: generic_check_item<2, 2, false>(in, c, R, q, slot); break;
    case BK_G23: generic_check_item<2, 3, false>(in, c, R, q, slot); break;
  }
}

// R and its state for one instance from its per-item partials (one CTA)
__device__ void batch_finalize_incr(const BatchInst& in, int r_mode, long long iter) {
  long long v = r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long x = ULLONG_MAX;
  for (unsigned long long i = threadIdx.x; i < in.items; i += blockDim.x) {
    const long long pv = __ldcg(&in.partials[i].v);
    const unsigned long long px = __ldcg(&in.partials[i].x);
    if (red_better(pv, px, v, x, r_mode)) v = pv, x = px;
  }
  RedPartial r;
  block_reduce_arg_to(v, x, r_mode, &r);  // only thread 0's copy is meaningful
  if (threadIdx.x == 0) {
    in.state->R = r.v;
    in.state->argmin = r.x;
    in.state->R_iter = iter;
  }
}

// E = max(0, max W) and the keep test for one instance (one CTA)
__device__ void batch_finalize_check(const BatchInst& in, long long iter) {
  long long v = 0;
  for (unsigned long long i = threadIdx.x; i < in.items; i += blockDim.x) v = max(v, __ldcg(&in.partials[i].v));
  RedPartial r;
  block_reduce_max_to(v, &r);
  if (threadIdx.x == 0) {
    DevState* st = in.state;
    const long long R = __ldcg(&st->R), E = max(0ll, r.v);
    st->E = E;
    st->E_iter = iter;
    st->have_check = 1;
    if (R - E >= st->r - st->eps) {
      st->r = R;
      st->eps = E;
      st->kept_iter = iter;
      st->kept_flag = 1;
    } else {
      st->kept_flag = 0;
    }
  }
}

// Hand out the items of one phase (sweep or check) dynamically.  Tickets are
// issued in order from one counter for the whole launch; ticket t belongs to
// phase t / total_items.  A CTA that draws a ticket of the next phase keeps
// it (s_pending) and serves it first in that phase, so every item of every
// phase is served exactly once and the counter never needs resetting inside
// the launch.
template <class F>
__device__ __forceinline__ void run_phase(BatchCtl* ctl, unsigned long long phase, unsigned long long total_items,
                                          unsigned long long& s_pending, F&& serve) {
  const unsigned long long lo = phase * total_items, hi = lo + total_items;
  for (;;) {
    if (threadIdx.x == 0 && s_pending == ULLONG_MAX) s_pending = atomicAdd(&ctl->ticket, 1ull);
    __syncthreads();
    const unsigned long long t = s_pending;
    if (t >= hi) break;  // a ticket of a later phase: keep it
    serve(t - lo);
    __syncthreads();
    if (threadIdx.x == 0) s_pending = ULLONG_MAX;
  }
  __syncthreads();
}

// MINB = CTAs per SM the compiler must fit: 2 lets every kind's body keep its
// registers (128); 4 caps them at 64 (the heaviest bodies spill) for twice the
// warps in flight.  The autotuner times both.
template <int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
    batch_kernel(const BatchInst* __restrict__ insts, int n_inst, unsigned long long total_items, long long n_iters,
                 int check_every, int r_mode, long long one, BatchCtl* ctl) {
  __shared__ BatchInst si[kMaxBatch];
  __shared__ int s_newest[kMaxBatch];
  __shared__ unsigned long long s_pending;
  if (threadIdx.x == 0) s_pending = ULLONG_MAX;
  unsigned long long phase = 0;
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    si[i] = insts[i];
    s_newest[i] = ((volatile int*)ctl->newest)[i];
  }
  const long long it0 = *(volatile long long*)&ctl->iter_done;
  const long long call_end = *(volatile long long*)&ctl->call_end;
  __syncthreads();
  bool ok = true;
  long long done = 0;
  for (long long local = 0; local < n_iters && ok; ++local) {
    const long long it = it0 + local + 1;
    const bool check = (check_every > 0 && it % check_every == 0) || it == call_end;
    run_phase(ctl, phase++, total_items, s_pending, [&](unsigned long long g) {
      int i = 0;
      while (i + 1 < n_inst && si[i + 1].item_begin <= g) ++i;
      batch_sweep_item(si[i], s_newest[i], g - si[i].item_begin, check, r_mode, one);
    });
    ok = grid_barrier(ctl);
    if (ok && check) {
      for (int i = blockIdx.x; i < n_inst; i += gridDim.x) batch_finalize_incr(si[i], r_mode, it);
      ok = grid_barrier(ctl);
      if (ok) {
        // the check reads u = the iterate just written
        for (int i = threadIdx.x; i < n_inst; i += blockDim.x) s_newest[i] = (s_newest[i] + 1) % si[i].rows;
        __syncthreads();
        run_phase(ctl, phase++, total_items, s_pending, [&](unsigned long long g) {
          int i = 0;
          while (i + 1 < n_inst && si[i + 1].item_begin <= g) ++i;
          batch_check_item(si[i], s_newest[i], g - si[i].item_begin, one);
        });
        ok = grid_barrier(ctl);
      }
      if (ok) {
        for (int i = blockIdx.x; i < n_inst; i += gridDim.x) batch_finalize_check(si[i], it);
        ok = grid_barrier(ctl);
      }
    } else if (ok) {
      for (int i = threadIdx.x; i < n_inst; i += blockDim.x) s_newest[i] = (s_newest[i] + 1) % si[i].rows;
      __syncthreads();
    }
    if (ok) ++done;
  }
  // every CTA has passed the reads above (at least one barrier per iteration)
  if (blockIdx.x == 0 && threadIdx.x == 0 && ok) {
    for (int i = 0; i < n_inst; ++i) ctl->newest[i] = s_newest[i];
    ctl->iter_done = it0 + done;
  }
}

__global__ void batch_init_kernel(DevState* st) {
  DevState z{};
  z.kept_iter = -1;
  *st = z;
}

// ---------------------------------------------------------------------------
// host side

// one instance in the concurrent mode (work-list position r)
struct ConcInst {
  const KernelSet* ks;
  int grid_sweep, grid_check;
  RedPartial* partials;  // max(grid_sweep, grid_check) entries
  cudaStream_t stream;
  cudaEvent_t join;
  int newest;            // ring slot of the newest iterate (host copy of the device ring state)
};

struct BatchState {
  int n;
  int slot[kMaxBatch];  // user index -> position in the work-list order
  int sigma[kMaxBatch], d[kMaxBatch], h[kMaxBatch];
  unsigned long long n_total[kMaxBatch];
  std::vector<BatchInst> inst;  // host copy (pointers are device pointers)
  BatchInst* d_inst;
  BatchCtl* d_ctl;
  long long* h_call_end;        // pinned host value read by the graph's copy node
  unsigned long long total_items;
  int grid;
  int check_every, r_mode;
  long long one;
  int frac_bits;
  long long iter_done_host;
  int newest_host_valid;
  void* (*alloc)(size_t, void*);
  void (*free)(void*, void*);
  void* ctx;
  std::vector<void*> owned;
  std::map<long long, cudaGraphExec_t> graphs;
  bool use_graph;
  long long graph_replays;  // launches that replayed a captured graph
  int variant;              // persistent kernel: 0 = batch_kernel<2>, 1 = batch_kernel<4>
  int max_grid[2];          // resident CTAs of each variant
  long long spin_budget;
  int tune_grid_choice, tune_units_choice;
  double tuned_ms;
  long long launches;
  int mode;  // 0 persistent launch, 1 concurrent single-instance kernels, 2 the same never captured
  // mode 1: graphs of whole iterate calls, keyed by the call's schedule
  // (length, check phase, every instance's ring slot); a schedule is
  // captured when it comes a second time, and replayed from then on
  std::map<std::vector<long long>, cudaGraphExec_t> conc_graphs;
  std::map<std::vector<long long>, int> conc_seen;
  double ms_persistent, ms_concurrent;
  ConcInst conc[kMaxBatch];
  cudaEvent_t fork;
};

static void* balloc(BatchState* B, size_t bytes) {
  void* p = nullptr;
  if (B->alloc) {
    p = B->alloc(bytes, B->ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) B->owned.push_back(p);
  return p;
}

void batch_destroy(BatchState* B) {
  if (!B) return;
  for (int r = 0; r < kMaxBatch; ++r) {
    if (B->conc[r].stream) {
      cudaStreamSynchronize(B->conc[r].stream);
      cudaStreamDestroy(B->conc[r].stream);
    }
    if (B->conc[r].join) cudaEventDestroy(B->conc[r].join);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  for (auto& g : B->graphs) cudaGraphExecDestroy(g.second);
  for (auto& g : B->conc_graphs) cudaGraphExecDestroy(g.second);
  for (void* p : B->owned) {
    if (B->alloc) {
      if (B->free) B->free(p, B->ctx);
    } else {
      cudaFree(p);
    }
  }
  if (B->h_call_end) cudaFreeHost(B->h_call_end);
  delete B;
}

static int kind_of(int sigma, int d, int h, int sym_opt) {
  const bool sym = sigma == 2 && sym_opt && h >= 2;
  if (sigma == 2 && d == 2 && sym && h >= 6) return BK_S2D2;
  if (sigma == 2 && d == 2) return sym ? BK_G22S : BK_G22;
  if (sigma == 2 && d == 3) return sym ? BK_G23S : BK_G23;
  if (sigma == 2 && d == 4 && sym) return BK_G24S;
  if (sigma == 3 && d == 2) return BK_G32;
  if (sigma == 4 && d == 2) return BK_G42;
  return -1;
}

// recompute the work list for a choice of units per item
static void layout_items(BatchState* B, int units_scale) {
  unsigned long long begin = 0;
  // the device table must list instances in work-list order: the kernel finds
  // an item's instance by scanning item_begin; order[] maps back to the user's index
  for (int r = 0; r < B->n; ++r) {
    BatchInst& in = B->inst[r];
    in.units_per_item = (unsigned long long)units_scale;
    in.items = (in.units + in.units_per_item - 1) / in.units_per_item;
    in.item_begin = begin;
    begin += in.items;
  }
  B->total_items = begin;
}

static lcs_status reset_zero(BatchState* B, cudaStream_t s) {
  for (int i = 0; i < B->n; ++i) {
    const BatchInst& in = B->inst[i];
    for (int k = 0; k < in.rows; ++k) B_CUDA(cudaMemsetAsync(in.ring[k], 0, in.n_stored * 8, s));
    batch_init_kernel<<<1, 1, 0, s>>>(in.state);
    B_CUDA(cudaGetLastError());
  }
  BatchCtl c{};
  c.spin_budget = B->spin_budget;
  for (int i = 0; i < B->n; ++i) c.newest[i] = B->inst[i].d - 1;  // v_{d-1} is the newest start vector
  B_CUDA(cudaMemcpyAsync(B->d_ctl, &c, sizeof c, cudaMemcpyHostToDevice, s));
  B_CUDA(cudaStreamSynchronize(s));
  B->iter_done_host = 0;
  for (int r = 0; r < B->n; ++r) B->conc[r].newest = B->inst[r].d - 1;
  return LCS_OK;
}

// ---------------------------------------------------------------------------
// concurrent mode

// the single-instance kernel set of a batch kind (the zero start is
// symmetric under exchanging strings, so d = 2 with sigma >= 3 and
// sigma = 2 with d = 3 take the kernels that use it)
static const KernelSet* conc_kernels(int kind, int h) {
  switch (kind) {
    case BK_S2D2: return find_kernels(2, 2, 2);
    case BK_G22S: return find_kernels(2, 2, 1);
    case BK_G23S: return find_kernels(2, 3, h >= d3s_min_h() && h <= d3s_max_h() ? 4 : 1, 0);
    case BK_G24S: return find_kernels(2, 4, 1);
    case BK_G32: return find_kernels(3, 2, h >= d2s_min_h(3) ? 3 : 0);
    case BK_G42: return find_kernels(4, 2, h >= d2s_min_h(4) ? 3 : 0);
    case BK_G22: return find_kernels(2, 2, 0);
    case BK_G23: return find_kernels(2, 3, 0);
  }
  return nullptr;
}

// one iteration of instance r on its stream: the sweep, and on a checked
// iteration the increment reduction, the check and the keep test -- the
// sequence lcs_bound_iterate issues for a single instance
static lcs_status conc_step(BatchState* B, int r, long long rel, bool check) {
  ConcInst& c = B->conc[r];
  const BatchInst& in = B->inst[r];
  const int rows = in.rows;
  SweepParams p{};
  for (int k = 1; k <= in.d; ++k) p.prev[k - 1] = in.ring[(c.newest - (k - 1) + rows) % rows];
  p.out = in.ring[(c.newest + 1) % rows];
  p.n_tail = in.n_tail;
  p.n_stored = in.n_stored;
  p.h = in.h;
  p.incr = check ? 1 : 0;
  p.r_mode = B->r_mode;
  p.one = B->one;
  p.partials = c.partials;
  c.ks->sweep(p, c.grid_sweep, c.stream);
  B_CUDA(cudaGetLastError());
  B->launches++;
  if (check) {
    launch_finalize_incr(c.partials, c.grid_sweep, B->r_mode, in.state, rel, c.stream, &B->d_ctl->iter_done);
    CheckParams q{};
    q.u = p.out;
    q.n_tail = in.n_tail;
    q.n_stored = in.n_stored;
    q.h = in.h;
    q.one = B->one;
    q.state = in.state;
    q.R_from_state = 1;
    q.R = 0;
    q.partials = c.partials;
    c.ks->check(q, c.grid_check, c.stream);
    launch_finalize_check(c.partials, c.grid_check, in.state, rel, c.stream, &B->d_ctl->iter_done);
    B_CUDA(cudaGetLastError());
    B->launches += 3;
  }
  c.newest = (c.newest + 1) % rows;
  return LCS_OK;
}

__global__ void advance_count_kernel(long long* count, long long n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *count += n;
}

// n_iters iterations of every instance, interleaved in rounds so that all
// streams are fed while the host enqueues.  Iteration numbers are relative
// to the device count ctl->iter_done, which the call advances at its end.
static lcs_status conc_enqueue(BatchState* B, cudaStream_t s, long long n_iters) {
  const long long call_end = B->iter_done_host + n_iters;
  B_CUDA(cudaEventRecord(B->fork, s));
  for (int r = 0; r < B->n; ++r) B_CUDA(cudaStreamWaitEvent(B->conc[r].stream, B->fork, 0));
  const long long round = 16;
  for (long long base = 0; base < n_iters; base += round) {
    const long long m = std::min(round, n_iters - base);
    for (int r = 0; r < B->n; ++r) {
      for (long long j = 0; j < m; ++j) {
        const long long rel = base + j + 1;
        const long long it = B->iter_done_host + rel;
        const bool check = (B->check_every > 0 && it % B->check_every == 0) || it == call_end;
        lcs_status st = conc_step(B, r, rel, check);
        if (st) return st;
      }
    }
  }
  for (int r = 0; r < B->n; ++r) {
    B_CUDA(cudaEventRecord(B->conc[r].join, B->conc[r].stream));
    B_CUDA(cudaStreamWaitEvent(s, B->conc[r].join, 0));
  }
  advance_count_kernel<<<1, 32, 0, s>>>(&B->d_ctl->iter_done, n_iters);
  B_CUDA(cudaGetLastError());
  B->launches++;
  B->iter_done_host = call_end;
  return LCS_OK;
}

static lcs_status conc_iterate(BatchState* B, cudaStream_t s, long long n_iters) {
  // what the enqueued work depends on besides the device state
  std::vector<long long> key{n_iters, B->check_every > 0 ? B->iter_done_host % B->check_every : 0};
  for (int r = 0; r < B->n; ++r) key.push_back(B->conc[r].newest);
  if (B->mode == 1) {
    auto it = B->conc_graphs.find(key);
    if (it == B->conc_graphs.end() && ++B->conc_seen[key] >= 2) {
      // the second call with this schedule: capture it (the host-side state
      // the enqueue advances is restored if the capture fails)
      int saved_newest[kMaxBatch];
      for (int r = 0; r < B->n; ++r) saved_newest[r] = B->conc[r].newest;
      const long long saved_iters = B->iter_done_host, saved_launches = B->launches;
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      bool captured = false;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        lcs_status st = conc_enqueue(B, s, n_iters);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        captured = st == LCS_OK && e == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      for (int r = 0; r < B->n; ++r) B->conc[r].newest = saved_newest[r];
      B->iter_done_host = saved_iters;
      B->launches = saved_launches;
      if (captured) {
        it = B->conc_graphs.emplace(key, ge).first;
      } else {
        cudaGetLastError();
        B->mode = 2;  // capture is not available here: enqueue directly from now on
      }
    }
    if (it != B->conc_graphs.end()) {
      B_CUDA(cudaGraphLaunch(it->second, s));
      B->launches++;
      B->graph_replays++;
      for (int r = 0; r < B->n; ++r) B->conc[r].newest = (B->conc[r].newest + (int)(n_iters % B->inst[r].rows)) % B->inst[r].rows;
      B->iter_done_host += n_iters;
      return LCS_OK;
    }
  }
  return conc_enqueue(B, s, n_iters);
}

static lcs_status conc_setup(BatchState* B, int sms) {
  B_CUDA(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming));
  for (int r = 0; r < B->n; ++r) {
    ConcInst& c = B->conc[r];
    const BatchInst& in = B->inst[r];
    c.ks = conc_kernels(in.kind, in.h);
    if (!c.ks) return bfail(LCS_EUNSUPPORTED, "no single-instance kernels for batch kind %d", in.kind);
    // the grids lcs_bound_create picks for the same shape
    const unsigned long long work = in.kind == BK_S2D2 ? 2ull * in.tn * in.tn * (unsigned long long)kBlock
                                    : c.ks->sym == 3   ? d2s_slots(c.ks->sigma, in.h) * kBlock
                                    : c.ks->sym == 4   ? d3s_tiles(in.h) * kBlock
                                                       : in.n_threads;
    c.grid_sweep = grid_for_work(c.ks->sweep_fn, sms, work);
    c.grid_check = grid_for_work(c.ks->check_fn, sms, work);
    c.partials = (RedPartial*)balloc(B, sizeof(RedPartial) * (size_t)std::max(c.grid_sweep, c.grid_check));
    if (!c.partials) return bfail(LCS_ENOMEM, "concurrent-mode partials");
    B_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    B_CUDA(cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming));
    c.newest = in.d - 1;
  }
  return LCS_OK;
}

static lcs_status launch_block(BatchState* B, cudaStream_t s, long long n_iters) {
  void* args[] = {(void*)&B->d_inst, (void*)&B->n, (void*)&B->total_items, (void*)&n_iters,
                  (void*)&B->check_every, (void*)&B->r_mode, (void*)&B->one, (void*)&B->d_ctl};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(B->grid);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const void* fn = B->variant ? (const void*)batch_kernel<4> : (const void*)batch_kernel<2>;
  B_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  B->launches++;
  return LCS_OK;
}

// the enqueued work of one iterate call: the call's last iteration, the
// barrier words, the persistent kernel
static lcs_status enqueue_call(BatchState* B, cudaStream_t s, long long n_iters) {
  B_CUDA(cudaMemcpyAsync(&B->d_ctl->call_end, B->h_call_end, sizeof(long long), cudaMemcpyHostToDevice, s));
  B_CUDA(cudaMemsetAsync(&B->d_ctl->bar_count, 0, 2 * sizeof(unsigned int) + sizeof(unsigned long long), s));
  return launch_block(B, s, n_iters);
}

lcs_status batch_iterate(BatchState* B, cudaStream_t s, long long n_iters) {
  if (n_iters <= 0) return LCS_OK;
  if (B->mode >= 1) return conc_iterate(B, s, n_iters);
  *B->h_call_end = B->iter_done_host + n_iters;
  if (B->use_graph) {
    auto it = B->graphs.find(n_iters);
    if (it == B->graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      bool captured = false;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        lcs_status st = enqueue_call(B, s, n_iters);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st == LCS_OK && e == cudaSuccess && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) captured = true;
        if (g) cudaGraphDestroy(g);
      }
      if (!captured) {
        // capture of a cooperative launch not available: launch directly
        cudaGetLastError();
        B->use_graph = false;
      } else {
        it = B->graphs.emplace(n_iters, ge).first;
      }
    }
    if (B->use_graph) {
      B_CUDA(cudaGraphLaunch(it->second, s));
      B->launches++;
      B->graph_replays++;
      B->iter_done_host += n_iters;
      return LCS_OK;
    }
  }
  lcs_status st = enqueue_call(B, s, n_iters);
  if (st) return st;
  B->iter_done_host += n_iters;
  return LCS_OK;
}

// autotuner: time a few iterations of each launch shape from the zero start,
// keep the fastest, then return every vector to the zero start
static lcs_status autotune(BatchState* B, cudaStream_t s, int sms) {
  const int grid_choices[] = {sms, 2 * sms, 4 * sms};
  const int unit_choices[] = {2, 4};
  double best = 1e30;
  int bg = B->max_grid[0], bu = 1, bv = 0;
  cudaEvent_t e0, e1;
  B_CUDA(cudaEventCreate(&e0));
  B_CUDA(cudaEventCreate(&e1));
  const bool saved_graph = B->use_graph;
  B->use_graph = false;
  // short probes: the candidates differ by far more than the noise of 4 iterations
  const long long probe_iters = 4;
  for (int var = 0; var < 2; ++var)
  for (int gc : grid_choices) {
    if (gc > B->max_grid[var] && gc != sms) continue;  // not resident: the cooperative launch would fail
    const int grid = std::min(gc, B->max_grid[var]);
    for (int uc : unit_choices) {
      layout_items(B, uc);
      B->grid = grid;
      B->variant = var;
      B_CUDA(cudaMemcpyAsync(B->d_inst, B->inst.data(), sizeof(BatchInst) * B->n, cudaMemcpyHostToDevice, s));
      lcs_status st = reset_zero(B, s);
      if (st) return st;
      st = batch_iterate(B, s, 1);  // warm-up
      if (st) return st;
      B_CUDA(cudaEventRecord(e0, s));
      st = batch_iterate(B, s, probe_iters);
      if (st) return st;
      B_CUDA(cudaEventRecord(e1, s));
      B_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      B_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms, bg = grid, bu = uc, bv = var;
    }
  }
  B->use_graph = saved_graph;
  B->grid = bg;
  B->variant = bv;
  B->tune_grid_choice = bg;
  B->tune_units_choice = bu;
  B->ms_persistent = best / (double)probe_iters;
  layout_items(B, bu);
  B_CUDA(cudaMemcpyAsync(B->d_inst, B->inst.data(), sizeof(BatchInst) * B->n, cudaMemcpyHostToDevice, s));
  // the concurrent mode, timed the same way
  {
    lcs_status st = reset_zero(B, s);
    if (st) return st;
    B->mode = 1;
    st = batch_iterate(B, s, 1);
    if (st) return st;
    B_CUDA(cudaEventRecord(e0, s));
    st = batch_iterate(B, s, probe_iters);
    if (st) return st;
    B_CUDA(cudaEventRecord(e1, s));
    B_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    B_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    B->ms_concurrent = ms / (double)probe_iters;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->mode = B->ms_concurrent < B->ms_persistent ? 1 : 0;
  B->tuned_ms = std::min(B->ms_concurrent, B->ms_persistent);
  B->launches = 0;
  return reset_zero(B, s);
}

lcs_status batch_create(int n, const int (*shapes)[3], const lcs_bound_opts& o, cudaStream_t s, BatchState** out) {
  *out = nullptr;
  if (n < 1 || n > kMaxBatch) return bfail(LCS_EINVAL, "batch size %d outside 1..%d", n, kMaxBatch);
  if (o.keep_u) return bfail(LCS_EUNSUPPORTED, "keep_u is not supported for batches");
  BatchState* B = new BatchState();
  B->n = n;
  B->alloc = o.alloc;
  B->free = o.free;
  B->ctx = o.alloc_ctx;
  B->check_every = o.check_every;
  B->r_mode = o.r_mode;
  B->frac_bits = o.frac_bits;
  B->one = 1ll << o.frac_bits;
  B->use_graph = true;
  // about 2 s at 2 GHz; a test may lower it through lcs_bound_batch_set_spin_budget
  B->spin_budget = 4000000000ll;
  B->inst.resize(n);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int i = 0; i < n; ++i) {
    const int sg = shapes[i][0], d = shapes[i][1], h = shapes[i][2];
    if (sg < 2 || d < 2 || h < 1 || d > kMaxD) {
      batch_destroy(B);
      return bfail(LCS_EINVAL, "instance %d: bad shape (%d,%d,%d)", i, sg, d, h);
    }
    unsigned long long nn = 1, sd = 1;
    for (int k = 0; k < d * h; ++k) {
      nn *= (unsigned long long)sg;
      if (nn >= (1ull << 36)) {
        batch_destroy(B);
        return bfail(LCS_EINVAL, "instance %d: batched instances must have fewer than 2^36 states", i);
      }
    }
    for (int k = 0; k < d; ++k) sd *= (unsigned long long)sg;
    const int kind = kind_of(sg, d, h, o.symmetry);
    if (kind < 0) {
      batch_destroy(B);
      return bfail(LCS_EUNSUPPORTED, "instance %d: (%d,%d,%d) has no batch kernel body", i, sg, d, h);
    }
    B->sigma[i] = sg;
    B->d[i] = d;
    B->h[i] = h;
    B->n_total[i] = nn;
    BatchInst& in = B->inst[i];
    std::memset(&in, 0, sizeof in);
    in.kind = kind;
    in.d = d;
    in.h = h;
    in.rows = d + 1;
    in.n_tail = nn / sd;
    const bool sym = kind == BK_S2D2 || kind == BK_G22S || kind == BK_G23S || kind == BK_G24S;
    in.n_stored = sym ? nn / 2 : nn;
    if (kind == BK_S2D2) {
      in.tn = (1u << (h - 2)) / kS2D2Tile;
      in.tri = (unsigned long long)in.tn * (in.tn + 1) / 2;
      in.units = 2 * in.tri;
      in.n_threads = 0;
      in.cost = kBlock * 20.0;  // 12 loads + 8 stores per orbit
    } else {
      in.n_threads = sym ? in.n_tail / 2 : in.n_tail;
      in.units = (in.n_threads + kBlock - 1) / kBlock;
      const double sd = std::pow((double)sg, (double)d);
      in.cost = kBlock * (2.0 * sd + sg * (std::pow((double)sg + 1.0, (double)d) - 1.0 - sd));
    }
    for (int k = 0; k < in.rows; ++k) {
      in.ring[k] = (long long*)balloc(B, in.n_stored * 8);
      if (!in.ring[k]) {
        batch_destroy(B);
        return bfail(LCS_ENOMEM, "instance %d: iterate vector", i);
      }
    }
    in.state = (DevState*)balloc(B, sizeof(DevState));
    // enough partial slots for one unit per item (the finest layout)
    in.partials = (RedPartial*)balloc(B, sizeof(RedPartial) * in.units);
    if (!in.state || !in.partials) {
      batch_destroy(B);
      return bfail(LCS_ENOMEM, "instance %d: state", i);
    }
  }
  // work-list order: heaviest items first (served first by the ticket counter)
  {
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return B->inst[a].cost > B->inst[b].cost; });
    std::vector<BatchInst> sorted(n);
    for (int r = 0; r < n; ++r) {
      sorted[r] = B->inst[idx[r]];
      B->slot[idx[r]] = r;
    }
    B->inst = sorted;
  }
  B->d_inst = (BatchInst*)balloc(B, sizeof(BatchInst) * n);
  B->d_ctl = (BatchCtl*)balloc(B, sizeof(BatchCtl));
  if (!B->d_inst || !B->d_ctl || cudaMallocHost(&B->h_call_end, sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    batch_destroy(B);
    return bfail(LCS_ENOMEM, "batch control");
  }
  for (int var = 0; var < 2; ++var) {
    int per_sm = 0;
    const void* fn = var ? (const void*)batch_kernel<4> : (const void*)batch_kernel<2>;
    B_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0));
    if (per_sm < 1) {
      batch_destroy(B);
      return bfail(LCS_ECUDA, "the batch kernel cannot be resident");
    }
    B->max_grid[var] = per_sm * sms;
  }
  layout_items(B, 1);
  B->variant = 0;
  B->grid = B->max_grid[0];
  lcs_status st = conc_setup(B, sms);
  if (st) {
    batch_destroy(B);
    return st;
  }
  st = autotune(B, s, sms);
  if (st) {
    batch_destroy(B);
    return st;
  }
  *out = B;
  return LCS_OK;
}

lcs_status batch_status(BatchState* B, cudaStream_t s, long long* status, long long* iter_done, int* newest, int i) {
  BatchCtl c;
  B_CUDA(cudaMemcpyAsync(&c, B->d_ctl, sizeof c, cudaMemcpyDeviceToHost, s));
  B_CUDA(cudaStreamSynchronize(s));
  if (status) *status = c.status;
  if (B->mode >= 1) {
    // the ring state lives on the host in the concurrent modes
    if (iter_done) *iter_done = B->iter_done_host;
    if (newest) *newest = B->conc[i].newest;
    return LCS_OK;
  }
  if (iter_done) *iter_done = c.iter_done;
  if (newest) *newest = c.newest[i];
  return LCS_OK;
}

lcs_status batch_report(BatchState* B, cudaStream_t s, int i, lcs_bound_report* out) {
  if (i < 0 || i >= B->n) return bfail(LCS_EINVAL, "instance %d outside 0..%d", i, B->n - 1);
  DevState st;
  B_CUDA(cudaMemcpyAsync(&st, B->inst[B->slot[i]].state, sizeof st, cudaMemcpyDeviceToHost, s));
  long long status = 0, iter_done = 0;
  lcs_status e = batch_status(B, s, &status, &iter_done, nullptr, B->slot[i]);
  if (e) return e;
  out->iters_done = iter_done;
  out->R = st.R;
  out->argmin = st.argmin;
  out->E = st.E;
  out->r = st.r;
  out->eps = st.eps;
  out->kept_iter = st.kept_iter;
  out->have_check = st.have_check;
  out->frac_bits = B->frac_bits;
  out->status = (int)(status ? status : st.status);
  return LCS_OK;
}

const long long* batch_vector(BatchState* B, cudaStream_t s, int i, int k, unsigned long long* n_stored,
                              unsigned long long* n_total, lcs_status* err) {
  *err = LCS_OK;
  if (i < 0 || i >= B->n || k < 0 || k >= B->d[i]) {
    *err = bfail(LCS_EINVAL, "instance %d / k %d out of range", i, k);
    return nullptr;
  }
  int newest = 0;
  *err = batch_status(B, s, nullptr, nullptr, &newest, B->slot[i]);
  if (*err) return nullptr;
  const BatchInst& in = B->inst[B->slot[i]];
  *n_stored = in.n_stored;
  *n_total = B->n_total[i];
  return in.ring[(newest - k + in.rows) % in.rows];
}

int batch_size(const BatchState* B) { return B->n; }
int batch_d(const BatchState* B, int i) { return B->d[i]; }

void batch_tuning(const BatchState* B, int* grid, int* units, double* ms, long long* launches, int* graph, int* mode,
                  double* ms_persistent, double* ms_concurrent, int* graph_captured, long long* graph_replays,
                  int* min_ctas_per_sm) {
  *grid = B->tune_grid_choice;
  *units = B->tune_units_choice;
  *ms = B->tuned_ms;
  *launches = B->launches;
  *graph = (B->mode == 0 && B->use_graph) ? 1 : 0;
  *graph_captured = (B->graphs.empty() && B->conc_graphs.empty()) ? 0 : 1;
  *graph_replays = B->graph_replays;
  *min_ctas_per_sm = B->variant ? 4 : 2;
  *mode = B->mode;
  *ms_persistent = B->ms_persistent;
  *ms_concurrent = B->ms_concurrent;
}

lcs_status batch_set_mode(BatchState* B, cudaStream_t s, int mode) {
  if (B->iter_done_host != 0) return bfail(LCS_EINVAL, "the mode can only be set before the first iteration");
  B->mode = mode;
  return reset_zero(B, s);
}

lcs_status batch_set_spin_budget(BatchState* B, cudaStream_t s, long long cycles) {
  B->spin_budget = cycles;
  B_CUDA(cudaMemcpyAsync(&B->d_ctl->spin_budget, &B->spin_budget, sizeof(long long), cudaMemcpyHostToDevice, s));
  B_CUDA(cudaMemsetAsync(&B->d_ctl->status, 0, sizeof(long long), s));
  B_CUDA(cudaStreamSynchronize(s));
  return LCS_OK;
}

lcs_status batch_clear_status(BatchState* B, cudaStream_t s) {
  B_CUDA(cudaMemsetAsync(&B->d_ctl->status, 0, sizeof(long long), s));
  B_CUDA(cudaStreamSynchronize(s));
  return LCS_OK;
}

}  // namespace lcs
