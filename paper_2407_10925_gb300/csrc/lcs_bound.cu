// lcs_bound.cu -- C ABI and host driver of the GB300 feasible-triplet library
// (Heineman et al., arXiv 2407.10925, section 2.1, Algorithm 2).
//
// The handle owns a ring of d+1 fixed-point iterate vectors on the device.
// One iteration launches the sweep (v_t = F(v_{t-1}, .., v_{t-d})); an
// iteration that is checked fuses the increment reduction into the sweep and
// then launches: the increment finalize (R, argmin), the check kernel (W, its
// max) and the check finalize (E, and Algorithm 2's keep test).  The results
// stay on the device (DevState) until lcs_bound_read synchronises.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <sys/mman.h>

#include "../../include/lcs_bound.h"
#include "batch.h"
#include "lcs_common.h"

namespace lcs {

// ---------------------------------------------------------------------------
// Errors

static thread_local std::string g_last_error;

static lcs_status fail(lcs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

// lets other translation units of the library set the message that
// lcs_bound_last_error() returns
__attribute__((visibility("hidden"))) void record_error(const char* msg) { g_last_error = msg; }

#define LCS_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(LCS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                   \
  } while (0)

// ---------------------------------------------------------------------------
// Small kernels: finalize reductions, conversions, copies.

__device__ __forceinline__ bool better_arg(long long v, unsigned long long x, long long bv, unsigned long long bx,
                                           int r_mode) {
  if (v != bv) return r_mode ? (v > bv) : (v < bv);
  return x < bx;
}

// R and its state from the per-CTA partials of a sweep (deterministic: fixed
// assignment of partials to threads and a fixed reduction tree).
// iter_base (may be null): a device count added to iter, so that a captured
// graph records the right iteration each time it is replayed
__global__ void __launch_bounds__(kFinalBlock) finalize_incr_kernel(const RedPartial* parts, int n, int r_mode,
                                                                     DevState* st, long long iter,
                                                                     const long long* iter_base = nullptr) {
  long long v = r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long x = ULLONG_MAX;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (better_arg(parts[i].v, parts[i].x, v, x, r_mode)) v = parts[i].v, x = parts[i].x;
  __shared__ long long sv[kFinalBlock / 32];
  __shared__ unsigned long long sx[kFinalBlock / 32];
  for (int o = 16; o > 0; o >>= 1) {
    long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    unsigned long long ox = __shfl_xor_sync(0xffffffffu, x, o);
    if (better_arg(ov, ox, v, x, r_mode)) v = ov, x = ox;
  }
  if ((threadIdx.x & 31) == 0) sv[threadIdx.x >> 5] = v, sx[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    v = threadIdx.x < nw ? sv[threadIdx.x] : sv[0];
    x = threadIdx.x < nw ? sx[threadIdx.x] : sx[0];
    for (int o = 16; o > 0; o >>= 1) {
      long long ov = __shfl_xor_sync(0xffffffffu, v, o);
      unsigned long long ox = __shfl_xor_sync(0xffffffffu, x, o);
      if (better_arg(ov, ox, v, x, r_mode)) v = ov, x = ox;
    }
    if (threadIdx.x == 0) {
      st->R = v;
      st->argmin = x;
      st->R_iter = iter + (iter_base ? *iter_base : 0);
    }
  }
}

// One record of the check history (the layout of lcs_bound_check_record).
struct CheckRecord {
  long long iter, R;
  unsigned long long argmin;
  long long E, kept, r, eps, kept_iter;
};
constexpr int kHistCap = 4096;  // records kept (a ring: the newest overwrite the oldest)

// E = max(0, max W) and Algorithm 2's keep test "R - E >= r - eps"; with a
// history buffer, the check's record is appended to it.
__global__ void __launch_bounds__(kFinalBlock) finalize_check_kernel(const RedPartial* parts, int n, DevState* st,
                                                                      long long iter, CheckRecord* hist = nullptr,
                                                                      unsigned long long* hist_count = nullptr,
                                                                      const long long* iter_base = nullptr) {
  long long v = 0;  // E = max(0, ...)
  for (int i = threadIdx.x; i < n; i += blockDim.x) v = max(v, parts[i].v);
  __shared__ long long sv[kFinalBlock / 32];
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sv[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    v = threadIdx.x < nw ? sv[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      if (iter_base) iter += *iter_base;
      const long long R = st->R, E = v;
      st->E = E;
      st->E_iter = iter;
      st->have_check = 1;
      // both sides are differences of int64 values far from the int64 limits
      // (the host keeps every value below 2^62 in magnitude)
      if (R - E >= st->r - st->eps) {
        st->r = R;
        st->eps = E;
        st->kept_iter = iter;
        st->kept_flag = 1;
      } else {
        st->kept_flag = 0;
      }
      if (hist) {
        const unsigned long long c = *hist_count;
        hist[c % kHistCap] = CheckRecord{iter, R, st->argmin, E, st->kept_flag, st->r, st->eps, st->kept_iter};
        *hist_count = c + 1;
      }
    }
  }
}

__global__ void copy_if_kept_kernel(const long long* __restrict__ src, long long* __restrict__ dst,
                                    unsigned long long n, const DevState* st) {
  if (!st->kept_flag) return;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Convert [off, off+len) of a full-length input vector (doubles rounded down to
// multiples of 2^-K, or fixed-point values) into the stored vector.  Indices at
// or above n_stored (complement-symmetric storage) are compared with their
// mirror instead; a mismatch sets st->status.
template <bool FROM_DOUBLE>
__global__ void ingest_kernel(const void* __restrict__ src, unsigned long long off, unsigned long long len,
                              long long* __restrict__ dst, unsigned long long n_stored, unsigned long long n_total,
                              double scale, DevState* st) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    long long q;
    if constexpr (FROM_DOUBLE) {
      const double v = static_cast<const double*>(src)[i] * scale;  // exact: scale is a power of two
      if (!(v >= -4.0e18 && v <= 4.0e18)) {                          // also catches NaN
        atomicExch((unsigned long long*)&st->status, (unsigned long long)LCS_EOVERFLOW);
        continue;
      }
      q = __double2ll_rd(v);
    } else {
      q = static_cast<const long long*>(src)[i];
    }
    const unsigned long long g = off + i;
    if (g < n_stored) {
      dst[g] = q;
    } else if (dst[n_total - 1 - g] != q) {
      atomicExch((unsigned long long*)&st->status, (unsigned long long)LCS_EINVAL);
    }
  }
}

// out[i] = value of state off+i (mirrored from the stored half when needed).
// With offset-normalised 32-bit storage (T = int) the vector's offset, read
// from the device, is added back.
template <bool TO_DOUBLE, class T = long long>
__global__ void export_kernel(const T* __restrict__ src, unsigned long long off, unsigned long long len,
                              unsigned long long n_stored, unsigned long long n_total, double scale,
                              void* __restrict__ out, const long long* offs = nullptr, int slot = 0) {
  const long long c = sizeof(T) == 4 ? offs[slot] : 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long g = off + i;
    const long long q = (long long)src[g < n_stored ? g : n_total - 1 - g] + c;
    if constexpr (TO_DOUBLE)
      static_cast<double*>(out)[i] = __ll2double_rn(q) * scale;
    else
      static_cast<long long*>(out)[i] = q;
  }
}

__global__ void maxabs_kernel(const long long* __restrict__ v, unsigned long long n, DevState* st) {
  long long m = 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const long long a = v[i];
    m = max(m, a == LLONG_MIN ? LLONG_MAX : (a < 0 ? -a : a));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&st->maxabs, m);
}

// sigma = d = 2: max |v| (as maxabs_kernel) and whether v is invariant under
// exchanging the two strings, in one pass over the stored values.  The swap
// exchanges the two bits of every position in the interleaved index; a swapped
// index in the upper half is read through the complement symmetry.  A warp's
// swapped indices fall in one 32-value block, so both reads are coalesced.
template <class T = long long>
__global__ void maxabs_swap_check_kernel(const T* __restrict__ v, unsigned long long n_stored,
                                         unsigned long long n_total, DevState* st, const long long* offs = nullptr,
                                         int slot = 0) {
  const long long c = sizeof(T) == 4 ? offs[slot] : 0;  // 32-bit storage: the swap test needs no offset
  long long m = 0;
  bool bad = false;
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_stored;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    const long long a = (long long)v[x] + c;
    m = max(m, a == LLONG_MIN ? LLONG_MAX : (a < 0 ? -a : a));
    unsigned long long y = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
    if (y >= n_stored) y = n_total - 1 - y;
    bad |= (long long)v[y] + c != a;
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&st->maxabs, m);
  if (bad) atomicExch((unsigned long long*)&st->swap_bad, 1ull);
}

// dst[i] = src[i] - c as 32-bit values (offset-normalised storage); a value
// outside 32 bits sets the overflow status; max |src| goes to st->maxabs
__global__ void narrow_kernel(const long long* __restrict__ src, int* __restrict__ dst, unsigned long long n,
                              long long c, DevState* st) {
  long long m = 0;
  bool bad = false;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const long long a = src[i], w = a - c;
    bad |= w < INT_MIN || w > INT_MAX;
    dst[i] = (int)w;
    m = max(m, a == LLONG_MIN ? LLONG_MAX : (a < 0 ? -a : a));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&st->maxabs, m);
  if (bad) atomicExch((unsigned long long*)&st->status, (unsigned long long)LCS_EOVERFLOW);
}

// dst[i] = src[i] + offs[slot] (32-bit storage back to fixed-point values)
__global__ void widen_kernel(const int* __restrict__ src, long long* __restrict__ dst, unsigned long long n,
                             const long long* offs, int slot) {
  const long long c = offs[slot];
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    dst[i] = (long long)src[i] + c;
}

__global__ void set_offset_kernel(long long* offs, int slot, long long c) {
  if (threadIdx.x == 0 && blockIdx.x == 0) offs[slot] = c;
}

// The prefix lift of a start: states [lo, hi) of the two newest rows from the
// source values src[0, len) holding states from src_off on of the shorter
// shape (sigma = d = 2): state x takes the value of state x >> 2s, its strings
// cut to their first h - s letters.  newest = value - sub_newest, older =
// value - sub_older; 32-bit rows flag a value outside 32 bits.  max |value|
// goes to st->maxabs.
template <class T>
__global__ void lift_kernel(const long long* __restrict__ src, unsigned long long src_off, int s2,
                            unsigned long long lo, unsigned long long hi, T* __restrict__ newest, T* __restrict__ older,
                            long long sub_newest, long long sub_older, DevState* st) {
  long long m = 0;
  bool bad = false;
  for (unsigned long long x = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < hi;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    const long long a = src[(x >> s2) - src_off];
    const long long wn = a - sub_newest, wo = a - sub_older;
    if (sizeof(T) == 4) bad |= wn < INT_MIN || wn > INT_MAX || wo < INT_MIN || wo > INT_MAX;
    newest[x] = (T)wn;
    older[x] = (T)wo;
    m = max(m, a == LLONG_MIN ? LLONG_MAX : (a < 0 ? -a : a));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&st->maxabs, m);
  if (bad) atomicExch((unsigned long long*)&st->status, (unsigned long long)LCS_EOVERFLOW);
}

__global__ void init_state_kernel(DevState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    DevState z{};
    z.kept_iter = -1;
    *st = z;
  }
}

}  // namespace lcs

// ---------------------------------------------------------------------------
// The handle.

using namespace lcs;

struct lcs_bound {
  int sigma, d, h;
  unsigned long long n_total, n_stored, n_tail;
  int sym;
  lcs_bound_opts opts;
  cudaStream_t stream;
  bool own_stream;
  int device;
  const KernelSet* ks;       // kernels for the storage scheme (complement-symmetric or full)
  const KernelSet* ks_swap;  // kernels that also use the string swap / permutations (d = 2, 3)
  bool swap_ok;              // the live iterates are swap-symmetric: ks_swap may run
  long long* ring[kMaxD + 1];  // element type: long long, or int with narrow storage
  int newest;  // ring slot of the newest iterate
  // opts.storage = 1: 32-bit offset-normalised rows, offs[slot] their offsets
  // (device); elem = bytes per stored value
  int narrow;
  size_t elem;
  long long* offs;
  // opts.host_slots: the ring rows placed in pinned host memory (read and
  // written by the kernels over the host link); host_base / host_len = their
  // mappings
  void* host_base[kMaxD + 1];
  size_t host_len[kMaxD + 1];
  void* host_ptr[kMaxD + 1];  // the registered (aligned) start of each
  long long* ubuf;
  DevState* dstate;
  RedPartial* partials;
  CheckRecord* hist;               // the check history (kHistCap records)
  unsigned long long* hist_count;  // checks recorded since creation or the last start
  int grid_sweep, grid_check, grid_sweep_swap, grid_check_swap, n_partials;
  // the check of a checked iteration may wait for the next sweep, which then
  // evaluates it in the same pass (KernelSet::sweep_check): pending_check marks
  // an iteration whose R is on the device but whose check has not run
  int grid_fused;
  RedPartial* check_partials;
  bool pending_check;
  long long pending_iter;
  // host transfers: a stream for the copies and two staging buffers, so the
  // copy of one piece overlaps the kernel that converts the previous one
  cudaStream_t xstream;
  void* stage[2];
  cudaEvent_t stage_ready[2], stage_free[2], xsync;
  bool stage_recorded[2];  // stage_free[i] marks the end of the last use of stage[i]
  long long iters_done;
  double vbound;  // upper bound of max |v| over the live iterates, in units of 2^-K
  long long one;
  BatchState* batch;  // non-null: a batch of instances (lcs_bound_batch_create)
  // timing
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> sweep_ev, check_ev;
  double sweep_ms, check_ms;
  // transfer timing: kXferH2D, kXferD2H (copies), kXferKernel (kernels moving transferred values)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> xfer_ev[3];
  double xfer_ms[3];
  unsigned long long h2d_bytes, d2h_bytes;
  long long sweep_n, check_n, launches;
  unsigned long long sweep_bytes, check_bytes;
  int last_check_grid;
  int d_batch_worst;  // batch handles: d of the instance with the largest sigma^d
  // general kernels in block form: the means table (sigma 2^d rows of n_tail
  // values) and the term offsets of every advance set
  long long* rt_means;
  unsigned short* rt_offs;
  unsigned* rt_start;
  unsigned long long* rt_tiles;  // the first phase's tiles with a task
  unsigned long long rt_n_tiles;
};

// Host memory for the device: an anonymous mapping aligned to 512 MiB,
// advised for transparent huge pages, then pinned and mapped into the
// device's address space (cudaHostRegister).  On this GB300's host link a
// transfer from such memory keeps the link's rate from its first use: in
// processes that followed heavy use of the machine, parts of ordinary pinned
// buffers (cudaHostAlloc) were read at 16-40 GB/s the first time, and a
// kernel gathering from 128 GiB of ordinary pages ran several times slower.
// Returns the registered start; *base / *len describe the mapping.
static void* host_map_alloc(size_t bytes, void** base, size_t* len) {
  const size_t align = (size_t)512 << 20;
  *len = bytes + align;
  void* m = mmap(nullptr, *len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (m == MAP_FAILED) return nullptr;
  char* hp = (char*)(((uintptr_t)m + align - 1) / align * align);
  madvise(hp, bytes, MADV_HUGEPAGE);  // a hint: without huge pages the memory still works
  if (cudaHostRegister(hp, bytes, cudaHostRegisterPortable | cudaHostRegisterMapped) != cudaSuccess) {
    cudaGetLastError();
    munmap(m, *len);
    return nullptr;
  }
  *base = m;
  return hp;
}

static void host_map_free(void* p, void* base, size_t len) {
  cudaHostUnregister(p);
  munmap(base, len);
}

static void* dev_alloc(lcs_bound* H, size_t bytes) {
  if (H->opts.alloc) return H->opts.alloc(bytes, H->opts.alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void dev_free(lcs_bound* H, void* p) {
  if (!p) return;
  if (H->opts.alloc) {
    if (H->opts.free) H->opts.free(p, H->opts.alloc_ctx);
  } else {
    cudaFree(p);
  }
}

static int grid_for(const void* fn, int sms, unsigned long long work_items) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  unsigned long long full = (unsigned long long)sms * (unsigned long long)per_sm;
  unsigned long long need = (work_items + kBlock - 1) / kBlock;
  if (need < 1) need = 1;
  return (int)std::min(full, need);
}

namespace lcs {

int grid_for_work(const void* fn, int sms, unsigned long long work_items) { return grid_for(fn, sms, work_items); }

void launch_finalize_incr(const RedPartial* parts, int n, int r_mode, DevState* st, long long iter, cudaStream_t s,
                          const long long* iter_base) {
  finalize_incr_kernel<<<1, kFinalBlock, 0, s>>>(parts, n, r_mode, st, iter, iter_base);
}

void launch_finalize_check(const RedPartial* parts, int n, DevState* st, long long iter, cudaStream_t s,
                           const long long* iter_base) {
  finalize_check_kernel<<<1, kFinalBlock, 0, s>>>(parts, n, st, iter, nullptr, nullptr, iter_base);
}

}  // namespace lcs

// headroom: every intermediate of a sweep or check is at most sigma^d times the
// largest |value| (plus lower-order terms); keep it below 2^62
static bool headroom_ok(const lcs_bound* H, double vb) {
  const double sd = std::pow((double)H->sigma, (double)(H->batch ? H->d_batch_worst : H->d));
  return sd * (vb + 4.0 * (double)H->one) * 2.0 < 4.6e18;
}

extern "C" {

lcs_status lcs_bound_default_opts(lcs_bound_opts* o) {
  if (!o) return fail(LCS_EINVAL, "opts is NULL");
  std::memset(o, 0, sizeof *o);
  o->check_every = 0;
  o->r_mode = 0;
  o->f_mode = 0;
  o->frac_bits = 44;
  o->keep_u = 0;
  o->symmetry = 1;
  o->timing = 0;
  o->storage = 0;
  o->host_slots = 0;
  return LCS_OK;
}

const char* lcs_bound_errstr(lcs_status st) {
  switch (st) {
    case LCS_OK: return "ok";
    case LCS_EINVAL: return "invalid argument";
    case LCS_ENOMEM: return "out of memory";
    case LCS_ECUDA: return "CUDA error";
    case LCS_ETIMEOUT: return "device wait timed out";
    case LCS_ENOBOUND: return "no feasibility check has run";
    case LCS_EOVERFLOW: return "fixed-point range exceeded";
    case LCS_EUNSUPPORTED: return "no kernel for this shape or mode";
    case LCS_EIO: return "file input/output failed";
  }
  return "unknown status";
}

const char* lcs_bound_last_error(void) { return g_last_error.c_str(); }

// buffers of lcs_host_alloc: registered start -> (mapping, length)
static std::mutex g_host_mutex;
static std::map<void*, std::pair<void*, size_t>> g_host_maps;

lcs_status lcs_host_alloc(size_t bytes, void** out) {
  if (!out) return fail(LCS_EINVAL, "out is NULL");
  *out = nullptr;
  if (bytes == 0) return fail(LCS_EINVAL, "0 bytes");
  void* base = nullptr;
  size_t len = 0;
  void* p = host_map_alloc(bytes, &base, &len);
  if (!p) return fail(LCS_ENOMEM, "%zu bytes of pinned host memory", bytes);
  std::lock_guard<std::mutex> lock(g_host_mutex);
  g_host_maps[p] = {base, len};
  *out = p;
  return LCS_OK;
}

lcs_status lcs_host_free(void* p) {
  if (!p) return LCS_OK;
  std::pair<void*, size_t> m;
  {
    std::lock_guard<std::mutex> lock(g_host_mutex);
    auto it = g_host_maps.find(p);
    if (it == g_host_maps.end()) return fail(LCS_EINVAL, "not a buffer of lcs_host_alloc");
    m = it->second;
    g_host_maps.erase(it);
  }
  host_map_free(p, m.first, m.second);
  return LCS_OK;
}

lcs_status lcs_bound_synchronize(lcs_bound_t* H) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  return LCS_OK;
}

void lcs_bound_destroy(lcs_bound_t* H) {
  if (!H) return;
  if (H->stream) cudaStreamSynchronize(H->stream);
  for (auto& e : H->sweep_ev) cudaEventDestroy(e.first), cudaEventDestroy(e.second);
  for (auto& e : H->check_ev) cudaEventDestroy(e.first), cudaEventDestroy(e.second);
  for (auto& v : H->xfer_ev)
    for (auto& e : v) cudaEventDestroy(e.first), cudaEventDestroy(e.second);
  if (H->xstream) {
    cudaStreamSynchronize(H->xstream);
    cudaStreamDestroy(H->xstream);
    for (int i = 0; i < 2; ++i) cudaEventDestroy(H->stage_ready[i]), cudaEventDestroy(H->stage_free[i]);
    cudaEventDestroy(H->xsync);
  }
  if (H->batch) batch_destroy(H->batch);
  for (int k = 0; k <= H->d; ++k) {
    if (H->host_base[k]) {
      host_map_free(H->host_ptr[k], H->host_base[k], H->host_len[k]);
    } else {
      dev_free(H, H->ring[k]);
    }
  }
  dev_free(H, H->offs);
  dev_free(H, H->rt_means);
  dev_free(H, H->rt_offs);
  dev_free(H, H->rt_start);
  dev_free(H, H->rt_tiles);
  dev_free(H, H->check_partials);
  dev_free(H, H->ubuf);
  dev_free(H, H->dstate);
  dev_free(H, H->partials);
  dev_free(H, H->hist);
  dev_free(H, H->hist_count);
  dev_free(H, H->stage[0]);
  dev_free(H, H->stage[1]);
  if (H->own_stream && H->stream) cudaStreamDestroy(H->stream);
  delete H;
}

lcs_status lcs_bound_create(int sigma, int d, int h, const lcs_bound_opts* opts_in, lcs_bound_t** out) {
  if (!out) return fail(LCS_EINVAL, "out is NULL");
  *out = nullptr;
  lcs_bound_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    lcs_bound_default_opts(&opts);
  if (opts.frac_bits == 0) opts.frac_bits = 44;
  if (sigma < 2 || d < 2 || h < 1 || d > kMaxD) return fail(LCS_EINVAL, "bad shape sigma=%d d=%d h=%d", sigma, d, h);
  if (opts.frac_bits < 8 || opts.frac_bits > 56) return fail(LCS_EINVAL, "frac_bits %d outside 8..56", opts.frac_bits);
  if (opts.r_mode != 0 && opts.r_mode != 1) return fail(LCS_EINVAL, "r_mode %d", opts.r_mode);
  if (opts.check_every < 0) return fail(LCS_EINVAL, "check_every %d", opts.check_every);
  if (opts.f_mode != 0 && opts.f_mode != 1) return fail(LCS_EINVAL, "f_mode %d", opts.f_mode);
  if (opts.alloc && !opts.free) return fail(LCS_EINVAL, "alloc given without free");
  if (opts.storage != 0 && opts.storage != 1) return fail(LCS_EINVAL, "storage %d", opts.storage);
  if (opts.host_slots < 0 || opts.host_slots > 1) return fail(LCS_EINVAL, "host_slots %d outside 0..1", opts.host_slots);
  if (opts.storage == 1) {
    if (sigma != 2 || d != 2 || h < 6 || !opts.symmetry || opts.f_mode != 0)
      return fail(LCS_EUNSUPPORTED,
                  "32-bit storage needs sigma = d = 2, h >= 6, complement-symmetric storage and f_mode 0");
    if (opts.keep_u) return fail(LCS_EUNSUPPORTED, "32-bit storage does not retain u (keep_u)");
    if (opts.frac_bits > 30) return fail(LCS_EINVAL, "32-bit storage needs frac_bits <= 30 (got %d)", opts.frac_bits);
  }
  // state count below 2^40
  unsigned long long n = 1;
  for (int i = 0; i < d * h; ++i) {
    n *= (unsigned long long)sigma;
    if (n >= (1ull << 40)) return fail(LCS_EINVAL, "sigma^(d h) must be below 2^40");
  }
  int sym = (sigma == 2 && opts.symmetry && h >= 2) ? 1 : 0;
  const KernelSet* ks = find_kernels(sigma, d, sym, opts.f_mode);
  if (!ks && opts.f_mode == 0) {
    // no specialised kernel: the general one, with full storage
    ks = kernels_rt(sigma);
    sym = 0;
  }
  if (!ks) return fail(LCS_EUNSUPPORTED, "no kernel compiled for sigma=%d d=%d f_mode=%d", sigma, d, opts.f_mode);
  // kernels that also use the swap symmetry (used while the iterates have it)
  const KernelSet* ks_swap = nullptr;
  if (d == 2 && opts.f_mode == 0) {
    if (sym && h >= 6)
      ks_swap = find_kernels(sigma, d, 2);
    else if (!sym && sigma >= 3 && h >= d2s_min_h(sigma))
      ks_swap = find_kernels(sigma, d, 3);
  }
  if (d == 3 && sigma == 2 && sym && h >= d3s_min_h() && h <= d3s_max_h()) ks_swap = find_kernels(sigma, d, 4, opts.f_mode);
  if (opts.storage == 1) ks = ks_swap = kernels_s2d2_narrow();  // the swap-aware sweep only

  lcs_bound* H = new (std::nothrow) lcs_bound();
  if (!H) return fail(LCS_ENOMEM, "host allocation");
  H->sigma = sigma;
  H->d = d;
  H->h = h;
  H->n_total = n;
  H->sym = sym;
  H->n_stored = sym ? n / 2 : n;
  unsigned long long sd = 1;
  for (int i = 0; i < d; ++i) sd *= (unsigned long long)sigma;
  H->n_tail = n / sd;
  H->opts = opts;
  H->ks = ks;
  H->ks_swap = ks_swap;
  H->swap_ok = ks_swap != nullptr;  // the zero start is swap-symmetric
  H->one = 1ll << opts.frac_bits;
  H->newest = d - 1;
  H->narrow = opts.storage == 1;
  H->elem = H->narrow ? sizeof(int) : sizeof(long long);

  cudaError_t e = cudaGetDevice(&H->device);
  if (e != cudaSuccess) {
    lcs_bound_destroy(H);
    return fail(LCS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  if (opts.stream) {
    H->stream = (cudaStream_t)opts.stream;
    H->own_stream = false;
  } else {
    e = cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      lcs_bound_destroy(H);
      return fail(LCS_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    H->own_stream = true;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H->device);
  if (sms < 1) sms = 1;
  // the general kernels: in block form where it applies (one thread per state
  // in the second phase), else one tail tuple per CTA or warp
  const bool rt_blocks = ks->tails_per_thread == 0 && rt_blocks_apply(sigma, d, h);
  const unsigned long long thread_items =
      ks->tails_per_thread == 0 ? rt_work_items(sigma, d, n, H->n_tail, rt_blocks) : (sym ? H->n_tail / 2 : H->n_tail);
  H->grid_sweep = grid_for(ks->sweep_fn, sms, thread_items);
  H->grid_check = grid_for(ks->check_fn, sms, thread_items);
  if (rt_blocks) {
    // the block form's second phase (one thread per state, few registers,
    // bound by the latency of its table reads): six CTAs per SM
    const unsigned long long need = std::max(1ull, (n + kBlock - 1) / kBlock);
    H->grid_sweep = H->grid_check = (int)std::min((unsigned long long)sms * 6, need);
  }
  H->n_partials = std::max(H->grid_sweep, H->grid_check);
  if (ks_swap) {
    // sigma = d = 2: one CTA per 16 x 16 tile of orbit representatives;
    // d = 2, sigma >= 3: one CTA per slot of tiles of (A, B) pairs
    const unsigned long long tiles = ks_swap->sym == 2   ? 2ull * (1ull << (h - 6)) * (1ull << (h - 6))
                                     : ks_swap->sym == 3 ? d2s_slots(sigma, h)
                                                         : d3s_tiles(h);
    H->grid_sweep_swap = grid_for(ks_swap->sweep_fn, sms, tiles * kBlock);
    H->grid_check_swap = grid_for(ks_swap->check_fn, sms, tiles * kBlock);
    H->n_partials = std::max(H->n_partials, std::max(H->grid_sweep_swap, H->grid_check_swap));
    if (ks_swap->sweep_check) {
      H->grid_fused = grid_for(ks_swap->sweep_check_fn, sms, tiles * kBlock);
      H->n_partials = std::max(H->n_partials, H->grid_fused);
    }
  }

  const size_t vbytes = (size_t)H->n_stored * H->elem;
  for (int k = 0; k <= d; ++k) {
    if (k >= d + 1 - opts.host_slots) {
      // A row in pinned host memory mapped into the device's address space
      // (host_map_alloc: the kernels gather from all of it at once, and large
      // pages keep the device's translations few -- a 128 GiB row of 64 KiB
      // pages needs two million).
      void* base = nullptr;
      size_t len = 0;
      void* hp = host_map_alloc(vbytes, &base, &len);
      void* dp = nullptr;
      if (hp && cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) {
        cudaGetLastError();
        host_map_free(hp, base, len);
        hp = nullptr;
      }
      if (!hp) {
        lcs_bound_destroy(H);
        return fail(LCS_ENOMEM, "iterate vector %d in pinned host memory (%zu bytes)", k, vbytes);
      }
      H->host_base[k] = base;
      H->host_len[k] = len;
      H->host_ptr[k] = hp;
      H->ring[k] = (long long*)dp;
      continue;
    }
    H->ring[k] = (long long*)dev_alloc(H, vbytes);
    if (!H->ring[k]) {
      lcs_bound_destroy(H);
      return fail(LCS_ENOMEM, "iterate vector %d (%zu bytes)", k, vbytes);
    }
  }
  if (opts.keep_u) {
    H->ubuf = (long long*)dev_alloc(H, vbytes);
    if (!H->ubuf) {
      lcs_bound_destroy(H);
      return fail(LCS_ENOMEM, "u vector (%zu bytes)", vbytes);
    }
  }
  H->dstate = (DevState*)dev_alloc(H, sizeof(DevState));
  H->partials = (RedPartial*)dev_alloc(H, sizeof(RedPartial) * (size_t)H->n_partials);
  H->hist = (CheckRecord*)dev_alloc(H, sizeof(CheckRecord) * kHistCap);
  H->hist_count = (unsigned long long*)dev_alloc(H, sizeof(unsigned long long));
  if (!H->dstate || !H->partials || !H->hist || !H->hist_count) {
    lcs_bound_destroy(H);
    return fail(LCS_ENOMEM, "state and reduction scratch");
  }
  if (ks_swap && ks_swap->sweep_check) {
    H->check_partials = (RedPartial*)dev_alloc(H, sizeof(RedPartial) * (size_t)H->n_partials);
    if (!H->check_partials) {
      lcs_bound_destroy(H);
      return fail(LCS_ENOMEM, "partials of the fused check");
    }
  }
  if (rt_blocks) {
    const size_t rows = (size_t)sigma << d;
    H->rt_means = (long long*)dev_alloc(H, sizeof(long long) * rows * (size_t)H->n_tail);
    H->rt_offs = (unsigned short*)dev_alloc(H, sizeof(unsigned short) * rt_offsets_len(sigma, d));
    H->rt_start = (unsigned*)dev_alloc(H, sizeof(unsigned) << d);
    if (!H->rt_means || !H->rt_offs || !H->rt_start) {
      lcs_bound_destroy(H);
      return fail(LCS_ENOMEM, "means table and term offsets of the general kernels (%zu bytes)",
                  sizeof(long long) * rows * (size_t)H->n_tail);
    }
    rt_offsets_fill(sigma, d, H->rt_offs, H->rt_start, H->stream);
    const std::vector<unsigned long long> tiles = rt_tile_list(sigma, d, h);
    H->rt_n_tiles = tiles.size();
    H->rt_tiles = (unsigned long long*)dev_alloc(H, sizeof(unsigned long long) * std::max<size_t>(1, tiles.size()));
    if (!H->rt_tiles) {
      lcs_bound_destroy(H);
      return fail(LCS_ENOMEM, "tile list of the general kernels");
    }
    e = cudaMemcpyAsync(H->rt_tiles, tiles.data(), sizeof(unsigned long long) * tiles.size(), cudaMemcpyHostToDevice,
                        H->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H->stream);  // the host list is freed on return
    if (e != cudaSuccess) {
      lcs_bound_destroy(H);
      return fail(LCS_ECUDA, "tile list: %s", cudaGetErrorString(e));
    }
  }
  if (H->narrow) {
    H->offs = (long long*)dev_alloc(H, sizeof(long long) * (size_t)(kMaxD + 1));
    if (!H->offs) {
      lcs_bound_destroy(H);
      return fail(LCS_ENOMEM, "offsets of the 32-bit rows");
    }
    e = cudaMemsetAsync(H->offs, 0, sizeof(long long) * (size_t)(kMaxD + 1), H->stream);
    if (e != cudaSuccess) {
      lcs_bound_destroy(H);
      return fail(LCS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
  }
  e = cudaMemsetAsync(H->hist_count, 0, sizeof(unsigned long long), H->stream);
  if (e != cudaSuccess) {
    lcs_bound_destroy(H);
    return fail(LCS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  // zero start (Algorithm 2: v <- 0)
  for (int k = 0; k < d; ++k) {
    e = cudaMemsetAsync(H->ring[k], 0, vbytes, H->stream);
    if (e != cudaSuccess) {
      lcs_bound_destroy(H);
      return fail(LCS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
  }
  if (H->ubuf) cudaMemsetAsync(H->ubuf, 0, vbytes, H->stream);
  init_state_kernel<<<1, 32, 0, H->stream>>>(H->dstate);
  e = cudaStreamSynchronize(H->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    lcs_bound_destroy(H);
    return fail(LCS_ECUDA, "create: %s", cudaGetErrorString(e));
  }
  H->vbound = 0.0;
  *out = H;
  return LCS_OK;
}

lcs_status lcs_bound_size(const lcs_bound_t* H, uint64_t* n_states, uint64_t* n_stored) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  if (n_states) *n_states = H->n_total;
  if (n_stored) *n_stored = H->n_stored;
  return LCS_OK;
}

lcs_status lcs_bound_shape(const lcs_bound_t* H, int* sigma, int* d, int* h) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: its instances have their own shapes");
  if (sigma) *sigma = H->sigma;
  if (d) *d = H->d;
  if (h) *h = H->h;
  return LCS_OK;
}

static void fold_events(lcs_bound* H) {
  for (auto& e : H->sweep_ev) {
    float ms = 0;
    cudaEventSynchronize(e.second);
    cudaEventElapsedTime(&ms, e.first, e.second);
    H->sweep_ms += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : H->check_ev) {
    float ms = 0;
    cudaEventSynchronize(e.second);
    cudaEventElapsedTime(&ms, e.first, e.second);
    H->check_ms += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  H->sweep_ev.clear();
  H->check_ev.clear();
  for (int c = 0; c < 3; ++c) {
    for (auto& e : H->xfer_ev[c]) {
      float ms = 0;
      cudaEventSynchronize(e.second);
      cudaEventElapsedTime(&ms, e.first, e.second);
      H->xfer_ms[c] += ms;
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    H->xfer_ev[c].clear();
  }
}

static lcs_status timed_begin(lcs_bound* H, cudaEvent_t* a) {
  if (!H->opts.timing) return LCS_OK;
  LCS_CUDA(cudaEventCreate(a));
  LCS_CUDA(cudaEventRecord(*a, H->stream));
  return LCS_OK;
}

static lcs_status timed_end(lcs_bound* H, cudaEvent_t a, bool sweep) {
  if (!H->opts.timing) return LCS_OK;
  cudaEvent_t b;
  LCS_CUDA(cudaEventCreate(&b));
  LCS_CUDA(cudaEventRecord(b, H->stream));
  (sweep ? H->sweep_ev : H->check_ev).emplace_back(a, b);
  if (H->sweep_ev.size() + H->check_ev.size() > 8192) fold_events(H);
  return LCS_OK;
}

enum { kXferH2D = 0, kXferD2H = 1, kXferKernel = 2 };

// events around one transfer operation on stream s (opts.timing only)
static lcs_status xfer_begin(lcs_bound* H, cudaStream_t s, cudaEvent_t* a) {
  *a = nullptr;
  if (!H->opts.timing) return LCS_OK;
  LCS_CUDA(cudaEventCreate(a));
  LCS_CUDA(cudaEventRecord(*a, s));
  return LCS_OK;
}

static lcs_status xfer_end(lcs_bound* H, cudaStream_t s, cudaEvent_t a, int cat) {
  if (!H->opts.timing) return LCS_OK;
  cudaEvent_t b;
  LCS_CUDA(cudaEventCreate(&b));
  LCS_CUDA(cudaEventRecord(b, s));
  H->xfer_ev[cat].emplace_back(a, b);
  if (H->xfer_ev[cat].size() > 4096) fold_events(H);
  return LCS_OK;
}

static lcs_status run_check(lcs_bound* H, const long long* u, bool R_from_state, long long R, long long iter,
                            bool finalize, bool allow_swap) {
  const bool use_swap = allow_swap && H->swap_ok && H->ks_swap;
  const KernelSet* K = use_swap ? H->ks_swap : H->ks;
  const int grid = use_swap ? H->grid_check_swap : H->grid_check;
  CheckParams c{};
  c.u = u;
  c.n_tail = H->n_tail;
  c.n_stored = H->n_stored;
  c.h = H->h;
  c.one = H->one;
  c.state = H->dstate;
  c.R_from_state = R_from_state ? 1 : 0;
  c.R = R;
  c.partials = H->partials;
  c.rt_means = H->rt_means;
  c.rt_offs = H->rt_offs;
  c.rt_start = H->rt_start;
  cudaEvent_t a = nullptr;
  lcs_status st = timed_begin(H, &a);
  if (st) return st;
  K->check(c, grid, H->stream);
  LCS_CUDA(cudaGetLastError());
  st = timed_end(H, a, false);
  if (st) return st;
  H->check_n++;
  H->check_bytes += (unsigned long long)K->check_algo_bytes * H->n_stored;
  H->launches += H->rt_means ? 2 : 1;
  H->last_check_grid = grid;
  if (finalize) {
    finalize_check_kernel<<<1, kFinalBlock, 0, H->stream>>>(H->partials, grid, H->dstate, iter, H->hist,
                                                            H->hist_count);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
  }
  return LCS_OK;
}

// the part of a check that follows its partials: E, the keep test (and the
// history record), then the copy of a kept u
static lcs_status finish_check(lcs_bound* H, const RedPartial* parts, int n_parts, const long long* u, long long iter) {
  finalize_check_kernel<<<1, kFinalBlock, 0, H->stream>>>(parts, n_parts, H->dstate, iter, H->hist, H->hist_count);
  LCS_CUDA(cudaGetLastError());
  H->launches++;
  if (H->ubuf) {
    copy_if_kept_kernel<<<H->grid_sweep, kBlock, 0, H->stream>>>(u, H->ubuf, H->n_stored, H->dstate);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
  }
  return LCS_OK;
}

// run a check that waits for the next sweep on its own (before anything that
// reads the results of Algorithm 2)
static lcs_status flush_pending(lcs_bound* H) {
  if (!H->pending_check) return LCS_OK;
  H->pending_check = false;
  const long long* u = H->ring[H->newest];
  if (lcs_status st = run_check(H, u, true, 0, H->pending_iter, false, true)) return st;
  return finish_check(H, H->partials, H->last_check_grid, u, H->pending_iter);
}

lcs_status lcs_bound_iterate(lcs_bound_t* H, int64_t n_iters) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  if (n_iters < 0) return fail(LCS_EINVAL, "n_iters < 0");
  if (n_iters == 0) return LCS_OK;
  if (H->batch) {
    const double vb_after = H->vbound + (double)n_iters * (double)H->one;
    if (!headroom_ok(H, vb_after)) return fail(LCS_EOVERFLOW, "iterates could exceed the fixed-point range");
    lcs_status st = batch_iterate(H->batch, H->stream, n_iters);
    if (st) return st;
    H->vbound = vb_after;
    H->iters_done += n_iters;
    return LCS_OK;
  }
  const double vb_after = H->vbound + (double)n_iters * (double)H->one;
  if (!headroom_ok(H, vb_after))
    return fail(LCS_EOVERFLOW, "iterates could exceed the fixed-point range (max |v| up to %.3g)",
                vb_after / (double)H->one);
  if (H->narrow && !H->swap_ok)
    return fail(LCS_EINVAL, "32-bit storage runs only the swap-aware sweep, and the start lacks the swap symmetry");
  const int rows = H->d + 1;
  for (int64_t i = 0; i < n_iters; ++i) {
    const long long it = H->iters_done + 1;
    const bool check = (H->opts.check_every > 0 && it % H->opts.check_every == 0) || i == n_iters - 1;
    const int out_slot = (H->newest + 1) % rows;
    SweepParams p{};
    for (int k = 1; k <= H->d; ++k) p.prev[k - 1] = H->ring[(H->newest - (k - 1) + rows) % rows];
    p.out = H->ring[out_slot];
    p.n_tail = H->n_tail;
    p.n_stored = H->n_stored;
    p.h = H->h;
    p.incr = check ? 1 : 0;
    p.r_mode = H->opts.r_mode;
    p.one = H->one;
    p.partials = H->partials;
    p.state = H->dstate;
    p.rt_means = H->rt_means;
    p.rt_offs = H->rt_offs;
    p.rt_start = H->rt_start;
    p.rt_tiles = H->rt_tiles;
    p.rt_n_tiles = H->rt_n_tiles;
    if (H->narrow) {
      p.offs = H->offs;
      p.slot_in0 = H->newest;
      p.slot_in1 = (H->newest - 1 + rows) % rows;
      p.slot_out = out_slot;
      p.step = 0;  // before the first increment the offsets stay put
    }
    const bool use_swap = H->swap_ok && H->ks_swap;
    const KernelSet* K = use_swap ? H->ks_swap : H->ks;
    // a check left by the previous iteration runs inside this sweep if the
    // kernels can fuse it, else on its own first
    const bool fuse = H->pending_check && K->sweep_check;
    if (H->pending_check && !fuse)
      if (lcs_status st = flush_pending(H)) return st;
    const int grid = fuse ? H->grid_fused : use_swap ? H->grid_sweep_swap : H->grid_sweep;
    cudaEvent_t a = nullptr;
    lcs_status st = timed_begin(H, &a);
    if (st) return st;
    if (fuse) {
      p.check_partials = H->check_partials;
      K->sweep_check(p, grid, H->stream);
    } else {
      K->sweep(p, grid, H->stream);
    }
    LCS_CUDA(cudaGetLastError());
    st = timed_end(H, a, true);
    if (st) return st;
    H->sweep_n++;
    // the general kernels: every output written once, each of the d inputs read once
    const int algo = K->tails_per_thread == 0 ? 8 * (H->d + 1) : K->sweep_algo_bytes;
    // a fused check adds one more read of the newest input's blocks: half of a check's bytes
    H->sweep_bytes += (unsigned long long)(algo + (fuse ? K->check_algo_bytes / 2 : 0)) * H->n_stored;
    H->launches += H->rt_means ? 2 : 1;  // the block form: the means table, then the states
    if (fuse) {  // the pending check's E and keep test, before this iteration's increment replaces R
      H->pending_check = false;
      if (lcs_status st2 = finish_check(H, H->check_partials, grid, p.prev[0], H->pending_iter)) return st2;
    }
    if (check) {
      finalize_incr_kernel<<<1, kFinalBlock, 0, H->stream>>>(H->partials, grid, H->opts.r_mode, H->dstate, it);
      LCS_CUDA(cudaGetLastError());
      H->launches++;
      if (use_swap && K->sweep_check) {
        H->pending_check = true;  // the next sweep, or the next call that reads results, runs it
        H->pending_iter = it;
      } else {
        st = run_check(H, p.out, true, 0, it, false, true);
        if (st) return st;
        if (lcs_status st2 = finish_check(H, H->partials, H->last_check_grid, p.out, it)) return st2;
      }
    }
    H->newest = out_slot;
    H->iters_done = it;
  }
  H->vbound = vb_after;
  return LCS_OK;
}

lcs_status lcs_bound_read_report(lcs_bound_t* H, lcs_bound_report* out) {
  if (!H || !out) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  if (lcs_status st = flush_pending(H)) return st;
  DevState s;
  LCS_CUDA(cudaMemcpyAsync(&s, H->dstate, sizeof s, cudaMemcpyDeviceToHost, H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  out->iters_done = H->iters_done;
  out->R = s.R;
  out->argmin = s.argmin;
  out->E = s.E;
  out->r = s.r;
  out->eps = s.eps;
  out->kept_iter = s.kept_iter;
  out->have_check = s.have_check;
  out->frac_bits = H->opts.frac_bits;
  out->status = (int)s.status;
  return LCS_OK;
}

// round-down conversion of a fixed-point value to double
static double fx_to_double_rd(long long a, int frac_bits) {
  double x = (double)a;  // round to nearest
  if (x >= 9223372036854775808.0)
    x = std::nextafter(x, -INFINITY);
  else if ((long double)x > (long double)a && (long long)x > a)
    x = std::nextafter(x, -INFINITY);
  return std::ldexp(x, -frac_bits);
}

lcs_status lcs_bound_read(lcs_bound_t* H, double* bound_rd, uint64_t* argmin_state, double* r, double* eps,
                          int64_t* at_iter) {
  lcs_bound_report rep;
  lcs_status st = lcs_bound_read_report(H, &rep);
  if (st) return st;
  if (rep.status) return fail((lcs_status)rep.status, "device status %d", rep.status);
  if (!rep.have_check) return fail(LCS_ENOBOUND, "no feasibility check has run");
  const int K = H->opts.frac_bits;
  const long long B = (long long)H->d * (rep.r - rep.eps);  // |r|, |eps| < 2^62 / d by the headroom rule
  if (bound_rd) *bound_rd = fx_to_double_rd(B, K);
  if (argmin_state) *argmin_state = rep.argmin;
  if (r) *r = std::ldexp((double)rep.r, -K);
  if (eps) *eps = std::ldexp((double)rep.eps, -K);
  if (at_iter) *at_iter = rep.kept_iter;
  return LCS_OK;
}

static const size_t kChunk = (size_t)32 << 20;    // values per staged piece (256 MiB)

// The copy stream, its events and the two staging buffers, made on the first
// host transfer of a handle.
static lcs_status ensure_xfer(lcs_bound* H, bool staging) {
  if (!H->xstream) {
    LCS_CUDA(cudaStreamCreateWithFlags(&H->xstream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      LCS_CUDA(cudaEventCreateWithFlags(&H->stage_ready[i], cudaEventDisableTiming));
      LCS_CUDA(cudaEventCreateWithFlags(&H->stage_free[i], cudaEventDisableTiming));
    }
    LCS_CUDA(cudaEventCreateWithFlags(&H->xsync, cudaEventDisableTiming));
  }
  for (int i = 0; staging && i < 2; ++i) {
    if (H->stage[i]) continue;
    H->stage[i] = dev_alloc(H, kChunk * 8);
    if (!H->stage[i]) return fail(LCS_ENOMEM, "staging buffer (%zu bytes)", kChunk * 8);
  }
  return LCS_OK;
}

// make stream `to` wait for everything enqueued on stream `from` so far
static lcs_status stream_after(lcs_bound* H, cudaStream_t to, cudaStream_t from) {
  LCS_CUDA(cudaEventRecord(H->xsync, from));
  LCS_CUDA(cudaStreamWaitEvent(to, H->xsync, 0));
  return LCS_OK;
}

// One copy between host and device on the copy stream, timed.
static lcs_status xfer_copy(lcs_bound* H, void* dst, const void* src, size_t bytes, bool h2d) {
  cudaEvent_t a;
  if (lcs_status st = xfer_begin(H, H->xstream, &a)) return st;
  LCS_CUDA(cudaMemcpyAsync(dst, src, bytes, h2d ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, H->xstream));
  (h2d ? H->h2d_bytes : H->d2h_bytes) += bytes;
  return xfer_end(H, H->xstream, a, h2d ? kXferH2D : kXferD2H);
}

// (templates: C++ linkage inside the extern "C" block)
extern "C++" {
// Host -> device through the two staging buffers: piece i is copied into
// stage[i % 2] on the copy stream while `consume` (kernels on the handle's
// stream) converts piece i - 1 out of the other buffer.  A staging buffer is
// refilled only after the last kernel that read it (stage_free), also across
// calls, so the copies of one call may run ahead while the handle's stream
// still works on an earlier one.
template <class Consume>
static lcs_status h2d_pipelined(lcs_bound* H, const void* src_host, unsigned long long n, Consume consume) {
  if (lcs_status st = ensure_xfer(H, true)) return st;
  int i = 0;
  for (unsigned long long off = 0; off < n; off += kChunk, ++i) {
    const int b = i & 1;
    const unsigned long long len = std::min<unsigned long long>(kChunk, n - off);
    if (H->stage_recorded[b]) LCS_CUDA(cudaStreamWaitEvent(H->xstream, H->stage_free[b], 0));
    if (lcs_status st = xfer_copy(H, H->stage[b], (const char*)src_host + off * 8, len * 8, true)) return st;
    LCS_CUDA(cudaEventRecord(H->stage_ready[b], H->xstream));
    LCS_CUDA(cudaStreamWaitEvent(H->stream, H->stage_ready[b], 0));
    cudaEvent_t a;
    if (lcs_status st = xfer_begin(H, H->stream, &a)) return st;
    if (lcs_status st = consume((const long long*)H->stage[b], off, len)) return st;
    if (lcs_status st = xfer_end(H, H->stream, a, kXferKernel)) return st;
    LCS_CUDA(cudaEventRecord(H->stage_free[b], H->stream));
    H->stage_recorded[b] = true;
  }
  return LCS_OK;
}

// Device -> host through the two staging buffers: `produce` (kernels on the
// handle's stream) fills stage[i % 2] with piece i while the copy stream
// moves piece i - 1 out.  The handle's stream waits for the last copy.
template <class Produce>
static lcs_status d2h_pipelined(lcs_bound* H, void* dst_host, unsigned long long n, Produce produce) {
  if (lcs_status st = ensure_xfer(H, true)) return st;
  int i = 0;
  for (unsigned long long off = 0; off < n; off += kChunk, ++i) {
    const int b = i & 1;
    const unsigned long long len = std::min<unsigned long long>(kChunk, n - off);
    if (H->stage_recorded[b]) LCS_CUDA(cudaStreamWaitEvent(H->stream, H->stage_free[b], 0));
    cudaEvent_t a;
    if (lcs_status st = xfer_begin(H, H->stream, &a)) return st;
    if (lcs_status st = produce((long long*)H->stage[b], off, len)) return st;
    if (lcs_status st = xfer_end(H, H->stream, a, kXferKernel)) return st;
    LCS_CUDA(cudaEventRecord(H->stage_ready[b], H->stream));
    LCS_CUDA(cudaStreamWaitEvent(H->xstream, H->stage_ready[b], 0));
    if (lcs_status st = xfer_copy(H, (char*)dst_host + off * 8, H->stage[b], len * 8, false)) return st;
    LCS_CUDA(cudaEventRecord(H->stage_free[b], H->xstream));
    H->stage_recorded[b] = true;
  }
  return stream_after(H, H->stream, H->xstream);
}

// dst[i] = src[i], 16 B at a time (both 16-byte aligned, n even) plus a tail
__global__ void copy_values_kernel(const long long* __restrict__ src, long long* __restrict__ dst,
                                   unsigned long long n) {
  const unsigned long long n2 = n / 2;
  const longlong2* s2 = reinterpret_cast<const longlong2*>(src);
  longlong2* d2 = reinterpret_cast<longlong2*>(dst);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (unsigned long long)gridDim.x * blockDim.x)
    d2[i] = s2[i];
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) dst[n - 1] = src[n - 1];
}

static lcs_status copy_values(lcs_bound* H, const long long* src, long long* dst, unsigned long long n) {
  const int grid = (int)std::min<unsigned long long>(1024, (n / 2 + kBlock - 1) / kBlock + 1);
  copy_values_kernel<<<grid, kBlock, 0, H->stream>>>(src, dst, n);
  LCS_CUDA(cudaGetLastError());
  H->launches++;
  return LCS_OK;
}

}  // extern "C++"

// n values between host memory and a device buffer with no conversion.  Even
// these go through the staging pipeline: on this GB300's link, copy-engine
// copies straight into (or out of) a buffer of many GiB were measured at a
// tenth to a half of the link's rate in some processes (after heavy earlier
// use of the machine), while copies through a 256 MiB buffer kept 210 GB/s in
// the same processes; the copy kernel on the device side costs a pass over
// the values at HBM speed, hidden behind the link.
static lcs_status h2d_copy(lcs_bound* H, long long* dst_dev, const void* src_host, unsigned long long n) {
  return h2d_pipelined(H, src_host, n, [&](const long long* stage, unsigned long long off, unsigned long long len) {
    return copy_values(H, stage, dst_dev + off, len);
  });
}

static lcs_status d2h_copy(lcs_bound* H, void* dst_host, const long long* src_dev, unsigned long long n) {
  return d2h_pipelined(H, dst_host, n, [&](long long* stage, unsigned long long off, unsigned long long len) {
    return copy_values(H, src_dev + off, stage, len);
  });
}

// Ingest [off, off+len) of an input vector.  Under complement-symmetric
// storage the part below n_stored is written before the part above it is
// compared with its mirror: two launches, ordered on the stream.
static lcs_status ingest_range(lcs_bound* H, const void* src, unsigned long long off, unsigned long long len,
                               long long* dst, bool from_double, double scale) {
  const unsigned long long split = std::min(std::max(H->n_stored, off), off + len);
  const unsigned long long parts[2][2] = {{off, split - off}, {split, off + len - split}};
  for (const auto& pr : parts) {
    if (pr[1] == 0) continue;
    const void* s = (const char*)src + (pr[0] - off) * 8;
    const int grid = (int)std::min<unsigned long long>(4096, (pr[1] + kBlock - 1) / kBlock);
    if (from_double)
      ingest_kernel<true><<<grid, kBlock, 0, H->stream>>>(s, pr[0], pr[1], dst, H->n_stored, H->n_total, scale,
                                                          H->dstate);
    else
      ingest_kernel<false><<<grid, kBlock, 0, H->stream>>>(s, pr[0], pr[1], dst, H->n_stored, H->n_total, scale,
                                                           H->dstate);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
  }
  return LCS_OK;
}

// the end of every start: read the checks of the start vectors, reset the
// results (the kept triplet returns to the initial (v_0, 0, 0)) and the ring
static lcs_status finish_start(lcs_bound* H) {
  DevState s;
  LCS_CUDA(cudaMemcpyAsync(&s, H->dstate, sizeof s, cudaMemcpyDeviceToHost, H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  init_state_kernel<<<1, 32, 0, H->stream>>>(H->dstate);
  LCS_CUDA(cudaGetLastError());
  if (H->ubuf) LCS_CUDA(cudaMemcpyAsync(H->ubuf, H->ring[0], H->n_stored * 8, cudaMemcpyDeviceToDevice, H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  H->newest = H->d - 1;
  H->iters_done = 0;
  H->pending_check = false;
  if (s.status == LCS_EINVAL)
    return fail(LCS_EINVAL, "start vectors are not complement-symmetric (v[N-1-x] != v[x])");
  if (s.status == LCS_EOVERFLOW) return fail(LCS_EOVERFLOW, "start values outside the fixed-point range");
  H->vbound = (double)s.maxabs;
  H->swap_ok = H->ks_swap != nullptr && s.swap_bad == 0;
  if (!headroom_ok(H, H->vbound)) return fail(LCS_EOVERFLOW, "start values too large for the fixed-point headroom");
  return LCS_OK;
}

// calls that 32-bit storage does not offer
static lcs_status wide_only(const lcs_bound* H, const char* what) {
  if (H && H->narrow) return fail(LCS_EUNSUPPORTED, "%s is not available with 32-bit storage", what);
  return LCS_OK;
}

// the checks of one start row: max |v|, and the symmetries the fast kernels use
static lcs_status start_row_checks(lcs_bound* H, int slot) {
  long long* dst = H->ring[slot];
  const int grid = (int)std::min<unsigned long long>(4096, (H->n_stored + kBlock - 1) / kBlock);
  if (H->narrow) {  // max |v| came with the narrowing
    maxabs_swap_check_kernel<int><<<grid, kBlock, 0, H->stream>>>((const int*)dst, H->n_stored, H->n_total,
                                                                  H->dstate, H->offs, slot);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
    return LCS_OK;
  }
  if (H->ks_swap && H->ks_swap->sym == 2) {
    maxabs_swap_check_kernel<<<grid, kBlock, 0, H->stream>>>(dst, H->n_stored, H->n_total, H->dstate);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
    return LCS_OK;
  }
  maxabs_kernel<<<grid, kBlock, 0, H->stream>>>(dst, H->n_stored, H->dstate);
  LCS_CUDA(cudaGetLastError());
  H->launches++;
  if (H->ks_swap) {
    if (H->ks_swap->sym == 3)
      launch_swap_check_d2s(H->sigma, dst, H->n_stored, H->h, H->dstate, grid, H->stream);
    else
      launch_perm_check_d3s(dst, H->n_stored, H->n_total, H->dstate, grid, H->stream);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
  }
  return LCS_OK;
}

// a stored-form row into 32-bit storage: offset c = the row's first value
static lcs_status narrow_row(lcs_bound* H, const void* src, int on_device, int slot) {
  long long c = 0;
  if (on_device)
    LCS_CUDA(cudaMemcpy(&c, src, sizeof c, cudaMemcpyDeviceToHost));
  else
    c = *static_cast<const long long*>(src);
  int* dst = reinterpret_cast<int*>(H->ring[slot]);
  auto conv = [&](const long long* from, unsigned long long off, unsigned long long len) {
    const int grid = (int)std::min<unsigned long long>(4096, (len + kBlock - 1) / kBlock);
    narrow_kernel<<<grid, kBlock, 0, H->stream>>>(from, dst + off, len, c, H->dstate);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
    return LCS_OK;
  };
  if (on_device) {
    if (lcs_status st = conv(static_cast<const long long*>(src), 0, H->n_stored)) return st;
  } else if (lcs_status st = h2d_pipelined(H, src, H->n_stored, conv)) {
    return st;
  }
  set_offset_kernel<<<1, 32, 0, H->stream>>>(H->offs, slot, c);
  LCS_CUDA(cudaGetLastError());
  H->launches++;
  return LCS_OK;
}

// stored = true: v[k] holds the n_stored stored values (the storage form), copied as they are
static lcs_status set_start_checked(lcs_bound* H, const void* const* v, int on_device, bool from_double,
                                    bool stored = false) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  if (!v) return fail(LCS_EINVAL, "NULL argument");
  if (!stored)
    if (lcs_status st = wide_only(H, "a start of full vectors (use the stored form)")) return st;
  const double scale = std::ldexp(1.0, H->opts.frac_bits);
  LCS_CUDA(cudaMemsetAsync(H->dstate, 0, sizeof(DevState), H->stream));
  LCS_CUDA(cudaMemsetAsync(H->hist_count, 0, sizeof(unsigned long long), H->stream));
  for (int k = 0; k < H->d; ++k)
    if (!v[k]) return fail(LCS_EINVAL, "start vector %d is NULL", k);
  for (int k = 0; k < H->d; ++k) {
    long long* dst = H->ring[H->d - 1 - k];
    if (H->narrow) {
      if (lcs_status st = narrow_row(H, v[k], on_device, H->d - 1 - k)) return st;
    } else if (stored && !on_device) {
      if (lcs_status st = h2d_copy(H, dst, v[k], H->n_stored)) return st;
    } else if (stored) {
      LCS_CUDA(cudaMemcpyAsync(dst, v[k], H->n_stored * 8, cudaMemcpyDeviceToDevice, H->stream));
    } else if (on_device) {
      lcs_status st = ingest_range(H, v[k], 0, H->n_total, dst, from_double, scale);
      if (st) return st;
    } else {
      lcs_status st = h2d_pipelined(H, v[k], H->n_total,
                                    [&](const long long* stage, unsigned long long off, unsigned long long len) {
                                      return ingest_range(H, stage, off, len, dst, from_double, scale);
                                    });
      if (st) return st;
    }
    if (lcs_status st = start_row_checks(H, H->d - 1 - k)) return st;
  }
  if (lcs_status st = finish_start(H)) return st;
  if (H->narrow && !H->swap_ok) return fail(LCS_EINVAL, "32-bit storage needs swap-symmetric start vectors");
  return LCS_OK;
}

lcs_status lcs_bound_set_start(lcs_bound_t* H, const double* const* v, int on_device) {
  return set_start_checked(H, (const void* const*)v, on_device, true);
}

lcs_status lcs_bound_set_start_fx(lcs_bound_t* H, const int64_t* const* v, int on_device) {
  return set_start_checked(H, (const void* const*)v, on_device, false);
}

lcs_status lcs_bound_set_start_stored_fx(lcs_bound_t* H, const int64_t* const* v, int on_device) {
  return set_start_checked(H, (const void* const*)v, on_device, false, true);
}

lcs_status lcs_bound_set_start_lift_fx(lcs_bound_t* H, int h_from, const int64_t* src, int on_device, int64_t r_hat) {
  if (!H || !src) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  if (H->sigma != 2 || H->d != 2 || !H->sym)
    return fail(LCS_EUNSUPPORTED, "the prefix lift needs sigma = d = 2 with complement-symmetric storage");
  if (h_from < 2 || h_from > H->h) return fail(LCS_EINVAL, "h_from %d outside 2..%d", h_from, H->h);
  const int s2 = 2 * (H->h - h_from);
  const unsigned long long n_src = H->n_stored >> s2;  // the stored half of the shorter shape
  long long first = 0;
  if (on_device)
    LCS_CUDA(cudaMemcpy(&first, src, sizeof first, cudaMemcpyDeviceToHost));
  else
    first = src[0];
  // 64-bit rows hold the values; 32-bit rows hold value - first (newest) and
  // value - r_hat - (first - r_hat) (older): the same numbers, two offsets
  const long long sub_new = H->narrow ? first : 0, sub_old = H->narrow ? first : (long long)r_hat;
  LCS_CUDA(cudaMemsetAsync(H->dstate, 0, sizeof(DevState), H->stream));
  LCS_CUDA(cudaMemsetAsync(H->hist_count, 0, sizeof(unsigned long long), H->stream));
  const int s_new = H->d - 1, s_old = H->d - 2;  // ring rows of v[0] (newest) and v[1]
  auto lift = [&](const long long* from, unsigned long long off, unsigned long long len) {
    const unsigned long long lo = off << s2, hi = (off + len) << s2;
    const int grid = (int)std::min<unsigned long long>(4096, (hi - lo + kBlock - 1) / kBlock);
    if (H->narrow)
      lift_kernel<int><<<grid, kBlock, 0, H->stream>>>(from, off, s2, lo, hi, (int*)H->ring[s_new],
                                                       (int*)H->ring[s_old], sub_new, sub_old, H->dstate);
    else
      lift_kernel<long long><<<grid, kBlock, 0, H->stream>>>(from, off, s2, lo, hi, H->ring[s_new], H->ring[s_old],
                                                             sub_new, sub_old, H->dstate);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
    return LCS_OK;
  };
  if (on_device) {
    if (lcs_status st = lift(reinterpret_cast<const long long*>(src), 0, n_src)) return st;
  } else if (lcs_status st = h2d_pipelined(H, src, n_src, lift)) {
    return st;
  }
  if (H->narrow) {
    set_offset_kernel<<<1, 32, 0, H->stream>>>(H->offs, s_new, first);
    set_offset_kernel<<<1, 32, 0, H->stream>>>(H->offs, s_old, first - (long long)r_hat);
    LCS_CUDA(cudaGetLastError());
    H->launches += 2;
  }
  for (int slot : {s_new, s_old})
    if (lcs_status st = start_row_checks(H, slot)) return st;
  if (lcs_status st = finish_start(H)) return st;
  if (H->narrow && !H->swap_ok) return fail(LCS_EINVAL, "32-bit storage needs swap-symmetric start vectors");
  return LCS_OK;
}

lcs_status lcs_bound_export_stored_fx(lcs_bound_t* H, int k, int64_t* dst, int on_device) {
  if (!H || !dst) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  if (k < -1 || k >= H->d) return fail(LCS_EINVAL, "k=%d outside -1..d-1", k);
  if (k == -1)
    if (lcs_status st = flush_pending(H)) return st;  // u is the kept iterate: its check must have run
  const long long* src;
  int slot = -1;
  if (k == -1) {
    if (!H->ubuf) return fail(LCS_EINVAL, "u is not retained (opts.keep_u = 0)");
    src = H->ubuf;
  } else {
    const int rows = H->d + 1;
    slot = (H->newest - k + rows) % rows;
    src = H->ring[slot];
  }
  if (H->narrow) {  // widen: value = stored + the row's offset (no u is kept with 32-bit storage)
    auto widen = [&](long long* to, unsigned long long off, unsigned long long len) {
      const int grid = (int)std::min<unsigned long long>(4096, (len + kBlock - 1) / kBlock);
      widen_kernel<<<grid, kBlock, 0, H->stream>>>(reinterpret_cast<const int*>(src) + off, to, len, H->offs, slot);
      LCS_CUDA(cudaGetLastError());
      H->launches++;
      return LCS_OK;
    };
    if (on_device) {
      if (lcs_status st = widen(reinterpret_cast<long long*>(dst), 0, H->n_stored)) return st;
    } else if (lcs_status st = d2h_pipelined(H, dst, H->n_stored, widen)) {
      return st;
    }
  } else if (on_device) {
    LCS_CUDA(cudaMemcpyAsync(dst, src, H->n_stored * 8, cudaMemcpyDeviceToDevice, H->stream));
  } else if (lcs_status st = d2h_copy(H, dst, src, H->n_stored)) {
    return st;
  }
  if (!on_device) LCS_CUDA(cudaStreamSynchronize(H->stream));
  return LCS_OK;
}

// the orbit form (kernels_orbit.cu): sigma = d = 2 with the sweep that uses
// the complement and the swap
static lcs_status orbit_supported(const lcs_bound* H) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  if (!H->ks_swap || H->ks_swap->sym != 2)
    return fail(LCS_EUNSUPPORTED, "the orbit form needs sigma = d = 2, complement-symmetric storage and h >= 6");
  if (lcs_status st = wide_only(H, "the orbit form")) return st;
  return LCS_OK;
}

lcs_status lcs_bound_orbit_size(const lcs_bound_t* H, uint64_t* n_orbit) {
  if (lcs_status st = orbit_supported(H)) return st;
  if (!n_orbit) return fail(LCS_EINVAL, "NULL argument");
  *n_orbit = orbit_len(H->h);
  return LCS_OK;
}

lcs_status lcs_bound_set_start_orbit_fx(lcs_bound_t* H, const int64_t* const* v, int on_device) {
  if (lcs_status st = orbit_supported(H)) return st;
  if (!v) return fail(LCS_EINVAL, "NULL argument");
  for (int k = 0; k < H->d; ++k) {
    if (!v[k]) return fail(LCS_EINVAL, "start vector %d is NULL", k);
    if (on_device && ((uintptr_t)v[k] & 15)) return fail(LCS_EINVAL, "device vector %d is not 16-byte aligned", k);
  }
  const unsigned long long n_orb = orbit_len(H->h);
  LCS_CUDA(cudaMemsetAsync(H->dstate, 0, sizeof(DevState), H->stream));
  LCS_CUDA(cudaMemsetAsync(H->hist_count, 0, sizeof(unsigned long long), H->stream));
  if (on_device) {
    for (int k = 0; k < H->d; ++k) {
      launch_orbit_unpack(reinterpret_cast<const long long*>(v[k]), H->ring[H->d - 1 - k], H->h, H->n_tail,
                          H->dstate, H->stream);
      LCS_CUDA(cudaGetLastError());
      H->launches++;
    }
  } else {
    // Host vectors land in rows the unpacking does not write yet (n_orb =
    // 4^(h-1) + 2^h <= n_stored = 2 4^(h-1)): v[0] in row 0, which v[1] fills
    // later, and v[1] in row 2, which the start leaves free.  While v[0] is
    // unpacked into row 1, the copy stream already moves the first pieces of
    // v[1]; unpacking v[1] into row 0 follows on the stream.
    long long* scratch[2] = {H->ring[0], H->ring[2]};
    for (int k = 0; k < 2; ++k) {
      if (lcs_status st = h2d_copy(H, scratch[k], v[k], n_orb)) return st;
      cudaEvent_t a;
      if (lcs_status st = xfer_begin(H, H->stream, &a)) return st;
      launch_orbit_unpack(scratch[k], H->ring[1 - k], H->h, H->n_tail, H->dstate, H->stream);
      LCS_CUDA(cudaGetLastError());
      if (lcs_status st = xfer_end(H, H->stream, a, kXferKernel)) return st;
      H->launches++;
    }
  }
  return finish_start(H);  // symmetric by construction: swap_bad stays 0
}

lcs_status lcs_bound_export_orbit_fx(lcs_bound_t* H, int k, int64_t* dst, int on_device) {
  if (lcs_status st = orbit_supported(H)) return st;
  if (!dst) return fail(LCS_EINVAL, "NULL argument");
  if (k < -1 || k >= H->d) return fail(LCS_EINVAL, "k=%d outside -1..d-1", k);
  if (k == -1)
    if (lcs_status st = flush_pending(H)) return st;  // u is the kept iterate: its check must have run
  if (!H->swap_ok) return fail(LCS_EINVAL, "the iterates are not swap-symmetric (the start lacked the symmetry)");
  if (on_device && ((uintptr_t)dst & 15)) return fail(LCS_EINVAL, "device destination is not 16-byte aligned");
  const int rows = H->d + 1;
  const long long* src;
  if (k == -1) {
    if (!H->ubuf) return fail(LCS_EINVAL, "u is not retained (opts.keep_u = 0)");
    src = H->ubuf;
  } else {
    src = H->ring[(H->newest - k + rows) % rows];
  }
  const unsigned long long n_orb = orbit_len(H->h);
  if (on_device) {
    launch_orbit_pack(src, reinterpret_cast<long long*>(dst), H->h, H->n_tail, H->stream);
    LCS_CUDA(cudaGetLastError());
    H->launches++;
    return LCS_OK;
  }
  // host: pack into the row the next sweep overwrites (it holds v_{t-d}, which
  // no export and no later sweep reads), then copy out
  long long* scratch = H->ring[(H->newest + 1) % rows];
  launch_orbit_pack(src, scratch, H->h, H->n_tail, H->stream);
  LCS_CUDA(cudaGetLastError());
  H->launches++;
  if (lcs_status st = d2h_copy(H, dst, scratch, n_orb)) return st;
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  return LCS_OK;
}

lcs_status lcs_bound_history(lcs_bound_t* H, lcs_bound_check_record* out, int64_t max_records, int64_t* n_checks) {
  if (!H) return fail(LCS_EINVAL, "handle is NULL");
  if (H->batch) return fail(LCS_EINVAL, "batch handles keep no history");
  if (lcs_status st = flush_pending(H)) return st;
  if (max_records < 0 || (max_records > 0 && !out)) return fail(LCS_EINVAL, "bad output buffer");
  static_assert(sizeof(CheckRecord) == sizeof(lcs_bound_check_record), "record layouts differ");
  unsigned long long count = 0;
  LCS_CUDA(cudaMemcpyAsync(&count, H->hist_count, sizeof count, cudaMemcpyDeviceToHost, H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  if (n_checks) *n_checks = (int64_t)count;
  const unsigned long long kept = std::min<unsigned long long>(count, kHistCap);
  const unsigned long long n = std::min<unsigned long long>(kept, (unsigned long long)max_records);
  // the newest n records, oldest first: ring slots (count - n) .. (count - 1)
  for (unsigned long long i = 0; i < n;) {
    const unsigned long long slot = (count - n + i) % kHistCap;
    const unsigned long long run = std::min<unsigned long long>(n - i, kHistCap - slot);
    LCS_CUDA(cudaMemcpyAsync(out + i, H->hist + slot, run * sizeof(CheckRecord), cudaMemcpyDeviceToHost, H->stream));
    i += run;
  }
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  return LCS_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume

namespace {

struct CkptHeader {
  char magic[8];  // "LCSCKPT1"
  int32_t version;
  int32_t sigma, d, h;
  int32_t frac_bits, sym, f_mode, r_mode, check_every, keep_u;
  int32_t swap_ok;
  int32_t devstate_bytes;
  int64_t iters_done;
  uint64_t n_stored;
  double vbound;
};

constexpr char kCkptMagic[8] = {'L', 'C', 'S', 'C', 'K', 'P', 'T', '1'};
constexpr size_t kFileChunk = (size_t)8 << 20;  // int64 values per file transfer (64 MiB)

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};

}  // namespace

static lcs_status write_vector(lcs_bound* H, FILE* f, const long long* src, std::vector<long long>& buf) {
  for (unsigned long long off = 0; off < H->n_stored; off += kFileChunk) {
    const size_t len = (size_t)std::min<unsigned long long>(kFileChunk, H->n_stored - off);
    LCS_CUDA(cudaMemcpyAsync(buf.data(), src + off, len * 8, cudaMemcpyDeviceToHost, H->stream));
    LCS_CUDA(cudaStreamSynchronize(H->stream));
    if (fwrite(buf.data(), 8, len, f) != len) return fail(LCS_EIO, "checkpoint write failed");
  }
  return LCS_OK;
}

static lcs_status read_vector(lcs_bound* H, FILE* f, long long* dst, std::vector<long long>& buf) {
  for (unsigned long long off = 0; off < H->n_stored; off += kFileChunk) {
    const size_t len = (size_t)std::min<unsigned long long>(kFileChunk, H->n_stored - off);
    if (fread(buf.data(), 8, len, f) != len) return fail(LCS_EIO, "checkpoint file is truncated");
    LCS_CUDA(cudaMemcpyAsync(dst + off, buf.data(), len * 8, cudaMemcpyHostToDevice, H->stream));
    LCS_CUDA(cudaStreamSynchronize(H->stream));
  }
  return LCS_OK;
}

lcs_status lcs_bound_save(lcs_bound_t* H, const char* path) {
  if (lcs_status st = wide_only(H, "lcs_bound_save")) return st;
  if (H && !H->batch)
    if (lcs_status st = flush_pending(H)) return st;
  if (!H || !path) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "batch handles have no checkpoint");
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.sigma = H->sigma;
  hd.d = H->d;
  hd.h = H->h;
  hd.frac_bits = H->opts.frac_bits;
  hd.sym = H->sym;
  hd.f_mode = H->opts.f_mode;
  hd.r_mode = H->opts.r_mode;
  hd.check_every = H->opts.check_every;
  hd.keep_u = H->ubuf ? 1 : 0;
  hd.swap_ok = H->swap_ok ? 1 : 0;
  hd.devstate_bytes = (int32_t)sizeof(DevState);
  hd.iters_done = H->iters_done;
  hd.n_stored = H->n_stored;
  hd.vbound = H->vbound;
  DevState ds;
  LCS_CUDA(cudaMemcpyAsync(&ds, H->dstate, sizeof ds, cudaMemcpyDeviceToHost, H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  if (ds.status) return fail((lcs_status)ds.status, "device status %lld: nothing to save", (long long)ds.status);
  FileCloser fc{fopen(path, "wb")};
  if (!fc.f) return fail(LCS_EIO, "cannot open %s for writing", path);
  if (fwrite(&hd, sizeof hd, 1, fc.f) != 1 || fwrite(&ds, sizeof ds, 1, fc.f) != 1)
    return fail(LCS_EIO, "checkpoint write failed");
  std::vector<long long> buf((size_t)std::min<unsigned long long>(kFileChunk, H->n_stored));
  const int rows = H->d + 1;
  for (int k = 0; k < H->d; ++k) {  // newest first
    lcs_status st = write_vector(H, fc.f, H->ring[(H->newest - k + rows) % rows], buf);
    if (st) return st;
  }
  if (H->ubuf) {
    lcs_status st = write_vector(H, fc.f, H->ubuf, buf);
    if (st) return st;
  }
  if (fflush(fc.f) != 0) return fail(LCS_EIO, "checkpoint write failed");
  return LCS_OK;
}

lcs_status lcs_bound_restore(lcs_bound_t* H, const char* path) {
  if (lcs_status st = wide_only(H, "lcs_bound_restore")) return st;
  if (!H || !path) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "batch handles have no checkpoint");
  FileCloser fc{fopen(path, "rb")};
  if (!fc.f) return fail(LCS_EIO, "cannot open %s", path);
  CkptHeader hd;
  DevState ds;
  if (fread(&hd, sizeof hd, 1, fc.f) != 1) return fail(LCS_EIO, "checkpoint file is truncated");
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1)
    return fail(LCS_EINVAL, "%s is not a checkpoint of this library", path);
  if (hd.devstate_bytes != (int32_t)sizeof(DevState)) return fail(LCS_EINVAL, "checkpoint layout differs");
  if (hd.sigma != H->sigma || hd.d != H->d || hd.h != H->h)
    return fail(LCS_EINVAL, "checkpoint of shape (%d,%d,%d), handle (%d,%d,%d)", hd.sigma, hd.d, hd.h, H->sigma,
                H->d, H->h);
  if (hd.frac_bits != H->opts.frac_bits || hd.sym != H->sym || hd.f_mode != H->opts.f_mode ||
      hd.r_mode != H->opts.r_mode || hd.check_every != H->opts.check_every || hd.keep_u != (H->ubuf ? 1 : 0) ||
      hd.n_stored != H->n_stored)
    return fail(LCS_EINVAL, "checkpoint options differ from the handle's");
  if (fread(&ds, sizeof ds, 1, fc.f) != 1) return fail(LCS_EIO, "checkpoint file is truncated");
  std::vector<long long> buf((size_t)std::min<unsigned long long>(kFileChunk, H->n_stored));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  for (int k = 0; k < H->d; ++k) {
    lcs_status st = read_vector(H, fc.f, H->ring[H->d - 1 - k], buf);
    if (st) return st;
  }
  if (H->ubuf) {
    lcs_status st = read_vector(H, fc.f, H->ubuf, buf);
    if (st) return st;
  }
  LCS_CUDA(cudaMemcpyAsync(H->dstate, &ds, sizeof ds, cudaMemcpyHostToDevice, H->stream));
  LCS_CUDA(cudaMemsetAsync(H->hist_count, 0, sizeof(unsigned long long), H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  H->newest = H->d - 1;
  H->iters_done = hd.iters_done;
  H->pending_check = false;  // a saved handle has run all its checks
  H->vbound = hd.vbound;
  H->swap_ok = H->ks_swap != nullptr && hd.swap_ok;
  return LCS_OK;
}

static lcs_status export_impl(lcs_bound* H, int k, void* dst, int on_device, bool to_double) {
  if (!H || !dst) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  if (k < -1 || k >= H->d) return fail(LCS_EINVAL, "k=%d outside -1..d-1", k);
  if (k == -1)
    if (lcs_status st = flush_pending(H)) return st;  // u is the kept iterate: its check must have run
  const long long* src;
  int slot = 0;
  if (k == -1) {
    if (!H->ubuf) return fail(LCS_EINVAL, "u is not retained (opts.keep_u = 0)");
    src = H->ubuf;
  } else {
    const int rows = H->d + 1;
    slot = (H->newest - k + rows) % rows;
    src = H->ring[slot];
  }
  const double scale = std::ldexp(1.0, -H->opts.frac_bits);
  // one launch of the conversion for [off, off + len) of the states into `to`
  auto conv = [&](void* to, unsigned long long off, unsigned long long len) {
    const int grid = (int)std::min<unsigned long long>(4096, (len + kBlock - 1) / kBlock);
    if (H->narrow) {
      const int* w = reinterpret_cast<const int*>(src);
      if (to_double)
        export_kernel<true, int><<<grid, kBlock, 0, H->stream>>>(w, off, len, H->n_stored, H->n_total, scale, to,
                                                                 H->offs, slot);
      else
        export_kernel<false, int><<<grid, kBlock, 0, H->stream>>>(w, off, len, H->n_stored, H->n_total, scale, to,
                                                                  H->offs, slot);
    } else if (to_double) {
      export_kernel<true><<<grid, kBlock, 0, H->stream>>>(src, off, len, H->n_stored, H->n_total, scale, to);
    } else {
      export_kernel<false><<<grid, kBlock, 0, H->stream>>>(src, off, len, H->n_stored, H->n_total, scale, to);
    }
    LCS_CUDA(cudaGetLastError());
    H->launches++;
    return LCS_OK;
  };
  if (on_device) return conv(dst, 0, H->n_total);
  lcs_status st = d2h_pipelined(H, dst, H->n_total,
                                [&](long long* stage, unsigned long long off, unsigned long long len) {
                                  return conv(stage, off, len);
                                });
  if (st) return st;
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  return LCS_OK;
}

lcs_status lcs_bound_export(lcs_bound_t* H, int k, double* dst, int on_device) {
  return export_impl(H, k, dst, on_device, true);
}

lcs_status lcs_bound_export_fx(lcs_bound_t* H, int k, int64_t* dst, int on_device) {
  return export_impl(H, k, dst, on_device, false);
}

lcs_status lcs_bound_check_vector(lcs_bound_t* H, const int64_t* u_dev, int64_t R, int64_t* E_out) {
  if (lcs_status st = wide_only(H, "lcs_bound_check_vector")) return st;
  if (!H || !u_dev || !E_out) return fail(LCS_EINVAL, "NULL argument");
  if (H->batch) return fail(LCS_EINVAL, "a batch handle: use the lcs_bound_batch_* calls");
  lcs_status st = run_check(H, (const long long*)u_dev, false, R, 0, false, false);
  if (st) return st;
  std::vector<RedPartial> parts((size_t)H->last_check_grid);
  LCS_CUDA(cudaMemcpyAsync(parts.data(), H->partials, sizeof(RedPartial) * parts.size(), cudaMemcpyDeviceToHost,
                           H->stream));
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  long long E = 0;
  for (const auto& q : parts) E = std::max(E, q.v);
  *E_out = E;
  return LCS_OK;
}

lcs_status lcs_bound_stats(lcs_bound_t* H, lcs_bound_stats_t* out, int reset) {
  if (!H || !out) return fail(LCS_EINVAL, "NULL argument");
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  fold_events(H);
  out->sweep_launches = H->sweep_n;
  out->sweep_ms = H->sweep_ms;
  out->check_launches = H->check_n;
  out->check_ms = H->check_ms;
  out->kernel_launches = H->launches;
  out->sweep_bytes = H->sweep_bytes;
  out->check_bytes = H->check_bytes;
  out->h2d_ms = H->xfer_ms[kXferH2D];
  out->h2d_bytes = H->h2d_bytes;
  out->d2h_ms = H->xfer_ms[kXferD2H];
  out->d2h_bytes = H->d2h_bytes;
  out->xfer_kernel_ms = H->xfer_ms[kXferKernel];
  if (reset) {
    H->sweep_n = H->check_n = H->launches = 0;
    H->sweep_ms = H->check_ms = 0;
    H->sweep_bytes = H->check_bytes = 0;
    H->xfer_ms[0] = H->xfer_ms[1] = H->xfer_ms[2] = 0;
    H->h2d_bytes = H->d2h_bytes = 0;
  }
  return LCS_OK;
}

lcs_status lcs_bound_batch_create(int n, const int (*shapes)[3], const lcs_bound_opts* opts_in, lcs_bound_t** out) {
  if (!out || !shapes) return fail(LCS_EINVAL, "NULL argument");
  *out = nullptr;
  lcs_bound_opts opts;
  if (opts_in)
    opts = *opts_in;
  else
    lcs_bound_default_opts(&opts);
  if (opts.frac_bits == 0) opts.frac_bits = 44;
  if (opts.frac_bits < 8 || opts.frac_bits > 56) return fail(LCS_EINVAL, "frac_bits %d outside 8..56", opts.frac_bits);
  if (opts.r_mode != 0 && opts.r_mode != 1) return fail(LCS_EINVAL, "r_mode %d", opts.r_mode);
  if (opts.check_every < 0) return fail(LCS_EINVAL, "check_every %d", opts.check_every);
  if (opts.f_mode != 0) return fail(LCS_EUNSUPPORTED, "f_mode %d has no GPU kernel", opts.f_mode);
  if (opts.alloc && !opts.free) return fail(LCS_EINVAL, "alloc given without free");
  lcs_bound* H = new (std::nothrow) lcs_bound();
  if (!H) return fail(LCS_ENOMEM, "host allocation");
  H->opts = opts;
  H->one = 1ll << opts.frac_bits;
  H->d = 0;  // the handle owns no ring of its own
  cudaError_t e = cudaGetDevice(&H->device);
  if (e == cudaSuccess) {
    if (opts.stream) {
      H->stream = (cudaStream_t)opts.stream;
    } else {
      e = cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking);
      H->own_stream = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    lcs_bound_destroy(H);
    return fail(LCS_ECUDA, "batch stream: %s", cudaGetErrorString(e));
  }
  // headroom is checked against the largest sigma^d of the batch
  int worst_sigma = 2, worst_d = 2;
  double worst = 0;
  for (int i = 0; i < n && i < kMaxBatch; ++i) {
    const double sd = std::pow((double)shapes[i][0], (double)shapes[i][1]);
    if (sd > worst) worst = sd, worst_sigma = shapes[i][0], worst_d = shapes[i][1];
  }
  H->sigma = worst_sigma;
  H->d_batch_worst = worst_d;
  lcs_status st = batch_create(n, shapes, opts, H->stream, &H->batch);
  if (st) {
    lcs_bound_destroy(H);
    return st;
  }
  *out = H;
  return LCS_OK;
}

lcs_status lcs_bound_batch_report(lcs_bound_t* H, int i, lcs_bound_report* out) {
  if (!H || !out) return fail(LCS_EINVAL, "NULL argument");
  if (!H->batch) return fail(LCS_EINVAL, "not a batch handle");
  return batch_report(H->batch, H->stream, i, out);
}

lcs_status lcs_bound_batch_read(lcs_bound_t* H, int i, double* bound_rd, uint64_t* argmin_state, double* r,
                                double* eps, int64_t* at_iter) {
  lcs_bound_report rep;
  lcs_status st = lcs_bound_batch_report(H, i, &rep);
  if (st) return st;
  if (rep.status) return fail((lcs_status)rep.status, "device status %d", rep.status);
  if (!rep.have_check) return fail(LCS_ENOBOUND, "no feasibility check has run");
  const int K = H->opts.frac_bits;
  const long long B = (long long)batch_d(H->batch, i) * (rep.r - rep.eps);
  if (bound_rd) *bound_rd = fx_to_double_rd(B, K);
  if (argmin_state) *argmin_state = rep.argmin;
  if (r) *r = std::ldexp((double)rep.r, -K);
  if (eps) *eps = std::ldexp((double)rep.eps, -K);
  if (at_iter) *at_iter = rep.kept_iter;
  return LCS_OK;
}

lcs_status lcs_bound_batch_export_fx(lcs_bound_t* H, int i, int k, int64_t* dst, int on_device) {
  if (!H || !dst) return fail(LCS_EINVAL, "NULL argument");
  if (!H->batch) return fail(LCS_EINVAL, "not a batch handle");
  unsigned long long n_stored = 0, n_total = 0;
  lcs_status st = LCS_OK;
  const long long* src = batch_vector(H->batch, H->stream, i, k, &n_stored, &n_total, &st);
  if (!src) return st;
  if (on_device) {
    const int grid = (int)std::min<unsigned long long>(4096, (n_total + kBlock - 1) / kBlock);
    export_kernel<false><<<grid, kBlock, 0, H->stream>>>(src, 0, n_total, n_stored, n_total, 1.0, dst);
    LCS_CUDA(cudaGetLastError());
    return LCS_OK;
  }
  st = d2h_pipelined(H, dst, n_total, [&](long long* stage, unsigned long long off, unsigned long long len) {
    const int grid = (int)std::min<unsigned long long>(4096, (len + kBlock - 1) / kBlock);
    export_kernel<false><<<grid, kBlock, 0, H->stream>>>(src, off, len, n_stored, n_total, 1.0, stage);
    LCS_CUDA(cudaGetLastError());
    return LCS_OK;
  });
  if (st) return st;
  LCS_CUDA(cudaStreamSynchronize(H->stream));
  return LCS_OK;
}

lcs_status lcs_bound_batch_info(lcs_bound_t* H, lcs_bound_batch_info_t* out) {
  if (!H || !out) return fail(LCS_EINVAL, "NULL argument");
  if (!H->batch) return fail(LCS_EINVAL, "not a batch handle");
  long long launches = 0, replays = 0;
  batch_tuning(H->batch, &out->grid, &out->units_per_item, &out->tuned_ms_per_iter, &launches, &out->graph,
               &out->mode, &out->persistent_ms_per_iter, &out->concurrent_ms_per_iter, &out->graph_captured, &replays,
               &out->min_ctas_per_sm);
  out->launches = launches;
  out->graph_replays = replays;
  out->n_instances = batch_size(H->batch);
  return LCS_OK;
}

lcs_status lcs_bound_batch_set_mode(lcs_bound_t* H, int mode) {
  if (!H) return fail(LCS_EINVAL, "NULL argument");
  if (!H->batch) return fail(LCS_EINVAL, "not a batch handle");
  if (mode < 0 || mode > 2)
    return fail(LCS_EINVAL, "mode %d (0 persistent, 1 concurrent, 2 concurrent without graph capture)", mode);
  if (H->iters_done != 0) return fail(LCS_EINVAL, "the mode can only be set before the first iteration");
  return batch_set_mode(H->batch, H->stream, mode);
}

lcs_status lcs_bound_batch_set_spin_budget(lcs_bound_t* H, int64_t cycles) {
  if (!H) return fail(LCS_EINVAL, "NULL argument");
  if (!H->batch) return fail(LCS_EINVAL, "not a batch handle");
  if (cycles < 0) return fail(LCS_EINVAL, "negative budget");
  return batch_set_spin_budget(H->batch, H->stream, cycles);
}

lcs_status lcs_sweep_fx(int sigma, int d, int h, int f_mode, int frac_bits, const int64_t* const* v_prev,
                        int64_t* v_out, void* stream) {
  if (sigma < 2 || d < 2 || h < 1 || d > kMaxD) return fail(LCS_EINVAL, "bad shape");
  if (f_mode != 0 && f_mode != 1) return fail(LCS_EINVAL, "f_mode %d", f_mode);
  if (frac_bits == 0) frac_bits = 44;
  if (frac_bits < 8 || frac_bits > 56) return fail(LCS_EINVAL, "frac_bits");
  if (!v_prev || !v_out) return fail(LCS_EINVAL, "NULL argument");
  unsigned long long n = 1, sd = 1;
  for (int i = 0; i < d * h; ++i) {
    n *= (unsigned long long)sigma;
    if (n >= (1ull << 40)) return fail(LCS_EINVAL, "sigma^(d h) must be below 2^40");
  }
  for (int i = 0; i < d; ++i) sd *= (unsigned long long)sigma;
  const KernelSet* ks = find_kernels(sigma, d, 0, f_mode);
  if (!ks && f_mode == 0) ks = kernels_rt(sigma);
  if (!ks) return fail(LCS_EUNSUPPORTED, "no kernel for sigma=%d d=%d f_mode=%d", sigma, d, f_mode);
  SweepParams p{};
  for (int k = 0; k < d; ++k) {
    if (!v_prev[k]) return fail(LCS_EINVAL, "v_prev[%d] is NULL", k);
    const uintptr_t a = (uintptr_t)v_prev[k], b = (uintptr_t)v_out;
    if (a < b + 8 * n && b < a + 8 * n) return fail(LCS_EINVAL, "v_out overlaps v_prev[%d]", k);
    p.prev[k] = (const long long*)v_prev[k];
  }
  p.out = (long long*)v_out;
  p.n_tail = n / sd;
  p.n_stored = n;
  p.h = h;
  p.incr = 0;
  p.one = 1ll << frac_bits;
  int dev = 0, sms = 1;
  LCS_CUDA(cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid =
      grid_for(ks->sweep_fn, std::max(sms, 1), ks->tails_per_thread == 0 ? rt_work_items(sigma, d, n, p.n_tail, false) : p.n_tail);
  ks->sweep(p, grid, (cudaStream_t)stream);
  LCS_CUDA(cudaGetLastError());
  return LCS_OK;
}

}  // extern "C"
