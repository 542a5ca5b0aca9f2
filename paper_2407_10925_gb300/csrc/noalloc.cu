// noalloc.cu -- an entry point that allocates no device memory.
//
// Who needs it: code that must not call cudaMalloc or any allocating library
// routine after start-up -- for example a caller running inside a memory pool
// it does not own, a plugin whose host forbids device allocations, or a
// process that has already handed every free byte of HBM to other buffers.
// Such a caller can still pass its own input and output vectors, but it
// cannot provide the per-CTA scratch that the fused increment reduction
// needs.  This file keeps that scratch in a fixed array that is part of the
// library image: it is reserved when the library is loaded onto a device and
// stays reserved, on every device that loads the library, until the process
// exits.
//
// The entry point runs the same sweep kernel as the library's handle (one
// evaluation of F fused with the min/argmin of the increment) and then a
// small kernel that reduces the per-CTA partials into caller-owned outputs.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdint>

#include "../../include/lcs_bound.h"
#include "lcs_common.h"

namespace lcs {

// Capacity of the static scratch: one 16-byte partial per CTA of the sweep.
// 4096 CTAs = 64 KiB; a GB300 (152 SMs) launches at most 152 x 8 = 1216.
constexpr int kNoAllocMaxPartials = 4096;

// The scratch itself.  In host code this name is only a stand-in for the
// device object, never a device address; host code obtains the address with
// cudaGetSymbolAddress (see noalloc_setup) and passes it to the kernels.
static __device__ __align__(256) RedPartial g_noalloc_partials[kNoAllocMaxPartials];

// defined in lcs_bound.cu: the message lcs_bound_last_error() returns
void record_error(const char* msg);

static lcs_status noalloc_fail(lcs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  record_error(buf);
  return st;
}

// With the calling thread's device current: the scratch's device address and
// the device's SM count.  The address is looked up on every call
// (cudaGetSymbolAddress allocates nothing): a cached one would go stale when
// the device's context is re-created (cudaDeviceReset), which reloads the
// library's device code and may move the array.  The first lookup on a device
// loads that device code.
static lcs_status noalloc_setup(int dev, RedPartial** ptr, int* sms) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess)
    return noalloc_fail(LCS_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
  int n = 0;
  e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(LCS_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
  *ptr = static_cast<RedPartial*>(p);
  *sms = n > 0 ? n : 1;
  return LCS_OK;
}

// [a, a + na) and [b, b + nb) share a byte
static bool overlaps(const void* a, unsigned long long na, const void* b, unsigned long long nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

// Reduce the sweep's per-CTA partials (min, or max with r_mode = 1, ties to
// the smallest state index) into the caller's outputs.  Every slot it reads
// was written by the sweep of the same call: nothing is carried over.
__global__ void __launch_bounds__(kFinalBlock) noalloc_finalize_kernel(const RedPartial* parts, int n, int r_mode,
                                                                        long long* R_out,
                                                                        unsigned long long* argmin_out) {
  long long v = r_mode ? LLONG_MIN : LLONG_MAX;
  unsigned long long x = ULLONG_MAX;
  auto better = [r_mode](long long a, unsigned long long ax, long long b, unsigned long long bx) {
    if (a != b) return r_mode ? (a > b) : (a < b);
    return ax < bx;
  };
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (better(parts[i].v, parts[i].x, v, x)) v = parts[i].v, x = parts[i].x;
  __shared__ long long sv[kFinalBlock / 32];
  __shared__ unsigned long long sx[kFinalBlock / 32];
  for (int o = 16; o > 0; o >>= 1) {
    long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    unsigned long long ox = __shfl_xor_sync(0xffffffffu, x, o);
    if (better(ov, ox, v, x)) v = ov, x = ox;
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
      if (better(ov, ox, v, x)) v = ov, x = ox;
    }
    if (threadIdx.x == 0) {
      *R_out = v;
      *argmin_out = x;
    }
  }
}

}  // namespace lcs

using namespace lcs;

extern "C" lcs_status lcs_sweep_incr_fx_noalloc(int sigma, int d, int h, int frac_bits, int r_mode,
                                                const int64_t* const* v_prev, int64_t* v_out, int64_t* R_out,
                                                uint64_t* argmin_out, void* stream) {
  if (sigma < 2 || d < 2 || h < 1 || d > kMaxD)
    return noalloc_fail(LCS_EINVAL, "bad shape sigma=%d d=%d h=%d", sigma, d, h);
  if (frac_bits == 0) frac_bits = 44;
  if (frac_bits < 8 || frac_bits > 56) return noalloc_fail(LCS_EINVAL, "frac_bits %d outside 8..56", frac_bits);
  if (r_mode != 0 && r_mode != 1) return noalloc_fail(LCS_EINVAL, "r_mode %d", r_mode);
  if (!v_prev || !v_out || !R_out || !argmin_out) return noalloc_fail(LCS_EINVAL, "NULL argument");
  unsigned long long n = 1, sd = 1;
  for (int i = 0; i < d * h; ++i) {
    n *= (unsigned long long)sigma;
    if (n >= (1ull << 40)) return noalloc_fail(LCS_EINVAL, "sigma^(d h) must be below 2^40");
  }
  for (int i = 0; i < d; ++i) sd *= (unsigned long long)sigma;
  const KernelSet* ks = find_kernels(sigma, d, 0);
  if (!ks) return noalloc_fail(LCS_EUNSUPPORTED, "no kernel for sigma=%d d=%d", sigma, d);
  // the output vector and the two 8-byte results must not share a byte with
  // any input or with each other (the inputs may share bytes: they are read only)
  SweepParams p{};
  const unsigned long long bytes = 8ull * n;
  for (int k = 0; k < d; ++k) {
    if (!v_prev[k]) return noalloc_fail(LCS_EINVAL, "v_prev[%d] is NULL", k);
    if (overlaps(v_prev[k], bytes, v_out, bytes)) return noalloc_fail(LCS_EINVAL, "v_out overlaps v_prev[%d]", k);
    if (overlaps(v_prev[k], bytes, R_out, 8)) return noalloc_fail(LCS_EINVAL, "R_out lies inside v_prev[%d]", k);
    if (overlaps(v_prev[k], bytes, argmin_out, 8))
      return noalloc_fail(LCS_EINVAL, "argmin_out lies inside v_prev[%d]", k);
    p.prev[k] = (const long long*)v_prev[k];
  }
  if (overlaps(v_out, bytes, R_out, 8)) return noalloc_fail(LCS_EINVAL, "R_out lies inside v_out");
  if (overlaps(v_out, bytes, argmin_out, 8)) return noalloc_fail(LCS_EINVAL, "argmin_out lies inside v_out");
  if (overlaps(R_out, 8, argmin_out, 8)) return noalloc_fail(LCS_EINVAL, "R_out and argmin_out overlap");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(LCS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  RedPartial* scratch = nullptr;
  int sms = 1;
  lcs_status st = noalloc_setup(dev, &scratch, &sms);
  if (st) return st;

  // the same launch shape as the handle: a persistent grid, capped by the work
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks->sweep_fn, kBlock, 0);
  if (e != cudaSuccess) return noalloc_fail(LCS_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
  const unsigned long long n_tail = n / sd;
  const unsigned long long need = std::max(1ull, (n_tail + kBlock - 1) / kBlock);
  const unsigned long long grid = std::min((unsigned long long)sms * (unsigned long long)std::max(per_sm, 1), need);
  if (grid > (unsigned long long)kNoAllocMaxPartials)
    return noalloc_fail(LCS_EINVAL,
                        "the sweep needs %llu CTA partials but the static scratch holds %d (64 KiB); "
                        "use the handle API, which allocates its scratch",
                        grid, kNoAllocMaxPartials);
  p.out = (long long*)v_out;
  p.n_tail = n_tail;
  p.n_stored = n;
  p.h = h;
  p.incr = 1;
  p.r_mode = r_mode;
  p.one = 1ll << frac_bits;
  p.partials = scratch;
  cudaStream_t s = (cudaStream_t)stream;
  ks->sweep(p, (int)grid, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(LCS_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
  noalloc_finalize_kernel<<<1, kFinalBlock, 0, s>>>(scratch, (int)grid, r_mode, (long long*)R_out,
                                                    (unsigned long long*)argmin_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(LCS_ECUDA, "finalize launch: %s", cudaGetErrorString(e));
  return LCS_OK;
}
