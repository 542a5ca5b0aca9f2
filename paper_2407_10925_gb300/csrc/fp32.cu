// fp32.cu -- experiment: iterates stored in 32-bit floats, offset-normalised.
//
// The library's iterates are exact int64 fixed point (8 bytes per state).
// This experiment stores w_t = v_t - t rho in float32 (4 bytes per state) and
// evaluates F in float32.  Because F is translation invariant (Lemma 1),
//   v_t = b + max_z mean(v_{t-k_z} over the advanced tuples)     (Eq. ineq3)
// becomes
//   w_t = b + max_z ( mean(w_{t-k_z}) - k_z rho ),   k_z = |N_z|,
// so the stored values stay near the spread of the iterate instead of growing
// by r per iteration.  rho is a guess of r (any value is exact in the
// mathematics; a good guess keeps w small).  Means are taken in float32 with
// the sum in Algorithm 1's loop order and a multiplication by 1 / sigma^k.
// No bound is reported from these iterates: float rounding is not directed,
// so only their error against the exact fixed-point iterates is measured.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../../include/lcs_bound.h"
#include "lcs_common.h"
#include "sweep_generic.cuh"

namespace lcs {

void record_error(const char* msg);

static lcs_status ffail(lcs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  record_error(buf);
  return st;
}

#define F_CUDA(call)                                                                                      \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return ffail(LCS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                        __FILE__, __LINE__);                                              \
  } while (0)

struct F32Params {
  const float* prev[kMaxD];
  float* out;
  unsigned long long n_tail;
  int h;
  float rho;
};

template <int SIG, int D, unsigned N, int Z>
__device__ __forceinline__ float f32_partial(const float* const* prev, const unsigned long long (&S)[D],
                                             unsigned long long n_tail) {
  using G = Geo<SIG, D>;
  constexpr int K = cpopc(N);
  const float* v = prev[K - 1];
  unsigned long long base = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (N >> j & 1u)
      base += S[j] * G::SD;
    else
      base += S[j] + (unsigned long long)Z * n_tail * G::wlast(j);
  }
  float acc = 0.f;
  static_for<0, (int)cpow(SIG, K)>([&](auto cc) {
    constexpr unsigned long long off = G::coff(N, decltype(cc)::value);
    acc += __ldg(v + base + off);
  });
  return acc;
}

template <int SIG, int D>
__global__ void __launch_bounds__(kBlock) f32_sweep_kernel(F32Params p) {
  using G = Geo<SIG, D>;
  const unsigned long long nt = p.n_tail;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long S[D];
    tail_fields<SIG, D>(t, p.h, S);
    float s_all = 0.f;
    {
      const float* vd = p.prev[D - 1];
      const unsigned long long b = t * G::SD;
      static_for<0, (int)G::SD>([&](auto c) { s_all += __ldg(vd + b + decltype(c)::value); });
    }
    float P[G::NP > 0 ? G::NP : 1];
    static_for<0, G::NP>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      P[i] = f32_partial<SIG, D, (unsigned)(i / SIG) + 1, i % SIG>(p.prev, S, nt);
    });
    static_for<0, (int)G::SD>([&](auto Hc) {
      constexpr int H = decltype(Hc)::value;
      float val;
      if constexpr (G::all_equal(H)) {
        val = 1.0f + (s_all * (1.0f / (float)G::SD) - (float)D * p.rho);
      } else {
        float best = -INFINITY;
        static_for<0, SIG>([&](auto zc) {
          constexpr int z = decltype(zc)::value;
          constexpr unsigned N = G::nz(H, z);
          float cand;
          if constexpr (N == G::FULL) {
            cand = s_all * (1.0f / (float)G::SD) - (float)D * p.rho;
          } else {
            constexpr int K = cpopc(N);
            cand = P[(int)(N - 1) * SIG + z] * (1.0f / (float)cpow(SIG, K)) - (float)K * p.rho;
          }
          best = fmaxf(best, cand);
        });
        val = best;
      }
      p.out[(unsigned long long)H * nt + t] = val;
    });
  }
}

__global__ void f32_init_kernel(float* v, unsigned long long n, float value) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    v[i] = value;
}

__global__ void f32_export_kernel(const float* __restrict__ w, unsigned long long n, double shift,
                                  double* __restrict__ out) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    out[i] = (double)w[i] + shift;
}

template <int SIG, int D>
static void launch_f32(const F32Params& p, int grid, cudaStream_t s) {
  f32_sweep_kernel<SIG, D><<<grid, kBlock, 0, s>>>(p);
}

}  // namespace lcs

using namespace lcs;

extern "C" lcs_status lcs_fp32_experiment(int sigma, int d, int h, int64_t n_iters, double rho, double* newest_dev,
                                          double* ms_per_sweep) {
  void (*launch)(const F32Params&, int, cudaStream_t) = nullptr;
  const void* fn = nullptr;
  if (sigma == 2 && d == 2) launch = &launch_f32<2, 2>, fn = (const void*)&f32_sweep_kernel<2, 2>;
  if (sigma == 2 && d == 3) launch = &launch_f32<2, 3>, fn = (const void*)&f32_sweep_kernel<2, 3>;
  if (sigma == 3 && d == 2) launch = &launch_f32<3, 2>, fn = (const void*)&f32_sweep_kernel<3, 2>;
  if (!launch) return ffail(LCS_EUNSUPPORTED, "no float32 kernel for sigma=%d d=%d", sigma, d);
  if (h < 1 || n_iters < 0 || !newest_dev) return ffail(LCS_EINVAL, "bad argument");
  unsigned long long n = 1, sd = 1;
  for (int i = 0; i < d * h; ++i) {
    n *= (unsigned long long)sigma;
    if (n >= (1ull << 36)) return ffail(LCS_EINVAL, "too many states");
  }
  for (int i = 0; i < d; ++i) sd *= (unsigned long long)sigma;
  float* ring[kMaxD + 1] = {};
  const int rows = d + 1;
  for (int k = 0; k < rows; ++k) {
    if (cudaMalloc(&ring[k], n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < k; ++j) cudaFree(ring[j]);
      return ffail(LCS_ENOMEM, "float32 vector");
    }
  }
  lcs_status st = LCS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  do {
    // zero start: v_k = 0 for k < d, i.e. w_k = -k rho
    for (int k = 0; k < d; ++k) f32_init_kernel<<<1024, 256>>>(ring[k], n, (float)(-k * rho));
    int per_sm = 0, dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0);
    const int grid = (int)std::min<unsigned long long>((unsigned long long)sms * std::max(per_sm, 1),
                                                       (n / sd + kBlock - 1) / kBlock);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      st = ffail(LCS_ECUDA, "events");
      break;
    }
    int newest = d - 1;
    cudaEventRecord(e0);
    for (int64_t it = 0; it < n_iters; ++it) {
      F32Params p{};
      for (int k = 1; k <= d; ++k) p.prev[k - 1] = ring[(newest - (k - 1) + rows) % rows];
      newest = (newest + 1) % rows;
      p.out = ring[newest];
      p.n_tail = n / sd;
      p.h = h;
      p.rho = (float)rho;
      launch(p, grid, nullptr);
    }
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      st = ffail(LCS_ECUDA, "float32 sweep: %s", cudaGetErrorString(e));
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_per_sweep) *ms_per_sweep = n_iters > 0 ? ms / (double)n_iters : 0.0;
    // the newest stored iterate is v_{d-1+n_iters} - (d-1+n_iters) rho
    f32_export_kernel<<<1024, 256>>>(ring[newest], n, (double)(d - 1 + n_iters) * rho, newest_dev);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = ffail(LCS_ECUDA, "float32 export: %s", cudaGetErrorString(e));
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int k = 0; k < rows; ++k) cudaFree(ring[k]);
  return st;
}
