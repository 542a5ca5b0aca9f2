// mlp_net.h -- shape, parameter layout and features of the warm-start network
// (shared by the training kernels and the tensor-core inference kernel).
// The network is not part of the paper's method; see mlp.cu.
#pragma once

#include <cuda_runtime.h>

namespace lcs {

constexpr int kHin = 12;                 // encoded positions per string
constexpr int kFeat = 4 * kHin + 1;      // 49
constexpr int kHid = 256;
constexpr long long kOffW1 = 0;
constexpr long long kOffB1 = kOffW1 + (long long)kHid * kFeat;
constexpr long long kOffW2 = kOffB1 + kHid;
constexpr long long kOffB2 = kOffW2 + (long long)kHid * kHid;
constexpr long long kOffW3 = kOffB2 + kHid;
constexpr long long kOffB3 = kOffW3 + kHid;
constexpr long long kNParams = kOffB3 + 1;

// ---------------------------------------------------------------------------
// features

__host__ __device__ inline unsigned long long mlp_canonical(unsigned long long x, int h) {
  const unsigned long long n1 = (h >= 32) ? ~0ull : ((1ull << (2 * h)) - 1);
  const unsigned long long c = n1 - x;
  const unsigned long long w = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
  const unsigned long long wc = n1 - w;
  unsigned long long m = x < c ? x : c;
  m = m < w ? m : w;
  return m < wc ? m : wc;
}

// indices of the active one-hot features (2 per encoded position)
__device__ __forceinline__ int mlp_active(unsigned long long x, int h, int* idx) {
  x = mlp_canonical(x, h);
  const int np = h < kHin ? h : kHin;
  for (int p = 0; p < np; ++p) {
    const unsigned pair = (unsigned)((x >> (2 * (h - 1 - p))) & 3ull);
    idx[2 * p] = 4 * p + (int)(pair >> 1);
    idx[2 * p + 1] = 4 * p + 2 + (int)(pair & 1u);
  }
  return 2 * np;
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

}  // namespace lcs
