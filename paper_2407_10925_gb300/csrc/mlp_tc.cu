// mlp_tc.cu -- BF16 inference of the warm-start network on the tensor cores
// (tcgen05, accumulators in tensor memory), one fused kernel per prediction
// table.
//
// Which rows.  The network sees a state only through the first np = min(h, 12)
// positions of its canonical form (and h).  The canonical form c, the
// smallest index of the orbit under complement and string swap, is below
// 4^h / 2 (c and its complement sum to 4^h - 1), so the first letter of
// string 0 is 0 and the prefix q = c >> 2 (h - np) is below 2^(2 np - 1).
// The kernel evaluates the network once per prefix into a table T[q]; a
// gather then writes a full-length vector by looking T up at each state's
// canonical prefix.  For h >= 12 the table has 2^23 rows whatever h is, of
// which about half can be canonical prefixes: tiles with none are skipped.
//
// One CTA per SM, persistent over tiles of 128 rows; 256 threads:
//   layer 1 (SIMT, fp32): thread j holds the 48 one-hot weights of hidden
//     unit j in registers and adds the selected ones in feature order (the
//     same sum the FP32 path forms; the part shared by a tile's rows once per
//     tile), applies GELU and stores the activation,
//     rounded to bf16, in shared memory in the no-swizzle K-major core-matrix
//     layout the tensor core reads (8 x 8 bf16 blocks of 128 contiguous bytes,
//     32 blocks per 8-row group);
//   layer 2 (tensor cores): 16 tcgen05.mma of M = 128, N = 256, K = 16,
//     A = the activations, B = W2 in bf16 (staged once per CTA, 128 KB),
//     fp32 accumulators in 256 columns of tensor memory, completion signalled
//     through an mbarrier by tcgen05.commit;
//   head (SIMT): warp w reads lanes 32 (w mod 4) .. +31 (one accumulator row
//     per thread) and columns 128 (w div 4) .. +127 with tcgen05.ld, adds b2,
//     applies GELU and dots with w3; the two half sums of a row meet in
//     shared memory and b3 is added.
// Every wait is bounded: if the mbarrier does not complete within the spin
// budget the kernel records an error, waits once more (bounded) for the
// tensor core, frees its tensor memory and returns.
#include <cstdint>

#include <cuda_bf16.h>

#include "../../include/lcs_bound.h"
#include "mlp_net.h"

namespace lcs {

namespace {

constexpr int kTileRows = 128;
constexpr int kTcThreads = 256;
constexpr uint32_t kW2Bytes = kHid * kHid * 2;         // 131072
constexpr uint32_t kABytes = kTileRows * kHid * 2;     // 65536
constexpr uint32_t kOffA = kW2Bytes;
constexpr uint32_t kOffVec = kOffA + kABytes;          // b2, w3, partial sums: 3 x 1 KB
constexpr uint32_t kOffBar = kOffVec + 3 * 1024;
constexpr uint32_t kTcSmem = kOffBar + 16;
constexpr uint32_t kTmemCols = 256;

// byte offset of element (row r, column k) in the core-matrix layout:
// 8 x 8 blocks of 128 bytes, row-major inside a block, 32 blocks along k per 8-row group
__host__ __device__ __forceinline__ uint32_t cm_off(int r, int k) {
  return ((uint32_t)(((r >> 3) << 5) + (k >> 3)) << 7) + ((uint32_t)(r & 7) << 4) + ((uint32_t)(k & 7) << 1);
}

// shared-memory matrix descriptor, no swizzle: leading (k) offset 128 B between
// adjacent blocks along k, stride offset 4096 B between 8-row groups,
// descriptor version 1 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(4096u >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}"
      :
      : "r"(d_tmem), "l"(a), "l"(b), "r"(accumulate), "r"(kIdesc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive fp32 columns of this thread's lane, waited for in the same statement
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// bounded wait on an mbarrier phase; false when the budget (in clock cycles) runs out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

// GELU(x) = x Phi(x) with Phi(x) = (1 + erf(x / sqrt 2)) / 2 and erf from
// Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7 for y >= 0):
//   erfc(y) ~ (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-y^2),  t = 1 / (1 + p y).
// Phi(-|x|) = erfc(|x| / sqrt 2) / 2 is formed directly (no cancellation for
// x << 0) and Phi(|x|) = 1 - Phi(-|x|).  The absolute error of the GELU is at
// most 1e-7 |x|, far below the bf16 rounding that follows it.
__device__ __forceinline__ float gelu_as(float x) {
  const float y = fabsf(x) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, y, 1.0f));
  const float poly =
      t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
  const float lower = 0.5f * poly * __expf(-y * y);  // Phi(-|x|)
  return x * (x >= 0.0f ? 1.0f - lower : lower);
}

struct TcParams {
  const float* P;       // FP32 parameters
  const uint4* w2c;     // W2 in bf16, core-matrix layout (kW2Bytes)
  float* table;         // rows predictions
  long long rows;
  int h;
  int np;               // encoded positions, min(h, 12)
  int* err;             // set to 1 when a wait ran out
  long long spin_budget;
};

__global__ void __launch_bounds__(kTcThreads, 1) mlp_table_tc_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sW2 = smem;
  unsigned char* sA = smem + kOffA;
  float* sb2 = reinterpret_cast<float*>(smem + kOffVec);
  float* sw3 = sb2 + kHid;
  float* spart = sw3 + kHid;  // [2][128]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + kOffBar);
  uint32_t* stmem = reinterpret_cast<uint32_t*>(smem + kOffBar + 8);
  int* sabort = reinterpret_cast<int*>(smem + kOffBar + 12);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < (int)(kW2Bytes / 16); i += kTcThreads) reinterpret_cast<uint4*>(sW2)[i] = p.w2c[i];
  sb2[tid] = p.P[kOffB2 + tid];
  sw3[tid] = p.P[kOffW3 + tid];
  const float b3 = p.P[kOffB3];

  // layer-1 weights of hidden unit tid: w[p][0..1] string 0 letter 0/1, w[p][2..3] string 1
  const float* W1 = p.P + kOffW1 + (long long)tid * kFeat;
  float w[kHin][4];
#pragma unroll
  for (int q = 0; q < kHin; ++q)
#pragma unroll
    for (int c = 0; c < 4; ++c) w[q][c] = q < p.np ? W1[4 * q + c] : 0.0f;
  const float z0 = p.P[kOffB1 + tid] + (float)p.h * (1.0f / 16.0f) * W1[kFeat - 1];

  const uint32_t bar_a = smem_u32(bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_a), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *sabort = 0;
  }
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(stmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W2 visible to the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *stmem;

  const int shift = 2 * (kHin - p.np);  // the prefix, left-aligned to 12 positions
  const long long n_tiles = (p.rows + kTileRows - 1) / kTileRows;
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sW2);
  uint32_t parity = 0;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (p.np == kHin) {
      // A canonical form c is at most its swap and its complemented swap, so
      // its prefix q is at most theirs; the 128 rows of a tile share positions
      // 0..7 (the top 16 bits X of q), and when X already exceeds the swap or
      // the complemented swap of X, no row of the tile is a canonical prefix:
      // the gather never reads it, and the tile is skipped (about half of them).
      const uint32_t X = (uint32_t)(tile * kTileRows) >> 8;
      const uint32_t sw = ((X >> 1) & 0x5555u) | ((X & 0x5555u) << 1);
      if (X > sw || X > 0xFFFFu - sw) continue;
    }
    // ---- layer 1 into shared memory (bf16); the sum runs over the features in
    // order, position 0 first, as in the FP32 path
    if (p.np == kHin) {
      // the 128 rows of a tile share positions 0..7 and the first letter of
      // position 8: that part of the sum is formed once per tile
      const uint32_t q0 = (uint32_t)(tile * kTileRows);
      float zf = z0;
#pragma unroll
      for (int pp = 0; pp < 8; ++pp) {
        const uint32_t pair = (q0 >> (2 * (kHin - 1 - pp))) & 3u;
        zf += (pair & 2u) ? w[pp][1] : w[pp][0];
        zf += (pair & 1u) ? w[pp][3] : w[pp][2];
      }
      zf += (q0 & 128u) ? w[8][1] : w[8][0];
      // row r = (b8, pair 9, pair 10, pair 11) in bits 6, 5..4, 3..2, 1..0:
      // the loops are unrolled, so every weight is chosen at compile time and
      // rows that share a prefix share its partial sum (the same additions,
      // in the same order, as one running sum per row)
      unsigned char* const a_col = sA + cm_off(0, tid);
#pragma unroll
      for (int b8 = 0; b8 < 2; ++b8) {
        const float z8 = zf + w[8][2 + b8];
#pragma unroll
        for (int p9 = 0; p9 < 4; ++p9) {
          const float z9 = (z8 + w[9][p9 >> 1]) + w[9][2 + (p9 & 1)];
#pragma unroll
          for (int p10 = 0; p10 < 4; ++p10) {
            const float z10 = (z9 + w[10][p10 >> 1]) + w[10][2 + (p10 & 1)];
#pragma unroll
            for (int p11 = 0; p11 < 4; ++p11) {
              const float z = (z10 + w[11][p11 >> 1]) + w[11][2 + (p11 & 1)];
              const int r = (b8 << 6) | (p9 << 4) | (p10 << 2) | p11;
              *reinterpret_cast<__nv_bfloat16*>(a_col + cm_off(r, 0)) = __float2bfloat16_rn(gelu_as(z));
            }
          }
        }
      }
    } else {
      for (int r = 0; r < kTileRows; ++r) {
        const uint32_t q = (uint32_t)(tile * kTileRows + r) << shift;
        float z = z0;
#pragma unroll
        for (int pp = 0; pp < kHin; ++pp) {
          const uint32_t pair = (q >> (2 * (kHin - 1 - pp))) & 3u;
          z += (pair & 2u) ? w[pp][1] : w[pp][0];
          z += (pair & 1u) ? w[pp][3] : w[pp][2];
        }
        *reinterpret_cast<__nv_bfloat16*>(sA + cm_off(r, tid)) = __float2bfloat16_rn(gelu_as(z));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    // ---- layer 2 on the tensor cores
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < kHid / 16; ++s)
        tc_mma(tmem, smem_desc(a_base + 256u * s), smem_desc(b_base + 256u * s), s > 0 ? 1u : 0u);
      tc_commit(bar_a);
      if (!mbar_wait(bar_a, parity, p.spin_budget)) {
        atomicExch(p.err, 1);
        *sabort = 1;
        mbar_wait(bar_a, parity, p.spin_budget);
      }
    }
    parity ^= 1u;
    __syncthreads();
    if (*sabort) break;
    tc_fence_after();
    // ---- head
    const int quarter = warp & 3, half = warp >> 2;
    float s = 0.f;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      const int col0 = half * 128 + c * 32;
      float v[32];
      tc_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) s += gelu_as(v[i] + sb2[col0 + i]) * sw3[col0 + i];
    }
    spart[half * kTileRows + quarter * 32 + lane] = s;
    tc_fence_before();
    __syncthreads();
    if (tid < kTileRows) {
      const long long q = tile * kTileRows + tid;
      if (q < p.rows) p.table[q] = spart[tid] + spart[kTileRows + tid] + b3;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

__global__ void mlp_w2_layout_kernel(const float* __restrict__ W2, __nv_bfloat16* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kHid * kHid; i += gridDim.x * blockDim.x) {
    const int n = i / kHid, k = i % kHid;
    out[cm_off(n, k) / 2] = __float2bfloat16_rn(W2[i]);
  }
}

}  // namespace

int mlp_table_rows(int h) {
  const int np = h < kHin ? h : kHin;
  return 1 << (2 * np - 1);
}

size_t mlp_w2c_bytes() { return kW2Bytes; }

// the prediction table of shape h (mlp_table_rows(h) floats) on stream s;
// err_dev (one int) is cleared and set by the kernel if a wait ran out
cudaError_t mlp_table_tc(const float* P, int h, float* table, void* w2c, int* err_dev, cudaStream_t s) {
  static int configured_device = -1;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device != dev) {
    e = cudaFuncSetAttribute(mlp_table_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int clock_khz = 0;
  cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
  mlp_w2_layout_kernel<<<64, 256, 0, s>>>(P + kOffW2, static_cast<__nv_bfloat16*>(w2c));
  e = cudaMemsetAsync(err_dev, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  TcParams p{};
  p.P = P;
  p.w2c = static_cast<const uint4*>(w2c);
  p.table = table;
  p.h = h;
  p.np = h < kHin ? h : kHin;
  p.rows = mlp_table_rows(h);
  p.err = err_dev;
  // about one second of clock cycles per wait
  p.spin_budget = (long long)(clock_khz > 0 ? clock_khz : 2000000) * 1000ll;
  const long long tiles = (p.rows + kTileRows - 1) / kTileRows;
  const int grid = (int)(tiles < sms ? tiles : sms);
  mlp_table_tc_kernel<<<grid, kTcThreads, kTcSmem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace lcs
