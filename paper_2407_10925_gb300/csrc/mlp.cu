// mlp.cu -- the learned warm start: a small MLP that predicts the relative
// value function of the binary two-string case (sigma = d = 2), trained on the
// converged iterates of smaller h and used to start the iteration at a larger
// h.  Not part of the paper's method: the paper starts from the zero vector.
// Lemma 1 (section 2.1) makes any start legitimate, because the bound comes
// only from a triplet whose feasibility the check verifies directly; the
// warm start can change how many iterations are needed, never the rigor.
//
// Network: 49 features -> 256 -> 256 -> 1, GELU (erf form) after each hidden
// layer, FP32 weights.  Features of a state of length h: for positions p < 12
// of each string, a one-hot of the letter (feature 4p + 2j + letter), zero
// when p >= h; feature 48 = h / 16.  The state is first replaced by the
// smallest index of its orbit under complement and string swap, so the
// prediction carries the iterate's exact symmetries.
//
// Training runs on the GPU with the kernels below: a tiled FP32 GEMM for the
// 256 x 256 layer (forward and both backward products), elementwise kernels
// for the first layer (a gather of one-hot columns), GELU and its derivative,
// deterministic column reductions for the bias and first-layer gradients, and
// Adam.  Parameters are laid out flat as W1 (256 x 49, row-major), b1, W2
// (256 x 256, row-major, out x in), b2, w3, b3.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/lcs_bound.h"
#include "lcs_common.h"
#include "mlp_net.h"

namespace lcs {

void record_error(const char* msg);
int mlp_table_rows(int h);
size_t mlp_w2c_bytes();
cudaError_t mlp_table_tc(const float* P, int h, float* table, void* w2c, int* err_dev, cudaStream_t s);

static lcs_status mfail(lcs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  record_error(buf);
  return st;
}

#define M_CUDA(call)                                                                                      \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return mfail(LCS_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                        __FILE__, __LINE__);                                              \
  } while (0)

// ---------------------------------------------------------------------------
// kernels

// first layer for rows [0, n): Z1 = b1 + sum of active columns of W1 + (h/16) W1[:, 48];
// A1 = GELU(Z1); the active-feature bit mask of each row goes to mask (for dW1)
__global__ void mlp_layer1_kernel(const float* __restrict__ P, const unsigned long long* __restrict__ states,
                                  const int* __restrict__ hs, int n, float* __restrict__ Z1, float* __restrict__ A1,
                                  unsigned long long* __restrict__ mask) {
  const int r = blockIdx.x;
  if (r >= n) return;
  __shared__ int idx[2 * kHin];
  __shared__ int cnt;
  if (threadIdx.x == 0) {
    cnt = mlp_active(states[r], hs[r], idx);
    if (mask) {
      unsigned long long m = 0;
      for (int i = 0; i < cnt; ++i) m |= 1ull << idx[i];
      mask[r] = m;
    }
  }
  __syncthreads();
  const int j = threadIdx.x;  // hidden unit
  const float* W1 = P + kOffW1;
  float z = P[kOffB1 + j] + (float)hs[r] * (1.0f / 16.0f) * W1[j * kFeat + (kFeat - 1)];
  for (int i = 0; i < cnt; ++i) z += W1[j * kFeat + idx[i]];
  Z1[(long long)r * kHid + j] = z;
  A1[(long long)r * kHid + j] = gelu_f(z);
}

// C[M x N] = op(A) op(B) + bias (bias per column, optional); row-major, 64 x 64 tiles
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       const float* __restrict__ B, int ldb,
                                                       const float* __restrict__ bias, float* __restrict__ C,
                                                       int ldc) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int gm = m0 + mm, gk = k0 + kk;
      float a = 0.f;
      if (gm < M && gk < K) a = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = a;
      const int gn = n0 + mm;
      float b = 0.f;
      if (gn < N && gk < K) b = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][mm] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i], bv[i] = Bs[kk][tx * 4 + i];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] += av[i] * bv[jj];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + jj;
      if (gm < M && gn < N) C[(long long)gm * ldc + gn] = acc[i][jj] + (bias ? bias[gn] : 0.f);
    }
}

// A2 = GELU(Z2); y = A2 w3 + b3; per row (one block of kHid threads)
__global__ void mlp_head_kernel(const float* __restrict__ P, const float* __restrict__ Z2, int n,
                                float* __restrict__ A2, float* __restrict__ y) {
  const int r = blockIdx.x;
  if (r >= n) return;
  const int j = threadIdx.x;
  const float a = gelu_f(Z2[(long long)r * kHid + j]);
  if (A2) A2[(long long)r * kHid + j] = a;
  float v = a * P[kOffW3 + j];
  __shared__ float red[kHid / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((j & 31) == 0) red[j >> 5] = v;
  __syncthreads();
  if (j == 0) {
    float s = 0.f;
    for (int w = 0; w < kHid / 32; ++w) s += red[w];
    y[r] = s + P[kOffB3];
  }
}

// dy = 2 (y - t) / n; dZ2 = dy w3 * GELU'(Z2); per row
__global__ void mlp_back_head_kernel(const float* __restrict__ P, const float* __restrict__ Z2,
                                     const float* __restrict__ y, const float* __restrict__ t, int n,
                                     float* __restrict__ dy, float* __restrict__ dZ2) {
  const int r = blockIdx.x;
  if (r >= n) return;
  const int j = threadIdx.x;
  const float g = 2.0f * (y[r] - t[r]) / (float)n;
  if (j == 0) dy[r] = g;
  dZ2[(long long)r * kHid + j] = g * P[kOffW3 + j] * gelu_grad_f(Z2[(long long)r * kHid + j]);
}

// in place: D = D * GELU'(Z)
__global__ void mlp_gelu_back_kernel(float* __restrict__ D, const float* __restrict__ Z, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    D[i] *= gelu_grad_f(Z[i]);
}

// column sums: out[j] = sum_r X[r][j] (* w[r] if w)
__global__ void mlp_colsum_kernel(const float* __restrict__ X, const float* __restrict__ w, int n, int cols,
                                  float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int r = 0; r < n; ++r) s += X[(long long)r * cols + j] * (w ? w[r] : 1.0f);
  out[j] = s;
}

// db3 = sum dy
__global__ void mlp_sum_kernel(const float* __restrict__ x, int n, float* __restrict__ out) {
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// dW1[j][f] = sum over rows with feature f active of dZ1[r][j]; f = 48: weighted by h/16
__global__ void mlp_dw1_kernel(const float* __restrict__ dZ1, const unsigned long long* __restrict__ mask,
                               const int* __restrict__ hs, int n, float* __restrict__ dW1) {
  const int j = threadIdx.x, f = blockIdx.x;
  float s = 0.f;
  if (f == kFeat - 1) {
    for (int r = 0; r < n; ++r) s += dZ1[(long long)r * kHid + j] * ((float)hs[r] * (1.0f / 16.0f));
  } else {
    for (int r = 0; r < n; ++r)
      if ((mask[r] >> f) & 1ull) s += dZ1[(long long)r * kHid + j];
  }
  dW1[j * kFeat + f] = s;
}

__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mm,
                                float* __restrict__ V, long long count, float lr, float b1, float b2, float eps,
                                float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * Mm[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    Mm[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// a training batch from converged iterates: row r takes set r % n_sets and a
// state drawn by SplitMix64; target = (v[x] - ref) * 2^-K
struct TrainSet {
  const long long* v;       // full-length fixed-point vector (device)
  unsigned long long n;     // states
  long long ref;            // value subtracted (v at state 0)
  int h;
};

__device__ __forceinline__ unsigned long long splitmix(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void mlp_sample_kernel(const TrainSet* __restrict__ sets, int n_sets, int n, unsigned long long seed,
                                  double scale, unsigned long long* __restrict__ states, int* __restrict__ hs,
                                  float* __restrict__ t) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const TrainSet S = sets[r % n_sets];
  const unsigned long long x = splitmix(seed, (unsigned long long)r) % S.n;
  states[r] = x;
  hs[r] = S.h;
  t[r] = (float)((double)(S.v[x] - S.ref) * scale);
}

// warm start: v_k[x] = u_hat[x] + k r_hat for the newest (k = d-1 .. ) convention of set_start
__global__ void mlp_to_start_kernel(const float* __restrict__ y, long long n, long long off, double r_hat, int d,
                                    double* __restrict__ v0, double* __restrict__ v1) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double u = (double)y[i];
    v1[off + i] = u;          // older start vector
    v0[off + i] = u + r_hat;  // newest
  }
}

// full-length vectors from the prediction table (mlp_tc.cu): the value of a
// state is the table entry of its canonical form's first np positions
__global__ void mlp_table_start_kernel(const float* __restrict__ T, int h, int np, long long n, double r_hat,
                                       double* __restrict__ newest, double* __restrict__ older) {
  const int shift = 2 * (h - np);
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const double u = (double)T[mlp_canonical((unsigned long long)x, h) >> shift];
    older[x] = u;
    newest[x] = u + r_hat;
  }
}

// the same start in the handle's stored form (states x < 4^h / 2) and fixed
// point, converted as set_start converts doubles (rounded down)
__global__ void mlp_table_start_fx_kernel(const float* __restrict__ T, int h, int np, long long n_stored, double r_hat,
                                          double scale, long long* __restrict__ newest, long long* __restrict__ older) {
  const int shift = 2 * (h - np);
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_stored;
       x += (long long)gridDim.x * blockDim.x) {
    const double u = (double)T[mlp_canonical((unsigned long long)x, h) >> shift];
    older[x] = __double2ll_rd(u * scale);
    newest[x] = __double2ll_rd((u + r_hat) * scale);
  }
}

__global__ void mlp_table_predict_kernel(const float* __restrict__ T, int h, int np, unsigned long long base,
                                         long long n, float* __restrict__ out) {
  const int shift = 2 * (h - np);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = T[mlp_canonical(base + (unsigned long long)i, h) >> shift];
}

// the prefix-truncation lift (the non-learned control of the warm start):
// dst[x] = src[x >> 2 (h_to - h_from)] - src[0], i.e. the value of the tuple
// cut to its first h_from letters, as doubles in units; both full length
__global__ void lift_prefix_kernel(const long long* __restrict__ src, int shift, long long n_to, double scale,
                                   double r_hat, double* __restrict__ newest, double* __restrict__ older) {
  const long long ref = src[0];
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n_to; x += (long long)gridDim.x * blockDim.x) {
    const double u = (double)(src[x >> shift] - ref) * scale;
    older[x] = u;
    newest[x] = u + r_hat;
  }
}

__global__ void iota_kernel(unsigned long long* __restrict__ s, long long n, unsigned long long base) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s[i] = base + (unsigned long long)i;
}

__global__ void fill_int_kernel(int* __restrict__ p, long long n, int v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace lcs

// ---------------------------------------------------------------------------
// host side

using namespace lcs;

struct lcs_mlp {
  float* P;       // parameters (device)
  float* G;       // gradient
  float* Mm;      // Adam moments
  float* V;
  long long adam_t;
  int cap;        // rows of the work buffers
  float *Z1, *A1, *Z2, *A2, *y, *t, *dy, *dZ2, *dA1;
  unsigned long long* states;
  unsigned long long* mask;
  int* hs;
  TrainSet* sets;
  cudaStream_t stream;
  // BF16 inference: W2 in bf16 (core-matrix layout), the prediction table, an error flag
  void* W2c;
  float* table;
  int* err;
  // device allocator (NULL alloc: cudaMalloc / cudaFree)
  void* (*alloc)(size_t, void*);
  void (*free)(void*, void*);
  void* alloc_ctx;
};

// every device buffer of the network goes through these two
template <class T>
static lcs_status mlp_alloc(lcs_mlp* M, T** p, size_t bytes) {
  void* q = nullptr;
  if (M->alloc) {
    q = M->alloc(bytes, M->alloc_ctx);
  } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    q = nullptr;
  }
  *p = static_cast<T*>(q);
  if (!q) return mfail(LCS_ENOMEM, "mlp: device allocation of %zu bytes failed", bytes);
  return LCS_OK;
}

static void mlp_free(lcs_mlp* M, void* p) {
  if (!p) return;
  if (M->alloc) {
    if (M->free) M->free(p, M->alloc_ctx);
  } else {
    cudaFree(p);
  }
}

static unsigned long long host_splitmix(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static lcs_status ensure_cap(lcs_mlp* M, int rows) {
  if (rows <= M->cap) return LCS_OK;
  M_CUDA(cudaStreamSynchronize(M->stream));  // the old buffers may still be in use
  M->cap = 0;
  float** bufs[] = {&M->Z1, &M->A1, &M->Z2, &M->A2, &M->dZ2, &M->dA1};
  for (float** b : bufs) {
    mlp_free(M, *b);
    *b = nullptr;
    if (lcs_status st = mlp_alloc(M, b, sizeof(float) * (size_t)rows * kHid)) return st;
  }
  float** small[] = {&M->y, &M->t, &M->dy};
  for (float** b : small) {
    mlp_free(M, *b);
    *b = nullptr;
    if (lcs_status st = mlp_alloc(M, b, sizeof(float) * (size_t)rows)) return st;
  }
  mlp_free(M, M->states);
  mlp_free(M, M->mask);
  mlp_free(M, M->hs);
  M->states = M->mask = nullptr;
  M->hs = nullptr;
  if (lcs_status st = mlp_alloc(M, &M->states, sizeof(unsigned long long) * (size_t)rows)) return st;
  if (lcs_status st = mlp_alloc(M, &M->mask, sizeof(unsigned long long) * (size_t)rows)) return st;
  if (lcs_status st = mlp_alloc(M, &M->hs, sizeof(int) * (size_t)rows)) return st;
  M->cap = rows;
  return LCS_OK;
}

// forward for rows [0, n) already in M->states / M->hs; fills Z1, A1, Z2, A2 (if keep), y
static lcs_status forward_rows(lcs_mlp* M, int n, bool keep) {
  cudaStream_t s = M->stream;
  mlp_layer1_kernel<<<n, kHid, 0, s>>>(M->P, M->states, M->hs, n, M->Z1, M->A1, keep ? M->mask : nullptr);
  dim3 g2((kHid + 63) / 64, (n + 63) / 64);
  mlp_gemm_kernel<false, true><<<g2, 256, 0, s>>>(n, kHid, kHid, M->A1, kHid, M->P + kOffW2, kHid, M->P + kOffB2,
                                                   M->Z2, kHid);
  mlp_head_kernel<<<n, kHid, 0, s>>>(M->P, M->Z2, n, keep ? M->A2 : nullptr, M->y);
  M_CUDA(cudaGetLastError());
  return LCS_OK;
}

// gradient of the mean squared error over rows [0, n) into M->G
static lcs_status backward_rows(lcs_mlp* M, int n) {
  cudaStream_t s = M->stream;
  float* G = M->G;
  mlp_back_head_kernel<<<n, kHid, 0, s>>>(M->P, M->Z2, M->y, M->t, n, M->dy, M->dZ2);
  mlp_colsum_kernel<<<1, kHid, 0, s>>>(M->A2, M->dy, n, kHid, G + kOffW3);  // dw3 = A2^T dy
  mlp_sum_kernel<<<1, 256, 0, s>>>(M->dy, n, G + kOffB3);
  mlp_colsum_kernel<<<1, kHid, 0, s>>>(M->dZ2, nullptr, n, kHid, G + kOffB2);
  // dW2 = dZ2^T A1 (256 x 256, out x in)
  dim3 gw((kHid + 63) / 64, (kHid + 63) / 64);
  mlp_gemm_kernel<true, false><<<gw, 256, 0, s>>>(kHid, kHid, n, M->dZ2, kHid, M->A1, kHid, nullptr, G + kOffW2,
                                                   kHid);
  // dA1 = dZ2 W2, then dZ1 = dA1 * GELU'(Z1)
  dim3 ga((kHid + 63) / 64, (n + 63) / 64);
  mlp_gemm_kernel<false, false><<<ga, 256, 0, s>>>(n, kHid, kHid, M->dZ2, kHid, M->P + kOffW2, kHid, nullptr, M->dA1,
                                                    kHid);
  mlp_gelu_back_kernel<<<1024, 256, 0, s>>>(M->dA1, M->Z1, (long long)n * kHid);
  mlp_colsum_kernel<<<1, kHid, 0, s>>>(M->dA1, nullptr, n, kHid, G + kOffB1);
  mlp_dw1_kernel<<<kFeat, kHid, 0, s>>>(M->dA1, M->mask, M->hs, n, G + kOffW1);
  M_CUDA(cudaGetLastError());
  return LCS_OK;
}

extern "C" {

int64_t lcs_mlp_param_count(void) { return kNParams; }

void lcs_mlp_destroy(lcs_mlp_t* M) {
  if (!M) return;
  if (M->stream) cudaStreamSynchronize(M->stream);
  void* ptrs[] = {M->P, M->G, M->Mm, M->V, M->Z1, M->A1, M->Z2, M->A2, M->y, M->t, M->dy, M->dZ2, M->dA1,
                  M->states, M->mask, M->hs, M->sets, M->W2c, M->table, M->err};
  for (void* p : ptrs) mlp_free(M, p);
  if (M->stream) cudaStreamDestroy(M->stream);
  delete M;
}

lcs_status lcs_mlp_create(uint64_t seed, lcs_mlp_t** out) {
  return lcs_mlp_create_with_allocator(seed, nullptr, nullptr, nullptr, out);
}

lcs_status lcs_mlp_create_with_allocator(uint64_t seed, void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*),
                                         void* alloc_ctx, lcs_mlp_t** out) {
  if (!out) return mfail(LCS_EINVAL, "out is NULL");
  *out = nullptr;
  if (alloc && !free_fn) return mfail(LCS_EINVAL, "alloc given without free");
  lcs_mlp* M = new (std::nothrow) lcs_mlp();
  if (!M) return mfail(LCS_ENOMEM, "host allocation");
  std::memset(M, 0, sizeof *M);
  M->alloc = alloc;
  M->free = free_fn;
  M->alloc_ctx = alloc_ctx;
  cudaError_t e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    lcs_mlp_destroy(M);
    return mfail(LCS_ECUDA, "mlp stream: %s", cudaGetErrorString(e));
  }
  lcs_status st = mlp_alloc(M, &M->P, sizeof(float) * kNParams);
  if (!st) st = mlp_alloc(M, &M->G, sizeof(float) * kNParams);
  if (!st) st = mlp_alloc(M, &M->Mm, sizeof(float) * kNParams);
  if (!st) st = mlp_alloc(M, &M->V, sizeof(float) * kNParams);
  if (!st) st = mlp_alloc(M, &M->sets, sizeof(TrainSet) * 8);
  if (st) {
    lcs_mlp_destroy(M);
    return st;
  }
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64; biases zero
  std::vector<float> h(kNParams, 0.f);
  auto fill = [&](long long off, long long count, int fan_in) {
    const double a = 1.0 / std::sqrt((double)fan_in);
    for (long long i = 0; i < count; ++i) {
      const double u = (double)(host_splitmix(seed, (unsigned long long)(off + i)) >> 11) * (1.0 / 9007199254740992.0);
      h[off + i] = (float)((2.0 * u - 1.0) * a);
    }
  };
  fill(kOffW1, (long long)kHid * kFeat, 2 * kHin + 1);  // at most 25 inputs are non-zero
  fill(kOffW2, (long long)kHid * kHid, kHid);
  fill(kOffW3, kHid, kHid);
  e = cudaMemcpy(M->P, h.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->Mm, 0, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMemset(M->V, 0, sizeof(float) * kNParams);
  if (e != cudaSuccess) {
    lcs_mlp_destroy(M);
    return mfail(LCS_ECUDA, "mlp init: %s", cudaGetErrorString(e));
  }
  *out = M;
  return LCS_OK;
}

lcs_status lcs_mlp_get_params(lcs_mlp_t* M, float* host_out) {
  if (!M || !host_out) return mfail(LCS_EINVAL, "NULL argument");
  M_CUDA(cudaMemcpyAsync(host_out, M->P, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, M->stream));
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

lcs_status lcs_mlp_set_params(lcs_mlp_t* M, const float* host_in) {
  if (!M || !host_in) return mfail(LCS_EINVAL, "NULL argument");
  M_CUDA(cudaMemcpyAsync(M->P, host_in, sizeof(float) * kNParams, cudaMemcpyHostToDevice, M->stream));
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

lcs_status lcs_mlp_gradient(lcs_mlp_t* M, int n, const int64_t* states, const int* hs, const float* targets,
                            float* loss_out, float* grad_out) {
  if (!M || !states || !hs || !targets || !grad_out || n < 1) return mfail(LCS_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i)
    if (hs[i] < 1 || hs[i] > 31) return mfail(LCS_EINVAL, "h %d outside 1..31", hs[i]);
  lcs_status st = ensure_cap(M, n);
  if (st) return st;
  M_CUDA(cudaMemcpyAsync(M->states, states, sizeof(int64_t) * n, cudaMemcpyHostToDevice, M->stream));
  M_CUDA(cudaMemcpyAsync(M->hs, hs, sizeof(int) * n, cudaMemcpyHostToDevice, M->stream));
  M_CUDA(cudaMemcpyAsync(M->t, targets, sizeof(float) * n, cudaMemcpyHostToDevice, M->stream));
  st = forward_rows(M, n, true);
  if (st) return st;
  st = backward_rows(M, n);
  if (st) return st;
  M_CUDA(cudaMemcpyAsync(grad_out, M->G, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, M->stream));
  std::vector<float> y(n);
  M_CUDA(cudaMemcpyAsync(y.data(), M->y, sizeof(float) * n, cudaMemcpyDeviceToHost, M->stream));
  M_CUDA(cudaStreamSynchronize(M->stream));
  if (loss_out) {
    double l = 0;
    for (int i = 0; i < n; ++i) l += ((double)y[i] - targets[i]) * ((double)y[i] - targets[i]);
    *loss_out = (float)(l / n);
  }
  return LCS_OK;
}

lcs_status lcs_mlp_predict(lcs_mlp_t* M, int h, int64_t n, const int64_t* states_dev, float* out_dev) {
  if (!M || !states_dev || !out_dev || n < 0 || h < 1 || h > 31) return mfail(LCS_EINVAL, "bad argument");
  const int chunk = 1 << 20;
  lcs_status st = ensure_cap(M, (int)std::min<int64_t>(std::max<int64_t>(n, 1), chunk));
  if (st) return st;
  for (int64_t off = 0; off < n; off += chunk) {
    const int m = (int)std::min<int64_t>(chunk, n - off);
    M_CUDA(cudaMemcpyAsync(M->states, states_dev + off, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, M->stream));
    fill_int_kernel<<<256, 256, 0, M->stream>>>(M->hs, m, h);
    st = forward_rows(M, m, false);
    if (st) return st;
    M_CUDA(cudaMemcpyAsync(out_dev + off, M->y, sizeof(float) * m, cudaMemcpyDeviceToDevice, M->stream));
  }
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

lcs_status lcs_mlp_train(lcs_mlp_t* M, int n_sets, const int64_t* const* vectors, const int* hs, int64_t steps,
                         int batch, float lr, uint64_t seed, int frac_bits, float* last_loss) {
  if (!M || !vectors || !hs || n_sets < 1 || n_sets > 8 || steps < 0 || batch < 1) return mfail(LCS_EINVAL, "bad argument");
  if (frac_bits == 0) frac_bits = 44;
  TrainSet sets[8];
  for (int i = 0; i < n_sets; ++i) {
    if (!vectors[i] || hs[i] < 1 || hs[i] > 15) return mfail(LCS_EINVAL, "training set %d", i);
    sets[i].v = (const long long*)vectors[i];
    sets[i].n = 1ull << (2 * hs[i]);
    sets[i].h = hs[i];
    long long ref = 0;
    M_CUDA(cudaMemcpyAsync(&ref, vectors[i], sizeof(long long), cudaMemcpyDeviceToHost, M->stream));
    M_CUDA(cudaStreamSynchronize(M->stream));
    sets[i].ref = ref;
  }
  M_CUDA(cudaMemcpyAsync(M->sets, sets, sizeof(TrainSet) * n_sets, cudaMemcpyHostToDevice, M->stream));
  lcs_status st = ensure_cap(M, batch);
  if (st) return st;
  const double scale = std::ldexp(1.0, -frac_bits);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t k = 0; k < steps; ++k) {
    mlp_sample_kernel<<<(batch + 255) / 256, 256, 0, M->stream>>>(M->sets, n_sets, batch,
                                                                   host_splitmix(seed, (unsigned long long)k), scale,
                                                                   M->states, M->hs, M->t);
    st = forward_rows(M, batch, true);
    if (st) return st;
    st = backward_rows(M, batch);
    if (st) return st;
    M->adam_t++;
    const float c1 = 1.f - std::pow(b1, (float)M->adam_t), c2 = 1.f - std::pow(b2, (float)M->adam_t);
    mlp_adam_kernel<<<128, 256, 0, M->stream>>>(M->P, M->G, M->Mm, M->V, kNParams, lr, b1, b2, eps, c1, c2);
    M_CUDA(cudaGetLastError());
  }
  if (last_loss) {
    // loss of one fresh batch after training
    mlp_sample_kernel<<<(batch + 255) / 256, 256, 0, M->stream>>>(M->sets, n_sets, batch, host_splitmix(seed, ~0ull),
                                                                   scale, M->states, M->hs, M->t);
    st = forward_rows(M, batch, false);
    if (st) return st;
    std::vector<float> y(batch), t(batch);
    M_CUDA(cudaMemcpyAsync(y.data(), M->y, sizeof(float) * batch, cudaMemcpyDeviceToHost, M->stream));
    M_CUDA(cudaMemcpyAsync(t.data(), M->t, sizeof(float) * batch, cudaMemcpyDeviceToHost, M->stream));
    M_CUDA(cudaStreamSynchronize(M->stream));
    double l = 0;
    for (int i = 0; i < batch; ++i) l += ((double)y[i] - t[i]) * ((double)y[i] - t[i]);
    *last_loss = (float)(l / batch);
  }
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

// the BF16 prediction table of shape h (mlp_tc.cu) into M->table
static lcs_status build_table(lcs_mlp* M, int h) {
  // made on first use; after a failed allocation the next call retries the missing ones
  if (!M->W2c)
    if (lcs_status st = mlp_alloc(M, &M->W2c, mlp_w2c_bytes())) return st;
  if (!M->table)
    if (lcs_status st = mlp_alloc(M, &M->table, sizeof(float) * (size_t)mlp_table_rows(kHin))) return st;
  if (!M->err)
    if (lcs_status st = mlp_alloc(M, &M->err, sizeof(int))) return st;
  M_CUDA(mlp_table_tc(M->P, h, M->table, M->W2c, M->err, M->stream));
  int err = 0;
  M_CUDA(cudaMemcpyAsync(&err, M->err, sizeof(int), cudaMemcpyDeviceToHost, M->stream));
  M_CUDA(cudaStreamSynchronize(M->stream));
  if (err) return mfail(LCS_ETIMEOUT, "tensor-core inference: a wait on the tensor core ran out");
  return LCS_OK;
}

// predictions for every state of length h, as two full-length double vectors
// of a start: older = u_hat, newest = u_hat + r_hat (device pointers)
lcs_status lcs_mlp_start_vectors(lcs_mlp_t* M, int h, double r_hat, double* newest_dev, double* older_dev) {
  if (!M || !newest_dev || !older_dev || h < 1 || h > 16) return mfail(LCS_EINVAL, "bad argument");
  lcs_status st = build_table(M, h);
  if (st) return st;
  mlp_table_start_kernel<<<4096, 256, 0, M->stream>>>(M->table, h, std::min(h, kHin), 1ll << (2 * h), r_hat,
                                                      newest_dev, older_dev);
  M_CUDA(cudaGetLastError());
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

lcs_status lcs_mlp_start_vectors_stored_fx(lcs_mlp_t* M, int h, double r_hat, int frac_bits, int64_t* newest_dev,
                                           int64_t* older_dev) {
  if (!M || !newest_dev || !older_dev || h < 1 || h > 16) return mfail(LCS_EINVAL, "bad argument");
  if (frac_bits == 0) frac_bits = 44;
  if (frac_bits < 8 || frac_bits > 56) return mfail(LCS_EINVAL, "frac_bits %d outside 8..56", frac_bits);
  lcs_status st = build_table(M, h);
  if (st) return st;
  mlp_table_start_fx_kernel<<<4096, 256, 0, M->stream>>>(M->table, h, std::min(h, kHin), 1ll << (2 * h - 1), r_hat,
                                                         std::ldexp(1.0, frac_bits), (long long*)newest_dev,
                                                         (long long*)older_dev);
  M_CUDA(cudaGetLastError());
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

lcs_status lcs_lift_prefix(int h_from, int h_to, const int64_t* src_dev, int frac_bits, double r_hat,
                           double* newest_dev, double* older_dev) {
  if (!src_dev || !newest_dev || !older_dev || h_from < 1 || h_to < h_from || h_to > 16)
    return mfail(LCS_EINVAL, "bad argument");
  if (frac_bits == 0) frac_bits = 44;
  const long long n_to = 1ll << (2 * h_to);
  lift_prefix_kernel<<<4096, 256>>>((const long long*)src_dev, 2 * (h_to - h_from), n_to,
                                    std::ldexp(1.0, -frac_bits), r_hat, newest_dev, older_dev);
  M_CUDA(cudaGetLastError());
  M_CUDA(cudaDeviceSynchronize());
  return LCS_OK;
}

// BF16 predictions for the consecutive states base .. base+n-1 (device output)
lcs_status lcs_mlp_predict_bf16(lcs_mlp_t* M, int h, uint64_t base, int64_t n, float* out_dev) {
  if (!M || !out_dev || n < 0 || h < 1 || h > 31) return mfail(LCS_EINVAL, "bad argument");
  if (h < 32 && base + (uint64_t)n > (1ull << (2 * h)) && n > 0) return mfail(LCS_EINVAL, "states out of range");
  lcs_status st = build_table(M, h);
  if (st) return st;
  if (n > 0) {
    mlp_table_predict_kernel<<<2048, 256, 0, M->stream>>>(M->table, h, std::min(h, kHin), base, n, out_dev);
    M_CUDA(cudaGetLastError());
  }
  M_CUDA(cudaStreamSynchronize(M->stream));
  return LCS_OK;
}

}  // extern "C"
