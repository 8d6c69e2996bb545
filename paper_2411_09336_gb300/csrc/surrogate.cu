// Learned surrogate for log K (not part of the paper's method).
//
// Network: f -> ReLU(W1 f + b1) -> ReLU(W2 h1 + b2) -> w3 . h2 + b3 on the
// symmetric pair features f(x, y) = [(x - y)^2, (x + y)/2].  Hand-written
// kernels: feature construction, a tiled GEMM whose operands are rounded to
// bf16 as they enter shared memory (FP32 accumulation, optional for exact
// FP32 parity checks), fused bias + ReLU epilogues, the MSE loss, the
// backward pass and Adam (Kingma & Ba) on FP32 master weights.  Predictions
// are accepted where a split-conformal bound holds; qk_gram_surrogate sends
// every other entry to the exact overlap kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "qk_internal.h"
#include "tc_ptx.cuh"

struct qk_surrogate {
  int device = 0;
  int in_dim = 0, hidden = 0;
  int bf16 = 1;
  int64_t n_params = 0;
  float* d_params = nullptr;  // W1[h][in], b1[h], W2[h][h], b2[h], W3[h], b3[1]
  float* d_m = nullptr;
  float* d_v = nullptr;
  int64_t step = 0;
  double t_mean = 0.0, t_scale = 1.0;
  bool calibrated = false;
  std::vector<double> edges, bounds;
};

namespace qk {

namespace {

constexpr int kTM = 64, kTN = 64, kTK = 16;

struct Off {
  int64_t W1, b1, W2, b2, W3, b3, total;
};
Off offsets(int in, int h) {
  Off o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)h * in;
  o.W2 = o.b1 + h;
  o.b2 = o.W2 + (int64_t)h * h;
  o.W3 = o.b2 + h;
  o.b3 = o.W3 + h;
  o.total = o.b3 + 1;
  return o;
}

__device__ inline float rnd(float x, int bf16) { return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x; }

// C[m][n] = act(sum_k A(m,k) B(k,n) + bias[n]); A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn]; operands rounded to bf16 when bf16 != 0.
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* A, int64_t sam, int64_t sak,
                                                   const float* B, int64_t sbk, int64_t sbn, float* C, int64_t ldc,
                                                   const float* bias, int relu, int bf16) {
  __shared__ float sA[kTK][kTM + 4];
  __shared__ float sB[kTK][kTN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kTK) {
    for (int e = threadIdx.x; e < kTK * kTM; e += 256) {
      const int kk = e / kTM, mm = e % kTM;
      const int m = m0 + mm, k = k0 + kk;
      sA[kk][mm] = (m < M && k < K) ? rnd(A[(int64_t)m * sam + (int64_t)k * sak], bf16) : 0.f;
    }
    for (int e = threadIdx.x; e < kTK * kTN; e += 256) {
      const int kk = e / kTN, nn = e % kTN;
      const int n = n0 + nn, k = k0 + kk;
      sB[kk][nn] = (n < N && k < K) ? rnd(B[(int64_t)k * sbk + (int64_t)n * sbn], bf16) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) {
        float v = acc[i][j] + (bias ? bias[n] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        C[(int64_t)m * ldc + n] = v;
      }
    }
}

__global__ void features_kernel(const double* Xa, const double* Xb, const int32_t* pairs, int64_t P, int n,
                                float* F) {
  const int64_t total = P * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / n;
    const int k = (int)(e % n);
    const double a = Xa[(int64_t)pairs[2 * p] * n + k], b = Xb[(int64_t)pairs[2 * p + 1] * n + k];
    F[p * 2 * n + k] = (float)((a - b) * (a - b));
    F[p * 2 * n + n + k] = (float)(0.5 * (a + b));
  }
}

// y[p] = sum_h H[p][h] w[h] + b (one warp per row)
__global__ void head_kernel(const float* H, int64_t P, int h, const float* w, const float* b, int bf16, float* y) {
  const int lane = threadIdx.x & 31;
  for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; p < P;
       p += (int64_t)gridDim.x * blockDim.x / 32) {
    float s = 0.f;
    for (int i = lane; i < h; i += 32) s = fmaf(rnd(H[p * h + i], bf16), rnd(w[i], bf16), s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[p] = s + b[0];
  }
}

// r = y - t'; dy = r / P; loss accumulates 0.5 r^2 / P
__global__ void loss_kernel(const float* y, const double* t, int64_t P, double mean, double scale, float* dy,
                            double* loss) {
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const double r = (double)y[p] - (t[p] - mean) / scale;
    dy[p] = (float)(r / (double)P);
    acc += 0.5 * r * r / (double)P;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// dZ[p][i] = dy[p] * w[i] * (Z[p][i] > 0)
__global__ void outer_mask_kernel(const float* dy, const float* w, const float* Z, int64_t P, int h, int bf16,
                                  float* dZ) {
  const int64_t total = P * h;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % h);
    dZ[e] = Z[e] > 0.f ? dy[e / h] * rnd(w[i], bf16) : 0.f;
  }
}

__global__ void relu_kernel(const float* Z, float* H, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    H[e] = fmaxf(Z[e], 0.f);
}

__global__ void mask_kernel(float* G, const float* Z, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (!(Z[e] > 0.f)) G[e] = 0.f;
}

// out[j] = sum_p M[p][j]   (bias gradients)
__global__ void colsum_kernel(const float* M, int64_t P, int cols, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int64_t p = 0; p < P; ++p) s += M[p * cols + j];
  out[j] = s;
}

// w3 gradient: g[i] = sum_p dy[p] H[p][i]
__global__ void gemv_t_kernel(const float* H, const float* dy, int64_t P, int h, int bf16, float* g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= h) return;
  float s = 0.f;
  for (int64_t p = 0; p < P; ++p) s = fmaf(dy[p], rnd(H[p * h + i], bf16), s);
  g[i] = s;
}

__global__ void sum_kernel(const float* v, int64_t P, float* out) {
  float s = 0.f;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s += v[p];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[0] = t;
  }
}

__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// counter-based uniform in [0, 1): SplitMix64 (Steele, Lea, Flood 2014)
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void init_kernel(float* w, int64_t n, float lim, uint64_t seed, int64_t base) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64(seed ^ (uint64_t)(base + i)) >> 11) * (1.0 / 9007199254740992.0);
    w[i] = (float)((2.0 * u - 1.0) * lim);
  }
}

__global__ void accept_kernel(const float* y, int64_t P, double mean, double scale, const double* edges,
                              const double* bounds, int nb, double tol, double* Kout, uint8_t* acc,
                              unsigned long long* n_rej, int32_t* rej_idx) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const double pred = (double)y[p] * scale + mean;
    int b = 0;
    while (b + 1 < nb && pred >= edges[b + 1]) ++b;
    const bool ok = bounds[b] <= tol;
    acc[p] = ok ? 1 : 0;
    if (ok) {
      Kout[p] = exp(pred);
    } else {
      const unsigned long long q = atomicAdd(n_rej, 1ull);
      rej_idx[q] = (int32_t)p;
    }
  }
}

__global__ void block_pairs_kernel(int64_t i0, int64_t cnt, int NB, int32_t* pairs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lin = i0 + e;
    pairs[2 * e] = (int32_t)(lin / NB);
    pairs[2 * e + 1] = (int32_t)(lin % NB);
  }
}

__global__ void gather_pairs_kernel(const int32_t* pairs, const int32_t* idx, int64_t n, int32_t* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    out[2 * e] = pairs[2 * idx[e]];
    out[2 * e + 1] = pairs[2 * idx[e] + 1];
  }
}

// exact values of the rejected entries of a chunk into K
__global__ void scatter_block_kernel(const double* vals, const int32_t* idx, int64_t n, int64_t i0, int NB, double* K,
                                     int64_t ldk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lin = i0 + idx[e];
    K[(lin / NB) * ldk + lin % NB] = vals[e];
  }
}

__global__ void copy_block_kernel(const double* v, int64_t i0, int64_t cnt, int NB, double* K, int64_t ldk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lin = i0 + e;
    K[(lin / NB) * ldk + lin % NB] = v[e];
  }
}

inline int blocks(int64_t n, int t = 256) { return (int)std::min<int64_t>((n + t - 1) / t, 4096); }

// ---- the same GEMM on the tensor cores (bf16 operands) ---------------------
// One CTA computes a 128 x 128 tile of C with one tcgen05.mma (kind::f16,
// M = N = 128, K = 16) per 16-wide K chunk, FP32 accumulation in TMEM.  The
// 128 threads stage chunk c of A (row m0 + tid) and B (column n0 + tid),
// rounded to bf16 as the SIMT kernel rounds them, into a 4-stage ring in the
// K-major core-matrix layout (8 rows x 16 bytes, no swizzle); thread 0 issues
// the MMA and commits it to the stage's mbarrier, which the threads wait for
// (bounded) before they overwrite that stage.  Epilogue: tcgen05.ld -> bias
// -> ReLU -> C.  A wait that runs out sets g_tc_gemm_err and the CTA drains
// its MMAs before it frees the TMEM.
constexpr int kGT = 128, kGStages = 4, kGThreads = 128;
constexpr int kGStageBytes = 2 * kGT * 16 * 2;  // A and B blocks, bf16

__device__ int g_tc_gemm_err;

struct __align__(8) GemmShared {
  uint64_t bar[kGStages];
  uint64_t done;
  uint32_t tmem;
  int abort;
};

__device__ inline int core_off(int r, int k) { return (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }

__global__ void __launch_bounds__(kGThreads, 4) tc_gemm_kernel(int M, int N, int K, const float* A, int64_t sam,
                                                                int64_t sak, const float* B, int64_t sbk,
                                                                int64_t sbn, float* C, int64_t ldc,
                                                                const float* bias, int relu) {
  using namespace tcx;
  extern __shared__ __align__(1024) char gdyn[];
  __shared__ GemmShared sh;
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  if (tid < 32) tmem_alloc(&sh.tmem, kGT);
  if (tid == 0) {
    for (int s = 0; s < kGStages; ++s) mbar_init(&sh.bar[s], 1);
    mbar_init(&sh.done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    sh.abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sh.tmem;
  const uint32_t idesc = make_idesc(kGT, kGT, 0);
  const int nk = (K + 15) / 16;
  const int m = m0 + tid, n = n0 + tid;
  float va[16], vb[16];
  auto fetch = [&](int c) {
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const int k = c * 16 + kk;
      va[kk] = (m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : 0.f;
      vb[kk] = (n < N && k < K) ? B[(int64_t)k * sbk + (int64_t)n * sbn] : 0.f;
    }
  };
  if (nk > 0) fetch(0);
  for (int c = 0; c < nk; ++c) {
    const int s = c % kGStages;
    __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(gdyn + s * kGStageBytes);
    __nv_bfloat16* sb = sa + kGT * 16;
    // the MMA that read this stage (chunk c - kGStages) must be done
    if (c >= kGStages && !wait_bar(&sh.bar[s], ((c / kGStages) - 1) & 1)) sh.abort = 1;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      __align__(16) __nv_bfloat16 ha[8], hb[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        ha[i] = __float2bfloat16_rn(va[8 * half + i]);
        hb[i] = __float2bfloat16_rn(vb[8 * half + i]);
      }
      *reinterpret_cast<uint4*>(sa + core_off(tid, 8 * half)) = *reinterpret_cast<const uint4*>(ha);
      *reinterpret_cast<uint4*>(sb + core_off(tid, 8 * half)) = *reinterpret_cast<const uint4*>(hb);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (sh.abort) break;
    if (c + 1 < nk) fetch(c + 1);  // overlaps the MMA below
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      mma(tmem, make_desc(smem_u32(sa)), make_desc(smem_u32(sb)), idesc, c > 0 ? 1u : 0u);
      commit(&sh.bar[s]);
    }
  }
  if (tid == 0) commit(&sh.done);  // arrives once every MMA issued above is done
  __syncthreads();
  if (!wait_bar(&sh.done, 0)) sh.abort = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (!sh.abort && nk > 0) {
    const int w = tid >> 5, lane = tid & 31;
    const int row = m0 + 32 * w + lane;
    const uint32_t lane_base = (uint32_t)(32 * w) << 16;
    for (int c0 = 0; c0 < kGT; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + lane_base + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < M)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = n0 + c0 + i;
          if (col < N) {
            float v = __uint_as_float(r[i]) + (bias ? bias[col] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            C[(int64_t)row * ldc + col] = v;
          }
        }
    }
  } else if (!sh.abort) {
    // K = 0: C = act(bias)
    const int row = m0 + tid;
    if (row < M)
      for (int col = n0; col < min(N, n0 + kGT); ++col) {
        float v = bias ? bias[col] : 0.f;
        if (relu) v = fmaxf(v, 0.f);
        C[(int64_t)row * ldc + col] = v;
      }
  }
  if (sh.abort && tid == 0) atomicExch(&g_tc_gemm_err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (tid < 32) tmem_dealloc(tmem, kGT);
}

void gemm(cudaStream_t st, int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B,
          int64_t sbk, int64_t sbn, float* C, int64_t ldc, const float* bias, int relu, int bf16) {
  if (bf16) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGStages * kGStageBytes);
      attr = true;
    }
    dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
    tc_gemm_kernel<<<grid, kGThreads, kGStages * kGStageBytes, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc,
                                                                    bias, relu);
    return;
  }
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
  gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu, bf16);
}

// Reads and clears the tensor-core GEMM's error word (synchronises the stream).
qk_status gemm_status(cudaStream_t st, const char* who) {
  int h = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&h, g_tc_gemm_err, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, who);
  if (h) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_gemm_err, &zero, sizeof(int));
    return fail(QK_ERR_TIMEOUT, std::string(who) + ": a bounded wait of the tensor-core GEMM ran out");
  }
  return QK_OK;
}

// Work buffers for a minibatch of P pairs.
struct Work {
  float *F = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *y = nullptr, *dy = nullptr,
        *dZ2 = nullptr, *dZ1 = nullptr, *g = nullptr;
  double* loss = nullptr;
  int64_t cap = 0;
  void release(cudaStream_t st) {
    for (float* p : {F, Z1, H1, Z2, H2, y, dy, dZ2, dZ1, g})
      if (p) cudaFreeAsync(p, st);
    if (loss) cudaFreeAsync(loss, st);
    *this = Work();
  }
};

qk_status alloc_work(Work& w, const qk_surrogate* net, int64_t P, bool grads, cudaStream_t st) {
  const int in = net->in_dim, h = net->hidden;
  auto A = [&](float** p, int64_t n) { return cudaMallocAsync(p, sizeof(float) * std::max<int64_t>(n, 1), st); };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = A(&w.F, P * in);
  if (e == cudaSuccess) e = A(&w.Z1, P * h);
  if (e == cudaSuccess) e = A(&w.H1, P * h);
  if (e == cudaSuccess) e = A(&w.Z2, P * h);
  if (e == cudaSuccess) e = A(&w.H2, P * h);
  if (e == cudaSuccess) e = A(&w.y, P);
  if (grads) {
    if (e == cudaSuccess) e = A(&w.dy, P);
    if (e == cudaSuccess) e = A(&w.dZ2, P * h);
    if (e == cudaSuccess) e = A(&w.dZ1, P * h);
    if (e == cudaSuccess) e = A(&w.g, net->n_params);
    if (e == cudaSuccess) e = cudaMallocAsync(&w.loss, sizeof(double), st);
  }
  w.cap = P;
  if (e != cudaSuccess) {
    w.release(st);
    return cuda_fail(e, "surrogate work buffers");
  }
  return QK_OK;
}

// forward for P pairs whose features are in w.F; y standardised
void forward(const qk_surrogate* net, Work& w, int64_t P, cudaStream_t st) {
  const int in = net->in_dim, h = net->hidden, bf = net->bf16;
  const Off o = offsets(in, h);
  const float* prm = net->d_params;
  // Z1 = F W1^T + b1 ; H1 = ReLU(Z1) ; Z2 = H1 W2^T + b2 ; H2 = ReLU(Z2)
  gemm(st, (int)P, h, in, w.F, in, 1, prm + o.W1, 1, in, w.Z1, h, prm + o.b1, 0, bf);
  relu_kernel<<<blocks(P * h), 256, 0, st>>>(w.Z1, w.H1, P * h);
  gemm(st, (int)P, h, h, w.H1, h, 1, prm + o.W2, 1, h, w.Z2, h, prm + o.b2, 0, bf);
  relu_kernel<<<blocks(P * h), 256, 0, st>>>(w.Z2, w.H2, P * h);
  head_kernel<<<blocks(P * 32), 256, 0, st>>>(w.H2, P, h, prm + o.W3, prm + o.b3, bf, w.y);
}

// loss + gradient into w.g (same layout as the parameters)
void backward(const qk_surrogate* net, Work& w, int64_t P, const double* t, cudaStream_t st) {
  const int in = net->in_dim, h = net->hidden, bf = net->bf16;
  const Off o = offsets(in, h);
  const float* prm = net->d_params;
  cudaMemsetAsync(w.loss, 0, sizeof(double), st);
  loss_kernel<<<blocks(P), 256, 0, st>>>(w.y, t, P, net->t_mean, net->t_scale, w.dy, w.loss);
  // head: g_w3 = H2^T dy, g_b3 = sum dy, dZ2 = dy w3 * 1[Z2 > 0]
  gemv_t_kernel<<<(h + 255) / 256, 256, 0, st>>>(w.H2, w.dy, P, h, bf, w.g + o.W3);
  sum_kernel<<<1, 1024, 0, st>>>(w.dy, P, w.g + o.b3);
  outer_mask_kernel<<<blocks(P * h), 256, 0, st>>>(w.dy, prm + o.W3, w.Z2, P, h, bf, w.dZ2);
  // g_W2[i][j] = sum_p dZ2[p][i] H1[p][j] ; g_b2 = colsum dZ2
  gemm(st, h, h, (int)P, w.dZ2, 1, h, w.H1, h, 1, w.g + o.W2, h, nullptr, 0, bf);
  colsum_kernel<<<(h + 255) / 256, 256, 0, st>>>(w.dZ2, P, h, w.g + o.b2);
  // dZ1 = (dZ2 W2) * 1[Z1 > 0]
  gemm(st, (int)P, h, h, w.dZ2, h, 1, prm + o.W2, h, 1, w.dZ1, h, nullptr, 0, bf);
  mask_kernel<<<blocks(P * h), 256, 0, st>>>(w.dZ1, w.Z1, P * h);
  // g_W1[i][j] = sum_p dZ1[p][i] F[p][j] ; g_b1 = colsum dZ1
  gemm(st, h, in, (int)P, w.dZ1, 1, h, w.F, in, 1, w.g + o.W1, in, nullptr, 0, bf);
  colsum_kernel<<<(h + 255) / 256, 256, 0, st>>>(w.dZ1, P, h, w.g + o.b1);
}

struct Inputs {
  const double *Xa = nullptr, *Xb = nullptr, *t = nullptr;
  const int32_t* pairs = nullptr;
  void* owned[4] = {nullptr, nullptr, nullptr, nullptr};
  void release(cudaStream_t st) {
    for (void* p : owned)
      if (p) cudaFreeAsync(p, st);
  }
};

qk_status stage_inputs(Inputs& in, const double* Xa, int64_t Na, const double* Xb, int64_t Nb, int n,
                       const int32_t* pairs, int64_t P, const double* t, cudaStream_t st) {
  const void* d = nullptr;
  qk_status rc = to_device(Xa, sizeof(double) * Na * n, st, &d, &in.owned[0]);
  if (rc != QK_OK) return rc;
  in.Xa = (const double*)d;
  rc = to_device(Xb, sizeof(double) * Nb * n, st, &d, &in.owned[1]);
  if (rc != QK_OK) return rc;
  in.Xb = (const double*)d;
  if (pairs) {
    rc = to_device(pairs, sizeof(int32_t) * 2 * P, st, &d, &in.owned[2]);
    if (rc != QK_OK) return rc;
    in.pairs = (const int32_t*)d;
  }
  if (t) {
    rc = to_device(t, sizeof(double) * P, st, &d, &in.owned[3]);
    if (rc != QK_OK) return rc;
    in.t = (const double*)d;
  }
  return QK_OK;
}

qk_status check_net(const qk_surrogate* net, int n, const char* who) {
  if (!net) return fail(QK_ERR_INVALID_ARG, std::string(who) + ": NULL net");
  if (net->in_dim != 2 * n) return fail(QK_ERR_INVALID_ARG, std::string(who) + ": in_dim must equal 2n");
  return QK_OK;
}

qk_status check_pairs_host(const int32_t* pairs, int64_t P, int64_t Na, int64_t Nb, cudaStream_t st,
                           const char* who) {
  std::vector<int32_t> hp;
  const int32_t* src = pairs;
  if (is_device_ptr(pairs)) {
    hp.resize(2 * P);
    QK_CUDA(cudaMemcpyAsync(hp.data(), pairs, sizeof(int32_t) * 2 * P, cudaMemcpyDeviceToHost, st));
    QK_CUDA(cudaStreamSynchronize(st));
    src = hp.data();
  }
  for (int64_t p = 0; p < P; ++p)
    if (src[2 * p] < 0 || src[2 * p] >= Na || src[2 * p + 1] < 0 || src[2 * p + 1] >= Nb)
      return fail(QK_ERR_INVALID_ARG, std::string(who) + ": pair index out of range");
  return QK_OK;
}

constexpr int64_t kChunk = 1 << 17;  // pairs per forward chunk

// standardised predictions for P pairs into d_y (float, device)
qk_status predict_std(const qk_surrogate* net, const Inputs& in, int n, int64_t P, float* d_y, cudaStream_t st) {
  Work w;
  qk_status rc = alloc_work(w, net, std::min(P, kChunk), false, st);
  if (rc != QK_OK) return rc;
  for (int64_t p0 = 0; p0 < P; p0 += kChunk) {
    const int64_t cnt = std::min(kChunk, P - p0);
    features_kernel<<<blocks(cnt * n), 256, 0, st>>>(in.Xa, in.Xb, in.pairs + 2 * p0, cnt, n, w.F);
    forward(net, w, cnt, st);
    cudaMemcpyAsync(d_y + p0, w.y, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, st);
  }
  cudaError_t e = cudaGetLastError();
  w.release(st);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate forward");
  return QK_OK;
}

}  // namespace

qk_status gram_pairs_exact(qk_prec prec, const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                           int64_t P, double* dK, cudaStream_t st);

}  // namespace qk

using namespace qk;

extern "C" qk_status qk_surrogate_create(int32_t in_dim, int32_t hidden, uint64_t seed, qk_surrogate** out) {
  if (!out) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_create: out is NULL");
  if (in_dim < 4 || in_dim > 4096 || (in_dim & 1)) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_create: in_dim must be even, in [4, 4096]");
  if (hidden < 16 || hidden > 1024 || hidden % 16) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_create: hidden must be a multiple of 16 in [16, 1024]");
  qk_surrogate* net = new qk_surrogate();
  cudaGetDevice(&net->device);
  net->in_dim = in_dim;
  net->hidden = hidden;
  const Off o = offsets(in_dim, hidden);
  net->n_params = o.total;
  cudaError_t e = cudaMalloc(&net->d_params, sizeof(float) * o.total);
  if (e == cudaSuccess) e = cudaMalloc(&net->d_m, sizeof(float) * o.total);
  if (e == cudaSuccess) e = cudaMalloc(&net->d_v, sizeof(float) * o.total);
  if (e != cudaSuccess) {
    cudaFree(net->d_params);
    cudaFree(net->d_m);
    cudaFree(net->d_v);
    delete net;
    return cuda_fail(e, "qk_surrogate_create");
  }
  cudaMemset(net->d_params, 0, sizeof(float) * o.total);
  cudaMemset(net->d_m, 0, sizeof(float) * o.total);
  cudaMemset(net->d_v, 0, sizeof(float) * o.total);
  // He-uniform: limit sqrt(6 / fan_in)
  init_kernel<<<blocks((int64_t)hidden * in_dim), 256>>>(net->d_params + o.W1, (int64_t)hidden * in_dim,
                                                         (float)std::sqrt(6.0 / in_dim), seed, o.W1);
  init_kernel<<<blocks((int64_t)hidden * hidden), 256>>>(net->d_params + o.W2, (int64_t)hidden * hidden,
                                                         (float)std::sqrt(6.0 / hidden), seed, o.W2);
  init_kernel<<<blocks(hidden), 256>>>(net->d_params + o.W3, hidden, (float)std::sqrt(6.0 / hidden), seed, o.W3);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    qk_surrogate_free(net);
    return cuda_fail(e, "qk_surrogate_create init");
  }
  *out = net;
  return QK_OK;
}

extern "C" qk_status qk_surrogate_free(qk_surrogate* net) {
  if (!net) return QK_OK;
  cudaFree(net->d_params);
  cudaFree(net->d_m);
  cudaFree(net->d_v);
  delete net;
  return QK_OK;
}

extern "C" int64_t qk_surrogate_param_count(const qk_surrogate* net) { return net ? net->n_params : 0; }

extern "C" qk_status qk_surrogate_get_params(const qk_surrogate* net, float* params) {
  if (!net || !params) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_get_params: NULL argument");
  QK_CUDA(cudaMemcpy(params, net->d_params, sizeof(float) * net->n_params, cudaMemcpyDefault));
  return QK_OK;
}

extern "C" qk_status qk_surrogate_set_params(qk_surrogate* net, const float* params) {
  if (!net || !params) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_set_params: NULL argument");
  QK_CUDA(cudaMemcpy(net->d_params, params, sizeof(float) * net->n_params, cudaMemcpyDefault));
  cudaMemset(net->d_m, 0, sizeof(float) * net->n_params);
  cudaMemset(net->d_v, 0, sizeof(float) * net->n_params);
  net->step = 0;
  return QK_OK;
}

extern "C" qk_status qk_surrogate_set_target_scale(qk_surrogate* net, double mean, double scale) {
  if (!net || !(scale > 0.0) || !std::isfinite(mean)) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_set_target_scale: bad arguments");
  net->t_mean = mean;
  net->t_scale = scale;
  return QK_OK;
}

extern "C" qk_status qk_surrogate_set_bf16(qk_surrogate* net, int32_t on) {
  if (!net) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_set_bf16: NULL net");
  net->bf16 = on ? 1 : 0;
  return QK_OK;
}

extern "C" qk_status qk_surrogate_loss_grad(qk_surrogate* net, const double* Xa, int64_t Na, const double* Xb,
                                            int64_t Nb, int32_t n, const int32_t* pairs, const double* target,
                                            int64_t P, float* grads, double* loss, void* stream) {
  qk_status rc = check_net(net, n, "qk_surrogate_loss_grad");
  if (rc != QK_OK) return rc;
  if (!Xa || !Xb || !pairs || !target || P < 1 || P > kChunk)
    return fail(QK_ERR_INVALID_ARG, "qk_surrogate_loss_grad: bad arguments (1 <= P <= 131072)");
  cudaStream_t st = (cudaStream_t)stream;
  rc = check_pairs_host(pairs, P, Na, Nb, st, "qk_surrogate_loss_grad");
  if (rc != QK_OK) return rc;
  Inputs in;
  rc = stage_inputs(in, Xa, Na, Xb, Nb, n, pairs, P, target, st);
  if (rc != QK_OK) {
    in.release(st);
    return rc;
  }
  Work w;
  rc = alloc_work(w, net, P, true, st);
  if (rc == QK_OK) {
    features_kernel<<<blocks(P * n), 256, 0, st>>>(in.Xa, in.Xb, in.pairs, P, n, w.F);
    forward(net, w, P, st);
    backward(net, w, P, in.t, st);
    if (grads) cudaMemcpyAsync(grads, w.g, sizeof(float) * net->n_params, cudaMemcpyDefault, st);
    double hl = 0.0;
    cudaMemcpyAsync(&hl, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_surrogate_loss_grad");
    if (loss) *loss = hl;
  }
  w.release(st);
  in.release(st);
  cudaStreamSynchronize(st);
  if (rc == QK_OK) rc = gemm_status(st, "qk_surrogate_loss_grad");
  return rc;
}

extern "C" qk_status qk_surrogate_train(qk_surrogate* net, const double* Xa, int64_t Na, const double* Xb,
                                        int64_t Nb, int32_t n, const int32_t* pairs, const double* target,
                                        int64_t P, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                        void* stream, double* loss_out) {
  qk_status rc = check_net(net, n, "qk_surrogate_train");
  if (rc != QK_OK) return rc;
  if (!Xa || !Xb || !pairs || !target || P < 1 || epochs < 1 || batch < 1 || batch > kChunk || !(lr > 0.f))
    return fail(QK_ERR_INVALID_ARG, "qk_surrogate_train: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  rc = check_pairs_host(pairs, P, Na, Nb, st, "qk_surrogate_train");
  if (rc != QK_OK) return rc;
  // shuffled copies of the pair list and targets per epoch (host permutation)
  std::vector<int32_t> hp(2 * P);
  std::vector<double> ht(P);
  QK_CUDA(cudaMemcpy(hp.data(), pairs, sizeof(int32_t) * 2 * P, cudaMemcpyDefault));
  QK_CUDA(cudaMemcpy(ht.data(), target, sizeof(double) * P, cudaMemcpyDefault));
  Inputs in;
  rc = stage_inputs(in, Xa, Na, Xb, Nb, n, nullptr, 0, nullptr, st);
  if (rc != QK_OK) {
    in.release(st);
    return rc;
  }
  int32_t* dp = nullptr;
  double* dt = nullptr;
  Work w;
  cudaError_t e = cudaMallocAsync(&dp, sizeof(int32_t) * 2 * P, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dt, sizeof(double) * P, st);
  if (e != cudaSuccess) rc = cuda_fail(e, "qk_surrogate_train buffers");
  if (rc == QK_OK) rc = alloc_work(w, net, batch, true, st);
  std::vector<int64_t> perm(P);
  std::vector<int32_t> sp(2 * P);
  std::vector<double> stt(P);
  double last = 0.0;
  for (int ep = 0; ep < epochs && rc == QK_OK; ++ep) {
    for (int64_t i = 0; i < P; ++i) perm[i] = i;
    for (int64_t i = P - 1; i > 0; --i) {  // Fisher-Yates with a counter-based generator
      const int64_t j = (int64_t)(splitmix64(seed * 0x9E3779B97F4A7C15ull + ep * 1000003ull + i) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    for (int64_t i = 0; i < P; ++i) {
      sp[2 * i] = hp[2 * perm[i]];
      sp[2 * i + 1] = hp[2 * perm[i] + 1];
      stt[i] = ht[perm[i]];
    }
    cudaMemcpyAsync(dp, sp.data(), sizeof(int32_t) * 2 * P, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dt, stt.data(), sizeof(double) * P, cudaMemcpyHostToDevice, st);
    // the host buffers are reused next epoch: wait for the copies
    cudaStreamSynchronize(st);
    for (int64_t p0 = 0; p0 < P; p0 += batch) {
      const int64_t cnt = std::min<int64_t>(batch, P - p0);
      features_kernel<<<blocks(cnt * n), 256, 0, st>>>(in.Xa, in.Xb, dp + 2 * p0, cnt, n, w.F);
      forward(net, w, cnt, st);
      backward(net, w, cnt, dt + p0, st);
      ++net->step;
      const float c1 = 1.f - std::pow(0.9f, (float)net->step), c2 = 1.f - std::pow(0.999f, (float)net->step);
      adam_kernel<<<blocks(net->n_params), 256, 0, st>>>(net->d_params, w.g, net->d_m, net->d_v, net->n_params, lr,
                                                         0.9f, 0.999f, 1e-8f, c1, c2);
      // last epoch's loss: batch means weighted by batch size
      double bl = 0.0;
      if (ep == epochs - 1) {
        cudaMemcpyAsync(&bl, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        last += bl * (double)cnt;
      }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_surrogate_train");
  }
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (rc == QK_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "qk_surrogate_train");
  if (loss_out) *loss_out = last / (double)P;
  w.release(st);
  if (dp) cudaFreeAsync(dp, st);
  if (dt) cudaFreeAsync(dt, st);
  in.release(st);
  cudaStreamSynchronize(st);
  if (rc == QK_OK) rc = gemm_status(st, "qk_surrogate_train");
  return rc;
}

extern "C" qk_status qk_surrogate_predict(const qk_surrogate* net, const double* Xa, int64_t Na, const double* Xb,
                                          int64_t Nb, int32_t n, const int32_t* pairs, int64_t P, double* y,
                                          void* stream) {
  qk_status rc = check_net(net, n, "qk_surrogate_predict");
  if (rc != QK_OK) return rc;
  if (!Xa || !Xb || !pairs || !y || P < 1) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_predict: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  rc = check_pairs_host(pairs, P, Na, Nb, st, "qk_surrogate_predict");
  if (rc != QK_OK) return rc;
  Inputs in;
  rc = stage_inputs(in, Xa, Na, Xb, Nb, n, pairs, P, nullptr, st);
  float* dy = nullptr;
  if (rc == QK_OK) {
    cudaError_t e = cudaMallocAsync(&dy, sizeof(float) * P, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_surrogate_predict");
  }
  if (rc == QK_OK) rc = predict_std(net, in, n, P, dy, st);
  if (rc == QK_OK) {
    std::vector<float> hy(P);
    cudaMemcpyAsync(hy.data(), dy, sizeof(float) * P, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    std::vector<double> out(P);
    for (int64_t p = 0; p < P; ++p) out[p] = (double)hy[p] * net->t_scale + net->t_mean;
    cudaError_t e = cudaMemcpy(y, out.data(), sizeof(double) * P, cudaMemcpyDefault);
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_surrogate_predict copy");
  }
  if (dy) cudaFreeAsync(dy, st);
  in.release(st);
  cudaStreamSynchronize(st);
  if (rc == QK_OK) rc = gemm_status(st, "qk_surrogate_predict");
  return rc;
}

extern "C" qk_status qk_surrogate_calibrate(qk_surrogate* net, const double* Xa, int64_t Na, const double* Xb,
                                            int64_t Nb, int32_t n, const int32_t* pairs, const double* truth,
                                            int64_t P, double alpha, int32_t n_bins, void* stream) {
  qk_status rc = check_net(net, n, "qk_surrogate_calibrate");
  if (rc != QK_OK) return rc;
  if (!truth || P < 1 || !(alpha > 0.0 && alpha < 1.0) || n_bins < 1 || n_bins > 1024)
    return fail(QK_ERR_INVALID_ARG, "qk_surrogate_calibrate: bad arguments");
  std::vector<double> pred(P), tr(P);
  rc = qk_surrogate_predict(net, Xa, Na, Xb, Nb, n, pairs, P, pred.data(), stream);
  if (rc != QK_OK) return rc;
  QK_CUDA(cudaMemcpy(tr.data(), truth, sizeof(double) * P, cudaMemcpyDefault));
  // equal-count bins of the predicted value
  std::vector<double> sorted = pred;
  std::sort(sorted.begin(), sorted.end());
  std::vector<double> edges(n_bins + 1);
  edges[0] = -INFINITY;
  edges[n_bins] = INFINITY;
  for (int b = 1; b < n_bins; ++b) edges[b] = sorted[(size_t)((double)b * P / n_bins)];
  std::vector<std::vector<double>> res(n_bins);
  for (int64_t p = 0; p < P; ++p) {
    int b = (int)(std::upper_bound(edges.begin() + 1, edges.end() - 1, pred[p]) - (edges.begin() + 1));
    res[b].push_back(std::fabs(pred[p] - tr[p]));
  }
  std::vector<double> bounds(n_bins, INFINITY);
  for (int b = 0; b < n_bins; ++b) {
    auto& r = res[b];
    std::sort(r.begin(), r.end());
    const int64_t m = (int64_t)r.size();
    const int64_t q = (int64_t)std::ceil((m + 1) * (1.0 - alpha));
    if (m > 0 && q <= m) bounds[b] = r[q - 1];
  }
  net->edges = edges;
  net->bounds = bounds;
  net->calibrated = true;
  return QK_OK;
}

extern "C" qk_status qk_surrogate_bins(const qk_surrogate* net, int32_t* n_bins, double* edges, double* bounds) {
  if (!net || !net->calibrated) return fail(QK_ERR_INVALID_ARG, "qk_surrogate_bins: net is not calibrated");
  if (n_bins) *n_bins = (int32_t)net->bounds.size();
  if (edges) std::copy(net->edges.begin(), net->edges.end(), edges);
  if (bounds) std::copy(net->bounds.begin(), net->bounds.end(), bounds);
  return QK_OK;
}

extern "C" qk_status qk_gram_surrogate(const qk_surrogate* net, const qk_mps_batch* A, const qk_mps_batch* B,
                                       const double* Xa, const double* Xb, double tol, double* K, int64_t ldk,
                                       uint8_t* accepted, qk_prec prec, void* stream, int64_t* n_accepted) {
  if (!net || !A || !B || !Xa || !Xb || !K) return fail(QK_ERR_INVALID_ARG, "qk_gram_surrogate: NULL argument");
  if (!net->calibrated) return fail(QK_ERR_INVALID_ARG, "qk_gram_surrogate: net is not calibrated");
  if (A->n != B->n || net->in_dim != 2 * A->n) return fail(QK_ERR_INVALID_ARG, "qk_gram_surrogate: shape mismatch");
  if (ldk < B->N || !(tol >= 0.0)) return fail(QK_ERR_INVALID_ARG, "qk_gram_surrogate: bad ldk or tol");
  if (prec != QK_PREC_FP64 && prec != QK_PREC_SPLIT_BF16 && prec != QK_PREC_SPLIT_BF16X3)
    return fail(QK_ERR_INVALID_ARG, "qk_gram_surrogate: bad precision");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = A->n;
  const int NB = (int)B->N;
  const int64_t total = A->N * B->N;
  Inputs in;
  qk_status rc = stage_inputs(in, Xa, A->N, Xb, B->N, n, nullptr, 0, nullptr, st);
  const int nb = (int)net->bounds.size();
  double *d_edges = nullptr, *d_bounds = nullptr, *d_Kc = nullptr, *d_ex = nullptr, *dK = K;
  int32_t *d_pairs = nullptr, *d_rej = nullptr, *d_rp = nullptr;
  uint8_t *d_acc = nullptr;
  float* d_y = nullptr;
  unsigned long long* d_nrej = nullptr;
  void* owned_k = nullptr;
  const bool host_k = !is_device_ptr(K);
  const int64_t chunk = std::min<int64_t>(total, (int64_t)1 << 21);
  auto M = [&](void** p, size_t b) {
    if (rc != QK_OK) return;
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(b, 16), st);
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_gram_surrogate buffers");
  };
  M((void**)&d_edges, sizeof(double) * (nb + 1));
  M((void**)&d_bounds, sizeof(double) * nb);
  M((void**)&d_Kc, sizeof(double) * chunk);
  M((void**)&d_ex, sizeof(double) * chunk);
  M((void**)&d_pairs, sizeof(int32_t) * 2 * chunk);
  M((void**)&d_rej, sizeof(int32_t) * chunk);
  M((void**)&d_rp, sizeof(int32_t) * 2 * chunk);
  M((void**)&d_acc, total);
  M((void**)&d_y, sizeof(float) * chunk);
  M((void**)&d_nrej, sizeof(unsigned long long));
  if (host_k) {
    M(&owned_k, sizeof(double) * (size_t)((A->N - 1) * ldk + B->N));
    dK = (double*)owned_k;
  }
  if (rc == QK_OK) {
    cudaMemcpyAsync(d_edges, net->edges.data(), sizeof(double) * (nb + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_bounds, net->bounds.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st);
  }
  int64_t n_acc = 0;
  for (int64_t i0 = 0; i0 < total && rc == QK_OK; i0 += chunk) {
    const int64_t cnt = std::min(chunk, total - i0);
    block_pairs_kernel<<<blocks(cnt), 256, 0, st>>>(i0, cnt, NB, d_pairs);
    Inputs ci = in;
    for (auto& o : ci.owned) o = nullptr;
    ci.pairs = d_pairs;
    rc = predict_std(net, ci, n, cnt, d_y, st);
    if (rc != QK_OK) break;
    cudaMemsetAsync(d_nrej, 0, sizeof(unsigned long long), st);
    accept_kernel<<<blocks(cnt), 256, 0, st>>>(d_y, cnt, net->t_mean, net->t_scale, d_edges, d_bounds, nb, tol,
                                               d_Kc, d_acc + i0, d_nrej, d_rej);
    unsigned long long nrej = 0;
    cudaMemcpyAsync(&nrej, d_nrej, sizeof(nrej), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    n_acc += cnt - (int64_t)nrej;
    copy_block_kernel<<<blocks(cnt), 256, 0, st>>>(d_Kc, i0, cnt, NB, dK, ldk);
    if (nrej > 0) {
      gather_pairs_kernel<<<blocks(nrej), 256, 0, st>>>(d_pairs, d_rej, (int64_t)nrej, d_rp);
      rc = gram_pairs_exact(prec, A, B, d_rp, (int64_t)nrej, d_ex, st);
      if (rc != QK_OK) break;
      scatter_block_kernel<<<blocks(nrej), 256, 0, st>>>(d_ex, d_rej, (int64_t)nrej, i0, NB, dK, ldk);
    }
  }
  if (rc == QK_OK && host_k) {
    cudaError_t e = cudaMemcpyAsync(K, dK, sizeof(double) * (size_t)((A->N - 1) * ldk + B->N), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_gram_surrogate K");
  }
  if (rc == QK_OK && accepted) {
    cudaError_t e = cudaMemcpyAsync(accepted, d_acc, total, cudaMemcpyDefault, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "qk_gram_surrogate accepted");
  }
  cudaStreamSynchronize(st);
  for (void* p : {(void*)d_edges, (void*)d_bounds, (void*)d_Kc, (void*)d_ex, (void*)d_pairs, (void*)d_rej, (void*)d_rp,
                  (void*)d_acc, (void*)d_y, (void*)d_nrej, owned_k})
    if (p) cudaFreeAsync(p, st);
  in.release(st);
  cudaStreamSynchronize(st);
  if (rc == QK_OK && n_accepted) *n_accepted = n_acc;
  if (rc == QK_OK) rc = gemm_status(st, "qk_gram_surrogate");
  return rc;
}
