// Self-overlaps <psi|psi> of stored (left-canonical) states without FP64
// arithmetic on the overlap sweep.
//
// For a left-canonical MPS the transfer sweep of a state with itself keeps
// the environment at the identity: with E_k = I + F_k,
//   E_{k+1} = sum_s A_k[s]^H E_k A_k[s] = I + G_k + sum_s A_k[s]^H F_k A_k[s],
//   G_k = sum_s A_k[s]^H A_k[s] - I          (the site's isometry defect),
// so F_{k+1} = G_k + sum_s A_k[s]^H F_k A_k[s], F_0 = 0, <psi|psi> = 1 + F_n.
// After complex64 rounding the defects are ~1e-7, so F stays small:
//   * G_k is formed from exact FP32 products (two-product via FMA) summed in
//     double-float arithmetic (Dekker 1971; Knuth two-sum), then rounded to
//     FP32 after the identity is subtracted -- its absolute error is ~1e-14;
//   * the recursion for F only needs relative accuracy ~1e-5 and runs in FP32.
// The resulting K_ii = |1 + F_n|^2 is within ~1e-10 of the FP64 sweep.  A
// state whose largest defect exceeds kDefectMax (not left-canonical) is
// flagged and its self-overlap is left to the FP64 kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "qk_internal.h"

namespace qk {

qk_status overlap_fp64(const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                       int64_t P, double* dK, int64_t ldk, bool sym, cudaStream_t st,
                       int ctas_per_sm = 4);

namespace {

constexpr int kThreads = 256;
constexpr float kDefectMax = 1e-4f;

struct DiagArgs {
  const uint64_t* site_ptr;  // [N][n], complex64 sites A[q][a][b]
  const int32_t* dims;       // [N][n+1]
  int n;
  int64_t N;
  double* K;
  int64_t ldk;
  int32_t* flag;             // [N]: 1 = not left-canonical, left to FP64
  float2* scratch;           // per CTA: F, Fn (cap each), T (2 cap)
  int64_t cap;
  int* queue;
};

// The error-free transformations below use the _rn intrinsics so that the
// compiler cannot contract a product into a neighbouring add.
// two-sum (Knuth): s + e == a + b exactly
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += p + q
__device__ inline void df_add(float& hi, float& lo, float p, float q) {
  float s, e;
  two_sum(hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, q));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// (hi, lo) += x * y, the product split exactly by FMA (Dekker's two-product)
__device__ inline void df_mac(float& hi, float& lo, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float q = fmaf(x, y, -p);
  df_add(hi, lo, p, q);
}

__global__ void __launch_bounds__(kThreads) diag_kernel(DiagArgs a) {
  __shared__ int s_state;
  __shared__ float s_defect;
  float2* F = a.scratch + (int64_t)blockIdx.x * 4 * a.cap;
  float2* Fn = F + a.cap;
  float2* T = Fn + a.cap;
  const int n = a.n;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_state = atomicAdd(a.queue, 1);
      s_defect = 0.f;
    }
    __syncthreads();
    const int64_t st = s_state;
    if (st >= a.N) break;
    const int32_t* dm = a.dims + st * (n + 1);
    if (threadIdx.x == 0) F[0] = make_float2(0.f, 0.f);
    __syncthreads();
    float local_defect = 0.f;
    for (int k = 0; k < n; ++k) {
      const int c0 = dm[k], c1 = dm[k + 1];
      const float2* A = reinterpret_cast<const float2*>(a.site_ptr[st * n + k]);
      // T[s][x][y] = sum_c F[x][c] A[s][c][y]   (FP32)
      for (int o = threadIdx.x; o < 2 * c0 * c1; o += kThreads) {
        const int s = o / (c0 * c1), rem = o % (c0 * c1), x = rem / c1, y = rem % c1;
        float re = 0.f, im = 0.f;
        for (int c = 0; c < c0; ++c) {
          const float2 f = F[x * c0 + c], v = A[(s * c0 + c) * c1 + y];
          re = fmaf(f.x, v.x, fmaf(-f.y, v.y, re));
          im = fmaf(f.x, v.y, fmaf(f.y, v.x, im));
        }
        T[o] = make_float2(re, im);
      }
      __syncthreads();
      // Fn[u][v] = G[u][v] + sum_s sum_x conj(A[s][x][u]) T[s][x][v]
      for (int o = threadIdx.x; o < c1 * c1; o += kThreads) {
        const int u = o / c1, v = o % c1;
        float gr = 0.f, grl = 0.f, gi = 0.f, gil = 0.f;  // double-float G
        float tr = 0.f, ti = 0.f;
        for (int s = 0; s < 2; ++s)
          for (int x = 0; x < c0; ++x) {
            const float2 au = A[(s * c0 + x) * c1 + u], av = A[(s * c0 + x) * c1 + v];
            // conj(au) * av
            df_mac(gr, grl, au.x, av.x);
            df_mac(gr, grl, au.y, av.y);
            df_mac(gi, gil, au.x, av.y);
            df_mac(gi, gil, -au.y, av.x);
            const float2 t = T[(s * c0 + x) * c1 + v];
            tr = fmaf(au.x, t.x, fmaf(au.y, t.y, tr));
            ti = fmaf(au.x, t.y, fmaf(-au.y, t.x, ti));
          }
        if (u == v) gr = __fsub_rn(gr, 1.f);  // exact (Sterbenz) when gr is in [0.5, 2]
        const float g_re = __fadd_rn(gr, grl), g_im = __fadd_rn(gi, gil);
        local_defect = fmaxf(local_defect, fmaxf(fabsf(g_re), fabsf(g_im)));
        Fn[o] = make_float2(g_re + tr, g_im + ti);
      }
      __syncthreads();
      float2* t = F;
      F = Fn;
      Fn = t;
    }
    // block max of the defect
    for (int off = 16; off > 0; off >>= 1) local_defect = fmaxf(local_defect, __shfl_xor_sync(0xffffffffu, local_defect, off));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(&s_defect), __float_as_int(local_defect));
    __syncthreads();
    if (threadIdx.x == 0) {
      const double zr = 1.0 + (double)F[0].x, zi = (double)F[0].y;
      a.K[st * a.ldk + st] = zr * zr + zi * zi;
      a.flag[st] = (s_defect > kDefectMax || !(s_defect == s_defect)) ? 1 : 0;
    }
    // the buffers swapped an odd or even number of times: restore the base
    F = a.scratch + (int64_t)blockIdx.x * 4 * a.cap;
    Fn = F + a.cap;
  }
}

}  // namespace

// A second, non-blocking stream per device for the self-overlaps, so that
// they run beside the FP64 re-evaluation of a split Gram (both are a few
// long-running CTAs); created on first use.
cudaStream_t side_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    streams[dev] = nullptr;
    cudaGetLastError();
  }
  return streams[dev];
}

// Launches diag_kernel for every state of a complex64 batch on `st` (no
// synchronisation); diag_finish reads the flags once `st` is done.
qk_status diag_launch(const qk_mps_batch* A, double* dK, int64_t ldk, cudaStream_t st, DiagPending* d) {
  d->st = st;
  d->flag = nullptr;
  d->N = A->N;
  if (A->N == 0 || A->store != QK_STORE_C64) return QK_OK;
  int dev = 0, sms = 0;
  QK_CUDA(cudaGetDevice(&dev));
  QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t N = A->N;
  const int64_t cap = (int64_t)A->chi_cap * A->chi_cap;
  const int64_t ctas = std::min<int64_t>((int64_t)4 * sms, N);
  float2* scratch = nullptr;
  int* queue = nullptr;
  QK_CUDA(cudaMallocAsync(&scratch, sizeof(float2) * 4 * cap * ctas, st));
  QK_CUDA(cudaMallocAsync(&queue, sizeof(int), st));
  QK_CUDA(cudaMallocAsync(&d->flag, sizeof(int32_t) * N, st));
  QK_CUDA(cudaMemsetAsync(queue, 0, sizeof(int), st));
  DiagArgs a;
  a.site_ptr = A->d_site_ptr;
  a.dims = A->d_dims;
  a.n = A->n;
  a.N = N;
  a.K = dK;
  a.ldk = ldk;
  a.flag = d->flag;
  a.scratch = scratch;
  a.cap = cap;
  a.queue = queue;
  timer_mark(false, st);
  diag_kernel<<<(int)ctas, kThreads, 0, st>>>(a);
  timer_mark(true, st);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(queue, st);
  if (e != cudaSuccess) return cuda_fail(e, "diag_kernel");
  return QK_OK;
}

// Waits for the launch, then re-does by the FP64 sweep (on st_fp64) every
// state that is not left-canonical, or every state of a complex128 batch.
qk_status diag_finish(const qk_mps_batch* A, double* dK, int64_t ldk, DiagPending* d, cudaStream_t st_fp64,
                      int64_t* n_fp64) {
  if (n_fp64) *n_fp64 = 0;
  const int64_t N = A->N;
  if (N == 0) return QK_OK;
  std::vector<int32_t> fallback;
  if (A->store != QK_STORE_C64) {
    for (int64_t i = 0; i < N; ++i) fallback.push_back((int32_t)i);
  } else {
    std::vector<int32_t> hf(N);
    cudaError_t e = cudaMemcpyAsync(hf.data(), d->flag, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, d->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->st);
    cudaFreeAsync(d->flag, d->st);
    d->flag = nullptr;
    if (e != cudaSuccess) return cuda_fail(e, "diag_kernel");
    for (int64_t i = 0; i < N; ++i)
      if (hf[i]) fallback.push_back((int32_t)i);
  }
  if (!fallback.empty()) {
    std::vector<int32_t> hp(2 * fallback.size());
    for (size_t i = 0; i < fallback.size(); ++i) hp[2 * i] = hp[2 * i + 1] = fallback[i];
    int32_t* dp = nullptr;
    QK_CUDA(cudaMallocAsync(&dp, sizeof(int32_t) * hp.size(), st_fp64));
    QK_CUDA(cudaMemcpyAsync(dp, hp.data(), sizeof(int32_t) * hp.size(), cudaMemcpyHostToDevice, st_fp64));
    qk_status rc = overlap_fp64(A, A, dp, (int64_t)fallback.size(), dK, ldk, false, st_fp64);
    cudaFreeAsync(dp, st_fp64);
    if (rc != QK_OK) return rc;
    if (n_fp64) *n_fp64 = (int64_t)fallback.size();
  }
  return QK_OK;
}

// K[i*ldk + i] for every state of a complex64 batch; states that are not
// left-canonical are re-done by the FP64 sweep.  Returns the FP64 count.
qk_status diag_self_overlaps(const qk_mps_batch* A, double* dK, int64_t ldk, cudaStream_t st,
                             int64_t* n_fp64) {
  DiagPending d;
  qk_status rc = diag_launch(A, dK, ldk, st, &d);
  if (rc != QK_OK) return rc;
  return diag_finish(A, dK, ldk, &d, st, n_fp64);
}

}  // namespace qk
