// Plain FP64 transfer sweep (Fig. 2) on the CUDA cores: one CTA per pair,
// persistent over a pair list.  Per site k the environment E (chi^a_k x
// chi^b_k, FP64 complex) absorbs the site pair in the cheaper of the two
// orders:
//   (a) T_s = E B_k[s],            E' = sum_s A_k[s]^H T_s
//   (b) F_s = A_k[s]^H E,          E' = sum_s F_s B_k[s]
// E and the intermediates live in a per-CTA scratch slice (L1/L2 resident).
// The storage precision of the states (complex64 or complex128) is read and
// widened to FP64; every product and sum is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "qk_internal.h"

namespace qk {
namespace {

constexpr int kThreads = 256;

template <typename C>
__device__ __forceinline__ double2 ld(const C* p, int64_t i);
template <>
__device__ __forceinline__ double2 ld<double2>(const double2* p, int64_t i) {
  return p[i];
}
template <>
__device__ __forceinline__ double2 ld<float2>(const float2* p, int64_t i) {
  float2 v = p[i];
  return make_double2((double)v.x, (double)v.y);
}

struct PairArgs {
  const uint64_t* a_ptr;   // [NA][n] site addresses of A
  const int32_t* a_dims;   // [NA][n+1]
  const uint64_t* b_ptr;
  const int32_t* b_dims;
  int n;
  const int32_t* pairs;    // [P][2]
  int64_t P;
  double* K;               // output
  int64_t ldk;             // >0: K[i*ldk + j] (and mirror if sym); 0: K[p]
  int sym;
  double2* scratch;        // per CTA 3 * cap
  int64_t cap;
  unsigned long long* queue;  // work counter (64-bit: it runs past P by the CTA count)
};

template <typename C>
__global__ void __launch_bounds__(kThreads) overlap_fp64_kernel(PairArgs a) {
  __shared__ long long s_pair;
  double2* E = a.scratch + (int64_t)blockIdx.x * 3 * a.cap;
  double2* T = E + a.cap;
  double2* E2 = T + a.cap;
  const int n = a.n;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_pair = (long long)atomicAdd(a.queue, 1ull);
    __syncthreads();
    const int64_t pi = s_pair;
    if (pi >= a.P) break;
    const int i = a.pairs[2 * pi], j = a.pairs[2 * pi + 1];
    const uint64_t* pa = a.a_ptr + (int64_t)i * n;
    const uint64_t* pb = a.b_ptr + (int64_t)j * n;
    const int32_t* da = a.a_dims + (int64_t)i * (n + 1);
    const int32_t* db = a.b_dims + (int64_t)j * (n + 1);
    if (threadIdx.x == 0) E[0] = make_double2(1.0, 0.0);
    __syncthreads();
    double2* Ecur = E;
    double2* Enext = E2;
    for (int k = 0; k < n; ++k) {
      const int xa = da[k], ua = da[k + 1], xb = db[k], yb = db[k + 1];
      const C* A = reinterpret_cast<const C*>(pa[k]);
      const C* B = reinterpret_cast<const C*>(pb[k]);
      const double costA = (double)xa * xb * yb + (double)ua * xa * yb;
      const double costB = (double)ua * xa * xb + (double)ua * xb * yb;
      if (costA <= costB) {
        // T[s][x][y] = sum_c E[x][c] B[s][c][y]
        for (int o = threadIdx.x; o < 2 * xa * yb; o += kThreads) {
          int s = o / (xa * yb), rem = o % (xa * yb), x = rem / yb, y = rem % yb;
          const double2* er = Ecur + (int64_t)x * xb;
          const C* bc = B + (int64_t)s * xb * yb + y;
          double re = 0.0, im = 0.0;
          for (int c = 0; c < xb; ++c) {
            double2 e = er[c], b = ld(bc, (int64_t)c * yb);
            re = fma(e.x, b.x, fma(-e.y, b.y, re));
            im = fma(e.x, b.y, fma(e.y, b.x, im));
          }
          T[o] = make_double2(re, im);
        }
        __syncthreads();
        // E'[u][y] = sum_s sum_x conj(A[s][x][u]) T[s][x][y]
        for (int o = threadIdx.x; o < ua * yb; o += kThreads) {
          int u = o / yb, y = o % yb;
          double re = 0.0, im = 0.0;
          for (int s = 0; s < 2; ++s)
            for (int x = 0; x < xa; ++x) {
              double2 av = ld(A, ((int64_t)s * xa + x) * ua + u);
              double2 t = T[((int64_t)s * xa + x) * yb + y];
              re = fma(av.x, t.x, fma(av.y, t.y, re));
              im = fma(av.x, t.y, fma(-av.y, t.x, im));
            }
          Enext[o] = make_double2(re, im);
        }
      } else {
        // F[s][u][c] = sum_x conj(A[s][x][u]) E[x][c]
        for (int o = threadIdx.x; o < 2 * ua * xb; o += kThreads) {
          int s = o / (ua * xb), rem = o % (ua * xb), u = rem / xb, c = rem % xb;
          double re = 0.0, im = 0.0;
          for (int x = 0; x < xa; ++x) {
            double2 av = ld(A, ((int64_t)s * xa + x) * ua + u);
            double2 e = Ecur[(int64_t)x * xb + c];
            re = fma(av.x, e.x, fma(av.y, e.y, re));
            im = fma(av.x, e.y, fma(-av.y, e.x, im));
          }
          T[o] = make_double2(re, im);
        }
        __syncthreads();
        // E'[u][y] = sum_s sum_c F[s][u][c] B[s][c][y]
        for (int o = threadIdx.x; o < ua * yb; o += kThreads) {
          int u = o / yb, y = o % yb;
          double re = 0.0, im = 0.0;
          for (int s = 0; s < 2; ++s)
            for (int c = 0; c < xb; ++c) {
              double2 f = T[((int64_t)s * ua + u) * xb + c];
              double2 b = ld(B, ((int64_t)s * xb + c) * yb + y);
              re = fma(f.x, b.x, fma(-f.y, b.y, re));
              im = fma(f.x, b.y, fma(f.y, b.x, im));
            }
          Enext[o] = make_double2(re, im);
        }
      }
      __syncthreads();
      double2* tmp = Ecur;
      Ecur = Enext;
      Enext = tmp;
    }
    if (threadIdx.x == 0) {
      double2 z = Ecur[0];
      double kv = z.x * z.x + z.y * z.y;
      if (a.ldk > 0) {
        a.K[(int64_t)i * a.ldk + j] = kv;
        if (a.sym) a.K[(int64_t)j * a.ldk + i] = kv;
      } else {
        a.K[pi] = kv;
      }
    }
  }
}

}  // namespace

// Contract the listed pairs in FP64.  ldk > 0 writes K[i*ldk + j] (mirrored
// when sym), ldk == 0 writes K[p].  ctas_per_sm bounds the grid (1 leaves
// room for a concurrent tensor-core kernel on every SM).
qk_status overlap_fp64(const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                       int64_t P, double* dK, int64_t ldk, bool sym, cudaStream_t st,
                       int ctas_per_sm) {
  if (P == 0) return QK_OK;
  int dev = 0, sms = 0;
  QK_CUDA(cudaGetDevice(&dev));
  QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int chi = std::max(A->chi_cap, B->chi_cap);
  int64_t cap = 2LL * chi * chi;
  int64_t ctas = std::min<int64_t>((int64_t)sms * ctas_per_sm, P);
  double2* scratch = nullptr;
  unsigned long long* queue = nullptr;
  QK_CUDA(cudaMallocAsync(&scratch, sizeof(double2) * 3 * cap * ctas, st));
  QK_CUDA(cudaMallocAsync(&queue, sizeof(unsigned long long), st));
  QK_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st));
  PairArgs a;
  a.a_ptr = A->d_site_ptr;
  a.a_dims = A->d_dims;
  a.b_ptr = B->d_site_ptr;
  a.b_dims = B->d_dims;
  a.n = A->n;
  a.pairs = d_pairs;
  a.P = P;
  a.K = dK;
  a.ldk = ldk;
  a.sym = sym ? 1 : 0;
  a.scratch = scratch;
  a.cap = cap;
  a.queue = queue;
  timer_mark(false, st);
  if (A->store == QK_STORE_C64)
    overlap_fp64_kernel<float2><<<(int)ctas, kThreads, 0, st>>>(a);
  else
    overlap_fp64_kernel<double2><<<(int)ctas, kThreads, 0, st>>>(a);
  timer_mark(true, st);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(queue, st);
  if (e != cudaSuccess) return cuda_fail(e, "overlap_fp64_kernel launch");
  return QK_OK;
}

}  // namespace qk

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP64 pair overlaps (qk_gram_pairs_noalloc).
// Its scratch is the file-scope array below instead of cudaMallocAsync
// buffers: one 256-byte control block (work counter) followed by one
// E / T / E' slice per CTA, sized for bond dimensions up to kNoAllocChi and
// kNoAllocCtas resident CTAs (37.7 MB, held by every device that loads the
// library until the process exits).
namespace qk {
namespace {

constexpr int kNoAllocChi = 64;
constexpr int kNoAllocCtas = 96;
constexpr int64_t kNoAllocCap = 2LL * kNoAllocChi * kNoAllocChi;          // double2 per buffer
constexpr int64_t kNoAllocCtl = 16;                                       // double2 = 256 bytes
constexpr int64_t kNoAllocElems = kNoAllocCtl + kNoAllocCtas * 3 * kNoAllocCap;

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocElems];

// Device address of g_noalloc_scratch per device, looked up once per device
// (host code may only use the symbol through cudaGetSymbolAddress).
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDevices] = {};

qk_status noalloc_scratch(int dev, double2** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<double2*>(g_noalloc_ptr[dev]);
  return QK_OK;
}

}  // namespace
}  // namespace qk

extern "C" qk_status qk_gram_pairs_noalloc(const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* pairs,
                                           int64_t P, double* K_out, void* stream) {
  using namespace qk;
  if (!A || !B) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: NULL batch");
  if (A->n != B->n) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: batches differ in n");
  if (A->store != B->store) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: batches differ in storage precision");
  if (P < 0 || P >= ((int64_t)1 << 31)) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: P out of range");
  if (P == 0) return QK_OK;
  if (A->chi_cap > kNoAllocChi || B->chi_cap > kNoAllocChi)
    return fail(QK_ERR_INVALID_ARG,
                "qk_gram_pairs_noalloc: a bond dimension exceeds 64, the limit of the static scratch "
                "(use qk_gram_pairs)");
  if (!pairs || !K_out || !is_device_ptr(pairs) || !is_device_ptr(K_out))
    return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: pairs and K_out must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  QK_CUDA(cudaGetDevice(&dev));
  if (dev != A->device || dev != B->device)
    return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: batches live on another device");
  double2* scratch = nullptr;
  qk_status rc = noalloc_scratch(dev, &scratch);
  if (rc != QK_OK) return rc;
  // index check through a fixed stack buffer (no allocation)
  int32_t chunk[2 * 2048];
  for (int64_t p0 = 0; p0 < P; p0 += 2048) {
    const int64_t cnt = std::min<int64_t>(2048, P - p0);
    QK_CUDA(cudaMemcpyAsync(chunk, pairs + 2 * p0, sizeof(int32_t) * 2 * cnt, cudaMemcpyDeviceToHost, st));
    QK_CUDA(cudaStreamSynchronize(st));
    for (int64_t q = 0; q < cnt; ++q)
      if (chunk[2 * q] < 0 || chunk[2 * q] >= A->N || chunk[2 * q + 1] < 0 || chunk[2 * q + 1] >= B->N)
        return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs_noalloc: pair index out of range");
  }
  int sms = 0;
  QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the work counter starts at zero on every call
  QK_CUDA(cudaMemsetAsync(scratch, 0, sizeof(double2) * kNoAllocCtl, st));
  PairArgs a;
  a.a_ptr = A->d_site_ptr;
  a.a_dims = A->d_dims;
  a.b_ptr = B->d_site_ptr;
  a.b_dims = B->d_dims;
  a.n = A->n;
  a.pairs = pairs;
  a.P = P;
  a.K = K_out;
  a.ldk = 0;
  a.sym = 0;
  a.scratch = scratch + kNoAllocCtl;
  a.cap = kNoAllocCap;
  a.queue = reinterpret_cast<unsigned long long*>(scratch);
  const int ctas = (int)std::min<int64_t>(std::min(kNoAllocCtas, 4 * sms), P);
  if (A->store == QK_STORE_C64)
    overlap_fp64_kernel<float2><<<ctas, kThreads, 0, st>>>(a);
  else
    overlap_fp64_kernel<double2><<<ctas, kThreads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "qk_gram_pairs_noalloc");
  return QK_OK;
}
