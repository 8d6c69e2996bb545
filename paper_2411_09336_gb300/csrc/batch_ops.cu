// Batch utilities: rotated copies of states (a final Z layer), host blobs
// for save/load, and the per-call kernel timings of qk_gram.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "qk_internal.h"

namespace qk {

// ---- per-call timing (CUDA events on the call's stream) -------------------
// Each phase keeps up to kSpans (start, end) event pairs; a phase's time is
// the sum of its spans, so several launches of one phase add up.
constexpr int kSpans = 8;
static thread_local cudaEvent_t g_ev[2][kSpans][2] = {};
static thread_local int g_nspan[2] = {0, 0};
static thread_local bool g_open[2] = {false, false};
static thread_local int g_phase = 0;  // 0: main sweep, 1: refinement
static thread_local double g_prof[3] = {0.0, 0.0, 0.0};

void timer_begin_call() {
  for (int p = 0; p < 2; ++p) {
    g_nspan[p] = 0;
    g_open[p] = false;
  }
  g_phase = 0;
  g_prof[0] = g_prof[1] = g_prof[2] = 0.0;
}
void timer_set_phase(int phase) { g_phase = phase; }
void timer_mark(bool end, cudaStream_t st) {
  const int p = g_phase;
  if (p < 0 || p > 1) return;  // launches outside the timed phases
  if (!end) {
    if (g_nspan[p] >= kSpans) return;  // further spans are not timed
    int i = g_nspan[p];
    for (int k = 0; k < 2; ++k)
      if (!g_ev[p][i][k]) cudaEventCreate(&g_ev[p][i][k]);
    cudaEventRecord(g_ev[p][i][0], st);
    g_open[p] = true;
  } else if (g_open[p]) {
    cudaEventRecord(g_ev[p][g_nspan[p]][1], st);
    g_open[p] = false;
    ++g_nspan[p];
  }
}
void timer_end_call(double total_ms) {
  for (int p = 0; p < 2; ++p) {
    double sum = 0.0;
    for (int i = 0; i < g_nspan[p]; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g_ev[p][i][0], g_ev[p][i][1]) == cudaSuccess) sum += ms;
    }
    g_prof[p] = sum;
  }
  g_prof[2] = total_ms;
  cudaGetLastError();
}

namespace {

__global__ void rz_copy_kernel(const uint64_t* src_ptr, const int32_t* dims, const double* phi, int n,
                               int64_t N, int store, const uint64_t* dst_ptr) {
  // grid: x = site, y = state, z = copy
  const int k = blockIdx.x;
  const int64_t s = blockIdx.y, c = blockIdx.z;
  const int cl = dims[s * (n + 1) + k], cr = dims[s * (n + 1) + k + 1];
  const int64_t o = (c * N + s) * n + k;
  double sp, cp;
  sincos(phi[c * n + k], &sp, &cp);
  const int cnt = 2 * cl * cr;
  if (store) {
    const float2* a = reinterpret_cast<const float2*>(src_ptr[s * n + k]);
    float2* b = reinterpret_cast<float2*>(dst_ptr[o]);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int q = i / (cl * cr);
      const double pr = cp, pi = q ? sp : -sp;  // exp(-i phi (1 - 2q))
      const float2 v = a[i];
      b[i] = make_float2((float)(v.x * pr - v.y * pi), (float)(v.x * pi + v.y * pr));
    }
  } else {
    const double2* a = reinterpret_cast<const double2*>(src_ptr[s * n + k]);
    double2* b = reinterpret_cast<double2*>(dst_ptr[o]);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int q = i / (cl * cr);
      const double pr = cp, pi = q ? sp : -sp;
      const double2 v = a[i];
      b[i] = make_double2(v.x * pr - v.y * pi, v.x * pi + v.y * pr);
    }
  }
}

__global__ void gather_kernel(const uint64_t* src_ptr, const uint64_t* dst_off, const int32_t* dims, int n,
                              size_t eb, char* dst) {
  const int k = blockIdx.x;
  const int64_t s = blockIdx.y;
  const int cl = dims[s * (n + 1) + k], cr = dims[s * (n + 1) + k + 1];
  const size_t bytes = (size_t)2 * cl * cr * eb;
  const char* a = reinterpret_cast<const char*>(src_ptr[s * n + k]);
  char* b = dst + dst_off[s * n + k];
  for (size_t i = threadIdx.x * 4; i < bytes; i += blockDim.x * 4)
    *reinterpret_cast<uint32_t*>(b + i) = *reinterpret_cast<const uint32_t*>(a + i);
}

const int64_t kMagic = 0x716b6d7073LL;

size_t dims_bytes(int64_t N, int n) { return ((size_t)N * (n + 1) * 4 + 32 + 255) & ~size_t(255); }

// site offsets (relative to the site area) in blob order
size_t site_offsets(const std::vector<int32_t>& dims, int64_t N, int n, size_t eb,
                    std::vector<uint64_t>& off) {
  off.resize((size_t)N * n);
  size_t o = 0;
  for (int64_t s = 0; s < N; ++s)
    for (int k = 0; k < n; ++k) {
      off[s * n + k] = o;
      o += (size_t)2 * dims[s * (n + 1) + k] * dims[s * (n + 1) + k + 1] * eb;
      o = (o + 255) & ~size_t(255);
    }
  return o;
}

qk_status finish_tables(qk_mps_batch* b, const std::vector<int32_t>& dims, const std::vector<uint64_t>& ptrs,
                        const std::vector<double>& w, cudaStream_t st) {
  QK_CUDA(cudaMalloc(&b->d_dims, sizeof(int32_t) * dims.size()));
  QK_CUDA(cudaMalloc(&b->d_site_ptr, sizeof(uint64_t) * ptrs.size()));
  QK_CUDA(cudaMalloc(&b->d_trunc_w, sizeof(double) * w.size()));
  QK_CUDA(cudaMemcpyAsync(b->d_dims, dims.data(), sizeof(int32_t) * dims.size(), cudaMemcpyHostToDevice, st));
  QK_CUDA(cudaMemcpyAsync(b->d_site_ptr, ptrs.data(), sizeof(uint64_t) * ptrs.size(), cudaMemcpyHostToDevice, st));
  QK_CUDA(cudaMemcpyAsync(b->d_trunc_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, st));
  QK_CUDA(cudaStreamSynchronize(st));
  b->h_dims = dims;
  b->h_site_ptr = ptrs;
  b->h_trunc_w = w;
  int cmax = 1;
  int64_t elems = 0;
  for (int64_t s = 0; s < b->N; ++s)
    for (int k = 0; k < b->n; ++k) {
      const int a = dims[s * (b->n + 1) + k], c = dims[s * (b->n + 1) + k + 1];
      cmax = std::max(cmax, std::max(a, c));
      elems += 2LL * a * c;
    }
  b->chi_cap = cmax;
  b->arena_bytes = elems * (int64_t)elem_bytes(b->store);
  return QK_OK;
}

}  // namespace
}  // namespace qk

using namespace qk;

extern "C" qk_status qk_last_profile(double* overlap_ms, double* refine_ms, double* total_ms) {
  if (overlap_ms) *overlap_ms = g_prof[0];
  if (refine_ms) *refine_ms = g_prof[1];
  if (total_ms) *total_ms = g_prof[2];
  return QK_OK;
}

extern "C" qk_status qk_mps_rz_copies(const qk_mps_batch* src, const double* phi, int64_t copies, void* stream,
                                      qk_mps_batch** out) {
  if (!src || !phi || !out) return fail(QK_ERR_INVALID_ARG, "qk_mps_rz_copies: NULL argument");
  if (copies < 1 || copies > 65535 || src->N > 65535)
    return fail(QK_ERR_INVALID_ARG, "qk_mps_rz_copies: copies and N must be in [1, 65535]");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = src->n;
  const int64_t N = src->N, M = N * copies;
  const size_t eb = elem_bytes(src->store);
  std::vector<int32_t> dims((size_t)M * (n + 1));
  for (int64_t c = 0; c < copies; ++c)
    memcpy(dims.data() + c * N * (n + 1), src->h_dims.data(), sizeof(int32_t) * N * (n + 1));
  std::vector<uint64_t> off;
  const size_t total = site_offsets(dims, M, n, eb, off);
  const void* dphi = nullptr;
  void* owned = nullptr;
  qk_status rc = to_device(phi, sizeof(double) * copies * n, st, &dphi, &owned);
  if (rc != QK_OK) return rc;
  qk_mps_batch* b = new qk_mps_batch();
  cudaGetDevice(&b->device);
  b->N = M;
  b->n = n;
  b->store = src->store;
  auto bail = [&](qk_status s) {
    if (owned) cudaFreeAsync(owned, st);
    free_batch_memory(b);
    delete b;
    return s;
  };
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, std::max<size_t>(total, 256));
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(rz copies)"));
  b->chunks.push_back(Chunk{arena, total});
  std::vector<uint64_t> ptrs(off.size());
  for (size_t i = 0; i < off.size(); ++i) ptrs[i] = (uint64_t)arena + off[i];
  std::vector<double> w((size_t)M);
  for (int64_t c = 0; c < copies; ++c) memcpy(w.data() + c * N, src->h_trunc_w.data(), sizeof(double) * N);
  rc = finish_tables(b, dims, ptrs, w, st);
  if (rc != QK_OK) return bail(rc);
  rz_copy_kernel<<<dim3(n, (unsigned)N, (unsigned)copies), 256, 0, st>>>(
      src->d_site_ptr, src->d_dims, (const double*)dphi, n, N, src->store == QK_STORE_C64 ? 1 : 0,
      b->d_site_ptr);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (owned) cudaFreeAsync(owned, st);
  owned = nullptr;
  if (e != cudaSuccess) return bail(cuda_fail(e, "rz_copy_kernel"));
  *out = b;
  return QK_OK;
}

extern "C" qk_status qk_mps_blob_bytes(const qk_mps_batch* b, int64_t* bytes) {
  if (!b || !bytes) return fail(QK_ERR_INVALID_ARG, "qk_mps_blob_bytes: NULL argument");
  std::vector<uint64_t> off;
  *bytes = (int64_t)(dims_bytes(b->N, b->n) + site_offsets(b->h_dims, b->N, b->n, elem_bytes(b->store), off));
  return QK_OK;
}

extern "C" qk_status qk_mps_save(const qk_mps_batch* b, void* blob, int64_t bytes) {
  if (!b || !blob) return fail(QK_ERR_INVALID_ARG, "qk_mps_save: NULL argument");
  const int n = b->n;
  const size_t eb = elem_bytes(b->store);
  std::vector<uint64_t> off;
  const size_t sites = site_offsets(b->h_dims, b->N, n, eb, off);
  const size_t head = dims_bytes(b->N, n);
  if ((size_t)bytes < head + sites) return fail(QK_ERR_INVALID_ARG, "qk_mps_save: blob too small");
  std::vector<char> h(head, 0);
  int64_t hdr[4] = {kMagic, b->N, n, (int64_t)b->store};
  memcpy(h.data(), hdr, sizeof(hdr));
  memcpy(h.data() + 32, b->h_dims.data(), sizeof(int32_t) * b->h_dims.size());
  char* dst = (char*)blob;
  const bool dev = is_device_ptr(blob);
  char* stage = nullptr;
  uint64_t* d_off = nullptr;
  QK_CUDA(cudaMalloc(&stage, std::max<size_t>(sites, 256)));
  cudaError_t e = cudaMalloc(&d_off, sizeof(uint64_t) * off.size());
  if (e == cudaSuccess) e = cudaMemcpy(d_off, off.data(), sizeof(uint64_t) * off.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    cudaMemset(stage, 0, sites);
    gather_kernel<<<dim3(n, (unsigned)b->N), 256>>>(b->d_site_ptr, d_off, b->d_dims, n, eb, stage);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(dst, h.data(), head, dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
  if (e == cudaSuccess) e = cudaMemcpy(dst + head, stage, sites, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  cudaFree(stage);
  cudaFree(d_off);
  if (e != cudaSuccess) return cuda_fail(e, "qk_mps_save");
  return QK_OK;
}

extern "C" qk_status qk_mps_load(const void* blob, int64_t bytes, void* stream, qk_mps_batch** out) {
  if (!blob || !out || bytes < 32) return fail(QK_ERR_INVALID_ARG, "qk_mps_load: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = is_device_ptr(blob);
  int64_t hdr[4];
  if (dev)
    QK_CUDA(cudaMemcpy(hdr, blob, sizeof(hdr), cudaMemcpyDeviceToHost));
  else
    memcpy(hdr, blob, sizeof(hdr));
  if (hdr[0] != kMagic || hdr[1] < 1 || hdr[2] < 2 || hdr[2] > 1024 || (hdr[3] != 0 && hdr[3] != 1))
    return fail(QK_ERR_INVALID_ARG, "qk_mps_load: not a qk MPS blob");
  const int64_t N = hdr[1];
  const int n = (int)hdr[2];
  const qk_store store = (qk_store)hdr[3];
  const size_t head = dims_bytes(N, n);
  if ((size_t)bytes < head) return fail(QK_ERR_INVALID_ARG, "qk_mps_load: blob too small");
  std::vector<int32_t> dims((size_t)N * (n + 1));
  if (dev)
    QK_CUDA(cudaMemcpy(dims.data(), (const char*)blob + 32, sizeof(int32_t) * dims.size(), cudaMemcpyDeviceToHost));
  else
    memcpy(dims.data(), (const char*)blob + 32, sizeof(int32_t) * dims.size());
  for (int64_t s = 0; s < N; ++s) {
    if (dims[s * (n + 1)] != 1 || dims[s * (n + 1) + n] != 1)
      return fail(QK_ERR_INVALID_ARG, "qk_mps_load: end bonds must be 1");
    for (int k = 0; k <= n; ++k)
      if (dims[s * (n + 1) + k] < 1 || dims[s * (n + 1) + k] > 128)
        return fail(QK_ERR_INVALID_ARG, "qk_mps_load: bond dimension out of range");
  }
  std::vector<uint64_t> off;
  const size_t sites = site_offsets(dims, N, n, elem_bytes(store), off);
  if ((size_t)bytes < head + sites) return fail(QK_ERR_INVALID_ARG, "qk_mps_load: blob too small");
  qk_mps_batch* b = new qk_mps_batch();
  cudaGetDevice(&b->device);
  b->N = N;
  b->n = n;
  b->store = store;
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, std::max<size_t>(sites, 256));
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaMalloc(qk_mps_load)");
  }
  b->chunks.push_back(Chunk{arena, sites});
  e = cudaMemcpyAsync(arena, (const char*)blob + head, sites, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  std::vector<uint64_t> ptrs(off.size());
  for (size_t i = 0; i < off.size(); ++i) ptrs[i] = (uint64_t)arena + off[i];
  std::vector<double> w((size_t)N, 0.0);
  qk_status rc = e == cudaSuccess ? finish_tables(b, dims, ptrs, w, st) : cuda_fail(e, "qk_mps_load copy");
  if (rc != QK_OK) {
    free_batch_memory(b);
    delete b;
    return rc;
  }
  *out = b;
  return QK_OK;
}
