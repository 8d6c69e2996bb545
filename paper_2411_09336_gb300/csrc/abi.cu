// C ABI of libqk: argument checking, batch ownership, host/device pointer
// handling, and dispatch to the builder and overlap kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "qk_internal.h"

namespace qk {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
qk_status fail(qk_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
qk_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? QK_ERR_OOM : QK_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

qk_status to_device(const void* src, size_t bytes, cudaStream_t st, const void** dev,
                    void** owned) {
  *owned = nullptr;
  if (is_device_ptr(src) || bytes == 0) {
    *dev = src;
    return QK_OK;
  }
  void* d = nullptr;
  QK_CUDA(cudaMallocAsync(&d, bytes, st));
  cudaError_t e = cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(d, st);
    return cuda_fail(e, "cudaMemcpyAsync(H2D)");
  }
  *dev = d;
  *owned = d;
  return QK_OK;
}

size_t elem_bytes(qk_store s) { return s == QK_STORE_C64 ? 8 : 16; }

void free_batch_memory(qk_mps_batch* b) {
  free_tc_cache(b);
  for (auto& c : b->chunks) cudaFree(c.ptr);
  b->chunks.clear();
  cudaFree(b->d_dims);
  cudaFree(b->d_site_ptr);
  cudaFree(b->d_trunc_w);
  b->d_dims = nullptr;
  b->d_site_ptr = nullptr;
  b->d_trunc_w = nullptr;
}

qk_status build_states_device(const double* dX, int64_t N, int n, int d, int reps, double gamma,
                              int chi_max, double eps, qk_store store, int32_t* rank_trace,
                              cudaStream_t st, qk_mps_batch* out);
qk_status overlap_fp64(const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                       int64_t P, double* dK, int64_t ldk, bool sym, cudaStream_t st,
                       int ctas_per_sm = 4);
qk_status gram_split(int parts, const qk_mps_batch* A, const qk_mps_batch* B, double* dK,
                     int64_t ldk, double refine_floor, cudaStream_t st, int64_t* n_refined);
qk_status pairs_split(int parts, const qk_mps_batch* A, const qk_mps_batch* B,
                      const int32_t* d_pairs, int64_t P, double* dK, cudaStream_t st);
static bool valid_prec(qk_prec p) {
  return p == QK_PREC_FP64 || p == QK_PREC_SPLIT_BF16 || p == QK_PREC_SPLIT_BF16X3;
}
static int split_parts(qk_prec p) { return p == QK_PREC_SPLIT_BF16X3 ? 3 : 2; }

// Host copies of the tables + derived sizes after the device tables are set.
static qk_status finish_batch(qk_mps_batch* b, cudaStream_t st) {
  b->h_dims.resize(b->N * (b->n + 1));
  b->h_site_ptr.resize(b->N * b->n);
  b->h_trunc_w.resize(b->N);
  QK_CUDA(cudaMemcpyAsync(b->h_dims.data(), b->d_dims, sizeof(int32_t) * b->h_dims.size(),
                          cudaMemcpyDeviceToHost, st));
  QK_CUDA(cudaMemcpyAsync(b->h_site_ptr.data(), b->d_site_ptr,
                          sizeof(uint64_t) * b->h_site_ptr.size(), cudaMemcpyDeviceToHost, st));
  QK_CUDA(cudaMemcpyAsync(b->h_trunc_w.data(), b->d_trunc_w, sizeof(double) * b->N,
                          cudaMemcpyDeviceToHost, st));
  QK_CUDA(cudaStreamSynchronize(st));
  int cmax = 1;
  int64_t elems = 0;
  for (int64_t s = 0; s < b->N; ++s)
    for (int k = 0; k < b->n; ++k) {
      int a = b->h_dims[s * (b->n + 1) + k], c = b->h_dims[s * (b->n + 1) + k + 1];
      cmax = std::max(cmax, std::max(a, c));
      elems += 2LL * a * c;
    }
  b->chi_cap = cmax;
  b->arena_bytes = elems * (int64_t)elem_bytes(b->store);
  return QK_OK;
}

}  // namespace qk

using namespace qk;

extern "C" const char* qk_last_error(void) { return g_err.c_str(); }

extern "C" qk_status qk_build_states(const double* X, int64_t N, int32_t n, int32_t d,
                                     int32_t reps, double gamma, int32_t chi_max, double eps,
                                     qk_store store, int32_t* rank_trace, void* stream,
                                     qk_mps_batch** out) {
  if (!out) return fail(QK_ERR_INVALID_ARG, "qk_build_states: out is NULL");
  if (!X) return fail(QK_ERR_INVALID_ARG, "qk_build_states: X is NULL");
  if (N < 1 || N > (int64_t)1 << 30) return fail(QK_ERR_INVALID_ARG, "qk_build_states: N out of range");
  if (n < 2 || n > 1024) return fail(QK_ERR_INVALID_ARG, "qk_build_states: n must be in [2, 1024]");
  if (d < 0 || d > n - 1) return fail(QK_ERR_INVALID_ARG, "qk_build_states: d must be in [0, n-1]");
  if (reps < 1 || reps > 1000) return fail(QK_ERR_INVALID_ARG, "qk_build_states: reps must be in [1, 1000]");
  if (!isfinite(gamma)) return fail(QK_ERR_INVALID_ARG, "qk_build_states: gamma is not finite");
  if (chi_max < 1 || chi_max > 128) return fail(QK_ERR_INVALID_ARG, "qk_build_states: chi_max must be in [1, 128]");
  if (!(eps >= 0.0) || !isfinite(eps)) return fail(QK_ERR_INVALID_ARG, "qk_build_states: eps must be finite and >= 0");
  if (store != QK_STORE_C64 && store != QK_STORE_C128) return fail(QK_ERR_INVALID_ARG, "qk_build_states: bad store");
  if (rank_trace && !is_device_ptr(rank_trace)) return fail(QK_ERR_INVALID_ARG, "qk_build_states: rank_trace must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t xb = sizeof(double) * (size_t)N * n;
  // finiteness of X is checked on the host copy
  std::vector<double> hx;
  const double* hsrc = X;
  if (is_device_ptr(X)) {
    hx.resize((size_t)N * n);
    QK_CUDA(cudaMemcpyAsync(hx.data(), X, xb, cudaMemcpyDeviceToHost, st));
    QK_CUDA(cudaStreamSynchronize(st));
    hsrc = hx.data();
  }
  for (size_t i = 0; i < (size_t)N * n; ++i)
    if (!isfinite(hsrc[i])) return fail(QK_ERR_INVALID_ARG, "qk_build_states: X holds a non-finite value");
  const void* dX = nullptr;
  void* owned = nullptr;
  qk_status rc = to_device(X, xb, st, &dX, &owned);
  if (rc != QK_OK) return rc;
  qk_mps_batch* b = new qk_mps_batch();
  cudaError_t de = cudaGetDevice(&b->device);
  if (de != cudaSuccess) {
    delete b;
    if (owned) cudaFreeAsync(owned, st);
    return cuda_fail(de, "cudaGetDevice");
  }
  b->N = N;
  b->n = n;
  b->store = store;
  rc = build_states_device((const double*)dX, N, n, d, reps, gamma, chi_max, eps, store,
                           rank_trace, st, b);
  if (owned) cudaFreeAsync(owned, st);
  if (rc == QK_OK || rc == QK_ERR_NUMERIC) {
    qk_status r2 = finish_batch(b, st);
    if (r2 != QK_OK) rc = r2;
  }
  if (rc != QK_OK) {
    free_batch_memory(b);
    delete b;
    return rc;
  }
  *out = b;
  return QK_OK;
}

extern "C" qk_status qk_mps_import(int64_t N, int32_t n, const int32_t* bond_dims,
                                   const double* re_im, qk_store store, void* stream,
                                   qk_mps_batch** out) {
  if (!out || !bond_dims || !re_im) return fail(QK_ERR_INVALID_ARG, "qk_mps_import: NULL argument");
  if (N < 1 || n < 2 || n > 1024) return fail(QK_ERR_INVALID_ARG, "qk_mps_import: bad N or n");
  if (store != QK_STORE_C64 && store != QK_STORE_C128) return fail(QK_ERR_INVALID_ARG, "qk_mps_import: bad store");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t elems = 0;
  for (int64_t s = 0; s < N; ++s) {
    const int32_t* dm = bond_dims + s * (n + 1);
    if (dm[0] != 1 || dm[n] != 1) return fail(QK_ERR_INVALID_ARG, "qk_mps_import: end bonds must be 1");
    for (int k = 0; k <= n; ++k)
      if (dm[k] < 1 || dm[k] > 128) return fail(QK_ERR_INVALID_ARG, "qk_mps_import: bond dimension out of [1, 128]");
    for (int k = 0; k < n; ++k) elems += 2LL * dm[k] * dm[k + 1];
  }
  const size_t eb = elem_bytes(store);
  qk_mps_batch* b = new qk_mps_batch();
  cudaGetDevice(&b->device);
  b->N = N;
  b->n = n;
  b->store = store;
  auto bail = [&](qk_status s) {
    free_batch_memory(b);
    delete b;
    return s;
  };
  // per-site 256-byte aligned placement
  std::vector<uint64_t> offs((size_t)N * n);
  size_t total = 0;
  for (int64_t s = 0; s < N; ++s)
    for (int k = 0; k < n; ++k) {
      offs[s * n + k] = total;
      total += 2ULL * bond_dims[s * (n + 1) + k] * bond_dims[s * (n + 1) + k + 1] * eb;
      total = (total + 255) & ~size_t(255);
    }
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, std::max<size_t>(total, 256));
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(arena)"));
  b->chunks.push_back(Chunk{arena, total});
  std::vector<char> host(total);
  size_t src = 0;
  for (int64_t s = 0; s < N; ++s)
    for (int k = 0; k < n; ++k) {
      int64_t cnt = 2LL * bond_dims[s * (n + 1) + k] * bond_dims[s * (n + 1) + k + 1];
      char* dst = host.data() + offs[s * n + k];
      for (int64_t i = 0; i < cnt; ++i) {
        double re = re_im[2 * (src + i)], im = re_im[2 * (src + i) + 1];
        if (store == QK_STORE_C64) {
          float v[2] = {(float)re, (float)im};
          memcpy(dst + 8 * i, v, 8);
        } else {
          double v[2] = {re, im};
          memcpy(dst + 16 * i, v, 16);
        }
      }
      src += cnt;
    }
  // the import layout is [a][q][b]; the device layout is [q][a][b]
  {
    std::vector<char> perm(total);
    for (int64_t s = 0; s < N; ++s)
      for (int k = 0; k < n; ++k) {
        int ca = bond_dims[s * (n + 1) + k], cb = bond_dims[s * (n + 1) + k + 1];
        char* in = host.data() + offs[s * n + k];
        char* o = perm.data() + offs[s * n + k];
        for (int a = 0; a < ca; ++a)
          for (int q = 0; q < 2; ++q)
            for (int bb = 0; bb < cb; ++bb)
              memcpy(o + ((q * ca + a) * cb + bb) * eb, in + ((a * 2 + q) * cb + bb) * eb, eb);
      }
    host.swap(perm);
  }
  std::vector<uint64_t> ptrs((size_t)N * n);
  for (size_t i = 0; i < ptrs.size(); ++i) ptrs[i] = (uint64_t)arena + offs[i];
  e = cudaMemcpy(arena, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpy(arena)"));
  if ((e = cudaMalloc(&b->d_dims, sizeof(int32_t) * N * (n + 1))) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  if ((e = cudaMalloc(&b->d_site_ptr, sizeof(uint64_t) * N * n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  if ((e = cudaMalloc(&b->d_trunc_w, sizeof(double) * N)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  if ((e = cudaMemcpy(b->d_dims, bond_dims, sizeof(int32_t) * N * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_site_ptr, ptrs.data(), sizeof(uint64_t) * N * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(b->d_trunc_w, 0, sizeof(double) * N)) != cudaSuccess)
    return bail(cuda_fail(e, "qk_mps_import tables"));
  qk_status rc = finish_batch(b, st);
  if (rc != QK_OK) return bail(rc);
  *out = b;
  return QK_OK;
}

extern "C" qk_status qk_mps_shape(const qk_mps_batch* b, int64_t* N, int32_t* n) {
  if (!b) return fail(QK_ERR_INVALID_ARG, "qk_mps_shape: NULL batch");
  if (N) *N = b->N;
  if (n) *n = b->n;
  return QK_OK;
}

extern "C" qk_status qk_mps_bond_dims(const qk_mps_batch* b, int32_t* dims) {
  if (!b || !dims) return fail(QK_ERR_INVALID_ARG, "qk_mps_bond_dims: NULL argument");
  memcpy(dims, b->h_dims.data(), sizeof(int32_t) * b->h_dims.size());
  return QK_OK;
}

extern "C" qk_status qk_mps_trunc_weight(const qk_mps_batch* b, double* w) {
  if (!b || !w) return fail(QK_ERR_INVALID_ARG, "qk_mps_trunc_weight: NULL argument");
  memcpy(w, b->h_trunc_w.data(), sizeof(double) * b->N);
  return QK_OK;
}

extern "C" qk_status qk_mps_bytes(const qk_mps_batch* b, int64_t* bytes) {
  if (!b || !bytes) return fail(QK_ERR_INVALID_ARG, "qk_mps_bytes: NULL argument");
  *bytes = b->arena_bytes;
  return QK_OK;
}

extern "C" qk_status qk_mps_export(const qk_mps_batch* b, int64_t s, double* re_im, int64_t cap) {
  if (!b || !re_im) return fail(QK_ERR_INVALID_ARG, "qk_mps_export: NULL argument");
  if (s < 0 || s >= b->N) return fail(QK_ERR_INVALID_ARG, "qk_mps_export: state index out of range");
  const int n = b->n;
  const int32_t* dm = b->h_dims.data() + s * (n + 1);
  int64_t need = 0;
  for (int k = 0; k < n; ++k) need += 2LL * 2 * dm[k] * dm[k + 1];
  if (cap < need) return fail(QK_ERR_INVALID_ARG, "qk_mps_export: buffer too small");
  const size_t eb = elem_bytes(b->store);
  int64_t o = 0;
  for (int k = 0; k < n; ++k) {
    int ca = dm[k], cb = dm[k + 1];
    std::vector<char> buf(2ULL * ca * cb * eb);
    QK_CUDA(cudaMemcpy(buf.data(), (const void*)b->h_site_ptr[s * n + k], buf.size(), cudaMemcpyDeviceToHost));
    for (int a = 0; a < ca; ++a)
      for (int q = 0; q < 2; ++q)
        for (int bb = 0; bb < cb; ++bb) {
          size_t src = ((size_t)(q * ca + a) * cb + bb);
          double re, im;
          if (b->store == QK_STORE_C64) {
            float v[2];
            memcpy(v, buf.data() + 8 * src, 8);
            re = v[0];
            im = v[1];
          } else {
            double v[2];
            memcpy(v, buf.data() + 16 * src, 16);
            re = v[0];
            im = v[1];
          }
          re_im[o++] = re;
          re_im[o++] = im;
        }
  }
  return QK_OK;
}

extern "C" qk_status qk_mps_free(qk_mps_batch* b) {
  if (!b) return QK_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  free_batch_memory(b);
  cudaSetDevice(cur);
  delete b;
  return QK_OK;
}

static qk_status check_pair(const qk_mps_batch* A, const qk_mps_batch* B, const char* who) {
  if (!A || !B) return fail(QK_ERR_INVALID_ARG, std::string(who) + ": NULL batch");
  if (A->n != B->n) return fail(QK_ERR_INVALID_ARG, std::string(who) + ": batches differ in n");
  if (A->store != B->store) return fail(QK_ERR_INVALID_ARG, std::string(who) + ": batches differ in storage precision");
  return QK_OK;
}

extern "C" qk_status qk_gram(const qk_mps_batch* A, const qk_mps_batch* B, double* K, int64_t ldk,
                             qk_prec prec, double refine_floor, void* stream, int64_t* n_refined) {
  qk_status rc = check_pair(A, B, "qk_gram");
  if (rc != QK_OK) return rc;
  if (!K) return fail(QK_ERR_INVALID_ARG, "qk_gram: K is NULL");
  if (ldk < B->N) return fail(QK_ERR_INVALID_ARG, "qk_gram: ldk < N_B");
  if (!valid_prec(prec)) return fail(QK_ERR_INVALID_ARG, "qk_gram: bad precision");
  if (!(refine_floor >= 0.0)) return fail(QK_ERR_INVALID_ARG, "qk_gram: refine_floor must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  timer_begin_call();
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, st);
  const bool sym = (A == B);
  const size_t kb = sizeof(double) * (size_t)((A->N - 1) * ldk + B->N);
  double* dK = K;
  void* owned = nullptr;
  const bool host_k = !is_device_ptr(K);
  if (host_k) {
    QK_CUDA(cudaMallocAsync(&owned, kb, st));
    dK = (double*)owned;
    if (ldk != B->N) QK_CUDA(cudaMemcpyAsync(dK, K, kb, cudaMemcpyHostToDevice, st));
  }
  if (n_refined) *n_refined = 0;
  if (prec == QK_PREC_FP64) {
    std::vector<int32_t> pairs;
    pairs.reserve(sym ? (size_t)A->N * (A->N + 1) : (size_t)2 * A->N * B->N);
    for (int64_t i = 0; i < A->N; ++i)
      for (int64_t j = sym ? i : 0; j < B->N; ++j) {
        pairs.push_back((int32_t)i);
        pairs.push_back((int32_t)j);
      }
    int64_t P = (int64_t)pairs.size() / 2;
    if (P >= ((int64_t)1 << 31)) return fail(QK_ERR_INVALID_ARG, "qk_gram: too many pairs for one call");
    int32_t* dp = nullptr;
    QK_CUDA(cudaMallocAsync(&dp, sizeof(int32_t) * pairs.size(), st));
    QK_CUDA(cudaMemcpyAsync(dp, pairs.data(), sizeof(int32_t) * pairs.size(), cudaMemcpyHostToDevice, st));
    rc = overlap_fp64(A, B, dp, P, dK, ldk, sym, st);
    cudaFreeAsync(dp, st);
  } else {
    rc = gram_split(split_parts(prec), A, B, dK, ldk, refine_floor, st, n_refined);
  }
  if (rc == QK_OK && host_k) {
    cudaError_t e = cudaMemcpyAsync(K, dK, kb, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(K D2H)");
  }
  if (owned) cudaFreeAsync(owned, st);
  cudaEventRecord(t1, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == QK_OK && e != cudaSuccess) rc = cuda_fail(e, "qk_gram");
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) ms = 0.f;
  timer_end_call(ms);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return rc;
}

extern "C" qk_status qk_tune_split(const qk_mps_batch* A, const qk_mps_batch* B, qk_prec prec, void* stream,
                                   int32_t* kets_per_tile, int32_t* band, double* us_per_pair) {
  qk_status rc = check_pair(A, B, "qk_tune_split");
  if (rc != QK_OK) return rc;
  if (prec != QK_PREC_SPLIT_BF16 && prec != QK_PREC_SPLIT_BF16X3)
    return fail(QK_ERR_INVALID_ARG, "qk_tune_split: prec must be a split precision");
  int32_t k = 0, b = 0;
  double us = 0.0;
  rc = split_schedule(split_parts(prec), A, B, (cudaStream_t)stream, true, &k, &b, &us);
  if (rc != QK_OK) return rc;
  if (kets_per_tile) *kets_per_tile = k;
  if (band) *band = b;
  if (us_per_pair) *us_per_pair = us;
  return QK_OK;
}

extern "C" qk_status qk_set_split_schedule(const qk_mps_batch* A, const qk_mps_batch* B, qk_prec prec,
                                           int32_t kets_per_tile, int32_t band) {
  qk_status rc = check_pair(A, B, "qk_set_split_schedule");
  if (rc != QK_OK) return rc;
  if (prec != QK_PREC_SPLIT_BF16 && prec != QK_PREC_SPLIT_BF16X3)
    return fail(QK_ERR_INVALID_ARG, "qk_set_split_schedule: prec must be a split precision");
  if (kets_per_tile < 1 || kets_per_tile > 4 || band < 1)
    return fail(QK_ERR_INVALID_ARG, "qk_set_split_schedule: kets_per_tile in 1..4, band >= 1");
  return set_split_schedule(split_parts(prec), A, B, kets_per_tile, band);
}

extern "C" qk_status qk_gram_pairs(const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* pairs,
                                   int64_t P, double* K_out, qk_prec prec, void* stream) {
  qk_status rc = check_pair(A, B, "qk_gram_pairs");
  if (rc != QK_OK) return rc;
  if (P < 0 || P >= ((int64_t)1 << 31)) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs: P out of range");
  if (P == 0) return QK_OK;
  if (!pairs || !K_out) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs: NULL argument");
  if (!valid_prec(prec)) return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs: bad precision");
  cudaStream_t st = (cudaStream_t)stream;
  timer_begin_call();
  // validate the indices on the host
  std::vector<int32_t> hp;
  const int32_t* hsrc = pairs;
  if (is_device_ptr(pairs)) {
    hp.resize(2 * P);
    QK_CUDA(cudaMemcpyAsync(hp.data(), pairs, sizeof(int32_t) * 2 * P, cudaMemcpyDeviceToHost, st));
    QK_CUDA(cudaStreamSynchronize(st));
    hsrc = hp.data();
  }
  for (int64_t p = 0; p < P; ++p)
    if (hsrc[2 * p] < 0 || hsrc[2 * p] >= A->N || hsrc[2 * p + 1] < 0 || hsrc[2 * p + 1] >= B->N)
      return fail(QK_ERR_INVALID_ARG, "qk_gram_pairs: pair index out of range");
  const void* dp = nullptr;
  void* owned_p = nullptr;
  rc = to_device(pairs, sizeof(int32_t) * 2 * P, st, &dp, &owned_p);
  if (rc != QK_OK) return rc;
  double* dK = K_out;
  void* owned_k = nullptr;
  const bool host_k = !is_device_ptr(K_out);
  if (host_k) {
    QK_CUDA(cudaMallocAsync(&owned_k, sizeof(double) * P, st));
    dK = (double*)owned_k;
  }
  if (prec == QK_PREC_FP64)
    rc = overlap_fp64(A, B, (const int32_t*)dp, P, dK, 0, false, st);
  else
    rc = pairs_split(split_parts(prec), A, B, (const int32_t*)dp, P, dK, st);
  if (rc == QK_OK && host_k) {
    cudaError_t e = cudaMemcpyAsync(K_out, dK, sizeof(double) * P, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(K D2H)");
  }
  if (owned_p) cudaFreeAsync(owned_p, st);
  if (owned_k) cudaFreeAsync(owned_k, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == QK_OK && e != cudaSuccess) rc = cuda_fail(e, "qk_gram_pairs");
  timer_end_call(0.0);
  return rc;
}

namespace qk {
// exact overlaps of a device pair list into a device vector (surrogate fallback)
qk_status gram_pairs_exact(qk_prec prec, const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                           int64_t P, double* dK, cudaStream_t st) {
  if (prec == QK_PREC_FP64) return overlap_fp64(A, B, d_pairs, P, dK, 0, false, st);
  return pairs_split(split_parts(prec), A, B, d_pairs, P, dK, st);
}
}  // namespace qk
