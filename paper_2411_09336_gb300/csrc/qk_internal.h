// Internal declarations shared by the libqk translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qk.h"

namespace qk {

// ---- error state (thread-local message, see qk_last_error) ----------------
void set_error(const std::string& msg);
qk_status fail(qk_status st, const std::string& msg);
qk_status cuda_fail(cudaError_t e, const char* what);

#define QK_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::qk::cuda_fail(e_, #call); \
  } while (0)

// ---- two-site op schedule (Sec. II-C) -------------------------------------
enum OpKind : int32_t { OP_RXX = 0, OP_SWAP_RXX = 1, OP_SWAP = 2 };
struct Op {
  int32_t kind;  // OpKind
  int32_t p;     // acts on positions (p, p+1)
  int32_t qi;    // Rxx qubits (qi, qj); -1 for a bare SWAP
  int32_t qj;
};
std::vector<Op> make_schedule(int n, int d);

// ---- device memory helpers --------------------------------------------------
// Copies `bytes` from a host-or-device pointer into a fresh device buffer when
// the source is host memory; returns the device pointer to use.  `owned`
// receives the buffer to free (nullptr when src is already device memory).
qk_status to_device(const void* src, size_t bytes, cudaStream_t st,
                    const void** dev, void** owned);
bool is_device_ptr(const void* p);

// ---- MPS batch -------------------------------------------------------------
// Site k of state s is the tensor A[q][a][b] (q < 2, a < chi_k,
// b < chi_{k+1}), row-major, complex (re, im) interleaved, in the storage
// precision; site_ptr[s*n + k] is its device address.
struct Chunk {
  void* ptr;
  size_t bytes;
};

}  // namespace qk

struct qk_mps_batch {
  int device = 0;
  int64_t N = 0;
  int32_t n = 0;
  qk_store store = QK_STORE_C64;
  int32_t chi_cap = 1;  // largest bond dimension present
  std::vector<qk::Chunk> chunks;     // arena allocations
  int32_t* d_dims = nullptr;         // [N][n+1]
  uint64_t* d_site_ptr = nullptr;    // [N][n]
  double* d_trunc_w = nullptr;       // [N]
  std::vector<int32_t> h_dims;       // host copy [N][n+1]
  std::vector<uint64_t> h_site_ptr;  // host copy [N][n]
  std::vector<double> h_trunc_w;
  int64_t arena_bytes = 0;
  // tensor-core operand cache (built on first split-precision use)
  void* tc_cache = nullptr;
};

namespace qk {
// kernel timings of the current qk_gram call (see qk_last_profile)
void timer_begin_call();
void timer_set_phase(int phase);  // 0: main sweep, 1: FP64 refinement
void timer_mark(bool end, cudaStream_t st);
void timer_end_call(double total_ms);
size_t elem_bytes(qk_store s);
void free_batch_memory(qk_mps_batch* b);
void free_tc_cache(qk_mps_batch* b);
// K[i*ldk + i] = |<psi_i|psi_i>|^2 for all states of a batch: the
// isometry-defect recursion for left-canonical complex64 states, the FP64
// sweep for the rest (their count in *n_fp64).  Synchronises the stream.
// Tile schedule of the split kernel's full-Gram modes for (A, B): the cached
// or set one, else (force, or a Gram large enough) one chosen by timing
// candidates on a sample; else the default (4 kets per tile, bands of 16).
qk_status split_schedule(int parts, const qk_mps_batch* A, const qk_mps_batch* B, cudaStream_t st,
                         bool force, int32_t* kets, int32_t* band, double* us_per_pair);
qk_status set_split_schedule(int parts, const qk_mps_batch* A, const qk_mps_batch* B, int32_t kets,
                             int32_t band);
qk_status diag_self_overlaps(const qk_mps_batch* A, double* dK, int64_t ldk, cudaStream_t st,
                             int64_t* n_fp64);
// The same in two parts: the launch on `st`, and the wait for it with the
// FP64 re-evaluation of the flagged states on `st_fp64`.
struct DiagPending {
  cudaStream_t st = nullptr;
  int32_t* flag = nullptr;
  int64_t N = 0;
};
qk_status diag_launch(const qk_mps_batch* A, double* dK, int64_t ldk, cudaStream_t st, DiagPending* d);
qk_status diag_finish(const qk_mps_batch* A, double* dK, int64_t ldk, DiagPending* d, cudaStream_t st_fp64,
                      int64_t* n_fp64);
// a non-blocking stream of the current device for work beside the call's stream
cudaStream_t side_stream();
}  // namespace qk
