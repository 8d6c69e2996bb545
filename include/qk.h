/*
 * qk.h - C ABI of libqk: quantum-kernel Gram matrices from MPS simulation on
 * one GB300 (sm_103a).
 *
 * The method (arXiv 2411.09336, Sec. II): every data vector x (m features ->
 * m qubits) is encoded as |psi(x)> = U(x)|+>^m with
 *   U(x) = (exp(-i H_XX) exp(-i H_Z))^r                               (Eq. 3)
 *   H_Z  = gamma sum_k x_k Z_k                                          (Eq. 4)
 *   H_XX = gamma^2 (pi/2) sum_{(i,j) in G} (1-x_i)(1-x_j) X_i X_j       (Eq. 5)
 * G = all qubit pairs at distance 1..d on a line (Sec. II-C).  The state is
 * simulated as a matrix product state, every two-qubit gate followed by an SVD
 * truncation (Sec. II-B, Fig. 1, Eq. 8), and the kernel is
 *   K_ij = |<psi(x_i)|psi(x_j)>|^2                                      (Eq. 1)
 * contracted by the left-to-right transfer sweep of Fig. 2.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a qk_status.  On failure the outputs are left
 *     untouched and qk_last_error() returns a message (thread-local).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; calls marked "synchronises" wait for
 *     the stream before returning.
 *   - Pointers marked "host or device" may point to either; the library looks
 *     the pointer up (cudaPointerGetAttributes) and copies host data itself.
 *   - Arguments are checked before any launch: a bad argument returns
 *     QK_ERR_INVALID_ARG and launches nothing.
 *   - Bounded device waits never trap: a wait that runs out sets an error word
 *     that the host reads back as QK_ERR_TIMEOUT.
 */
#ifndef QK_H_
#define QK_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QK_OK = 0,
  QK_ERR_INVALID_ARG = 1,
  QK_ERR_OOM = 2,
  QK_ERR_CUDA = 3,
  QK_ERR_NUMERIC = 4,  /* SVD sweep cap reached or a non-finite value */
  QK_ERR_TIMEOUT = 5   /* a bounded device wait ran out */
} qk_status;

/* Overlap arithmetic. */
typedef enum {
  QK_PREC_FP64 = 0,         /* plain FP64 transfer sweep on the CUDA cores */
  QK_PREC_SPLIT_BF16 = 1,   /* tcgen05 tensor cores: operands split into bf16
                               hi + lo (residual <= 2^-17), products
                               hi*hi + hi*lo + lo*hi, FP32 accumulation */
  QK_PREC_SPLIT_BF16X3 = 2  /* as above with three bf16 parts (exact for
                               FP32 values) and the six products of order
                               >= 2^-16: FP32-level accuracy, twice the MMAs */
} qk_prec;

/* The split path's error is relative to |<a|b>| (FP32 accumulation in the
 * tensor cores truncates, a bias that grows with n), so entries with
 * K > QK_SPLIT_REFINE_ABOVE are always re-evaluated in FP64; this keeps
 * |dK| <= 1e-5 absolute for n up to a few hundred qubits. */
#define QK_SPLIT_REFINE_ABOVE 1e-3

/* Storage precision of the packed states (the build itself is FP64). */
typedef enum { QK_STORE_C128 = 0, QK_STORE_C64 = 1 } qk_store;

/* Opaque batch of N MPS states on one device, owned by the library. */
typedef struct qk_mps_batch qk_mps_batch;
/* Opaque surrogate network, owned by the library. */
typedef struct qk_surrogate qk_surrogate;

/* Message of the last failed call on this thread ("" if none). */
const char* qk_last_error(void);

/* ------------------------------------------------------------------------
 * qk_build_states - simulate |psi(x_s)> for s = 0..N-1 as MPS (Sec. II-B).
 *
 *   X        host or device, N x n float64, row-major (row s = x_s).  Used as
 *            given: no rescaling is applied inside the method.
 *   n        qubits = features, 2 <= n <= 1024.
 *   d        interaction distance, 0 <= d <= n-1 (d = 0: product states).
 *   reps     circuit repetitions r >= 1.
 *   gamma    kernel bandwidth (finite).
 *   chi_max  bond-dimension cap, 1 <= chi_max <= 128.
 *   eps      truncation tolerance >= 0: after each two-site gate keep the
 *            fewest singular values whose discarded squared tail is
 *            <= eps^2 * (sum of all squares), then at most chi_max; the kept
 *            values are rescaled to unit norm.  eps = 0: no truncation below
 *            chi_max.  (Eq. 8: the discarded weight bounds the infidelity.)
 *   store    storage precision of the result.
 *   rank_trace  optional device int32 [N][reps * n_ops] (NULL to skip): the
 *            rank kept after every two-site op, in execution order;
 *            n_ops = qk_schedule_length(n, d).
 *   out      receives the new batch (free with qk_mps_free).
 * The build runs in FP64: every two-site op is a Householder QR with column
 * pivoting followed by a one-sided Jacobi SVD of its R factor.  Two-site ops
 * follow the SWAP-routed schedule:
 * for each qubit i, Rxx(i,i+t) (t < k) fused with the following SWAP, then
 * Rxx(i,i+k) and k-1 SWAPs back, k = min(d, n-1-i) (Sec. II-C).  Final
 * states are left-canonical.  Synchronises.
 * Errors: INVALID_ARG (ranges above, non-finite X or gamma), OOM, CUDA,
 * NUMERIC (an SVD did not converge in its sweep cap).
 * ---------------------------------------------------------------------- */
qk_status qk_build_states(const double* X, int64_t N, int32_t n, int32_t d,
                          int32_t reps, double gamma, int32_t chi_max,
                          double eps, qk_store store, int32_t* rank_trace,
                          void* stream, qk_mps_batch** out);

/* Device-side profile of the last qk_build_states call on this thread:
 *   kernel_ms       CUDA-event time of the build kernel launches;
 *   phase_sm_ms     host double [6]: SM-milliseconds (clock64 cycles of each
 *                   CTA / SM clock, summed over CTAs) spent in: theta formation
 *                   and gate, QR with column pivoting, Jacobi sweeps, writing
 *                   the factors (isometry + GEMM), centre moves, other (Z
 *                   layers, packing);
 *   ctas            CTAs launched; sweeps  Jacobi sweeps summed over all
 *                   factorisations; factorisations  their number;
 *   fp64_flops      FP64 flops the kernel executed (an FMA counts 2): theta
 *                   formation and gate, QR updates, Jacobi inner products and
 *                   rotations, the GEMMs that form the factors.
 * Any pointer may be NULL.  No synchronisation. */
qk_status qk_last_build_profile(double* kernel_ms, double* phase_sm_ms,
                                int64_t* ctas, int64_t* sweeps,
                                int64_t* factorisations, double* fp64_flops);

/* Number of two-site ops in one repetition: sum_i (2 min(d, n-1-i) - 1). */
int64_t qk_schedule_length(int32_t n, int32_t d);

/* ------------------------------------------------------------------------
 * qk_mps_import - wrap caller-supplied MPS as a batch (tests and tooling).
 *   bond_dims  host int32 [N][n+1], chi_0 = chi_n = 1, each 1..chi_max_cap.
 *   re_im      host float64, the sites of all states back to back: for state
 *              s, site k, entry (a, q, b) of the tensor A_k[a][q][b]
 *              (a < chi_k, q < 2, b < chi_{k+1}) stored as (re, im) at
 *              2 * (off_s + off_k + (a*2 + q)*chi_{k+1} + b).
 *   store      storage precision used for the batch.
 * Synchronises.  Errors: INVALID_ARG, OOM, CUDA.
 * ---------------------------------------------------------------------- */
qk_status qk_mps_import(int64_t N, int32_t n, const int32_t* bond_dims,
                        const double* re_im, qk_store store, void* stream,
                        qk_mps_batch** out);

/* Shape queries (host, no synchronisation). */
qk_status qk_mps_shape(const qk_mps_batch* b, int64_t* N, int32_t* n);
/* dims: host int32 [N][n+1].  Synchronises. */
qk_status qk_mps_bond_dims(const qk_mps_batch* b, int32_t* dims);
/* w: host float64 [N], summed discarded weight per state.  Synchronises. */
qk_status qk_mps_trunc_weight(const qk_mps_batch* b, double* w);
/* Stored bytes of the packed states (arena only). */
qk_status qk_mps_bytes(const qk_mps_batch* b, int64_t* bytes);
/* Copy state `s` to host in the qk_mps_import layout; `cap` is the length of
 * re_im in doubles (>= 2 * sum_k chi_k * 2 * chi_{k+1}).  Synchronises. */
qk_status qk_mps_export(const qk_mps_batch* b, int64_t s, double* re_im,
                        int64_t cap);
qk_status qk_mps_free(qk_mps_batch* b);

/* ------------------------------------------------------------------------
 * qk_mps_rz_copies - `copies` rotated copies of every state of `src`:
 * copy c of state s (output index c * N + s) is exp(-i sum_k phi[c][k] Z_k)
 * applied to |psi_s>, i.e. a final single-qubit Z layer (Eq. 4, Fig. 1a)
 * contracted into the sites: slice q of site k times exp(-i phi (1 - 2q)).
 * Bond dimensions are unchanged.  phi: host or device float64
 * [copies][n].  Synchronises.  Errors: INVALID_ARG, OOM, CUDA.
 * ---------------------------------------------------------------------- */
qk_status qk_mps_rz_copies(const qk_mps_batch* src, const double* phi,
                           int64_t copies, void* stream, qk_mps_batch** out);

/* Serialise a batch to one host blob / rebuild it on the current device.
 * Blob: int64 header {magic 0x716b6d7073, N, n, store}, int32 bond dims
 * [N][n+1] (padded to 8 bytes), then every site of every state in the
 * device layout A[q][a][b] (complex, storage precision), each site padded
 * to 256 bytes.  qk_mps_blob_bytes gives the size; `blob` for qk_mps_load
 * may be host (pinned or pageable) or device memory; load issues one copy
 * of the arena.  Synchronises.  Errors: INVALID_ARG (bad header or size),
 * OOM, CUDA. */
qk_status qk_mps_blob_bytes(const qk_mps_batch* b, int64_t* bytes);
qk_status qk_mps_save(const qk_mps_batch* b, void* blob, int64_t bytes);
qk_status qk_mps_load(const void* blob, int64_t bytes, void* stream,
                      qk_mps_batch** out);

/* Device time of the kernels of the last qk_gram / qk_gram_pairs call on
 * this thread, from CUDA events on the call's stream: the overlap kernel
 * (tensor-core or FP64 sweep over all pairs), the FP64 re-evaluation, and
 * the whole call.  Milliseconds; 0 where a part did not run. */
qk_status qk_last_profile(double* overlap_ms, double* refine_ms,
                          double* total_ms);

/* ------------------------------------------------------------------------
 * qk_gram - K[i][j] = |<psi(a_i)|psi(b_j)>|^2 for all i < N_A, j < N_B
 * (Eq. 1) by the transfer sweep of Fig. 2.
 *   A, B     batches with equal n.  B == A (same pointer) selects the
 *            symmetric case: only i <= j is contracted and mirrored
 *            (Sec. II-D: half of the entries).
 *   K        host or device float64, row-major with leading dimension ldk
 *            >= N_B; K[i*ldk + j].
 *   prec     QK_PREC_FP64, QK_PREC_SPLIT_BF16 or QK_PREC_SPLIT_BF16X3.
 *   refine_floor  split path only: entries with K < refine_floor are
 *            contracted again in FP64 (0 disables); entries with
 *            K > QK_SPLIT_REFINE_ABOVE always are.
 *   n_refined     optional host out: entries not taken from the split
 *            product -- those re-evaluated in FP64 and, when B == A, the
 *            N self-overlaps.
 * Split path, B == A: the self-overlaps K_ii come from the recursion
 * E_k = I + F_k, F_k+1 = G_k + sum_s A_k[s]^H F_k A_k[s] with the site's
 * isometry defect G_k = sum_s A_k[s]^H A_k[s] - I formed in double-float
 * arithmetic (exact for a left-canonical state, which keeps E = I; within
 * ~1e-10 of the FP64 sweep); states whose defect exceeds 1e-4 (not
 * left-canonical) take the FP64 sweep.
 * Synchronises.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT.
 * ---------------------------------------------------------------------- */
qk_status qk_gram(const qk_mps_batch* A, const qk_mps_batch* B, double* K,
                  int64_t ldk, qk_prec prec, double refine_floor, void* stream,
                  int64_t* n_refined);

/* K_out[p] = |<psi(a_{pairs[2p]})|psi(b_{pairs[2p+1]})>|^2 for p < P.
 * The split path re-evaluates entries above QK_SPLIT_REFINE_ABOVE in FP64.
 * pairs: host or device int32 [P][2]; K_out: host or device float64 [P].
 * Synchronises.  Errors: INVALID_ARG (index out of range), OOM, CUDA. */
qk_status qk_gram_pairs(const qk_mps_batch* A, const qk_mps_batch* B,
                        const int32_t* pairs, int64_t P, double* K_out,
                        qk_prec prec, void* stream);

/* ------------------------------------------------------------------------
 * Tile schedule of the split-precision Gram (qk_gram with a split prec).
 * Sec. II-D distributes square tiles of the Gram matrix over GPUs; on one
 * GPU the kernel takes tiles of one bra and `kets_per_tile` kets (1, 2 or
 * 4), in bands of `band` bras whose tiles run side by side and share the
 * kets in L2.  The paper has no tuner: here the schedule is chosen by
 * measurement.
 *
 * qk_tune_split times six candidate schedules (4 kets in bands of 16, 2 in
 * bands of 64, 1 in bands of 16/32/64/128) on one sample of the Gram of
 * (A, B) -- the pairs of the first 128 bras with the first ~290 kets (160
 * when B != A), at least four tiles per CTA; each candidate runs twice
 * and its faster run counts) and keeps the fastest, the default (4 kets,
 * bands of 16) unless another beats it by more than 3 %, for later qk_gram
 * calls on the same A, B and split depth (cached with A's
 * tensor-core operands, dropped by qk_mps_free(A), and for the rest of the
 * process for any Gram of the same shape: device, N_A, N_B, n, largest bond
 * dimensions, split depth, symmetric or not).  qk_gram tunes by itself
 * when the Gram has at least 64 default tiles per CTA; smaller Grams use 4
 * kets per tile in bands of 16 unless a schedule was tuned or set.
 *   prec     QK_PREC_SPLIT_BF16 or QK_PREC_SPLIT_BF16X3.
 *   kets_per_tile, band, us_per_pair   optional host outs: the chosen
 *            schedule and its device time per pair on the sample.
 * A schedule already cached (tuned or set) is returned without timing.
 * Synchronises.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT.
 *
 * qk_set_split_schedule fixes the schedule for (A, B, prec) instead:
 * kets_per_tile in 1..4, band >= 1.  Every schedule computes the same
 * entries; only their order and grouping on the GPU change.
 * ---------------------------------------------------------------------- */
qk_status qk_tune_split(const qk_mps_batch* A, const qk_mps_batch* B,
                        qk_prec prec, void* stream, int32_t* kets_per_tile,
                        int32_t* band, double* us_per_pair);
qk_status qk_set_split_schedule(const qk_mps_batch* A, const qk_mps_batch* B,
                                qk_prec prec, int32_t kets_per_tile,
                                int32_t band);

/* Test hook for the failure path (the paper has no counterpart): when `on`,
 * the next launch of the tensor-core overlap kernel lets one bounded wait of
 * CTA 0 run out (a 10 ms wait on a barrier nothing arrives at, in the middle
 * of a GEMM with bulk copies and MMAs in flight).  The CTA then drains what
 * it issued, frees its TMEM and exits, and the call returns QK_ERR_TIMEOUT;
 * the device stays usable.  Consumed by that launch. */
qk_status qk_debug_stall_next_split(int32_t on);

/* Profiling switch of the tensor-core overlap kernel (the paper has no
 * counterpart).  While `on`, every launch of the kernel sums per-CTA clock64
 * cycles by phase; qk_last_tc_profile returns those of the last launch on
 * this thread: counters[11] = thread 0's cycles inside the MMA-issue loop,
 * waiting for operand copies, waiting for ring space; the CTA's cycles
 * waiting for the MMAs, in the epilogue, at the barrier after it (all seen
 * by thread 0, summed over CTAs); GEMMs, K-chunks and tiles processed; and
 * thread 0's cycles in the ring bookkeeping and copy issue (ring waits
 * included) and in issuing the MMAs of a chunk.
 * ctas: CTAs of that launch.  No synchronisation. */
qk_status qk_debug_tc_profile(int32_t on);
/* Test knob: caps the grid of the tensor-core overlap kernel at `ctas` CTAs
 * (0 restores the default of one wave at full residency).  Results do not
 * depend on it; only the schedule's spread over the SMs changes. */
qk_status qk_debug_tc_max_ctas(int32_t ctas);
/* Operand-stream variant of the next tensor-core overlap launches (the
 * paper has no counterpart): a bit set in `flags` (0..15) turns on
 *   1  an L2 prefetch of a GEMM's whole static operand block when its first
 *      chunk is issued,
 *   2  an L2 prefetch of the next site's static blocks when a site starts,
 *   4  the normal L2 priority for the static operands (default: evict-first),
 *   8  dropping the L2 lines of a consumed environment or half-step block
 *      without write-back (the next reader finds it rewritten in full).
 * Results do not depend on it (the same MMAs on the same data); only where
 * the operand bytes come from changes.  The default is 8 (the fastest
 * measured).  QK_ERR_INVALID_ARG outside 0..15. */
qk_status qk_debug_tc_variant(int32_t flags);
qk_status qk_last_tc_profile(double* counters, int32_t* ctas);

/* ------------------------------------------------------------------------
 * qk_gram_pairs_noalloc - the FP64 pair overlaps of qk_gram_pairs
 * (QK_PREC_FP64) without any device or host allocation inside the call.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate during the work, e.g. a host application that owns the
 * whole device memory pool through its own allocator, or a latency-bound
 * loop that cannot afford the device-wide synchronisation a cudaMalloc /
 * cudaFree may cause.
 *   A, B     batches on the current device with equal n and storage
 *            precision; every bond dimension must be <= 64.
 *   pairs    device int32 [P][2], indices in range (checked through a fixed
 *            stack buffer before the launch).
 *   K_out    device float64 [P].
 * Scratch is a file-scope device array of 37.7 MB (a 256-byte work counter
 * plus one 384 KiB slice per CTA for 96 CTAs), which every device that loads
 * the library holds until the process exits.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, once per
 * device); make that first call before any stream capture.  Every call
 * shares the array: the work counter is cleared at the start of each call,
 * and calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it, so serialise them.  Synchronises.
 * Errors: INVALID_ARG (bond dimension above 64, host pointers, index out of
 * range, mismatched batches), CUDA.
 * ---------------------------------------------------------------------- */
qk_status qk_gram_pairs_noalloc(const qk_mps_batch* A, const qk_mps_batch* B,
                                const int32_t* pairs, int64_t P, double* K_out,
                                void* stream);

/* ------------------------------------------------------------------------
 * Learned surrogate for log K (not in the paper).  A 3-layer MLP
 *   f -> ReLU(W1 f + b1) -> ReLU(W2 h + b2) -> w3 . h + b3
 * on the symmetric pair features f(x, y) = [(x - y)^2, (x + y)/2] (2n values),
 * bf16 weights and activations in the products, FP32 accumulation and FP32
 * master weights, Adam.  Its predictions of log K are accepted only where a
 * split-conformal bound (per bin of predicted value) is within `tol`; every
 * other entry falls back to the exact MPS overlap.
 * ---------------------------------------------------------------------- */
/* in_dim must be 2n, 16 <= in_dim <= 4096; hidden a multiple of 16 in
 * [16, 1024].  Weights are He-uniform from a counter-based generator seeded
 * by `seed`; biases zero. */
qk_status qk_surrogate_create(int32_t in_dim, int32_t hidden, uint64_t seed,
                              qk_surrogate** out);
qk_status qk_surrogate_free(qk_surrogate* net);
/* Parameter transfer in FP32, order W1[h][in], b1[h], W2[h][h], b2[h],
 * W3[h], b3[1]; host buffers of qk_surrogate_param_count() floats. */
int64_t qk_surrogate_param_count(const qk_surrogate* net);
qk_status qk_surrogate_get_params(const qk_surrogate* net, float* params);
qk_status qk_surrogate_set_params(qk_surrogate* net, const float* params);
/* Arithmetic of the products: on (default) rounds every GEMM operand to bf16
 * (FP32 accumulation); off keeps FP32 operands (used to check the kernels
 * against an FP64 reference without the bf16 rounding). */
qk_status qk_surrogate_set_bf16(qk_surrogate* net, int32_t on);
/* Target standardisation: the network fits (t - mean) / scale. */
qk_status qk_surrogate_set_target_scale(qk_surrogate* net, double mean,
                                        double scale);

/* Loss and gradient of one batch, no update (for parity checks).
 *   Xa, Xb   host or device float64 [Na][n], [Nb][n]; pairs [P][2] int32;
 *   target   host or device float64 [P] (log K, before standardisation).
 *   grads    optional host float32 [param_count], same order as params.
 *   loss     optional host out: (1/2P) sum (yhat - t')^2 on standardised t'. */
qk_status qk_surrogate_loss_grad(qk_surrogate* net, const double* Xa,
                                 int64_t Na, const double* Xb, int64_t Nb,
                                 int32_t n, const int32_t* pairs,
                                 const double* target, int64_t P,
                                 float* grads, double* loss, void* stream);
/* Adam training: `epochs` passes over the P pairs in shuffled minibatches of
 * `batch` (seeded by `seed`), learning rate lr, betas (0.9, 0.999), eps 1e-8.
 * loss_out optional host float64: mean loss of the last epoch. */
qk_status qk_surrogate_train(qk_surrogate* net, const double* Xa, int64_t Na,
                             const double* Xb, int64_t Nb, int32_t n,
                             const int32_t* pairs, const double* target,
                             int64_t P, int32_t epochs, int32_t batch,
                             float lr, uint64_t seed, void* stream,
                             double* loss_out);
/* Predicted log K (de-standardised) for P pairs; y: host or device float64. */
qk_status qk_surrogate_predict(const qk_surrogate* net, const double* Xa,
                               int64_t Na, const double* Xb, int64_t Nb,
                               int32_t n, const int32_t* pairs, int64_t P,
                               double* y, void* stream);
/* Split-conformal calibration on held-out exact log K: n_bins equal-count
 * bins of predicted value, per-bin bound = ceil((m+1)(1-alpha))-th smallest
 * |pred - truth| (inf where a bin is too small).  Synchronises. */
qk_status qk_surrogate_calibrate(qk_surrogate* net, const double* Xa,
                                 int64_t Na, const double* Xb, int64_t Nb,
                                 int32_t n, const int32_t* pairs,
                                 const double* truth, int64_t P, double alpha,
                                 int32_t n_bins, void* stream);
/* Per-bin bounds after calibration: edges host [n_bins+1], bounds [n_bins]. */
qk_status qk_surrogate_bins(const qk_surrogate* net, int32_t* n_bins,
                            double* edges, double* bounds);

/* ------------------------------------------------------------------------
 * qk_gram_surrogate - the N_A x N_B block K[i][j] (test-vs-train use) with
 * the surrogate first: where the calibrated bound of the predicted log K is
 * <= tol the entry is exp(prediction), otherwise it is the exact overlap of
 * states A[i], B[j] computed with `prec`.
 *   Xa, Xb    the data vectors of A and B (host or device, float64 [N][n]).
 *   K         host or device float64, leading dimension ldk.
 *   accepted  optional host or device uint8 [N_A][N_B]: 1 where the surrogate
 *             value was used.
 *   n_accepted optional host out.
 * Synchronises.  Errors: INVALID_ARG (uncalibrated net, shape mismatch), OOM,
 * CUDA.
 * ---------------------------------------------------------------------- */
qk_status qk_gram_surrogate(const qk_surrogate* net, const qk_mps_batch* A,
                            const qk_mps_batch* B, const double* Xa,
                            const double* Xb, double tol, double* K,
                            int64_t ldk, uint8_t* accepted, qk_prec prec,
                            void* stream, int64_t* n_accepted);

#ifdef __cplusplus
}
#endif

#endif /* QK_H_ */
