// Split-precision transfer sweep (Fig. 2) on the tcgen05 tensor cores.
//
// Per site k every pair (i, j) updates its environment E (chi^i_k x chi^j_k)
// in two half-steps, both complex GEMMs:
//   HS1 (ket side):  T_s[a][b'] = sum_b E[a][b] B_j[s][b][b']
//   HS2 (bra side):  E'[a'][b'] = sum_{s,a} conj(A_i[s][a][a']) T_s[a][b']
// A CTA takes one bra i and up to kG kets (the tile schedule's choice);
// HS2 stacks the kets' columns so the bra tensor is read once for all of them.  Operands as GEMM factors:
//   HS1: D1[(s,b'), a]   = Bt_j[(s,b'), b] . Et[b, a]        (A static, B = E)
//   HS2: D2[a', (j,b')]  = Ah_i[a', (s,a)] . T[(s,a), (j,b')] (A static, B = T)
// Every operand is stored K-major in 16-wide K chunks of 8x(16 B) core
// matrices (no swizzle), as bf16 parts of re and im, each value split into
// P parts x = x0 + x1 (+ x2), x_{k+1} = bf16(x - x0 - .. - x_k):
//   P = 2: residual <= 2^-17 |x|; products 00, 01, 10 (order >= 2^-8 kept,
//          lo*lo dropped);
//   P = 3: exact for any FP32 value; products 00, 01, 10, 02, 11, 20 (order
//          >= 2^-16 kept).
// The static (per-state) operands Bt/Ah are packed once per batch
// (tc_pack_kernel) as 2P planes (re parts, im parts).  The dynamic operands
// E^T and T hold, per part, the rows [re; im; -re], so one MMA of width 2N
// over rows [re; im] and one with the A-negate bit over rows [im; -re] add
// [Ar Br - Ai Bi | Ar Bi + Ai Br] into a single FP32 accumulator [re | im]
// in TMEM: 2 MMAs per product and K chunk.  E and T live in a per-CTA global
// scratch that the epilogue writes (tcgen05.ld -> split -> st.global) and
// the next GEMM streams back with 1-D bulk copies.  Within a CTA one producer
// thread (warp 1) issues the bulk copies into a byte ring of up to eight
// chunks and reclaims the space of chunks whose MMAs have completed, while
// thread 0 waits for each chunk and issues its MMAs, so copy issue and MMA
// issue overlap; four CTAs per SM (P = 2; three at P = 3) overlap one
// another's epilogues and copy waits.  Every
// wait is bounded in time and reports QK_ERR_TIMEOUT instead of hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qk_internal.h"
#include "tc_ptx.cuh"

namespace qk {

qk_status overlap_fp64(const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                       int64_t P, double* dK, int64_t ldk, bool sym, cudaStream_t st,
                       int ctas_per_sm = 4);

namespace {

constexpr int kThreads = 128;
constexpr int kG = 4;            // kets per tile at most
// Residency: QK_TC_CTAS CTAs per SM share its 512 TMEM columns and shared
// memory; the N of one MMA (kNMax) is sized so re and im accumulators fit.
#ifndef QK_TC_CTAS
#define QK_TC_CTAS 4
#endif
constexpr int kCtas = QK_TC_CTAS;
// complex columns of one MMA (its N' is 2 kNMax: [re | im]); the accumulator
// takes 2 kNMax TMEM columns
#ifndef QK_TC_NMAX
#define QK_TC_NMAX (QK_TC_CTAS <= 2 ? 128 : 64)
#endif
constexpr int kNMax = QK_TC_NMAX;
constexpr int kTmemCols = 2 * kNMax;
static_assert(kNMax == 64 || kNMax == 128, "one MMA covers 64 or 128 complex columns");
static_assert(kCtas * kTmemCols <= 512, "the CTAs of an SM share its 512 TMEM columns");
#ifndef QK_TC_RING_MIN
#define QK_TC_RING_MIN 1
#endif
template <int P>
struct Stage {
  static constexpr int A = 128 * 32 * 2 * P;    // 128 rows of one 16-wide K chunk, all planes
  static constexpr int B = kNMax * 32 * 3 * P;  // up to kNMax complex rows, [re; im; -re] per part
  static constexpr int want = P == 2 ? kCtas : (kCtas < 3 ? kCtas : 3);
  static constexpr int fit = ((220 * 1024 / want) / 1024) * 1024;
  // ring: what the SM's shared memory allows per CTA, at least QK_TC_RING_MIN
  // chunks of the largest size (one is enough for correctness: the producer
  // restarts an empty ring at offset 0)
  static constexpr int ring = fit > QK_TC_RING_MIN * (A + B) ? fit : QK_TC_RING_MIN * (A + B);
  static_assert(QK_TC_RING_MIN >= 1, "the ring holds at least one chunk of the largest size");
  // CTAs that actually fit an SM with that ring (static shared memory and the
  // per-CTA reservation included), at most the requested count
  static constexpr int fits = (228 * 1024) / (ring + 2048);
  static constexpr int ctas_per_sm = want < fits ? want : fits;
};

__host__ __device__ inline int pad16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int mrows_of(int rows) { return rows <= 64 ? 64 : 128; }
__host__ __device__ inline int ntiles_of(int rows) { return rows <= 64 ? 1 : (rows + 127) / 128; }
// rows stored for M tile t of a static operand with `rows` rows (no padding)
__host__ __device__ inline int tile_rows(int rows, int t) { return rows - 128 * t < 128 ? rows - 128 * t : 128; }

// element offset of (complex row, k) in a dynamic B operand (E^T or T).
// Layout: [kchunk][kNMax-row tile t][part][3 rows_t x 16], rows_t =
// min(kNMax, rows - kNMax t), where the 3 rows_t rows of a part block are the
// part's re rows, then its im rows, then its re rows negated (which = 0, 1,
// 2), each block in the K-major core-matrix layout.  One N slice of one chunk
// is then one contiguous block, and the MMA pair of a complex product reads
// rows [0, 2 rows_t) = [re; im] and rows [rows_t, 3 rows_t) = [im; -re].
template <int P>
__host__ __device__ inline int64_t dyn_off(int row, int k, int part, int which, int rows) {
  const int kc = k >> 4, k16 = k & 15;
  const int t = (int)((unsigned)row / kNMax), r = (int)((unsigned)row % kNMax);  // row >= 0
  const int rows_t = min(kNMax, rows - kNMax * t);
  const int R = which * rows_t + r;
  return (int64_t)kc * P * 3 * rows * 16 + (int64_t)t * P * 3 * kNMax * 16 + (int64_t)part * 3 * rows_t * 16 +
         (R >> 3) * 128 + (k16 >> 3) * 64 + (R & 7) * 8 + (k16 & 7);
}

// element offset of (row, k) in a [kchunk][plane][rows x 16] block
template <int PL>
__host__ __device__ inline int64_t blk_off(int row, int k, int plane, int rows) {
  const int kc = k >> 4, k16 = k & 15;
  return ((int64_t)kc * PL + plane) * rows * 16 + (row >> 3) * 128 + (k16 >> 3) * 64 + (row & 7) * 8 +
         (k16 & 7);
}

// ---------------------------------------------------------------- packing
struct PackArgs {
  const uint64_t* site_ptr;  // [N][n]
  const int32_t* dims;       // [N][n+1]
  int n;
  int store;                 // 1: complex64, 0: complex128
  const int64_t* bt_off;     // [N][n] byte offsets
  const int64_t* ah_off;
  char* arena;
};

template <int P>
__device__ inline void splitp(float x, __nv_bfloat16* o) {
  float r = x;
#pragma unroll
  for (int i = 0; i < P; ++i) {
    o[i] = __float2bfloat16_rn(r);
    r -= __bfloat162float(o[i]);
  }
}

template <int P>
__global__ void tc_pack_kernel(PackArgs p) {
  constexpr int kParts = P, kPlanes = 2 * P;
  const int s = blockIdx.y, k = blockIdx.x;
  const int n = p.n;
  const int c0 = p.dims[(int64_t)s * (n + 1) + k], c1 = p.dims[(int64_t)s * (n + 1) + k + 1];
  const int p0 = pad16(c0), p1 = pad16(c1);
  const void* src = (const void*)p.site_ptr[(int64_t)s * n + k];
  auto val = [&](int q, int a, int b) -> float2 {  // A[q][a][b]
    int64_t idx = ((int64_t)q * c0 + a) * c1 + b;
    if (p.store) return reinterpret_cast<const float2*>(src)[idx];
    double2 v = reinterpret_cast<const double2*>(src)[idx];
    return make_float2((float)v.x, (float)v.y);
  };
  // ket form Bt[(q, b'), b] = A[q][b][b'], rows 2*p1 in M tiles of 128 rows
  // stored without padding rows (tile t holds tile_rows(rows, t) rows), K = p0
  {
    const int rows = 2 * p1;
    __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(p.arena + p.bt_off[(int64_t)s * n + k]);
    const int total = rows * p0;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int R = e / p0, b = e % p0;
      const int t = R / 128, r = R % 128;
      const int rt = tile_rows(rows, t);
      float2 v = make_float2(0.f, 0.f);
      const int q = R / p1, bp = R % p1;
      if (bp < c1 && b < c0) v = val(q, b, bp);
      __nv_bfloat16* blk = base + (int64_t)t * 128 * p0 * kPlanes;
      __nv_bfloat16 h[kPlanes];
      splitp<P>(v.x, h);
      splitp<P>(v.y, h + kParts);
      for (int pl = 0; pl < kPlanes; ++pl) blk[blk_off<kPlanes>(r, b, pl, rt)] = h[pl];
    }
  }
  // bra form Ah[a', (q, a)] = conj(A[q][a][a']), rows p1 (<= 128), K = 2*p0
  {
    __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(p.arena + p.ah_off[(int64_t)s * n + k]);
    const int total = p1 * 2 * p0;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int r = e / (2 * p0), K = e % (2 * p0);
      const int q = K / p0, a = K % p0;
      float2 v = make_float2(0.f, 0.f);
      if (r < c1 && a < c0) {
        v = val(q, a, r);
        v.y = -v.y;
      }
      __nv_bfloat16 h[kPlanes];
      splitp<P>(v.x, h);
      splitp<P>(v.y, h + kParts);
      for (int pl = 0; pl < kPlanes; ++pl) base[blk_off<kPlanes>(r, K, pl, p1)] = h[pl];
    }
  }
}

// ---------------------------------------------------------------- PTX helpers
using namespace tcx;  // smem_u32, make_desc, make_idesc, mma, commit, now_ns, wait_bar (tc_ptx.cuh)

// L2 policies: streamed static operands go first, the per-CTA E/T scratch last
__device__ inline uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ inline uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ inline void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 prefetch of a byte range (16-byte aligned start, size a multiple of 16),
// in pieces of at most 32 KB; nothing waits for it
__device__ inline void prefetch_l2(const void* src, uint32_t bytes) {
  const char* p = static_cast<const char*>(src);
  for (uint32_t o = 0; o < bytes; o += 32768u) {
    const uint32_t b = bytes - o < 32768u ? bytes - o : 32768u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(b) : "memory");
  }
}

// Drops the whole 128-byte L2 lines of [p, p + bytes) without writing them
// back (p 128-byte aligned); threads of the CTA take the lines in turn.
__device__ inline void discard_l2(const char* p, int64_t bytes) {
  for (int64_t o = (int64_t)threadIdx.x * 128; o + 128 <= bytes; o += (int64_t)blockDim.x * 128)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p + o) : "memory");
}

__device__ inline uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ inline void st_v4_last(void* p, uint4 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(policy)
               : "memory");
}

__device__ inline void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 16 consecutive accumulator columns of this thread's lane from each of two
// TMEM addresses (the re and im halves), one wait for both loads
__device__ inline void tmem_ld16x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[16], q[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
        "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(q[i]);
  }
}

// split 16 floats into P bf16 planes, two values per cvt.rn.bf16x2
template <int P>
__device__ inline void split16(const float* x, uint32_t (*o)[8]) {
  float r[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = x[i];
#pragma unroll
  for (int part = 0; part < P; ++part) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      __nv_bfloat162 b = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
      o[part][i] = *reinterpret_cast<uint32_t*>(&b);
      if (part + 1 < P) {
        float2 f = __bfloat1622float2(b);
        r[2 * i] -= f.x;
        r[2 * i + 1] -= f.y;
      }
    }
  }
}

// store 16 consecutive K values (re, im) of one row as the 2P bf16 planes
template <int P>
__device__ inline void store_row16(__nv_bfloat16* blk, int row, int k, int rows, const float* re,
                                   const float* im, uint64_t policy) {
  uint32_t hr[P][8], hi[P][8];
  split16<P>(re, hr);
  split16<P>(im, hi);
#pragma unroll
  for (int part = 0; part < P; ++part) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const uint32_t* r4 = hr[part] + 4 * half;
      const uint32_t* i4 = hi[part] + 4 * half;
      // splitting is odd-symmetric, so the parts of -re are the negated parts of re
      const uint32_t sgn = 0x80008000u;
      st_v4_last(blk + dyn_off<P>(row, k + 8 * half, part, 0, rows), make_uint4(r4[0], r4[1], r4[2], r4[3]),
                 policy);
      st_v4_last(blk + dyn_off<P>(row, k + 8 * half, part, 1, rows), make_uint4(i4[0], i4[1], i4[2], i4[3]),
                 policy);
      st_v4_last(blk + dyn_off<P>(row, k + 8 * half, part, 2, rows),
                 make_uint4(r4[0] ^ sgn, r4[1] ^ sgn, r4[2] ^ sgn, r4[3] ^ sgn), policy);
    }
  }
}

// ---------------------------------------------------------------- overlap kernel
struct TcArgs {
  const int32_t* a_dims;
  const int64_t* a_ah;
  const char* a_arena;
  const int32_t* b_dims;
  const int64_t* b_bt;
  const char* b_arena;
  int n;
  int mode;                  // 0 symmetric full, 1 rectangular full, 2 pair list
  int kets;                  // kets per tile, 1..kG (modes 0/1)
  int64_t n_tiles;
  const int32_t* tiles;      // modes 0/1: (bra i, first ket j0) per tile, banded order
  int NA, NB;
  const int32_t* pairs;      // mode 2
  double* K;
  int64_t ldk;
  char* scratch;
  int64_t scratch_stride;
  int64_t et_stride;
  unsigned long long* queue;
  int* err;
  int stall;                 // test hook: CTA 0 lets one bounded wait run out mid-GEMM
  int flags;                 // kPrefetchGemm | kPrefetchSite | kStaticNormal | kDiscardScratch
  unsigned long long* prof;  // optional [kProfN] cycle counters summed over CTAs
};

// Phase counters of the profiling switch (qk_debug_tc_profile): clock64
// cycles of thread 0 in its copy waits, ring waits and issue loop, and of
// the CTA (as seen by thread 0) waiting for the MMAs, in the epilogue and at
// the barrier after it; plus GEMM, chunk and tile counts.
enum TcProfIdx { TP_ISSUE = 0, TP_WFULL, TP_WRING, TP_DONE, TP_EPI, TP_SYNC, TP_GEMMS, TP_CHUNKS, TP_TILES, TP_TOPUP,
                 TP_MMA, kProfN };
struct TcProf {  // in shared memory, written by thread 0 only
  unsigned long long v[kProfN];
  unsigned long long t;  // last mark
};

constexpr int kSlots = 8;  // chunks in flight at most (one mbarrier pair each)
// Operand-stream variants (qk_debug_tc_variant): L2 prefetch of a GEMM's
// whole static block when its first chunk is issued (the ring holds only
// two or three chunks); L2 prefetch of the next site's static blocks (bra
// and kets) when a site starts; static operands loaded with the normal L2
// priority instead of evict-first; dropping the L2 lines of a consumed
// E^T / T block without write-back (its next reader finds it rewritten in
// full by the epilogue that precedes it).
constexpr int kPrefetchGemm = 1, kPrefetchSite = 2, kStaticNormal = 4, kDiscardScratch = 8;
#ifndef QK_TC_VARIANT
#define QK_TC_VARIANT 8  // kDiscardScratch: the measured best (0.9 % over none)
#endif
constexpr int kProducer = 32;  // the thread (lane 0 of warp 1) that issues the bulk copies

// test hook (qk_debug_stall_next_split): the next tensor-core launch lets one
// bounded wait run out
std::atomic<int> g_stall_next{0};
// profiling switch (qk_debug_tc_profile) and the counters of the last
// profiled launch on this thread
std::atomic<int> g_tc_profile{0};
// test knob (qk_debug_tc_max_ctas): cap on the grid of the tensor-core kernel (0: none)
std::atomic<int> g_tc_max_ctas{0};
// operand-stream variant flags of the next launches (kPrefetchGemm, ...)
std::atomic<int> g_tc_variant{QK_TC_VARIANT};
thread_local unsigned long long g_tc_prof_last[kProfN] = {};
thread_local int g_tc_prof_ctas = 0;
thread_local unsigned long long* g_tc_prof_pending = nullptr;

struct __align__(8) TcShared {
  uint64_t full[kSlots];
  uint64_t empty[kSlots];
  uint64_t done;
  uint64_t drain;   // tcgen05.commit target when an aborting CTA drains its MMAs
  uint64_t stall;   // never arrived at (test hook)
  uint32_t tmem;
  int abort;
  int64_t tile;
  uint32_t roff[kSlots];  // ring offset of the chunk in each slot (producer -> MMA thread)
  uint32_t issued;        // chunks whose copies were issued (for the abort drain)
};

// Byte ring of operand chunks in shared memory (thread 0's bookkeeping).
// Chunk g (a running count over all GEMMs of the CTA) uses mbarrier slot
// g % kSlots; its A and B blocks sit contiguously at off[slot], len[slot]
// bytes including any padding skipped at the ring's end.  Chunks are
// reclaimed in order once the MMAs that read them have completed.
struct Ring {  // producer state
  uint32_t produced = 0, released = 0;  // chunks issued / reclaimed so far
  // The live chunks occupy the `used` bytes (padding included) that end at
  // the write position `wpos`, circularly.  Both stay below the ring size, so
  // nothing wraps however many bytes a CTA streams (a byte counter taken
  // modulo the ring size, as an earlier version did, jumps when the counter
  // wraps at 2^32 and places new chunks on live ones).
  uint32_t wpos = 0, used = 0;
  uint32_t len[kSlots];
};

// Operands of one GEMM: `nchunks` 16-wide K chunks of a static A block
// (a_rows rows of 2P planes, a_bytes per chunk, consecutive) and a dynamic B
// block (N complex rows as [re; im; -re] per part, b_bytes per chunk, chunk
// stride b_stride); M accumulator rows.
struct Gemm {
  const char* gA;
  uint32_t a_bytes;
  int a_rows;
  const char* gB;
  uint32_t b_bytes;
  int64_t b_stride;
  int nchunks, M, N;
};

// The MMA reads M rows of every A plane; the planes hold a_rows <= M rows, so
// the last plane's read runs (M - a_rows) rows past the A block.  The ring
// reserves that span (the extra rows feed unused accumulator rows).
template <int P>
__device__ inline uint32_t a_span_of(const Gemm& g) {
  return (uint32_t)(2 * P - 1) * g.a_rows * 32 + (uint32_t)g.M * 32;
}

// Bounded wait that also gives up once another thread of the CTA has aborted.
__device__ inline bool wait_or_abort(TcShared& sh, uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 0) {
      if (*(volatile int*)&sh.abort) return false;
      const unsigned long long t = now_ns();
      if (it == 0)
        t0 = t;
      else if (t - t0 > kTimeoutNs)
        return false;
    }
  }
}

// Producer (one thread of warp 1): streams the chunks of one GEMM through the
// ring with bulk copies, as far ahead as the ring's bytes and mbarrier slots
// allow, and reclaims the space of chunks whose MMAs have completed.  Every
// issued chunk is consumed in order by the MMA thread, so waiting for the
// oldest live chunk always ends.
template <int P>
__device__ bool gemm_produce(TcShared& sh, char* ring, Ring& rg, const Gemm& g, uint64_t pol_a, uint64_t pol_b,
                             bool prefetch, TcProf* pf) {
  const unsigned long long t_in = pf ? clock64() : 0ull;
  // the static chunks beyond the ring's depth then come from L2
  if (prefetch && g.nchunks > 1) prefetch_l2(g.gA, (uint32_t)g.nchunks * g.a_bytes);
  constexpr uint32_t R = Stage<P>::ring;
  const uint32_t a_span = a_span_of<P>(g), size = a_span + g.b_bytes;
  const uint32_t g0 = rg.produced;
  for (int p = 0; p < g.nchunks; ++p) {
    const uint32_t gi = g0 + p;
    uint32_t pad, need;
    for (;;) {
      if (rg.used == 0) rg.wpos = 0;  // an empty ring restarts at its start
      pad = rg.wpos + size > R ? R - rg.wpos : 0;  // a chunk never straddles the end
      need = pad + size;
      // fits, or wait for the oldest live chunk (one exists whenever the
      // ring is not empty or the slots are all taken; an empty ring always
      // fits a chunk since R >= size)
      if (rg.used + need <= R && gi - rg.released < (uint32_t)kSlots) break;
      const uint32_t j = rg.released, js = j % kSlots;
      const unsigned long long t0 = pf ? clock64() : 0ull;
      if (!wait_or_abort(sh, &sh.empty[js], (j / kSlots) & 1)) return false;
      if (pf) pf->v[TP_WRING] += clock64() - t0;
      rg.used -= rg.len[js];
      ++rg.released;
    }
    const uint32_t slot = gi % kSlots, off = pad ? 0u : rg.wpos;
    sh.roff[slot] = off;
    rg.len[slot] = need;
    rg.used += need;
    rg.wpos = off + size == R ? 0u : off + size;
    expect_tx(&sh.full[slot], g.a_bytes + g.b_bytes);
    bulk_load(ring + off, g.gA + (int64_t)p * g.a_bytes, g.a_bytes, &sh.full[slot], pol_a);
    bulk_load(ring + off + a_span, g.gB + (int64_t)p * g.b_stride, g.b_bytes, &sh.full[slot], pol_b);
    sh.issued = gi + 1;
  }
  rg.produced = g0 + g.nchunks;
  if (pf) pf->v[TP_TOPUP] += clock64() - t_in;
  return true;
}

// Consumer (thread 0): waits for each chunk and issues its split products,
// 2 MMAs of width 2N per product into the accumulator [re | im] (TMEM columns
// [0, 2N)), commits each chunk to its `empty` barrier and the GEMM to `done`.
template <int P>
__device__ bool gemm_consume(TcShared& sh, char* ring, uint32_t& consumed, uint32_t& waited, const Gemm& g,
                             bool& stall, TcProf* pf) {
  const unsigned long long t_in = pf ? clock64() : 0ull;
  if (pf) {
    pf->v[TP_GEMMS] += 1;
    pf->v[TP_CHUNKS] += g.nchunks;
  }
  const uint32_t id_pos = make_idesc(g.M, 2 * g.N, 0), id_neg = make_idesc(g.M, 2 * g.N, 1);
  const uint32_t t_acc = sh.tmem;
  const uint32_t a_span = a_span_of<P>(g);
  // bytes per plane: A is stored with a_rows rows (rows of the M tile past
  // a_rows read other data and only feed accumulator rows that are unused);
  // B part y is the block [re; im; -re] of 3N rows (32 bytes per row)
  const uint32_t pa = (uint32_t)g.a_rows * 32, pbp = (uint32_t)g.N * 96;
  const uint32_t g0 = consumed;
  for (int c = 0; c < g.nchunks; ++c) {
    const uint32_t gi = g0 + c, slot = gi % kSlots;
    if (stall && c == 1) {
      // test hook: a wait on a barrier nothing arrives at runs out while
      // chunk 0's MMAs and the later chunks' copies are in flight
      stall = false;
      if (!wait_bar(&sh.stall, 0, 10000000ull)) return false;
    }
    {
      const unsigned long long tw = pf ? clock64() : 0ull;
      if (!wait_or_abort(sh, &sh.full[slot], (gi / kSlots) & 1)) return false;
      if (pf) pf->v[TP_WFULL] += clock64() - tw;
    }
    waited = gi + 1;
    const unsigned long long t_mma = pf ? clock64() : 0ull;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t off = *(volatile uint32_t*)&sh.roff[slot];
    const uint32_t a0 = smem_u32(ring + off), b0 = a0 + a_span;
    // cross terms (x part, y part) kept
    constexpr int NT = P == 2 ? 3 : 6;
    const int xs[6] = {0, 0, 1, 0, 1, 2};
    const int ys[6] = {0, 1, 0, 2, 1, 0};
    const uint32_t acc = c > 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const uint64_t ar = make_desc(a0 + xs[t] * pa), ai = make_desc(a0 + (P + xs[t]) * pa);
      const uint32_t bp = b0 + ys[t] * pbp;
      // [re | im] += Ar [Br; Bi]^T ;  [re | im] += -Ai [Bi; -Br]^T
      mma(t_acc, ar, make_desc(bp), id_pos, t > 0 || acc);
      mma(t_acc, ai, make_desc(bp + (uint32_t)g.N * 32), id_neg, 1);
    }
    commit(&sh.empty[slot]);
    if (pf) pf->v[TP_MMA] += clock64() - t_mma;
  }
  commit(&sh.done);
  consumed = g0 + g.nchunks;
  if (pf) pf->v[TP_ISSUE] += clock64() - t_in;
  return true;
}

// lane -> accumulator row for M = 64 / 128 (64: rows 16w..16w+15 sit in the
// first 16 lanes of warp w)
__device__ inline int acc_row(int M) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (M == 128) return 32 * w + l;
  return l < 16 ? 16 * w + l : -1;
}

__device__ inline void sync_after_epilogue() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
}

template <int P>
__global__ void __launch_bounds__(kThreads, Stage<P>::ctas_per_sm) tc_overlap_kernel(TcArgs a) {
  constexpr int kPlanes = 2 * P;
  constexpr int kRowBytes = 32 * kPlanes;   // static operand: bytes per row of a 16-wide K chunk
  constexpr int kRowBytesB = 96 * P;        // dynamic operand: [re; im; -re] per part
  extern __shared__ __align__(1024) char dyn[];
  __shared__ TcShared sh;
  char* stage = dyn;
  const int tid = threadIdx.x;
  const int n = a.n;
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.done)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.drain)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.stall)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sh.abort = 0;
    sh.issued = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sh.tmem;
  const uint64_t pol_first = (a.flags & kStaticNormal) ? policy_evict_normal() : policy_evict_first();
  const uint64_t pol_last = policy_evict_last();
  const bool pf_gemm = (a.flags & kPrefetchGemm) != 0;
  Ring rg;                       // operand ring (the producer thread's state)
  uint32_t consumed = 0, waited = 0;  // the MMA thread's chunk counts
  bool stall = a.stall && blockIdx.x == 0;  // test hook, first GEMM of >= 2 chunks
  __shared__ TcProf s_prof;
  TcProf* pf = a.prof ? &s_prof : nullptr;  // written by thread 0 and the producer (disjoint counters)
  if (a.prof && tid == 0) {
    for (int f = 0; f < kProfN; ++f) s_prof.v[f] = 0ull;
    s_prof.t = clock64();
  }
  auto mark = [&](int what) {
    if (a.prof && tid == 0) {
      const unsigned long long t = clock64();
      s_prof.v[what] += t - s_prof.t;
      s_prof.t = t;
    }
  };
  uint32_t done_phase = 0;  // completed GEMMs (all threads)
  char* scr = a.scratch + (int64_t)blockIdx.x * a.scratch_stride;
  char* T_buf = scr + (int64_t)a.kets * a.et_stride;

  while (true) {
    if (tid == 0) sh.tile = (int64_t)atomicAdd(a.queue, 1ull);
    __syncthreads();
    const int64_t tile = sh.tile;
    if (tile >= a.n_tiles || sh.abort) break;
    if (a.prof && tid == 0) s_prof.v[TP_TILES] += 1;
    // ---- decode the tile: bra i, kets j[0..nk), output slots
    int i, nk = 0;
    int jj[kG];
    int64_t outp[kG];
    if (a.mode == 2) {
      i = a.pairs[2 * tile];
      jj[0] = a.pairs[2 * tile + 1];
      outp[0] = tile;
      nk = 1;
    } else {
      i = a.tiles[2 * tile];
      const int j0 = a.tiles[2 * tile + 1];
      // symmetric: only kets above the diagonal (the self-overlaps run separately)
      for (int j = (a.mode == 0 ? max(j0, i + 1) : j0); j < min(j0 + a.kets, a.NB); ++j) {
        jj[nk] = j;
        outp[nk] = (int64_t)i * a.ldk + j;
        ++nk;
      }
    }
    // ---- E_0 = [1]: Et blocks of 16 x 16 (one chunk), only (0, 0) = 1
    for (int q = 0; q < nk; ++q) {
      __nv_bfloat16* et = reinterpret_cast<__nv_bfloat16*>(scr + q * a.et_stride);
      for (int e = tid; e < 3 * P * 16 * 16; e += kThreads) et[e] = __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    if (tid < nk) {
      __nv_bfloat16* et = reinterpret_cast<__nv_bfloat16*>(scr + tid * a.et_stride);
      et[dyn_off<P>(0, 0, 0, 0, 16)] = __float2bfloat16_rn(1.f);    // re part 0
      et[dyn_off<P>(0, 0, 0, 2, 16)] = __float2bfloat16_rn(-1.f);   // its negation
    }
    sync_after_epilogue();
    const int32_t* da = a.a_dims + (int64_t)i * (n + 1);
    for (int k = 0; k < n; ++k) {
      const int ap = pad16(da[k]), ap1 = pad16(da[k + 1]);
      if ((a.flags & kPrefetchSite) && tid == kProducer && k + 1 < n) {
        // the next site's bra block Ah (p1 x 2 p0) and ket blocks Bt (2 p1 x p0)
        prefetch_l2(a.a_arena + a.a_ah[(int64_t)i * n + k + 1], (uint32_t)(ap1 * 2 * pad16(da[k + 2]) * 2 * kPlanes));
        for (int q = 0; q < nk; ++q) {
          const int32_t* db = a.b_dims + (int64_t)jj[q] * (n + 1);
          prefetch_l2(a.b_arena + a.b_bt[(int64_t)jj[q] * n + k + 1],
                      (uint32_t)(2 * pad16(db[k + 2]) * pad16(db[k + 1]) * 2 * kPlanes));
        }
      }
      int q0 = 0;
      while (q0 < nk) {
        // group kets while their stacked columns fit one MMA (<= kNMax); a
        // ket wider than kNMax forms a group of its own, split into slices
        int q1 = q0, ntot = 0;
        int nb[kG];
        while (q1 < nk) {
          const int w = pad16(a.b_dims[(int64_t)jj[q1] * (n + 1) + k + 1]);
          if (q1 > q0 && ntot + w > kNMax) break;
          nb[q1] = ntot;
          ntot += w;
          ++q1;
          if (ntot > kNMax) break;
        }
        // ---- HS1 for each ket of the group: D1[(s,b'), a] over N slices of a
        for (int q = q0; q < q1; ++q) {
          const int32_t* db = a.b_dims + (int64_t)jj[q] * (n + 1);
          const int bp = pad16(db[k]), bp1 = pad16(db[k + 1]);
          const int rows = 2 * bp1, mr = mrows_of(rows), nt = ntiles_of(rows);
          const char* bt = a.b_arena + a.b_bt[(int64_t)jj[q] * n + k];
          const char* et = scr + q * a.et_stride;
          for (int t = 0; t < nt; ++t) {
            for (int h0 = 0; h0 < ap; h0 += kNMax) {
              const int nh = min(kNMax, ap - h0);
              if (tid == 0 || tid == kProducer) {
                const int rt = tile_rows(rows, t);
                const Gemm g{bt + (int64_t)t * (bp / 16) * 128 * kRowBytes, (uint32_t)(rt * kRowBytes), rt,
                             et + (int64_t)h0 * kRowBytesB, (uint32_t)(nh * kRowBytesB),
                             (int64_t)ap * kRowBytesB, bp / 16, mr, nh};
                const bool ok = tid == 0 ? gemm_consume<P>(sh, stage, consumed, waited, g, stall, pf)
                                         : gemm_produce<P>(sh, stage, rg, g, pol_first, pol_last, pf_gemm, pf);
                if (!ok) {
                  sh.abort = 1;
                  atomicExch(a.err, 1);
                }
              }
              __syncthreads();
              if (sh.abort) goto finish;
              if (a.prof && tid == 0) s_prof.t = clock64();
              if (!wait_bar(&sh.done, done_phase & 1)) {
                sh.abort = 1;
                atomicExch(a.err, 1);
              }
              ++done_phase;
              asm volatile("tcgen05.fence::after_thread_sync;");
              mark(TP_DONE);
              {
                const int r = acc_row(mr);
                const int R = t * 128 + r;
                const uint32_t lane_base = (uint32_t)((tid >> 5) * 32) << 16;
                __nv_bfloat16* Tb = reinterpret_cast<__nv_bfloat16*>(T_buf);
                for (int c = 0; c < nh; c += 16) {
                  float re[16], im[16];
                  tmem_ld16x2(tmem + lane_base + c, tmem + lane_base + nh + c, re, im);
                  if (r >= 0 && R < rows) {
                    const int s = R / bp1, b1 = R % bp1;
                    store_row16<P>(Tb, nb[q] + b1, s * ap + h0 + c, ntot, re, im, pol_last);
                  }
                }
              }
              mark(TP_EPI);
              sync_after_epilogue();
              mark(TP_SYNC);
              if (sh.abort) goto finish;
            }
          }
        }
        // E^T of the group's kets is dead until the HS2 epilogue rewrites it
        // (every element of the next site's block, padding included)
        if (a.flags & kDiscardScratch)
          for (int q = q0; q < q1; ++q)
            discard_l2(scr + q * a.et_stride,
                       (int64_t)pad16(a.b_dims[(int64_t)jj[q] * (n + 1) + k]) * ap * 3 * P * 2);
        // ---- HS2 for the group: D2[a', (j,b')] over kNMax-row slices of T
        {
          const int mr = mrows_of(ap1);
          const char* ah = a.a_arena + a.a_ah[(int64_t)i * n + k];
          for (int h0 = 0; h0 < ntot; h0 += kNMax) {
            const int nh = min(kNMax, ntot - h0);
            if (tid == 0 || tid == kProducer) {
              const Gemm g{ah, (uint32_t)(ap1 * kRowBytes), ap1, T_buf + (int64_t)h0 * kRowBytesB,
                           (uint32_t)(nh * kRowBytesB), (int64_t)ntot * kRowBytesB, (2 * ap) / 16, mr, nh};
              const bool ok = tid == 0 ? gemm_consume<P>(sh, stage, consumed, waited, g, stall, pf)
                                       : gemm_produce<P>(sh, stage, rg, g, pol_first, pol_last, pf_gemm, pf);
              if (!ok) {
                sh.abort = 1;
                atomicExch(a.err, 1);
              }
            }
            __syncthreads();
            if (sh.abort) goto finish;
            if (a.prof && tid == 0) s_prof.t = clock64();
            if (!wait_bar(&sh.done, done_phase & 1)) {
              sh.abort = 1;
              atomicExch(a.err, 1);
            }
            ++done_phase;
            asm volatile("tcgen05.fence::after_thread_sync;");
            mark(TP_DONE);
            const int r = acc_row(mr);
            const uint32_t lane_base = (uint32_t)((tid >> 5) * 32) << 16;
            for (int q = q0; q < q1; ++q) {
              const int bp1 = pad16(a.b_dims[(int64_t)jj[q] * (n + 1) + k + 1]);
              // columns of this slice that belong to ket q
              const int c0 = max(nb[q], h0) - h0, c1 = min(nb[q] + bp1, h0 + nh) - h0;
              if (c0 >= c1) continue;
              if (k + 1 < n) {
                __nv_bfloat16* et = reinterpret_cast<__nv_bfloat16*>(scr + q * a.et_stride);
                for (int c = c0; c < c1; c += 16) {
                  float re[16], im[16];
                  tmem_ld16x2(tmem + lane_base + c, tmem + lane_base + nh + c, re, im);
                  if (r >= 0 && r < ap1) store_row16<P>(et, r, h0 + c - nb[q], ap1, re, im, pol_last);
                }
              } else if (nb[q] >= h0) {
                // last site: 1 x 1 environments, z = E[0][0]
                float re[16], im[16];
                tmem_ld16x2(tmem + lane_base + c0, tmem + lane_base + nh + c0, re, im);
                if (r == 0) {
                  const double zr = re[0], zi = im[0];
                  const double kv = zr * zr + zi * zi;
                  a.K[outp[q]] = kv;
                  if (a.mode == 0) a.K[(int64_t)jj[q] * a.ldk + i] = kv;
                }
              }
            }
            mark(TP_EPI);
            sync_after_epilogue();
            mark(TP_SYNC);
            if (sh.abort) goto finish;
          }
        }
        // T is dead until the next HS1 epilogue rewrites it (the barrier
        // after that GEMM's issue orders these drops before the writes)
        if (a.flags & kDiscardScratch) discard_l2(T_buf, (int64_t)2 * ap * ntot * 3 * P * 2);
        q0 = q1;
      }
    }
  }
finish:
  __syncthreads();
  if (tid == 0 && sh.abort) {
    // An aborting CTA may still have bulk copies landing in its ring and MMAs
    // writing its TMEM: wait (bounded) for every copy issued but not yet
    // waited for, then for every MMA this thread issued, before the TMEM is
    // freed and the CTA's shared memory is released.
    const uint32_t issued = *(volatile uint32_t*)&sh.issued;
    for (uint32_t gi = waited; gi < issued; ++gi) wait_bar(&sh.full[gi % kSlots], (gi / kSlots) & 1);
    commit(&sh.drain);
    wait_bar(&sh.drain, 0);
  }
  if (a.prof && tid == 0)
    for (int f = 0; f < kProfN; ++f) atomicAdd(a.prof + f, s_prof.v[f]);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// compaction of the entries that go to FP64: K < floor_v or K > ceil_v
__global__ void select_refine_kernel(const double* K, int64_t ldk, int NA, int NB, int sym, double floor_v,
                                     double ceil_v, int32_t* pairs, unsigned long long* count,
                                     unsigned long long cap) {
  const int64_t total = (int64_t)NA * NB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / NB), j = (int)(e % NB);
    if (sym && j <= i) continue;  // the self-overlaps are computed separately
    const double v = K[(int64_t)i * ldk + j];
    if (v < floor_v || v > ceil_v) {
      unsigned long long p = atomicAdd(count, 1ull);
      if (p < cap) {
        pairs[2 * p] = i;
        pairs[2 * p + 1] = j;
      }
    }
  }
}

// pair-list variant: positions p with K[p] > ceil_v
__global__ void select_refine_list_kernel(const double* K, const int32_t* pairs, int64_t P, double ceil_v,
                                          int32_t* sel_pairs, int64_t* sel_pos, unsigned long long* count) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    if (K[p] > ceil_v) {
      unsigned long long q = atomicAdd(count, 1ull);
      sel_pairs[2 * q] = pairs[2 * p];
      sel_pairs[2 * q + 1] = pairs[2 * p + 1];
      sel_pos[q] = p;
    }
  }
}

__global__ void scatter_kernel(const int32_t* pairs, const double* v, int64_t P, double* K, int64_t ldk, int sym) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    K[(int64_t)i * ldk + j] = v[p];
    if (sym) K[(int64_t)j * ldk + i] = v[p];
  }
}

__global__ void scatter_list_kernel(const int64_t* pos, const double* v, int64_t P, double* K) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
    K[pos[p]] = v[p];
}

// Per-batch packed operands, one arena per split depth (index P - 2).
struct TcArena {
  char* arena = nullptr;
  int64_t* d_bt = nullptr;
  int64_t* d_ah = nullptr;
  int64_t bytes = 0;
};
// Tile schedule of the full-Gram modes: kets per tile and bras per band.
struct TcSchedule {
  int kets = kG;
  int band = 16;
};
// A schedule chosen by measurement for (this batch as A, B, split depth, mode).
struct TcTuned {
  const qk_mps_batch* B;
  int P, mode;
  TcSchedule sch;
  double us_per_pair;
};
struct TcCache {
  TcArena part[2];
  std::vector<TcTuned> tuned;
};

// Tiles (bra i, first ket j0) of the pairs with i < i_lim and j0 < j_lim, in
// bands of sch.band bras; within a band the ket groups are the outer loop,
// so the CTAs running at the same time share kets (and bras) in L2.
// Symmetric (mode 0): strict upper triangle only.  Returns the number of
// pairs the tiles cover.
int64_t make_tiles(int mode, int64_t NB, const TcSchedule& sch, int64_t i_lim, int64_t j_lim,
                   std::vector<int32_t>& tiles) {
  tiles.clear();
  int64_t pairs = 0;
  for (int64_t i0 = 0; i0 < i_lim; i0 += sch.band) {
    const int64_t i1 = std::min<int64_t>(i_lim, i0 + sch.band);
    const int64_t jstart = mode == 0 ? i0 + 1 : 0;
    for (int64_t j0 = jstart; j0 < j_lim; j0 += sch.kets)
      for (int64_t i = i0; i < i1; ++i) {
        const int64_t jend = std::min<int64_t>(j0 + sch.kets, NB);
        const int64_t jbeg = mode == 0 ? std::max<int64_t>(j0, i + 1) : j0;
        if (jend <= jbeg) continue;  // no ket above the diagonal
        tiles.push_back((int32_t)i);
        tiles.push_back((int32_t)j0);
        pairs += jend - jbeg;
      }
  }
  return pairs;
}

template <int P>
qk_status ensure_tc_arena(qk_mps_batch* b, cudaStream_t st) {
  constexpr int kPlanes = 2 * P;
  if (!b->tc_cache) b->tc_cache = new TcCache();
  TcArena& c = ((TcCache*)b->tc_cache)->part[P - 2];
  if (c.arena) return QK_OK;
  const int n = b->n;
  const int64_t N = b->N;
  std::vector<int64_t> bt((size_t)N * n), ah((size_t)N * n);
  int64_t off = 0;
  for (int64_t s = 0; s < N; ++s)
    for (int k = 0; k < n; ++k) {
      const int c0 = b->h_dims[s * (n + 1) + k], c1 = b->h_dims[s * (n + 1) + k + 1];
      const int p0 = pad16(c0), p1 = pad16(c1);
      bt[s * n + k] = off;
      off += (int64_t)2 * p1 * p0 * 2 * kPlanes;
      ah[s * n + k] = off;
      off += (int64_t)p1 * 2 * p0 * 2 * kPlanes;
    }
  auto bail = [&](cudaError_t e, const char* w) {
    cudaFree(c.arena);
    cudaFree(c.d_bt);
    cudaFree(c.d_ah);
    c = TcArena();
    return cuda_fail(e, w);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&c.arena, off)) != cudaSuccess) return bail(e, "cudaMalloc(tc arena)");
  if ((e = cudaMalloc(&c.d_bt, sizeof(int64_t) * N * n)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMalloc(&c.d_ah, sizeof(int64_t) * N * n)) != cudaSuccess) return bail(e, "cudaMalloc");
  cudaMemcpyAsync(c.d_bt, bt.data(), sizeof(int64_t) * N * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(c.d_ah, ah.data(), sizeof(int64_t) * N * n, cudaMemcpyHostToDevice, st);
  PackArgs p;
  p.site_ptr = b->d_site_ptr;
  p.dims = b->d_dims;
  p.n = n;
  p.store = b->store == QK_STORE_C64 ? 1 : 0;
  p.bt_off = c.d_bt;
  p.ah_off = c.d_ah;
  p.arena = c.arena;
  for (int64_t s0 = 0; s0 < N; s0 += 65535) {
    const int64_t cnt = std::min<int64_t>(65535, N - s0);
    PackArgs q = p;
    q.site_ptr = p.site_ptr + s0 * n;
    q.dims = p.dims + s0 * (n + 1);
    q.bt_off = p.bt_off + s0 * n;
    q.ah_off = p.ah_off + s0 * n;
    tc_pack_kernel<P><<<dim3(n, (unsigned)cnt), 256, 0, st>>>(q);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "tc_pack_kernel");
  // the host offset tables must outlive the asynchronous copies
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "tc_pack_kernel");
  c.bytes = off;
  return QK_OK;
}

// Enqueues the kernel on `st` without waiting for it; *err_out receives the
// device error word for tc_finish (nullptr when nothing was launched).
// Modes 0/1 cover the tiles of make_tiles(sch, i_lim, j_lim); the full Gram
// is i_lim = N_A, j_lim = N_B.
template <int P>
qk_status launch_tc(const qk_mps_batch* A, const qk_mps_batch* B, int mode, const int32_t* d_pairs,
                    int64_t P_pairs, double* dK, int64_t ldk, cudaStream_t st, int** err_out,
                    const TcSchedule& sch, int64_t i_lim, int64_t j_lim) {
  *err_out = nullptr;
  qk_status rc = ensure_tc_arena<P>(const_cast<qk_mps_batch*>(A), st);
  if (rc != QK_OK) return rc;
  rc = ensure_tc_arena<P>(const_cast<qk_mps_batch*>(B), st);
  if (rc != QK_OK) return rc;
  const TcArena& ca = ((const TcCache*)A->tc_cache)->part[P - 2];
  const TcArena& cb = ((const TcCache*)B->tc_cache)->part[P - 2];
  int dev = 0, sms = 0;
  QK_CUDA(cudaGetDevice(&dev));
  QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  std::vector<int32_t> tiles;
  int64_t n_tiles = 0;
  const int kets = mode == 2 ? 1 : std::max(1, std::min(kG, sch.kets));
  if (mode == 2) {
    n_tiles = P_pairs;
  } else {
    TcSchedule s2 = sch;
    s2.kets = kets;
    s2.band = std::max(1, sch.band);
    make_tiles(mode, B->N, s2, std::min<int64_t>(i_lim, A->N), std::min<int64_t>(j_lim, B->N), tiles);
    n_tiles = (int64_t)tiles.size() / 2;
  }
  if (n_tiles == 0) return QK_OK;
  // scratch: `kets` Et blocks (<= 128 x 128) + T (<= 128 rows x 256 K), bf16 planes
  const int chi = std::max(A->chi_cap, B->chi_cap);
  const int cp = pad16(chi);
  // dynamic operands hold [re; im; -re] per part: 3 P bf16 rows per complex row
  const int64_t et_stride = (int64_t)cp * cp * 2 * 3 * P + 256;
  const int64_t t_bytes = (int64_t)128 * 2 * cp * 2 * 3 * P;
  const int64_t stride = ((kets * et_stride + t_bytes) + 1023) & ~int64_t(1023);
  int64_t ctas = std::min<int64_t>((int64_t)Stage<P>::ctas_per_sm * sms, n_tiles);
  if (g_tc_max_ctas.load() > 0) ctas = std::min<int64_t>(ctas, g_tc_max_ctas.load());
  char* scratch = nullptr;
  int32_t* d_tiles = nullptr;
  unsigned long long* queue = nullptr;
  int* err = nullptr;
  QK_CUDA(cudaMallocAsync(&scratch, stride * ctas, st));
  QK_CUDA(cudaMallocAsync(&queue, sizeof(unsigned long long), st));
  QK_CUDA(cudaMallocAsync(&err, sizeof(int), st));
  QK_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st));
  QK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  if (!tiles.empty()) {
    QK_CUDA(cudaMallocAsync(&d_tiles, sizeof(int32_t) * tiles.size(), st));
    QK_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int32_t) * tiles.size(), cudaMemcpyHostToDevice, st));
  }
  TcArgs a;
  a.a_dims = A->d_dims;
  a.a_ah = ca.d_ah;
  a.a_arena = ca.arena;
  a.b_dims = B->d_dims;
  a.b_bt = cb.d_bt;
  a.b_arena = cb.arena;
  a.n = A->n;
  a.mode = mode;
  a.kets = kets;
  a.n_tiles = n_tiles;
  a.tiles = d_tiles;
  a.NA = (int)A->N;
  a.NB = (int)B->N;
  a.pairs = d_pairs;
  a.K = dK;
  a.ldk = ldk;
  a.scratch = scratch;
  a.scratch_stride = stride;
  a.et_stride = et_stride;
  a.queue = queue;
  a.err = err;
  a.stall = g_stall_next.exchange(0);
  a.flags = g_tc_variant.load();
  a.prof = nullptr;
  if (g_tc_profile.load() && !g_tc_prof_pending) {
    QK_CUDA(cudaMallocAsync(&a.prof, sizeof(unsigned long long) * kProfN, st));
    QK_CUDA(cudaMemsetAsync(a.prof, 0, sizeof(unsigned long long) * kProfN, st));
    g_tc_prof_pending = a.prof;
    g_tc_prof_ctas = (int)ctas;
  }
  const int smem = Stage<P>::ring;
  QK_CUDA(cudaFuncSetAttribute(tc_overlap_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  QK_CUDA(cudaFuncSetAttribute(tc_overlap_kernel<P>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  timer_mark(false, st);
  tc_overlap_kernel<P><<<(int)ctas, kThreads, smem, st>>>(a);
  timer_mark(true, st);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(scratch, st);
  cudaFreeAsync(queue, st);
  if (d_tiles) cudaFreeAsync(d_tiles, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(err, st);
    return cuda_fail(e, "tc_overlap_kernel");
  }
  *err_out = err;  // read (and freed) by tc_finish after the stream is synchronised
  return QK_OK;
}

// Reads the kernel's error word once the stream has been synchronised.
qk_status tc_finish(int* err, cudaStream_t st) {
  if (!err) return QK_OK;
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (g_tc_prof_pending) {
    if (e == cudaSuccess)
      e = cudaMemcpy(g_tc_prof_last, g_tc_prof_pending, sizeof(g_tc_prof_last), cudaMemcpyDeviceToHost);
    cudaFree(g_tc_prof_pending);
    g_tc_prof_pending = nullptr;
  }
  if (e != cudaSuccess) return cuda_fail(e, "tc_overlap_kernel");
  if (herr) return fail(QK_ERR_TIMEOUT, "tc_overlap_kernel: a bounded wait ran out");
  return QK_OK;
}

qk_status launch_tc_parts(int parts, const qk_mps_batch* A, const qk_mps_batch* B, int mode,
                          const int32_t* d_pairs, int64_t P_pairs, double* dK, int64_t ldk, cudaStream_t st,
                          int** err_out, const TcSchedule& sch = TcSchedule(), int64_t i_lim = INT64_MAX,
                          int64_t j_lim = INT64_MAX) {
  return parts == 3 ? launch_tc<3>(A, B, mode, d_pairs, P_pairs, dK, ldk, st, err_out, sch, i_lim, j_lim)
                    : launch_tc<2>(A, B, mode, d_pairs, P_pairs, dK, ldk, st, err_out, sch, i_lim, j_lim);
}

// ---- schedule tuning ------------------------------------------------------
// Candidate schedules are timed on one sample of the Gram: the pairs with bra
// i < 128 and first ket j0 < i_lim + 160 (symmetric) or < 160, i.e. >= 4 tiles
// per CTA at 4 kets per tile, enough to fill every SM several times and to
// hold the largest band.  Each candidate runs twice (the first warms L2 and
// the instruction cache) and the faster run counts; the result is cached on
// A's operand cache for (B, P, mode).  One ket per tile keeps the least
// per-CTA scratch live, so the bands are explored at that width.
constexpr int kTuneBras = 128, kTuneKets = 160;
constexpr int kTuneCands = 6;
const TcSchedule kCands[kTuneCands] = {{4, 16}, {2, 64}, {1, 16}, {1, 32}, {1, 64}, {1, 128}};
// A candidate replaces the default (the first) only when it is faster by
// more than the sample's run-to-run noise.
constexpr double kTuneMargin = 0.97;

// Full Grams at least this many default tiles per CTA are tuned on the fly.
constexpr int64_t kTuneMinTilesPerCta = 64;

qk_status tune_schedule(int parts, const qk_mps_batch* A, const qk_mps_batch* B, int mode, cudaStream_t st,
                        TcSchedule* best, double* best_us_per_pair) {
  const int64_t i_lim = std::min<int64_t>(A->N, kTuneBras);
  const int64_t j_lim = std::min<int64_t>(B->N, (mode == 0 ? i_lim : 0) + kTuneKets);
  // a scratch K holding every row and column the sample writes (the
  // symmetric mirror writes rows j < j_lim + kG)
  const int64_t rows = std::min<int64_t>(A->N, std::max<int64_t>(i_lim, j_lim + kG));
  if (rows == 0 || B->N == 0) return QK_OK;  // nothing to time: the default stands
  double* Ks = nullptr;
  QK_CUDA(cudaMallocAsync(&Ks, sizeof(double) * rows * B->N, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  qk_status rc = QK_OK;
  double best_us = 0.0, default_us = 0.0;
  std::vector<int32_t> tiles;
  timer_set_phase(2);  // not one of the call's timed phases
  for (int c = 0; c < kTuneCands && rc == QK_OK; ++c) {
    const int64_t pairs = make_tiles(mode, B->N, kCands[c], i_lim, j_lim, tiles);
    if (pairs == 0) continue;
    float ms_min = 0.f;
    for (int rep = 0; rep < 2 && rc == QK_OK; ++rep) {
      int* err = nullptr;
      cudaEventRecord(e0, st);
      rc = launch_tc_parts(parts, A, B, mode, nullptr, 0, Ks, B->N, st, &err, kCands[c], i_lim, j_lim);
      cudaEventRecord(e1, st);
      qk_status rc2 = tc_finish(err, st);  // synchronises
      if (rc == QK_OK) rc = rc2;
      float ms = 0.f;
      if (rc == QK_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (rep == 0 || ms < ms_min))
        ms_min = ms;
    }
    const double us = 1000.0 * ms_min / (double)pairs;
    if (rc != QK_OK) break;
    if (c == 0) {
      best_us = default_us = us;
      *best = kCands[0];
    } else if (us < best_us && us < kTuneMargin * default_us) {
      best_us = us;
      *best = kCands[c];
    }
  }
  timer_set_phase(0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(Ks, st);
  if (best_us_per_pair) *best_us_per_pair = best_us;
  return rc;
}

// The schedule for a full Gram of (A, B): the cached choice, else a tuned
// one when the Gram is large enough to repay the sample, else the default.
// Tuned schedules by the shape of the Gram (device, N_A, N_B, n, largest
// bonds, split depth, mode), so that a new batch of the same shape -- a
// reloaded or re-rotated copy -- reuses the choice without timing again.
using TuneKey = std::tuple<int, int64_t, int64_t, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<TcSchedule, double>> g_tuned;

TuneKey tune_key(int parts, const qk_mps_batch* A, const qk_mps_batch* B, int mode) {
  return TuneKey(A->device, A->N, B->N, A->n, A->chi_cap, B->chi_cap, parts, mode);
}

qk_status schedule_for(int parts, const qk_mps_batch* A, const qk_mps_batch* B, int mode, cudaStream_t st,
                       bool force, TcSchedule* out, double* us_per_pair) {
  *out = TcSchedule();
  if (us_per_pair) *us_per_pair = 0.0;
  TcCache* c = (TcCache*)A->tc_cache;
  if (c)
    for (const TcTuned& t : c->tuned)
      if (t.B == B && t.P == parts && t.mode == mode) {
        *out = t.sch;
        if (us_per_pair) *us_per_pair = t.us_per_pair;
        return QK_OK;
      }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(parts, A, B, mode));
    if (it != g_tuned.end()) {
      *out = it->second.first;
      if (us_per_pair) *us_per_pair = it->second.second;
      return QK_OK;
    }
  }
  if (!force) {
    int dev = 0, sms = 0;
    QK_CUDA(cudaGetDevice(&dev));
    QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const double pairs = mode == 0 ? 0.5 * (double)A->N * (double)(A->N - 1) : (double)A->N * (double)B->N;
    if (pairs / kG < (double)kTuneMinTilesPerCta * 4 * sms) return QK_OK;
  }
  TcSchedule best;
  double us = 0.0;
  qk_status rc = tune_schedule(parts, A, B, mode, st, &best, &us);
  if (rc != QK_OK) return rc;
  c = (TcCache*)A->tc_cache;  // created by the tuning launches
  if (c) c->tuned.push_back({B, parts, mode, best, us});
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(parts, A, B, mode)] = {best, us};
  }
  *out = best;
  if (us_per_pair) *us_per_pair = us;
  return QK_OK;
}

}  // namespace

void free_tc_cache(qk_mps_batch* b) {
  if (!b->tc_cache) return;
  TcCache* c = (TcCache*)b->tc_cache;
  for (auto& a : c->part) {
    cudaFree(a.arena);
    cudaFree(a.d_bt);
    cudaFree(a.d_ah);
  }
  delete c;
  b->tc_cache = nullptr;
}

qk_status split_schedule(int parts, const qk_mps_batch* A, const qk_mps_batch* B, cudaStream_t st,
                         bool force, int32_t* kets, int32_t* band, double* us_per_pair) {
  TcSchedule sch;
  qk_status rc = schedule_for(parts, A, B, A == B ? 0 : 1, st, force, &sch, us_per_pair);
  if (rc != QK_OK) return rc;
  if (kets) *kets = sch.kets;
  if (band) *band = sch.band;
  return QK_OK;
}

qk_status set_split_schedule(int parts, const qk_mps_batch* A, const qk_mps_batch* B, int32_t kets,
                             int32_t band) {
  qk_mps_batch* a = const_cast<qk_mps_batch*>(A);
  if (!a->tc_cache) a->tc_cache = new TcCache();
  TcCache* c = (TcCache*)a->tc_cache;
  const int mode = A == B ? 0 : 1;
  TcSchedule sch;
  sch.kets = kets;
  sch.band = band;
  for (TcTuned& t : c->tuned)
    if (t.B == B && t.P == parts && t.mode == mode) {
      t.sch = sch;
      t.us_per_pair = 0.0;
      return QK_OK;
    }
  c->tuned.push_back({B, parts, mode, sch, 0.0});
  return QK_OK;
}

qk_status gram_split(int parts, const qk_mps_batch* A, const qk_mps_batch* B, double* dK, int64_t ldk,
                     double refine_floor, cudaStream_t st, int64_t* n_refined) {
  const bool sym = (A == B);
  int* tc_err = nullptr;
  TcSchedule sch;
  qk_status rc = schedule_for(parts, A, B, sym ? 0 : 1, st, false, &sch, nullptr);
  if (rc != QK_OK) return rc;
  rc = launch_tc_parts(parts, A, B, sym ? 0 : 1, nullptr, 0, dK, ldk, st, &tc_err, sch);
  // The off-diagonal entries below the floor and above the ceiling go to
  // FP64; they are selected right behind the split kernel.
  const unsigned long long cap = sym ? (unsigned long long)A->N * (A->N + 1) / 2
                                     : (unsigned long long)A->N * B->N;
  int32_t* pairs = nullptr;
  unsigned long long* cnt = nullptr;
  unsigned long long hc = 0;
  cudaError_t e = cudaSuccess;
  if (rc == QK_OK) {
    e = cudaMallocAsync(&pairs, sizeof(int32_t) * 2 * cap, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&cnt, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
      select_refine_kernel<<<1024, 256, 0, st>>>(dK, ldk, (int)A->N, (int)B->N, sym ? 1 : 0, refine_floor,
                                                 QK_SPLIT_REFINE_ABOVE, pairs, cnt, cap);
      e = cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
    }
  }
  // synchronises st: the split kernel and the selection are done
  qk_status rc2 = tc_finish(tc_err, st);
  if (rc == QK_OK) rc = rc2;
  if (rc == QK_OK && e != cudaSuccess) rc = cuda_fail(e, "gram_split: refinement selection");
  if (rc == QK_OK && hc > 0) {
    double* vals = nullptr;
    e = cudaMallocAsync(&vals, sizeof(double) * hc, st);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaMallocAsync");
    } else {
      timer_set_phase(1);
      rc = overlap_fp64(A, B, pairs, (int64_t)hc, vals, 0, false, st);
      timer_set_phase(0);
      if (rc == QK_OK) scatter_kernel<<<1024, 256, 0, st>>>(pairs, vals, (int64_t)hc, dK, ldk, sym ? 1 : 0);
      cudaFreeAsync(vals, st);
    }
  }
  int64_t n_diag = 0;
  if (rc == QK_OK && sym) {
    // The diagonal (K_ii ~ 1, above the refinement ceiling by construction)
    // comes from the isometry-defect recursion, which needs no FP64 sweep for
    // left-canonical states.  It runs on a side stream beside the FP64
    // re-evaluation just launched (the two write disjoint entries; both are
    // a few long CTAs), and the flagged states then take the FP64 sweep on st.
    cudaStream_t side = side_stream();
    DiagPending dp;
    n_diag = A->N;
    timer_set_phase(1);
    rc = diag_launch(A, dK, ldk, side ? side : st, &dp);
    if (rc == QK_OK) rc = diag_finish(A, dK, ldk, &dp, st, nullptr);
    timer_set_phase(0);
  }
  if (n_refined) *n_refined = (int64_t)hc + n_diag;
  if (pairs) cudaFreeAsync(pairs, st);
  if (cnt) cudaFreeAsync(cnt, st);
  return rc;
}

qk_status pairs_split(int parts, const qk_mps_batch* A, const qk_mps_batch* B, const int32_t* d_pairs,
                      int64_t P, double* dK, cudaStream_t st) {
  int* tc_err = nullptr;
  qk_status rc = launch_tc_parts(parts, A, B, 2, d_pairs, P, dK, 0, st, &tc_err);
  qk_status rc2 = tc_finish(tc_err, st);
  if (rc == QK_OK) rc = rc2;
  if (rc != QK_OK) return rc;
  int32_t* sel = nullptr;
  int64_t* pos = nullptr;
  unsigned long long* cnt = nullptr;
  QK_CUDA(cudaMallocAsync(&sel, sizeof(int32_t) * 2 * P, st));
  QK_CUDA(cudaMallocAsync(&pos, sizeof(int64_t) * P, st));
  QK_CUDA(cudaMallocAsync(&cnt, sizeof(unsigned long long), st));
  QK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  select_refine_list_kernel<<<256, 256, 0, st>>>(dK, d_pairs, P, QK_SPLIT_REFINE_ABOVE, sel, pos, cnt);
  unsigned long long hc = 0;
  QK_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
  QK_CUDA(cudaStreamSynchronize(st));
  if (hc > 0) {
    double* vals = nullptr;
    QK_CUDA(cudaMallocAsync(&vals, sizeof(double) * hc, st));
    timer_set_phase(1);
    rc = overlap_fp64(A, B, sel, (int64_t)hc, vals, 0, false, st);
    timer_set_phase(0);
    if (rc == QK_OK) scatter_list_kernel<<<256, 256, 0, st>>>(pos, vals, (int64_t)hc, dK);
    cudaFreeAsync(vals, st);
  }
  cudaFreeAsync(sel, st);
  cudaFreeAsync(pos, st);
  cudaFreeAsync(cnt, st);
  return rc;
}

}  // namespace qk

extern "C" qk_status qk_debug_stall_next_split(int32_t on) {
  qk::g_stall_next.store(on ? 1 : 0);
  return QK_OK;
}

extern "C" qk_status qk_debug_tc_profile(int32_t on) {
  qk::g_tc_profile.store(on ? 1 : 0);
  return QK_OK;
}

extern "C" qk_status qk_last_tc_profile(double* counters, int32_t* ctas) {
  if (counters)
    for (int f = 0; f < qk::kProfN; ++f) counters[f] = (double)qk::g_tc_prof_last[f];
  if (ctas) *ctas = qk::g_tc_prof_ctas;
  return QK_OK;
}

extern "C" qk_status qk_debug_tc_variant(int32_t flags) {
  if (flags < 0 || flags > 15) return qk::fail(QK_ERR_INVALID_ARG, "qk_debug_tc_variant: flags must be in [0, 15]");
  qk::g_tc_variant.store(flags);
  return QK_OK;
}

extern "C" qk_status qk_debug_tc_max_ctas(int32_t ctas) {
  qk::g_tc_max_ctas.store(ctas > 0 ? ctas : 0);
  return QK_OK;
}
