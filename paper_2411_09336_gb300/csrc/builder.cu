// Batched MPS simulation of the feature-map circuit in FP64 (Sec. II-B/C).
//
// One CTA builds one state at a time and takes the next sample index from a
// global counter (persistent launch).  The state being built lives in the
// CTA's slice of a workspace in HBM (FP64 complex site tensors at a fixed
// capacity per site) next to three (2 chi_max)^2 scratch matrices.
//
// Every two-site op (Fig. 1b) and every move of the orthogonality centre is
// one factorisation of a matrix Z whose column space must become an isometry
// (the left factor when the singular values move right, the right factor,
// through Z = theta^H, when they move left).  Z is factorised in two steps:
//
//  1. Householder QR with column pivoting of Y = Z^H (Businger-Golub), so
//     that the rows of R are ordered by decreasing norm;
//  2. one-sided (Hestenes) Jacobi on the rows of R, which then converges in a
//     few sweeps even though the Schmidt spectrum of theta spans ten or more
//     decades (the QR-preconditioned Jacobi SVD of Drmac and Veselic, SIAM J.
//     Matrix Anal. Appl. 29 (2008)).  After convergence the rows w_j of the
//     rotated R satisfy W = conj(w) = P^T Z Q J, so the isometry is
//     U[perm[c]][j] = conj(w_j[c]) / |w_j| and sigma_j = |w_j|; the other
//     factor is one GEMM with Z, so no rotation matrix is accumulated and no
//     small singular value is divided into the kept part.
//
// The Jacobi rotates a pair of rows when |w_p^H w_q| exceeds
// tol |w_p||w_q| (tol = max(m, 32) eps), the standard relative test, while
// both rows carry more than kappa of the squared Frobenius norm F, with
// kappa = eps_trunc^2 / (1000 L): rows below it lie in the discarded tail in
// any case (their total is under 1e-3 of the truncation threshold), so only
// their total weight matters, which rotations among them do not change; a
// pair involving such a row is rotated only while the change exceeds a few
// ulps of sqrt(F).  Without this test those rows, which hold rounding noise,
// never satisfy the relative test and the sweep count triples.
//
// Truncation (Eq. 8, read as a discarded-weight rule): with s sorted
// descending, keep r = min{r >= 1 : sum_{i >= r} s_i^2 <= eps^2 sum_i s_i^2}
// (the tail summed from the smallest value upward), then r <= chi_max, and
// rescale the kept values to unit norm.  eps = 0 keeps everything up to
// chi_max.  The orthogonality centre follows the gate: after an op at
// (p, p+1) the singular values go to site p+1 if the next op lies to the
// right, else to site p; between repetitions the centre walks back by
// untruncated factorisations, and finally walks to the last site, so the
// stored state is left-canonical.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "qk_internal.h"

namespace qk {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSweeps = 60;
constexpr int kMaxCols = 256;   // 2 * chi_max
constexpr int kMaxN = 1024;     // qubits
#ifndef QK_BUILD_CTAS
#define QK_BUILD_CTAS 2
#endif
constexpr int kCtas = QK_BUILD_CTAS;  // CTAs per SM
// complex doubles of the shared-memory copy of Y; larger Y live in HBM/L2
constexpr int kSmemElems = kCtas == 1 ? 12800 : 5504;
constexpr double kEps = 2.220446049250313e-16;
constexpr unsigned kFull = 0xffffffffu;

// per-CTA profile counters (clock64 cycles per phase, counts)
enum Prof { PF_THETA = 0, PF_QR, PF_JACOBI, PF_OUT, PF_MOVE, PF_OTHER, PF_SWEEPS, PF_FACTOR, PF_FLOPS, PF_N };

struct BuildArgs {
  const double* X;         // [N][n]
  int64_t n_items;         // samples in this launch
  const int32_t* items;    // optional sample list (nullptr: item = sample)
  int n, d, reps, n_ops;
  double gamma, eps;
  int chi_max;
  const Op* ops;           // [n_ops]
  // workspace
  double2* ws;
  int64_t ws_stride;       // double2 per CTA
  const int64_t* cap_off;  // [n+1] double2 offsets of each site inside the slice
  int64_t w_off;           // offset of scratch Th (then T0, Yg at +wcap, +2 wcap)
  int64_t wcap;
  // output pool
  char* pool;
  unsigned long long pool_cap;
  unsigned long long* pool_used;
  int store;               // 0 c128, 1 c64
  int32_t* dims;           // [N][n+1]
  uint64_t* site_ptr;      // [N][n]
  double* trunc_w;         // [N]
  int32_t* status;         // [N]: bit0 numeric, bit1 pool overflow
  int64_t* need_bytes;     // [N]
  int32_t* rank_trace;     // optional [N][reps*n_ops]
  int* queue;
  unsigned long long* prof;  // optional [gridDim.x][PF_N]
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

struct Shared {
  double nrm[kMaxCols];     // QR column norms^2, then Jacobi row norms^2
  double2 hv[kMaxCols];     // Householder vector
  double sv[kMaxCols];      // singular values, sorted descending
  double sinv[kMaxCols];    // 1 / sv of the kept values (0: to be completed)
  double tail[kMaxCols + 1];
  int qperm[kMaxCols];      // QR column position -> row of Z
  int ipos[kMaxCols];       // row of Z -> QR column position
  int order[kMaxCols];      // sorted position -> row of R
  int chi[kMaxN + 1];
  double F;                 // squared Frobenius norm of the factorised matrix
  double hinv;
  double nrm_inv;
  double wsum;
  int kq;                   // rows of R that are not zero
  int rotated;
  int r;
  int sample;
  int bad;
  int need;                 // kept columns to be completed
  int sweeps;
  unsigned long long flops; // FP64 flops executed (FMA = 2), flushed per state
};

struct Work {
  double2* slice;  // site tensors
  double2* Th;     // the matrix being factorised (row-major), or theta
  double2* T0;     // temporary
  double2* Yg;     // Y when it does not fit in shared memory
  double2* Ys;     // Y in shared memory
  unsigned long long* prof;
};

__device__ __forceinline__ void prof_add(const Work& w, int what, unsigned long long& t0) {
  if (w.prof && threadIdx.x == 0) {
    const unsigned long long t = clock64();
    w.prof[what] += t - t0;
    t0 = t;
  }
}

// ---------------------------------------------------------------- QR (CP)
// Householder QR with column pivoting of Y (n x m, row-major).  On return
// rows 0..kq-1 of Y hold R (zeros below its diagonal; rows kq.. are zero),
// qperm[c] is the original column at position c, F the squared Frobenius
// norm.  The pivot is the column of largest remaining norm (ties: the lower
// index); the norms are recomputed exactly while the reflector is applied.
__device__ void qrcp(double2* Y, int n, int m, Shared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = min(n, m);
  if (tid == 0) sh.flops += 4ull * n * m;
  for (int c = tid; c < m; c += kThreads) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      const double2 y = Y[(int64_t)i * m + c];
      s = fma(y.x, y.x, fma(y.y, y.y, s));
    }
    sh.nrm[c] = s;
    sh.qperm[c] = c;
  }
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
    for (int c = lane; c < m; c += 32) s += sh.nrm[c];
    s = warp_sum(s);
    if (lane == 0) {
      sh.F = s;
      sh.kq = k;
    }
  }
  for (int j = 0; j < k; ++j) {
    if (warp == 0) {
      double bv = -1.0;
      int bi = m;
      for (int c = j + lane; c < m; c += 32) {
        const double v = sh.nrm[c];
        if (v > bv) {
          bv = v;
          bi = c;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(kFull, bv, o);
        const int oi = __shfl_xor_sync(kFull, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (bi != j) {
        for (int i = lane; i < n; i += 32) {
          double2* r = Y + (int64_t)i * m;
          const double2 t = r[j];
          r[j] = r[bi];
          r[bi] = t;
        }
        if (lane == 0) {
          const double t = sh.nrm[j];
          sh.nrm[j] = sh.nrm[bi];
          sh.nrm[bi] = t;
          const int q = sh.qperm[j];
          sh.qperm[j] = sh.qperm[bi];
          sh.qperm[bi] = q;
        }
      }
      __syncwarp();
      double xs = 0.0;
      for (int i = j + lane; i < n; i += 32) {
        const double2 y = Y[(int64_t)i * m + j];
        xs = fma(y.x, y.x, fma(y.y, y.y, xs));
      }
      xs = warp_sum(xs);
      const double2 al = Y[(int64_t)j * m + j];
      __syncwarp();  // every lane has read alpha before it is overwritten
      double hinv = 0.0;
      if (xs > 0.0) {
        // H = I - v v^H / h, v = x - beta e_1, beta = -e^{i arg alpha} |x|,
        // h = v^H v / 2 = |x| (|x| + |alpha|): H x = beta e_1
        const double xn = sqrt(xs), aa = sqrt(al.x * al.x + al.y * al.y);
        const double2 ph = aa > 0.0 ? make_double2(al.x / aa, al.y / aa) : make_double2(1.0, 0.0);
        const double2 beta = make_double2(-ph.x * xn, -ph.y * xn);
        hinv = 1.0 / (xn * (xn + aa));
        for (int i = j + lane; i < n; i += 32) {
          double2* y = Y + (int64_t)i * m + j;
          if (i == j) {
            sh.hv[i] = make_double2(al.x - beta.x, al.y - beta.y);
            *y = beta;
          } else {
            sh.hv[i] = *y;
            *y = make_double2(0.0, 0.0);
          }
        }
      }
      if (lane == 0) {
        sh.hinv = hinv;
        if (!(xs > 0.0)) sh.kq = j;  // every remaining column is zero
      }
    }
    __syncthreads();
    const double hinv = sh.hinv;
    if (hinv == 0.0) break;
    const int nc = m - j - 1, nr = n - j;
    if (tid == 0) sh.flops += 20ull * nr * (nc > 0 ? nc : 0) + 8ull * nr;
    if (nc > 0) {
      int G = 1;  // lanes per column
      while (G < 32 && 2 * G * nc <= kThreads && G < nr) G <<= 1;
      const int per = kThreads / G, g = tid % G;
      for (int c0 = j + 1; c0 < m; c0 += per) {
        const int c = c0 + tid / G;
        const bool ok = c < m;
        double wr = 0.0, wi = 0.0;
        if (ok)
          for (int i = j + g; i < n; i += G) {
            const double2 v = sh.hv[i], y = Y[(int64_t)i * m + c];
            wr = fma(v.x, y.x, fma(v.y, y.y, wr));
            wi = fma(v.x, y.y, fma(-v.y, y.x, wi));
          }
        for (int o = G >> 1; o > 0; o >>= 1) {
          wr += __shfl_xor_sync(kFull, wr, o);
          wi += __shfl_xor_sync(kFull, wi, o);
        }
        wr *= hinv;
        wi *= hinv;
        double ns = 0.0;
        if (ok)
          for (int i = j + g; i < n; i += G) {
            const double2 v = sh.hv[i];
            double2* yp = Y + (int64_t)i * m + c;
            double2 y = *yp;
            y.x -= v.x * wr - v.y * wi;
            y.y -= v.x * wi + v.y * wr;
            *yp = y;
            if (i > j) ns = fma(y.x, y.x, fma(y.y, y.y, ns));
          }
        for (int o = G >> 1; o > 0; o >>= 1) ns += __shfl_xor_sync(kFull, ns, o);
        if (ok && g == 0) sh.nrm[c] = ns;
      }
    }
    __syncthreads();
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Jacobi
// One-sided Jacobi on rows 0..kq-1 of Y (vectors of length m), round-robin
// ordering; a team of T lanes owns one pair per round: it forms w_p^H w_q,
// its leader turns it into the rotation (row norms are carried along:
// a' = a - t|g|, b' = b + t|g|, recomputed exactly every sweep), and the
// team applies it.  One barrier per round.  Returns false at the sweep cap.
__device__ bool jacobi_rows(double2* Y, int kq, int m, double kappa, Shared& sh) {
  if (kq < 2) return true;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npad = kq + (kq & 1), npairs = npad / 2;
  int T = 1;
  while (T < 32 && 2 * T * npairs <= kThreads) T <<= 1;
  const int per = kThreads / T, team = tid / T, tl = tid % T, leader = lane - tl;
  const double tol = (double)(m > 32 ? m : 32) * kEps;
  const double F = sh.F, kF = kappa * F, absf = 4.0 * kEps * sqrt(F);
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    for (int j = warp; j < kq; j += kWarps) {
      const double2* x = Y + (int64_t)j * m;
      double s = 0.0;
      for (int i = lane; i < m; i += 32) {
        const double2 v = x[i];
        s = fma(v.x, v.x, fma(v.y, v.y, s));
      }
      s = warp_sum(s);
      if (lane == 0) sh.nrm[j] = s;
    }
    if (tid == 0) {
      sh.rotated = 0;
      sh.flops += 4ull * kq * m;
    }
    __syncthreads();
    for (int round = 0; round < npad - 1; ++round) {
      for (int k0 = 0; k0 < npairs; k0 += per) {
        const int kk = k0 + team;
        int p = npad, q = npad;
        if (kk < npairs) {
          if (kk == 0) {
            p = npad - 1;
            q = round;
          } else {
            p = (round + kk) % (npad - 1);
            q = (round - kk + (npad - 1)) % (npad - 1);
          }
        }
        const bool valid = p < kq && q < kq;
        double2* xp = Y + (int64_t)(valid ? p : 0) * m;
        double2* xq = Y + (int64_t)(valid ? q : 0) * m;
        double gr = 0.0, gi = 0.0;
        if (valid)
          for (int i = tl; i < m; i += T) {
            const double2 u = xp[i], v = xq[i];
            gr = fma(u.x, v.x, fma(u.y, v.y, gr));   // Re(conj(u) v)
            gi = fma(u.x, v.y, fma(-u.y, v.x, gi));  // Im(conj(u) v)
          }
        for (int o = T >> 1; o > 0; o >>= 1) {
          gr += __shfl_xor_sync(kFull, gr, o);
          gi += __shfl_xor_sync(kFull, gi, o);
        }
        int rot = 0;
        double c = 1.0, sx = 0.0, sy = 0.0;
        if (valid && tl == 0) {
          atomicAdd(&sh.flops, 8ull * m);  // w_p^H w_q
          const double a = sh.nrm[p], b = sh.nrm[q];
          const double g = sqrt(gr * gr + gi * gi);
          if (a > 0.0 && b > 0.0 && g > 0.0) {
            const bool sig = fmin(a, b) > kF;
            rot = sig ? (g > tol * sqrt(a) * sqrt(b)) : (g > absf * sqrt(fmax(a, b)));
            if (rot) {
              // [[c, s e^{i phi}], [-s e^{-i phi}, c]] zeroes w_p^H w_q
              const double zeta = (b - a) / (2.0 * g);
              const double t = fabs(zeta) > 1e100
                                   ? 0.5 / zeta
                                   : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
              if (t == 0.0) {
                rot = 0;
              } else {
                c = 1.0 / sqrt(1.0 + t * t);
                const double s = c * t;
                sx = s * gr / g;
                sy = s * gi / g;
                sh.nrm[p] = fmax(a - t * g, 0.0);
                sh.nrm[q] = b + t * g;
                atomicAdd(&sh.rotated, 1);
                atomicAdd(&sh.flops, 20ull * m);  // the rotation of both rows
              }
            }
          }
        }
        rot = __shfl_sync(kFull, rot, leader);
        c = __shfl_sync(kFull, c, leader);
        sx = __shfl_sync(kFull, sx, leader);
        sy = __shfl_sync(kFull, sy, leader);
        if (rot)
          for (int i = tl; i < m; i += T) {
            const double2 u = xp[i], v = xq[i];
            // w_p' = c w_p - s e^{-i phi} w_q ;  w_q' = s e^{i phi} w_p + c w_q
            xp[i] = make_double2(c * u.x - (sx * v.x + sy * v.y), c * u.y - (sx * v.y - sy * v.x));
            xq[i] = make_double2(c * v.x + (sx * u.x - sy * u.y), c * v.y + (sx * u.y + sy * u.x));
          }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) sh.sweeps += 1;
    if (sh.rotated == 0) return true;
    __syncthreads();
  }
  return false;
}

// Singular values (row norms of R after the Jacobi) sorted descending, ties
// by row index; sv[i] = 0 for the zero rows kq..k-1.
__device__ void sort_rows(const double2* Y, int kq, int k, int m, Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < k; j += kWarps) {
    double s = 0.0;
    if (j < kq) {
      const double2* x = Y + (int64_t)j * m;
      for (int i = lane; i < m; i += 32) s = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, s));
      s = warp_sum(s);
    }
    if (lane == 0) sh.nrm[j] = s;
  }
  __syncthreads();
  // non-negative doubles order like their bit patterns: compare as integers
  for (int i = threadIdx.x; i < k; i += kThreads) {
    const unsigned long long v = (unsigned long long)__double_as_longlong(sh.nrm[i]);
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const unsigned long long u = (unsigned long long)__double_as_longlong(sh.nrm[j]);
      rank += (u > v) || (u == v && j < i);
    }
    sh.order[rank] = i;
  }
  for (int c = threadIdx.x; c < m; c += kThreads) sh.ipos[sh.qperm[c]] = c;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += kThreads) sh.sv[i] = sqrt(sh.nrm[sh.order[i]]);
  __syncthreads();
}

// QR + Jacobi + sort of Y (n x m): singular values of Z (m x n, Y = Z^H).
__device__ void factor(const Work& w, double2* Y, int n, int m, double eps, Shared& sh,
                       unsigned long long& t0) {
  const int k = min(n, m);
  const double kappa = (eps > 0.0 ? eps * eps : 1e-28) / (1000.0 * (double)k);
  qrcp(Y, n, m, sh);
  prof_add(w, PF_QR, t0);
  const int kq = sh.kq;
  if (!jacobi_rows(Y, kq, m, kappa, sh) && threadIdx.x == 0) sh.bad |= 1;
  __syncthreads();
  prof_add(w, PF_JACOBI, t0);
  sort_rows(Y, kq, k, m, sh);
  if (threadIdx.x == 0) {
    if (!(sh.F > 0.0) || !isfinite(sh.F)) sh.bad |= 1;
    if (w.prof) w.prof[PF_FACTOR] += 1;
  }
}

// Truncation rank by the discarded-weight rule (single thread); kept values
// whose weight is at the rounding level of F are marked for completion.
__device__ void choose_rank(int L, int chi_max, double eps, bool truncate, double kappa, Shared& sh) {
  if (threadIdx.x == 0) {
    sh.tail[L] = 0.0;
    for (int i = L - 1; i >= 0; --i) sh.tail[i] = sh.tail[i + 1] + sh.sv[i] * sh.sv[i];
    const double tot = sh.tail[0];
    int r = L;
    if (truncate && eps > 0.0) {
      const double thr = eps * eps * tot;
      for (int c = 1; c <= L; ++c)
        if (sh.tail[c] <= thr) {
          r = c;
          break;
        }
    }
    if (truncate && r > chi_max) r = chi_max;
    double kept = 0.0;
    for (int i = 0; i < r; ++i) kept += sh.sv[i] * sh.sv[i];
    if (!(tot > 0.0) || !isfinite(tot)) sh.bad |= 1;
    sh.r = r;
    sh.nrm_inv = (kept > 0.0) ? 1.0 / sqrt(kept) : 0.0;
    if (truncate && tot > 0.0) sh.wsum += sh.tail[r] / tot;
    int need = 0;
    const double zero2 = kappa * sh.F;
    for (int i = 0; i < r; ++i) {
      const bool z = !(sh.sv[i] * sh.sv[i] > zero2);
      sh.sinv[i] = z ? 0.0 : 1.0 / sh.sv[i];
      need |= z;
    }
    sh.need = need;
  }
  __syncthreads();
}

// Isometry column j, element e, in a site tensor: the left-canonical form
// A[s][a][j] with e = 2a + s (ColL), or the stored conjugate of a right
// isometry A[t][j][b] with e = t chi + b (ColR).
struct ColL {
  double2* A;
  int cl, r;
  __device__ double2* at(int e, int j) const { return A + ((int64_t)(e & 1) * cl + (e >> 1)) * r + j; }
};
struct ColR {
  double2* A;
  int cr, r;
  __device__ double2* at(int e, int j) const { return A + ((int64_t)(e / cr) * r + j) * cr + (e % cr); }
};

// Replace the kept columns j < r with sinv[j] = 0 (weight at the rounding
// level) by unit vectors orthogonal to every other kept column (classical
// Gram-Schmidt, twice).  Rare; one warp.
template <class Col>
__device__ void complete_columns(const Col& U, int m, int r, Shared& sh) {
  if (!sh.need) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    int e = 0;
    for (int j = 0; j < r; ++j) {
      if (sh.sinv[j] != 0.0) continue;
      for (; e < m; ++e) {
        for (int i = lane; i < m; i += 32) *U.at(i, j) = make_double2(i == e ? 1.0 : 0.0, 0.0);
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int jj = 0; jj < r; ++jj) {
            if (jj == j || (sh.sinv[jj] == 0.0 && jj > j)) continue;
            double pr = 0.0, pi = 0.0;
            for (int i = lane; i < m; i += 32) {
              const double2 o = *U.at(i, jj), c = *U.at(i, j);
              pr += o.x * c.x + o.y * c.y;
              pi += o.x * c.y - o.y * c.x;
            }
            pr = warp_sum(pr);
            pi = warp_sum(pi);
            for (int i = lane; i < m; i += 32) {
              const double2 o = *U.at(i, jj);
              double2* c = U.at(i, j);
              c->x -= pr * o.x - pi * o.y;
              c->y -= pr * o.y + pi * o.x;
            }
            __syncwarp();
          }
        }
        double nn = 0.0;
        for (int i = lane; i < m; i += 32) {
          const double2 c = *U.at(i, j);
          nn += c.x * c.x + c.y * c.y;
        }
        nn = warp_sum(nn);
        if (nn > 0.25) {
          const double inv = 1.0 / sqrt(nn);
          for (int i = lane; i < m; i += 32) {
            double2* c = U.at(i, j);
            *c = make_double2(c->x * inv, c->y * inv);
          }
          __syncwarp();
          ++e;
          break;
        }
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double2* site(const BuildArgs& a, double2* slice, int k) {
  return slice + a.cap_off[k];
}

__device__ __forceinline__ double kappa_of(double eps, int k) {
  return (eps > 0.0 ? eps * eps : 1e-28) / (1000.0 * (double)k);
}

// Centre from site c to c+1 (no truncation): A_c = Q, A_{c+1} <- (Q^H A_c) A_{c+1}.
__device__ void move_right(const BuildArgs& a, Work& w, int c, Shared& sh, unsigned long long& t0) {
  const int cl = sh.chi[c], cr = sh.chi[c + 1], cn = sh.chi[c + 2];
  const int m = 2 * cl, n = cr;  // Z = M[(a, q)][b] = A_c[q][a][b]
  double2* Ac = site(a, w.slice, c);
  double2* An = site(a, w.slice, c + 1);
  double2* Y = (int64_t)m * n <= kSmemElems ? w.Ys : w.Yg;
  for (int i = threadIdx.x; i < m * n; i += kThreads) {
    const int row = i / n, b = i % n;
    const double2 v = Ac[((int64_t)(row & 1) * cl + (row >> 1)) * cr + b];
    w.T0[i] = v;
    Y[(int64_t)b * m + row] = conjd(v);
  }
  __syncthreads();
  factor(w, Y, n, m, a.eps, sh, t0);
  const int k = min(m, n);
  choose_rank(k, k, a.eps, false, kappa_of(a.eps, k), sh);
  // site c = U: U[row][j] = conj(w_{o_j}[ipos[row]]) / s_j
  for (int i = threadIdx.x; i < m * k; i += kThreads) {
    const int row = i / k, j = i % k;
    const double2 v = Y[(int64_t)sh.order[j] * m + sh.ipos[row]];
    const double s = sh.sinv[j];
    Ac[((int64_t)(row & 1) * cl + (row >> 1)) * k + j] = make_double2(v.x * s, -v.y * s);
  }
  __syncthreads();
  complete_columns(ColL{Ac, cl, k}, m, k, sh);
  // T = U^H M (k x n) -> Th
  for (int i = threadIdx.x; i < k * n; i += kThreads) {
    const int j = i / n, b = i % n;
    double2 acc = make_double2(0.0, 0.0);
    for (int row = 0; row < m; ++row) {
      const double2 u = Ac[((int64_t)(row & 1) * cl + (row >> 1)) * k + j];
      const double2 t = cmulc(u, w.T0[(int64_t)row * n + b]);
      acc.x += t.x;
      acc.y += t.y;
    }
    w.Th[i] = acc;
  }
  __syncthreads();
  // site c+1 = T A_{c+1}: [q][j][b'] = sum_b T[j][b] A[q][b][b']
  for (int i = threadIdx.x; i < 2 * k * cn; i += kThreads) {
    const int q = i / (k * cn), rem = i % (k * cn), j = rem / cn, bb = rem % cn;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < cr; ++b) {
      const double2 t = cmul(w.Th[(int64_t)j * n + b], An[((int64_t)q * cr + b) * cn + bb]);
      acc.x += t.x;
      acc.y += t.y;
    }
    w.T0[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * k * cn; i += kThreads) An[i] = w.T0[i];
  if (threadIdx.x == 0) {
    sh.chi[c + 1] = k;
    sh.flops += 8ull * k * m * n + 16ull * k * cn * cr;
  }
  __syncthreads();
  prof_add(w, PF_MOVE, t0);
}

// Centre from site c to c-1 (no truncation): A_c = V^H, A_{c-1} <- A_{c-1} (A_c V).
__device__ void move_left(const BuildArgs& a, Work& w, int c, Shared& sh, unsigned long long& t0) {
  const int cp = sh.chi[c - 1], cl = sh.chi[c], cr = sh.chi[c + 1];
  const int ncol = 2 * cr;  // M[a][(q, b)] = A_c[q][a][b]; Z = M^H (m = 2 cr, n = cl)
  const int m = ncol, n = cl;
  double2* Ac = site(a, w.slice, c);
  double2* Ap = site(a, w.slice, c - 1);
  double2* Y = (int64_t)m * n <= kSmemElems ? w.Ys : w.Yg;
  for (int i = threadIdx.x; i < cl * ncol; i += kThreads) {
    const int aa = i / ncol, col = i % ncol;
    const int q = col / cr, b = col % cr;
    const double2 v = Ac[((int64_t)q * cl + aa) * cr + b];
    w.T0[i] = v;
    Y[i] = v;  // Y = Z^H = M, row-major cl x ncol
  }
  __syncthreads();
  factor(w, Y, n, m, a.eps, sh, t0);
  const int k = min(m, n);
  choose_rank(k, k, a.eps, false, kappa_of(a.eps, k), sh);
  // site c = V^H: [q][j][b] = conj(V[q cr + b][j]) = w_{o_j}[ipos[col]] / s_j
  for (int i = threadIdx.x; i < 2 * k * cr; i += kThreads) {
    const int q = i / (k * cr), rem = i % (k * cr), j = rem / cr, b = rem % cr;
    const double2 v = Y[(int64_t)sh.order[j] * m + sh.ipos[q * cr + b]];
    const double s = sh.sinv[j];
    Ac[i] = make_double2(v.x * s, v.y * s);
  }
  __syncthreads();
  complete_columns(ColR{Ac, cr, k}, m, k, sh);
  // T = M V (cl x k) -> Th
  for (int i = threadIdx.x; i < cl * k; i += kThreads) {
    const int aa = i / k, j = i % k;
    double2 acc = make_double2(0.0, 0.0);
    for (int col = 0; col < ncol; ++col) {
      const int q = col / cr, b = col % cr;
      const double2 vh = Ac[((int64_t)q * k + j) * cr + b];  // conj(V[col][j])
      const double2 t = cmul(w.T0[(int64_t)aa * ncol + col], conjd(vh));
      acc.x += t.x;
      acc.y += t.y;
    }
    w.Th[i] = acc;
  }
  __syncthreads();
  // site c-1 = A_{c-1} T: [q][a'][j] = sum_a A[q][a'][a] T[a][j]
  for (int i = threadIdx.x; i < 2 * cp * k; i += kThreads) {
    const int q = i / (cp * k), rem = i % (cp * k), ap = rem / k, j = rem % k;
    double2 acc = make_double2(0.0, 0.0);
    for (int aa = 0; aa < cl; ++aa) {
      const double2 t = cmul(Ap[((int64_t)q * cp + ap) * cl + aa], w.Th[(int64_t)aa * k + j]);
      acc.x += t.x;
      acc.y += t.y;
    }
    w.T0[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * cp * k; i += kThreads) Ap[i] = w.T0[i];
  if (threadIdx.x == 0) {
    sh.chi[c] = k;
    sh.flops += 8ull * cl * k * ncol + 16ull * cp * k * cl;
  }
  __syncthreads();
  prof_add(w, PF_MOVE, t0);
}

// One scheduled two-site op at (p, p+1); `right`: singular values go right.
__device__ void two_site(const BuildArgs& a, Work& w, const double* x, const Op op, bool right, Shared& sh,
                         unsigned long long& t0) {
  const int p = op.p;
  const int cl = sh.chi[p], cm = sh.chi[p + 1], cr = sh.chi[p + 2];
  const int rows = 2 * cl, cols = 2 * cr;
  double2* Ap = site(a, w.slice, p);
  double2* Aq = site(a, w.slice, p + 1);
  // theta0[(a,s)][(t,b)] = sum_c A_p[s][a][c] A_{p+1}[t][c][b]  -> T0 (row-major)
  for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
    const int row = i / cols, col = i % cols;
    const int aa = row >> 1, s = row & 1, t = col / cr, b = col % cr;
    const double2* ar = Ap + ((int64_t)s * cl + aa) * cm;
    const double2* bc = Aq + (int64_t)t * cm * cr + b;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < cm; ++c) {
      const double2 u = cmul(ar[c], bc[(int64_t)c * cr]);
      acc.x += u.x;
      acc.y += u.y;
    }
    w.T0[i] = acc;
  }
  __syncthreads();
  // gate on the physical pair (s, t): theta -> Th, and Y = Z^H with
  // Z = theta (right: m = rows) or Z = theta^H (left: m = cols)
  double cs = 1.0, sn = 0.0;
  if (op.kind != OP_SWAP) {
    const double th = a.gamma * a.gamma * (M_PI / 2.0) * (1.0 - x[op.qi]) * (1.0 - x[op.qj]);
    sincos(th, &sn, &cs);
  }
  const bool swap = op.kind != OP_RXX;
  const int m = right ? rows : cols, n = right ? cols : rows;
  double2* Y = (int64_t)m * n <= kSmemElems ? w.Ys : w.Yg;
  for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
    const int row = i / cols, col = i % cols;
    const int aa = row >> 1, s = row & 1, t = col / cr, b = col % cr;
    const int s0 = swap ? t : s, t0_ = swap ? s : t;  // SWAP after Rxx: read (t, s)
    const double2 v = w.T0[((int64_t)aa * 2 + s0) * cols + t0_ * cr + b];
    const double2 f = w.T0[((int64_t)aa * 2 + (1 - s0)) * cols + (1 - t0_) * cr + b];
    // cs * v - i sn * f
    const double2 th = make_double2(cs * v.x + sn * f.y, cs * v.y - sn * f.x);
    w.Th[i] = th;
    if (right)
      Y[(int64_t)col * m + row] = conjd(th);
    else
      Y[i] = th;
  }
  if (threadIdx.x == 0) sh.flops += 8ull * rows * cols * cm + 6ull * rows * cols;
  __syncthreads();
  prof_add(w, PF_THETA, t0);
  factor(w, Y, n, m, a.eps, sh, t0);
  const int L = min(rows, cols);
  choose_rank(L, a.chi_max, a.eps, true, kappa_of(a.eps, L), sh);
  const int r = sh.r;
  const double nrm = sh.nrm_inv;
  if (right) {
    // site p = U_r : [s][a][j] = conj(w_{o_j}[ipos[(a,s)]]) / s_j
    for (int i = threadIdx.x; i < rows * r; i += kThreads) {
      const int row = i / r, j = i % r;
      const double2 v = Y[(int64_t)sh.order[j] * m + sh.ipos[row]];
      const double s = sh.sinv[j];
      Ap[((int64_t)(row & 1) * cl + (row >> 1)) * r + j] = make_double2(v.x * s, -v.y * s);
    }
    __syncthreads();
    complete_columns(ColL{Ap, cl, r}, rows, r, sh);
    // site p+1 = U_r^H theta / nrm : [t][j][b]
    for (int i = threadIdx.x; i < r * cols; i += kThreads) {
      const int j = i / cols, col = i % cols;
      const int t = col / cr, b = col % cr;
      double2 acc = make_double2(0.0, 0.0);
      for (int row = 0; row < rows; ++row) {
        const double2 u = Ap[((int64_t)(row & 1) * cl + (row >> 1)) * r + j];
        const double2 v = cmulc(u, w.Th[(int64_t)row * cols + col]);
        acc.x += v.x;
        acc.y += v.y;
      }
      Aq[((int64_t)t * r + j) * cr + b] = make_double2(acc.x * nrm, acc.y * nrm);
    }
  } else {
    // site p+1 = V_r^H : [t][j][b] = conj(V[(t,b)][j]) = w_{o_j}[ipos[(t,b)]] / s_j
    for (int i = threadIdx.x; i < r * cols; i += kThreads) {
      const int t = i / (r * cr), rem = i % (r * cr), j = rem / cr, b = rem % cr;
      const double2 v = Y[(int64_t)sh.order[j] * m + sh.ipos[t * cr + b]];
      const double s = sh.sinv[j];
      Aq[i] = make_double2(v.x * s, v.y * s);
    }
    __syncthreads();
    complete_columns(ColR{Aq, cr, r}, cols, r, sh);
    // site p = theta V_r / nrm : [s][a][j]
    for (int i = threadIdx.x; i < rows * r; i += kThreads) {
      const int row = i / r, j = i % r;
      const double2* g = w.Th + (int64_t)row * cols;
      double2 acc = make_double2(0.0, 0.0);
      for (int col = 0; col < cols; ++col) {
        const int t = col / cr, b = col % cr;
        const double2 vh = Aq[((int64_t)t * r + j) * cr + b];
        const double2 v = cmul(g[col], conjd(vh));
        acc.x += v.x;
        acc.y += v.y;
      }
      Ap[((int64_t)(row & 1) * cl + (row >> 1)) * r + j] = make_double2(acc.x * nrm, acc.y * nrm);
    }
  }
  if (threadIdx.x == 0) {
    sh.chi[p + 1] = r;
    sh.flops += 8ull * r * rows * cols;
  }
  __syncthreads();
  prof_add(w, PF_OUT, t0);
}

__global__ void __launch_bounds__(kThreads, kCtas) build_kernel(BuildArgs a) {
  __shared__ Shared sh;
  extern __shared__ __align__(16) double2 ys_dyn[];
  Work w;
  w.slice = a.ws + (int64_t)blockIdx.x * a.ws_stride;
  w.Th = w.slice + a.w_off;
  w.T0 = w.Th + a.wcap;
  w.Yg = w.T0 + a.wcap;
  w.Ys = ys_dyn;
  w.prof = a.prof ? a.prof + (int64_t)blockIdx.x * PF_N : nullptr;
  unsigned long long t0 = clock64();
  const int n = a.n;
  if (threadIdx.x == 0) {
    sh.sweeps = 0;
    sh.flops = 0ull;
  }
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) sh.sample = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = sh.sample;
    if (item >= a.n_items) break;
    const int smp = a.items ? a.items[item] : item;
    const double* x = a.X + (int64_t)smp * n;
    if (threadIdx.x == 0) {
      sh.bad = 0;
      sh.wsum = 0.0;
    }
    // |+>^n (Hadamard layer, Eq. 2)
    for (int k = threadIdx.x; k <= n; k += kThreads) sh.chi[k] = 1;
    for (int k = threadIdx.x; k < n; k += kThreads) {
      double2* A = site(a, w.slice, k);
      A[0] = make_double2(M_SQRT1_2, 0.0);
      A[1] = make_double2(M_SQRT1_2, 0.0);
    }
    __syncthreads();
    int centre = 0;
    for (int rep = 0; rep < a.reps; ++rep) {
      // exp(-i H_Z): slice q of site k times exp(-i phi_k (1 - 2q)) (Eq. 4)
      for (int k = 0; k < n; ++k) {
        const int cl = sh.chi[k], cr = sh.chi[k + 1];
        double sp, cp;
        sincos(a.gamma * x[k], &sp, &cp);
        double2* A = site(a, w.slice, k);
        for (int i = threadIdx.x; i < 2 * cl * cr; i += kThreads) {
          const int q = i / (cl * cr);
          A[i] = cmul(A[i], make_double2(cp, q ? sp : -sp));
        }
      }
      __syncthreads();
      prof_add(w, PF_OTHER, t0);
      for (int oi = 0; oi < a.n_ops; ++oi) {
        const Op op = a.ops[oi];
        while (centre < op.p) {
          move_right(a, w, centre, sh, t0);
          ++centre;
        }
        while (centre > op.p + 1) {
          move_left(a, w, centre, sh, t0);
          --centre;
        }
        int nxt;
        if (oi + 1 < a.n_ops)
          nxt = a.ops[oi + 1].p;
        else if (rep + 1 < a.reps)
          nxt = a.ops[0].p;
        else
          nxt = n;
        const bool right = nxt > op.p;
        two_site(a, w, x, op, right, sh, t0);
        centre = right ? op.p + 1 : op.p;
        if (a.rank_trace && threadIdx.x == 0)
          a.rank_trace[(int64_t)smp * a.reps * a.n_ops + (int64_t)rep * a.n_ops + oi] = sh.r;
      }
    }
    while (centre < n - 1) {
      move_right(a, w, centre, sh, t0);
      ++centre;
    }
    // pack into the output pool in the storage precision
    __shared__ unsigned long long s_off;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
      unsigned long long elems = 0;
      for (int k = 0; k < n; ++k) elems += 2ull * sh.chi[k] * sh.chi[k + 1];
      unsigned long long bytes = elems * (a.store ? 8ull : 16ull);
      bytes = (bytes + 255ull) & ~255ull;
      const unsigned long long off = atomicAdd(a.pool_used, bytes);
      s_ok = (off + bytes <= a.pool_cap);
      s_off = off;
      a.need_bytes[smp] = (int64_t)bytes;
      a.status[smp] = sh.bad | (s_ok ? 0 : 2);
      a.trunc_w[smp] = sh.wsum;
      for (int k = 0; k <= n; ++k) a.dims[(int64_t)smp * (n + 1) + k] = sh.chi[k];
    }
    __syncthreads();
    if (s_ok) {
      unsigned long long off = s_off;
      for (int k = 0; k < n; ++k) {
        const int cnt = 2 * sh.chi[k] * sh.chi[k + 1];
        const double2* A = site(a, w.slice, k);
        char* dst = a.pool + off;
        if (threadIdx.x == 0) a.site_ptr[(int64_t)smp * n + k] = (uint64_t)dst;
        if (a.store) {
          float2* D = reinterpret_cast<float2*>(dst);
          for (int i = threadIdx.x; i < cnt; i += kThreads)
            D[i] = make_float2(__double2float_rn(A[i].x), __double2float_rn(A[i].y));
          off += (unsigned long long)cnt * 8ull;
        } else {
          double2* D = reinterpret_cast<double2*>(dst);
          for (int i = threadIdx.x; i < cnt; i += kThreads) D[i] = A[i];
          off += (unsigned long long)cnt * 16ull;
        }
      }
    }
    prof_add(w, PF_OTHER, t0);
  }
  if (w.prof && threadIdx.x == 0) {
    w.prof[PF_SWEEPS] += sh.sweeps;
    w.prof[PF_FLOPS] += sh.flops;
  }
}

// profile of the last qk_build_states call on this thread
struct BuildProfile {
  double kernel_ms = 0.0;
  double sm_ms[PF_OTHER + 1] = {};  // per phase, SM-milliseconds summed over CTAs
  int64_t ctas = 0, sweeps = 0, factors = 0;
  double flops = 0.0;  // FP64 flops executed
};
thread_local BuildProfile g_bprof;

}  // namespace

// Host side: validates nothing (qk_build_states does), sizes the workspace,
// launches the persistent kernel, grows the pool for states that did not fit.
qk_status build_states_device(const double* dX, int64_t N, int n, int d, int reps,
                              double gamma, int chi_max, double eps, qk_store store,
                              int32_t* rank_trace, cudaStream_t st, qk_mps_batch* out) {
  std::vector<Op> ops = make_schedule(n, d);
  const int n_ops = (int)ops.size();
  int dev = 0;
  QK_CUDA(cudaGetDevice(&dev));
  int sms = 0, clock_khz = 0;
  QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QK_CUDA(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
  // per-site capacity: chi_k <= min(2^k, 2^(n-k), chi_max)
  std::vector<int64_t> capchi(n + 1);
  for (int k = 0; k <= n; ++k) {
    int64_t c = chi_max;
    int e = std::min(k, n - k);
    if (e < 30) c = std::min<int64_t>(c, (int64_t)1 << e);
    capchi[k] = c;
  }
  std::vector<int64_t> cap_off(n + 1);
  int64_t o = 0;
  for (int k = 0; k < n; ++k) {
    cap_off[k] = o;
    o += 2 * capchi[k] * capchi[k + 1];
    o = (o + 15) & ~int64_t(15);
  }
  cap_off[n] = o;
  const int64_t wcap = (int64_t)(2 * chi_max) * (2 * chi_max);
  const int64_t ws_stride = ((o + 3 * wcap) + 31) & ~int64_t(31);
  int64_t n_ctas = std::min<int64_t>((int64_t)kCtas * sms, N);
  size_t free_b = 0, total_b = 0;
  QK_CUDA(cudaMemGetInfo(&free_b, &total_b));
  while (n_ctas > 1 && (size_t)(n_ctas * ws_stride * 16) > free_b / 3) n_ctas /= 2;
  if ((size_t)(n_ctas * ws_stride * 16) > free_b / 2)
    return fail(QK_ERR_OOM, "qk_build_states: workspace does not fit in device memory");
  const int smem = kSmemElems * (int)sizeof(double2);
  QK_CUDA(cudaFuncSetAttribute(build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));

  double2* ws = nullptr;
  Op* d_ops = nullptr;
  int64_t* d_cap = nullptr;
  int32_t* d_status = nullptr;
  int64_t* d_need = nullptr;
  int* d_queue = nullptr;
  unsigned long long* d_used = nullptr;
  unsigned long long* d_prof = nullptr;
  qk_status rc = QK_OK;
  auto cleanup = [&]() {
    cudaFree(ws);
    cudaFree(d_ops);
    cudaFree(d_cap);
    cudaFree(d_status);
    cudaFree(d_need);
    cudaFree(d_queue);
    cudaFree(d_used);
    cudaFree(d_prof);
  };
#define QK_TRY(call)                        \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) {                \
      rc = cuda_fail(e_, #call);            \
      cleanup();                            \
      return rc;                            \
    }                                       \
  } while (0)
  QK_TRY(cudaMalloc(&ws, (size_t)n_ctas * ws_stride * sizeof(double2)));
  QK_TRY(cudaMalloc(&d_ops, sizeof(Op) * std::max(1, n_ops)));
  QK_TRY(cudaMalloc(&d_cap, sizeof(int64_t) * (n + 1)));
  QK_TRY(cudaMalloc(&d_status, sizeof(int32_t) * N));
  QK_TRY(cudaMalloc(&d_need, sizeof(int64_t) * N));
  QK_TRY(cudaMalloc(&d_queue, sizeof(int)));
  QK_TRY(cudaMalloc(&d_used, sizeof(unsigned long long)));
  QK_TRY(cudaMalloc(&d_prof, sizeof(unsigned long long) * PF_N * n_ctas));
  QK_TRY(cudaMemsetAsync(d_prof, 0, sizeof(unsigned long long) * PF_N * n_ctas, st));
  if (n_ops) QK_TRY(cudaMemcpyAsync(d_ops, ops.data(), sizeof(Op) * n_ops, cudaMemcpyHostToDevice, st));
  QK_TRY(cudaMemcpyAsync(d_cap, cap_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
  QK_TRY(cudaMalloc(&out->d_dims, sizeof(int32_t) * N * (n + 1)));
  QK_TRY(cudaMalloc(&out->d_site_ptr, sizeof(uint64_t) * N * n));
  QK_TRY(cudaMalloc(&out->d_trunc_w, sizeof(double) * N));

  // first pool: a guess of the final size, grown for the states that overflow
  const size_t eb = store == QK_STORE_C64 ? 8 : 16;
  size_t worst = 0;
  for (int k = 0; k < n; ++k) worst += 2 * capchi[k] * capchi[k + 1] * eb;
  worst = (worst + 255) & ~size_t(255);
  QK_TRY(cudaMemGetInfo(&free_b, &total_b));
  size_t pool_cap = std::min<size_t>(worst * (size_t)N, free_b / 3);
  pool_cap = std::max<size_t>(pool_cap, 256);

  std::vector<int32_t> items;  // empty: all samples
  int32_t* d_items = nullptr;
  int64_t n_items = N;
  bool any_numeric = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  float kernel_ms = 0.f;
  for (int pass = 0; pass < 8 && n_items > 0; ++pass) {
    void* pool = nullptr;
    QK_TRY(cudaMalloc(&pool, pool_cap));
    out->chunks.push_back(Chunk{pool, pool_cap});
    QK_TRY(cudaMemsetAsync(d_queue, 0, sizeof(int), st));
    QK_TRY(cudaMemsetAsync(d_used, 0, sizeof(unsigned long long), st));
    BuildArgs a;
    a.X = dX;
    a.n_items = n_items;
    a.items = d_items;
    a.n = n;
    a.d = d;
    a.reps = reps;
    a.n_ops = n_ops;
    a.gamma = gamma;
    a.eps = eps;
    a.chi_max = chi_max;
    a.ops = d_ops;
    a.ws = ws;
    a.ws_stride = ws_stride;
    a.cap_off = d_cap;
    a.w_off = o;
    a.wcap = wcap;
    a.pool = (char*)pool;
    a.pool_cap = pool_cap;
    a.pool_used = d_used;
    a.store = store == QK_STORE_C64 ? 1 : 0;
    a.dims = out->d_dims;
    a.site_ptr = out->d_site_ptr;
    a.trunc_w = out->d_trunc_w;
    a.status = d_status;
    a.need_bytes = d_need;
    a.rank_trace = rank_trace;
    a.queue = d_queue;
    a.prof = d_prof;
    int grid = (int)std::min<int64_t>(n_ctas, n_items);
    cudaEventRecord(ev0, st);
    build_kernel<<<grid, kThreads, smem, st>>>(a);
    cudaEventRecord(ev1, st);
    QK_TRY(cudaGetLastError());
    std::vector<int32_t> status(N);
    std::vector<int64_t> need(N);
    QK_TRY(cudaMemcpyAsync(status.data(), d_status, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    QK_TRY(cudaMemcpyAsync(need.data(), d_need, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, st));
    QK_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) kernel_ms += ms;
    std::vector<int32_t> redo;
    size_t redo_bytes = 0;
    auto consider = [&](int64_t s) {
      if (status[s] & 1) any_numeric = true;
      if (status[s] & 2) {
        redo.push_back((int32_t)s);
        redo_bytes += (size_t)need[s];
      }
    };
    if (items.empty())
      for (int64_t s = 0; s < N; ++s) consider(s);
    else
      for (int32_t s : items) consider(s);
    cudaFree(d_items);
    d_items = nullptr;
    items = redo;
    n_items = (int64_t)redo.size();
    if (n_items) {
      QK_TRY(cudaMalloc(&d_items, sizeof(int32_t) * n_items));
      QK_TRY(cudaMemcpyAsync(d_items, items.data(), sizeof(int32_t) * n_items, cudaMemcpyHostToDevice, st));
      pool_cap = redo_bytes + 256;
    }
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaFree(d_items);
  if (n_items > 0) {
    cleanup();
    return fail(QK_ERR_OOM, "qk_build_states: could not place every state in device memory");
  }
  {
    std::vector<unsigned long long> hp((size_t)PF_N * n_ctas);
    QK_TRY(cudaMemcpy(hp.data(), d_prof, sizeof(unsigned long long) * hp.size(), cudaMemcpyDeviceToHost));
    BuildProfile bp;
    bp.kernel_ms = kernel_ms;
    bp.ctas = n_ctas;
    for (int64_t c = 0; c < n_ctas; ++c) {
      const unsigned long long* row = hp.data() + (size_t)c * PF_N;
      // clock64 cycles -> milliseconds at the SM clock
      for (int f = PF_THETA; f <= PF_OTHER; ++f) bp.sm_ms[f] += (double)row[f] / (double)clock_khz;
      bp.sweeps += (int64_t)row[PF_SWEEPS];
      bp.factors += (int64_t)row[PF_FACTOR];
      bp.flops += (double)row[PF_FLOPS];
    }
    g_bprof = bp;
  }
#undef QK_TRY
  cleanup();
  if (any_numeric) return fail(QK_ERR_NUMERIC, "qk_build_states: an SVD reached its sweep cap or met a non-finite value");
  return QK_OK;
}

}  // namespace qk

extern "C" qk_status qk_last_build_profile(double* kernel_ms, double* phase_sm_ms, int64_t* ctas,
                                          int64_t* sweeps, int64_t* factorisations, double* fp64_flops) {
  const qk::BuildProfile& b = qk::g_bprof;
  if (fp64_flops) *fp64_flops = b.flops;
  if (kernel_ms) *kernel_ms = b.kernel_ms;
  if (phase_sm_ms)
    for (int f = 0; f <= qk::PF_OTHER; ++f) phase_sm_ms[f] = b.sm_ms[f];
  if (ctas) *ctas = b.ctas;
  if (sweeps) *sweeps = b.sweeps;
  if (factorisations) *factorisations = b.factors;
  return QK_OK;
}
