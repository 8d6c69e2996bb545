// Batched MPS simulation of the feature-map circuit in FP64 (Sec. II-B/C).
//
// One CTA builds one state at a time and takes the next sample index from a
// global counter (persistent launch, one or two CTAs per SM).  The state
// being built lives in the CTA's slice of a workspace in HBM (FP64 complex
// site tensors at a fixed capacity per site); three (2 chi_max)^2 scratch
// matrices hold the two-site tensor theta, its gated copy and GEMM results.
// The hot loop is the one-sided (Hestenes) Jacobi SVD of every gated theta,
// run on the CUDA cores in FP64: parallel round-robin ordering, one warp per
// column pair, rotation when |c_p^H c_q| > tol ||c_p|| ||c_q||.  The side that
// must be an isometry is always taken from the Jacobi columns themselves and
// the side carrying the singular values from one GEMM with the gated theta,
// so no rotation matrix is accumulated and no small singular value is
// divided by.
//
// Truncation (Eq. 8, read as a discarded-weight rule): with s sorted
// descending, keep r = min{r >= 1 : sum_{i >= r} s_i^2 <= eps^2 sum_i s_i^2}
// (the tail summed from the smallest value upward), then r <= chi_max, and
// rescale the kept values to unit norm.  eps = 0 keeps everything up to
// chi_max.  The orthogonality centre follows the gate: after an op at
// (p, p+1) the singular values go to site p+1 if the next op lies to the
// right, else to site p; between repetitions the centre walks back by
// orthogonal factorisations without truncation, and finally walks to the
// last site, so the stored state is left-canonical.
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
  int64_t w_off;           // offset of scratch W (then G, T at +wcap, +2 wcap)
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
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct Shared {
  double s2[kMaxCols];   // column norms^2 after convergence
  double sv[kMaxCols];   // singular values, sorted descending
  int perm[kMaxCols];    // sorted position -> column
  double tail[kMaxCols + 1];
  int chi[kMaxN + 1];
  double pa[kMaxCols / 2], pb[kMaxCols / 2], pgr[kMaxCols / 2], pgi[kMaxCols / 2];
  double pc[kMaxCols / 2], psx[kMaxCols / 2], psy[kMaxCols / 2];
  int pidx[kMaxCols / 2];
  int rotated;
  int r;
  int sample;
  int bad;
  double nrm_inv;
  double wsum;
};

// One-sided Jacobi on the `cols` columns (length `rows`, column-major) of W.
// A round of the round-robin ordering rotates up to cols/2 disjoint pairs in
// three phases: (A) a team of T lanes forms |c_p|^2, |c_q|^2 and c_p^H c_q
// for each pair, (B) one thread per pair turns them into the rotation (so the
// FP64 divisions and square roots are done once per pair, not once per lane),
// (C) the team applies it.  Returns false if the sweep cap was reached.
__device__ bool jacobi(double2* W, int rows, int cols, Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int npad = cols + (cols & 1);
  const int npairs = npad / 2;
  const double tol = (double)(rows > 32 ? rows : 32) * 2.220446049250313e-16;
  if (cols < 2) return true;
  // team size: about 8 rows per lane, 4..32 lanes
  int T = 4;
  while (T < 32 && T * 8 < rows) T <<= 1;
  const int per_warp = 32 / T;
  const int team = warp * per_warp + lane / T;
  const int tl = lane % T;
  const int nteams = kWarps * per_warp;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) sh.rotated = 0;
    __syncthreads();
    for (int round = 0; round < npad - 1; ++round) {
      // (A) inner products; the loop is uniform across the warp so every
      // lane reaches the team shuffles
      for (int kb = warp * per_warp; kb < npairs; kb += nteams) {
        const int k = kb + lane / T;
        int p = npad, q = npad;
        if (k < npairs) {
          if (k == 0) {
            p = npad - 1;
            q = round;
          } else {
            p = (round + k) % (npad - 1);
            q = (round - k + (npad - 1)) % (npad - 1);
          }
        }
        const bool valid = p < cols && q < cols;
        double a = 0.0, b = 0.0, gr = 0.0, gi = 0.0;
        if (valid) {
          const double2* cp = W + (int64_t)p * rows;
          const double2* cq = W + (int64_t)q * rows;
          for (int i = tl; i < rows; i += T) {
            double2 u = cp[i], v = cq[i];
            a = fma(u.x, u.x, fma(u.y, u.y, a));
            b = fma(v.x, v.x, fma(v.y, v.y, b));
            gr = fma(u.x, v.x, fma(u.y, v.y, gr));   // Re(conj(u) v)
            gi = fma(u.x, v.y, fma(-u.y, v.x, gi));  // Im(conj(u) v)
          }
        }
        for (int o = T >> 1; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gi += __shfl_xor_sync(0xffffffffu, gi, o);
        }
        if (tl == 0 && k < npairs) {
          sh.pa[k] = a;
          sh.pb[k] = b;
          sh.pgr[k] = gr;
          sh.pgi[k] = gi;
          sh.pidx[k] = valid ? (p | (q << 16)) : -1;
        }
      }
      __syncthreads();
      // (B) rotation parameters, one thread per pair
      for (int k = threadIdx.x; k < npairs; k += kThreads) {
        double a = sh.pa[k], b = sh.pb[k], gr = sh.pgr[k], gi = sh.pgi[k];
        double g = sqrt(gr * gr + gi * gi);
        bool rot = sh.pidx[k] >= 0 && a != 0.0 && b != 0.0 && g > tol * sqrt(a) * sqrt(b);
        double c = 1.0, sx = 0.0, sy = 0.0;
        if (rot) {
          // [[c, s e^{i phi}], [-s e^{-i phi}, c]] zeroes conj(c_p) c_q
          double zeta = (b - a) / (2.0 * g);
          double t = fabs(zeta) > 1e100
                         ? 0.5 / zeta
                         : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          if (t == 0.0) {
            rot = false;
          } else {
            c = 1.0 / sqrt(1.0 + t * t);
            double s = c * t;
            sx = s * gr / g;  // s e^{i phi} = (sx, sy)
            sy = s * gi / g;
          }
        }
        sh.pc[k] = rot ? c : 0.0;  // 0 marks "no rotation"
        sh.psx[k] = sx;
        sh.psy[k] = sy;
        if (rot) atomicAdd(&sh.rotated, 1);
      }
      __syncthreads();
      // (C) apply: c_p' = c c_p - s e^{-i phi} c_q ;  c_q' = s e^{i phi} c_p + c c_q
      for (int k = team; k < npairs; k += nteams) {
        const double c = sh.pc[k];
        if (c == 0.0) continue;
        const int pq = sh.pidx[k];
        const int p = pq & 0xffff, q = pq >> 16;
        const double sx = sh.psx[k], sy = sh.psy[k];
        double2* cp = W + (int64_t)p * rows;
        double2* cq = W + (int64_t)q * rows;
        for (int i = tl; i < rows; i += T) {
          double2 u = cp[i], v = cq[i];
          // s e^{-i phi} v = (sx v.x + sy v.y, sx v.y - sy v.x)
          cp[i] = make_double2(c * u.x - (sx * v.x + sy * v.y), c * u.y - (sx * v.y - sy * v.x));
          cq[i] = make_double2(c * v.x + (sx * u.x - sy * u.y), c * v.y + (sx * u.y + sy * u.x));
        }
      }
      __syncthreads();
    }
    if (sh.rotated == 0) return true;
    __syncthreads();
  }
  return false;
}

// Column norms, descending sort (ties by column index).
__device__ void sort_columns(const double2* W, int rows, int cols, Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < cols; j += kWarps) {
    const double2* c = W + (int64_t)j * rows;
    double a = 0.0;
    for (int i = lane; i < rows; i += 32) a = fma(c[i].x, c[i].x, fma(c[i].y, c[i].y, a));
    a = warp_sum(a);
    if (lane == 0) sh.s2[j] = a;
  }
  __syncthreads();
  // non-negative doubles order like their bit patterns: compare as integers
  // (keeps the O(cols^2) ranking off the FP64 pipe)
  for (int i = threadIdx.x; i < cols; i += kThreads) {
    const unsigned long long v = (unsigned long long)__double_as_longlong(sh.s2[i]);
    int rank = 0;
    for (int j = 0; j < cols; ++j) {
      const unsigned long long u = (unsigned long long)__double_as_longlong(sh.s2[j]);
      rank += (u > v) || (u == v && j < i);
    }
    sh.perm[rank] = i;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cols; i += kThreads) sh.sv[i] = sqrt(sh.s2[sh.perm[i]]);
  __syncthreads();
}

// Replace kept columns whose singular value is (numerically) zero by unit
// vectors orthogonal to the other kept columns (classical Gram-Schmidt,
// twice).  Columns are normalised in place (divided by their singular value)
// beforehand by the caller's convention: here W column perm[j] is scaled to
// unit norm for j < k.
__device__ void normalise_and_complete(double2* W, int rows, int k, Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_need;
  if (threadIdx.x == 0) s_need = 0;
  __syncthreads();
  for (int j = warp; j < k; j += kWarps) {
    double sv = sh.sv[j];
    double2* c = W + (int64_t)sh.perm[j] * rows;
    if (sv > 1e-280) {
      double inv = 1.0 / sv;
      for (int i = lane; i < rows; i += 32) c[i] = cscale(c[i], inv);
    } else if (lane == 0) {
      s_need = 1;
    }
  }
  __syncthreads();
  if (!s_need) return;
  // rare path: one warp completes the basis serially
  if (warp == 0) {
    int e = 0;
    for (int j = 0; j < k; ++j) {
      if (sh.sv[j] > 1e-280) continue;
      double2* c = W + (int64_t)sh.perm[j] * rows;
      for (; e < rows; ++e) {
        for (int i = lane; i < rows; i += 32) c[i] = make_double2(i == e ? 1.0 : 0.0, 0.0);
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass) {
          for (int jj = 0; jj < k; ++jj) {
            if (jj == j || (sh.sv[jj] <= 1e-280 && jj > j)) continue;
            const double2* o = W + (int64_t)sh.perm[jj] * rows;
            double pr = 0.0, pi = 0.0;
            for (int i = lane; i < rows; i += 32) {
              pr += o[i].x * c[i].x + o[i].y * c[i].y;
              pi += o[i].x * c[i].y - o[i].y * c[i].x;
            }
            pr = warp_sum(pr);
            pi = warp_sum(pi);
            for (int i = lane; i < rows; i += 32) {
              double2 oi = o[i];
              c[i].x -= pr * oi.x - pi * oi.y;
              c[i].y -= pr * oi.y + pi * oi.x;
            }
            __syncwarp();
          }
        }
        double nn = 0.0;
        for (int i = lane; i < rows; i += 32) nn += c[i].x * c[i].x + c[i].y * c[i].y;
        nn = warp_sum(nn);
        if (nn > 0.25) {
          double inv = 1.0 / sqrt(nn);
          for (int i = lane; i < rows; i += 32) c[i] = cscale(c[i], inv);
          __syncwarp();
          ++e;
          break;
        }
      }
    }
  }
  __syncthreads();
}

// Truncation rank by the discarded-weight rule (single thread).
__device__ void choose_rank(int L, int chi_max, double eps, bool truncate, Shared& sh) {
  if (threadIdx.x == 0) {
    sh.tail[L] = 0.0;
    for (int i = L - 1; i >= 0; --i) sh.tail[i] = sh.tail[i + 1] + sh.sv[i] * sh.sv[i];
    double tot = sh.tail[0];
    int r = L;
    if (truncate && eps > 0.0) {
      double thr = eps * eps * tot;
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
  }
  __syncthreads();
}

__device__ __forceinline__ double2* site(const BuildArgs& a, double2* slice, int k) {
  return slice + a.cap_off[k];
}

// Centre from site c to c+1 (no truncation).
__device__ void move_right(const BuildArgs& a, double2* slice, int c, Shared& sh) {
  double2* W = slice + a.w_off;
  double2* G = W + a.wcap;
  double2* T = G + a.wcap;
  const int cl = sh.chi[c], cr = sh.chi[c + 1], cn = sh.chi[c + 2];
  const int rows = 2 * cl;
  double2* Ac = site(a, slice, c);
  double2* An = site(a, slice, c + 1);
  // G[row][b] = A_c[q][a][b], row = a*2 + q ; W = column-major copy
  for (int i = threadIdx.x; i < rows * cr; i += kThreads) {
    int row = i / cr, b = i % cr;
    int aa = row >> 1, q = row & 1;
    double2 v = Ac[(q * cl + aa) * cr + b];
    G[i] = v;
    W[(int64_t)b * rows + row] = v;
  }
  __syncthreads();
  if (!jacobi(W, rows, cr, sh) && threadIdx.x == 0) sh.bad |= 1;
  __syncthreads();
  sort_columns(W, rows, cr, sh);
  const int k = rows < cr ? rows : cr;
  normalise_and_complete(W, rows, k, sh);
  // T = U_k^H G  (k x cr)
  for (int i = threadIdx.x; i < k * cr; i += kThreads) {
    int j = i / cr, b = i % cr;
    const double2* u = W + (int64_t)sh.perm[j] * rows;
    double2 acc = make_double2(0.0, 0.0);
    for (int row = 0; row < rows; ++row) acc = cadd(acc, cmulc(u[row], G[row * cr + b]));
    T[i] = acc;
  }
  // site c = U_k
  for (int i = threadIdx.x; i < rows * k; i += kThreads) {
    int row = i / k, j = i % k;
    int aa = row >> 1, q = row & 1;
    Ac[(q * cl + aa) * k + j] = W[(int64_t)sh.perm[j] * rows + row];
  }
  __syncthreads();
  // site c+1 = T * A_{c+1}: [q][j][b'] = sum_b T[j][b] A[q][b][b']
  for (int i = threadIdx.x; i < 2 * k * cn; i += kThreads) {
    int q = i / (k * cn), rem = i % (k * cn), j = rem / cn, bb = rem % cn;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < cr; ++b) acc = cadd(acc, cmul(T[j * cr + b], An[(q * cr + b) * cn + bb]));
    G[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * k * cn; i += kThreads) An[i] = G[i];
  if (threadIdx.x == 0) sh.chi[c + 1] = k;
  __syncthreads();
}

// Centre from site c to c-1 (no truncation).
__device__ void move_left(const BuildArgs& a, double2* slice, int c, Shared& sh) {
  double2* W = slice + a.w_off;
  double2* G = W + a.wcap;
  double2* T = G + a.wcap;
  const int cp = sh.chi[c - 1], cl = sh.chi[c], cr = sh.chi[c + 1];
  const int ncol = 2 * cr;  // columns of the matrix M[a][(q, b)]
  double2* Ac = site(a, slice, c);
  double2* Ap = site(a, slice, c - 1);
  // G[a][q*cr + b] = A_c[q][a][b]; W = conj(G) read as column-major with cl
  // columns of length ncol (the columns of M^H)
  for (int i = threadIdx.x; i < cl * ncol; i += kThreads) {
    int aa = i / ncol, col = i % ncol;
    int q = col / cr, b = col % cr;
    double2 v = Ac[(q * cl + aa) * cr + b];
    G[i] = v;
    W[i] = make_double2(v.x, -v.y);
  }
  __syncthreads();
  if (!jacobi(W, ncol, cl, sh) && threadIdx.x == 0) sh.bad |= 1;
  __syncthreads();
  sort_columns(W, ncol, cl, sh);
  const int k = cl < ncol ? cl : ncol;
  normalise_and_complete(W, ncol, k, sh);
  // T = G V_k (cl x k)
  for (int i = threadIdx.x; i < cl * k; i += kThreads) {
    int aa = i / k, j = i % k;
    const double2* v = W + (int64_t)sh.perm[j] * ncol;
    double2 acc = make_double2(0.0, 0.0);
    for (int col = 0; col < ncol; ++col) acc = cadd(acc, cmul(G[aa * ncol + col], v[col]));
    T[i] = acc;
  }
  // site c = V_k^H: [q][j][b] = conj(v_j[q*cr + b])
  for (int i = threadIdx.x; i < 2 * k * cr; i += kThreads) {
    int q = i / (k * cr), rem = i % (k * cr), j = rem / cr, b = rem % cr;
    double2 v = W[(int64_t)sh.perm[j] * ncol + q * cr + b];
    Ac[i] = make_double2(v.x, -v.y);
  }
  __syncthreads();
  // site c-1 = A_{c-1} T: [q][a'][j] = sum_a A[q][a'][a] T[a][j]
  for (int i = threadIdx.x; i < 2 * cp * k; i += kThreads) {
    int q = i / (cp * k), rem = i % (cp * k), ap = rem / k, j = rem % k;
    double2 acc = make_double2(0.0, 0.0);
    for (int aa = 0; aa < cl; ++aa) acc = cadd(acc, cmul(Ap[(q * cp + ap) * cl + aa], T[aa * k + j]));
    G[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * cp * k; i += kThreads) Ap[i] = G[i];
  if (threadIdx.x == 0) sh.chi[c] = k;
  __syncthreads();
}

// One scheduled two-site op at (p, p+1); `right`: singular values go right.
__device__ void two_site(const BuildArgs& a, double2* slice, const double* x, const Op op,
                         bool right, Shared& sh) {
  double2* W = slice + a.w_off;
  double2* G = W + a.wcap;
  const int p = op.p;
  const int cl = sh.chi[p], cm = sh.chi[p + 1], cr = sh.chi[p + 2];
  const int rows = 2 * cl, cols = 2 * cr;
  double2* Ap = site(a, slice, p);
  double2* Aq = site(a, slice, p + 1);
  // theta0[(a,s)][(t,b)] = sum_c A_p[s][a][c] A_{p+1}[t][c][b]  -> W (row-major)
  for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
    int row = i / cols, col = i % cols;
    int aa = row >> 1, s = row & 1, t = col / cr, b = col % cr;
    const double2* ar = Ap + (s * cl + aa) * cm;
    const double2* bc = Aq + t * cm * cr + b;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < cm; ++c) acc = cadd(acc, cmul(ar[c], bc[c * cr]));
    W[i] = acc;
  }
  __syncthreads();
  // gate on the physical pair (s, t): theta[a,s,t,b] from theta0
  double cs = 1.0, sn = 0.0;
  if (op.kind != OP_SWAP) {
    double th = a.gamma * a.gamma * (M_PI / 2.0) * (1.0 - x[op.qi]) * (1.0 - x[op.qj]);
    sincos(th, &sn, &cs);
  }
  const bool swap = op.kind != OP_RXX;
  for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
    int row = i / cols, col = i % cols;
    int aa = row >> 1, s = row & 1, t = col / cr, b = col % cr;
    int s0 = swap ? t : s, t0 = swap ? s : t;  // SWAP after Rxx: read (t, s)
    double2 v = W[(aa * 2 + s0) * cols + t0 * cr + b];
    double2 f = W[(aa * 2 + (1 - s0)) * cols + (1 - t0) * cr + b];
    // cs * v - i sn * f
    G[i] = make_double2(cs * v.x + sn * f.y, cs * v.y - sn * f.x);
  }
  __syncthreads();
  // Jacobi orientation: right -> columns of theta; left -> columns of theta^H
  const int jr = right ? rows : cols;  // column length
  const int jc = right ? cols : rows;  // number of columns
  for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
    int row = i / cols, col = i % cols;
    double2 v = G[i];
    if (right)
      W[(int64_t)col * rows + row] = v;
    else
      W[i] = make_double2(v.x, -v.y);
  }
  __syncthreads();
  if (!jacobi(W, jr, jc, sh) && threadIdx.x == 0) sh.bad |= 1;
  __syncthreads();
  sort_columns(W, jr, jc, sh);
  const int L = jr < jc ? jr : jc;
  choose_rank(L, a.chi_max, a.eps, true, sh);
  const int r = sh.r;
  const double nrm = sh.nrm_inv;
  normalise_and_complete(W, jr, r, sh);
  if (right) {
    // site p = U_r : [s][a][k] = u_k[(a,s)]
    for (int i = threadIdx.x; i < rows * r; i += kThreads) {
      int row = i / r, k = i % r;
      int aa = row >> 1, s = row & 1;
      Ap[(s * cl + aa) * r + k] = W[(int64_t)sh.perm[k] * rows + row];
    }
    // site p+1 = U_r^H theta / nrm : [t][k][b]
    for (int i = threadIdx.x; i < r * cols; i += kThreads) {
      int k = i / cols, col = i % cols;
      int t = col / cr, b = col % cr;
      const double2* u = W + (int64_t)sh.perm[k] * rows;
      double2 acc = make_double2(0.0, 0.0);
      for (int row = 0; row < rows; ++row) acc = cadd(acc, cmulc(u[row], G[row * cols + col]));
      Aq[(t * r + k) * cr + b] = cscale(acc, nrm);
    }
  } else {
    // site p+1 = V_r^H : [t][k][b] = conj(v_k[(t,b)])
    for (int i = threadIdx.x; i < r * cols; i += kThreads) {
      int k = i / cols, col = i % cols;
      int t = col / cr, b = col % cr;
      double2 v = W[(int64_t)sh.perm[k] * cols + col];
      Aq[(t * r + k) * cr + b] = make_double2(v.x, -v.y);
    }
    // site p = theta V_r / nrm : [s][a][k]
    for (int i = threadIdx.x; i < rows * r; i += kThreads) {
      int row = i / r, k = i % r;
      int aa = row >> 1, s = row & 1;
      const double2* v = W + (int64_t)sh.perm[k] * cols;
      const double2* g = G + (int64_t)row * cols;
      double2 acc = make_double2(0.0, 0.0);
      for (int col = 0; col < cols; ++col) acc = cadd(acc, cmul(g[col], v[col]));
      Ap[(s * cl + aa) * r + k] = cscale(acc, nrm);
    }
  }
  if (threadIdx.x == 0) sh.chi[p + 1] = r;
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) build_kernel(BuildArgs a) {
  __shared__ Shared sh;
  double2* slice = a.ws + (int64_t)blockIdx.x * a.ws_stride;
  const int n = a.n;
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
      double2* A = site(a, slice, k);
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
        double2* A = site(a, slice, k);
        for (int i = threadIdx.x; i < 2 * cl * cr; i += kThreads) {
          int q = i / (cl * cr);
          double2 ph = make_double2(cp, q ? sp : -sp);
          A[i] = cmul(A[i], ph);
        }
      }
      __syncthreads();
      for (int oi = 0; oi < a.n_ops; ++oi) {
        const Op op = a.ops[oi];
        while (centre < op.p) {
          move_right(a, slice, centre, sh);
          ++centre;
        }
        while (centre > op.p + 1) {
          move_left(a, slice, centre, sh);
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
        two_site(a, slice, x, op, right, sh);
        centre = right ? op.p + 1 : op.p;
        if (a.rank_trace && threadIdx.x == 0)
          a.rank_trace[(int64_t)smp * a.reps * a.n_ops + (int64_t)rep * a.n_ops + oi] = sh.r;
      }
    }
    while (centre < n - 1) {
      move_right(a, slice, centre, sh);
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
      unsigned long long off = atomicAdd(a.pool_used, bytes);
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
        const double2* A = site(a, slice, k);
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
  }
}

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
  int sms = 0;
  QK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
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
  int64_t n_ctas = std::min<int64_t>((int64_t)2 * sms, N);
  size_t free_b = 0, total_b = 0;
  QK_CUDA(cudaMemGetInfo(&free_b, &total_b));
  while (n_ctas > 1 && (size_t)(n_ctas * ws_stride * 16) > free_b / 3) n_ctas /= 2;
  if ((size_t)(n_ctas * ws_stride * 16) > free_b / 2)
    return fail(QK_ERR_OOM, "qk_build_states: workspace does not fit in device memory");

  double2* ws = nullptr;
  Op* d_ops = nullptr;
  int64_t* d_cap = nullptr;
  int32_t* d_status = nullptr;
  int64_t* d_need = nullptr;
  int* d_queue = nullptr;
  unsigned long long* d_used = nullptr;
  qk_status rc = QK_OK;
  auto cleanup = [&]() {
    cudaFree(ws);
    cudaFree(d_ops);
    cudaFree(d_cap);
    cudaFree(d_status);
    cudaFree(d_need);
    cudaFree(d_queue);
    cudaFree(d_used);
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
    int grid = (int)std::min<int64_t>(n_ctas, n_items);
    build_kernel<<<grid, kThreads, 0, st>>>(a);
    QK_TRY(cudaGetLastError());
    std::vector<int32_t> status(N);
    std::vector<int64_t> need(N);
    QK_TRY(cudaMemcpyAsync(status.data(), d_status, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    QK_TRY(cudaMemcpyAsync(need.data(), d_need, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, st));
    QK_TRY(cudaStreamSynchronize(st));
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
  cudaFree(d_items);
  if (n_items > 0) {
    cleanup();
    return fail(QK_ERR_OOM, "qk_build_states: could not place every state in device memory");
  }
#undef QK_TRY
  cleanup();
  if (any_numeric) return fail(QK_ERR_NUMERIC, "qk_build_states: an SVD reached its sweep cap or met a non-finite value");
  return QK_OK;
}

}  // namespace qk
