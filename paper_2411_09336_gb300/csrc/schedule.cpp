// Two-site op schedule of one repetition of exp(-i H_XX) (Sec. II-C).
//
// Every Rxx(i, j) with j - i = t > 1 needs its qubits adjacent, which the
// paper arranges with t - 1 SWAPs before the gate and the reverse SWAPs after
// it.  Taking the gates of one block {(i, i+1), ..., (i, i+k)} in order, the
// SWAPs that bring qubit i back after gate t and forward again before gate
// t + 1 cancel pairwise, so qubit i walks right once and back once:
//   position p = i + t - 1, t = 1..k-1 : Rxx(i, i+t) followed by SWAP (fused)
//   position p = i + k - 1             : Rxx(i, i+k)
//   positions i + k - 2 down to i      : SWAP
// with k = min(d, n - 1 - i).  The state produced is exactly the paper's; each
// listed op is one two-site gate and one SVD truncation.
#include "qk_internal.h"

namespace qk {

std::vector<Op> make_schedule(int n, int d) {
  std::vector<Op> ops;
  for (int i = 0; i + 1 < n; ++i) {
    int k = d < (n - 1 - i) ? d : (n - 1 - i);
    if (k <= 0) continue;
    for (int t = 1; t < k; ++t) ops.push_back(Op{OP_SWAP_RXX, i + t - 1, i, i + t});
    ops.push_back(Op{OP_RXX, i + k - 1, i, i + k});
    for (int p = i + k - 2; p >= i; --p) ops.push_back(Op{OP_SWAP, p, -1, -1});
  }
  return ops;
}

}  // namespace qk

extern "C" int64_t qk_schedule_length(int32_t n, int32_t d) {
  if (n < 2 || d < 0) return 0;
  int64_t c = 0;
  for (int i = 0; i + 1 < n; ++i) {
    int k = d < (n - 1 - i) ? d : (n - 1 - i);
    if (k > 0) c += 2 * k - 1;
  }
  return c;
}
