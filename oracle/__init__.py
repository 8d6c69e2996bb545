"""CPU oracle for the quantum-kernel Gram path (TEST INFRASTRUCTURE ONLY).

A plain, slow, FP64 restatement of what the method computes, written from the
paper (arXiv 2411.09336, Sec. II) and sharing no code with the CUDA library:

  circuit.py      edge set G, gate angles (Eqs. 4-5) and the 2-site op schedule
                  with SWAP routing (Sec. II-C).
  statevector.py  brute-force 2^n statevector of U(x)|+>^m (Eqs. 2-5), n <= 14.
  mps.py          MPS simulation with per-gate SVD truncation (Sec. II-B, Fig. 1,
                  Eq. 8), numpy's LAPACK SVD.
  overlap.py      MPS inner products by the left-to-right transfer sweep
                  (Fig. 2), the right-to-left sweep as a cross-check, the Gram
                  matrix (Eq. 1) and the d=0 product-state closed form.
  mlp.py          the learned surrogate's MLP (not in the paper): forward,
                  backward, Adam, split-conformal calibration.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
arm may import or run anything in this package.  The product path (the
paper_2411_09336_gb300 package and libqk) never calls it.

Parity status per function:
  statevector.*      pinned (closed form at d=0, gate identities, invariants).
  circuit.*          pinned (op counts, qubit-permutation replay, statevector).
  mps.build_mps      pinned against statevector at n <= 12 (eps = 0) and the
                     truncation bound of Eq. 8 at eps > 0.  Exact ranks at
                     eps > 0 where a tail sum sits on the threshold (near
                     ties) are parity unpinned: only agreement can be checked.
  overlap.*          pinned (closed form, statevector, two sweep orders).
  mlp.*              pinned (finite differences, closed-form cases).
"""
