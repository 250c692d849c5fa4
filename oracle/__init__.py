"""Plain, slow, FP64 CPU oracle for the structured-sketch hot path (arxiv 2508.21189).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py (its
cpu_baseline leg and its ``--impl reference`` arm) may import anything from this package.
The product package ``paper_2508_21189_gb300`` never imports it, and this package imports
nothing from the product: the two share no code, headers, tables or constants.  The only
module both sides use is ``synthetic`` (seeded input generators, none of the method's
arithmetic).

Modules, each citing the passage it follows:
  philox       Philox4x32-10 (Salmon et al., SC'11); pinned by the published known-answer
               vectors.
  sparse_sign  SparseUniform (Def. "SparseUniform", Sec. 3.2.1) as the left sketch S = Psi^T,
               Floyd sampling without replacement; pinned by uniformity of subsets, the
               zeta/d marginals, isotropy E[S^T S] = I, dense brute force, and the injectivity /
               dilation of the adversarial coordinate subspace against the Gaussian asymptotes.
  srtt         Omega = D F S with the WHT (Eq. "intro-srtt", Sec. 1.6; cost steps 1-3 of
               Sec. 4.x); pinned by scipy's Sylvester Hadamard matrix, H^T H = n I,
               the unsubsampled case being orthogonal, isotropy by Monte Carlo.
  lsq          sketch-and-solve (Alg. 3) warm start + preconditioned LSQR refinement; pinned
               by k = 1 closed form, orthonormal columns (x* = A^T b), consistent systems,
               agreement with LAPACK least squares, and the warm start's residual within the
               sketch-and-solve bound (Sec. 2.3).
  rsvd         Alg. 1 with power iterations; pinned by exact recovery of low-rank matrices,
               the Eckart-Young lower bound, the HMT-style upper bound, and agreement with a
               Gaussian test matrix's error (Fig. 1's comparison).
Every function above is pinned; none is "parity unpinned".
"""
