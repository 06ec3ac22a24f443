"""Plain FP64 CPU oracle for HaTT (Hadamard-avoiding TT recompression).

TEST INFRASTRUCTURE ONLY. Only the test suite, `__graft_entry__.smoke()` and
`bench.py`'s CPU-baseline / reference leg may import or call anything in this
package. The CUDA product path never imports it and shares no code with it:
the only common module is the seeded input generator
`paper_2410_04385_gb300.workloads`, which holds none of the method's arithmetic.

Every function follows the paper's definitions step by step in float64 numpy,
with numpy/LAPACK routines (matmul, QR, SVD) as the only library steps:

  philox.py    counter-based RNG (Salmon et al., SC'11) + Box-Muller sketch TT
               (Definition 2.1 random Gaussian TT).
  tt.py        TT basics (Section 2.1-2.2): dense expansion, PKP (Hadamard via
               partial Kronecker product), inner product, stable difference norm.
  rounding.py  TT-Rounding (Algorithm 1) and the truncation rule.
  randorth.py  RandOrth (Algorithm 2) on explicit cores.
  hatt.py      HPCRL-1 (Section 3.1, Eq. (3.3)-(3.6), Algorithm 3) in two
               independent codings, the HaTT left-to-right pass (Section 3.2,
               Eq. (3.8)-(3.10), Algorithm 4), the rank plan, the truncation
               sweep and the end-to-end recompression.
  flops.py     the Section 4 / Table 4.1 cost model.

Parity status: every function is pinned by a `-m "not gpu"` test
(tests/test_oracle_*.py) against brute force, closed forms, library routines
or known-answer vectors. The accuracy of HaTT at a target rank below the
numerical rank, which the paper does not bound, is held to a bound assembled
from published results (the Gaussian range finder's expected error per bond,
Halko, Martinsson and Tropp 2011, and the root-sum-of-squares accumulation of
bond errors in a TT, Oseledets 2011), with a factor 2 over several seeds.
"""
