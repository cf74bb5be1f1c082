"""FP64 CPU oracle for the FFT bin-averaged bispectrum estimator (Sec. 2).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only the tests, the package's smoke entry
(`__graft_entry__.smoke`) and the CPU-baseline leg of `bench.py` may import or run
anything here. The CUDA path shares no code with this package and never calls it.

Modules
  plan      shells, mode counts, shell means, triplet enumeration, (mu, t) labels and
            cells, the aliasing cap (Sec. 2.1, Eqs. (2.2), (2.4), (2.12))
  fbe       the FFT estimator written out plainly in float64 (Eqs. (2.7)-(2.11))
  dbe       the direct estimator: a literal loop over k-mode pairs (Eqs. (2.3), (2.9))
  analytic  Eq. (3.2), Eq. (3.3), the exact grid expectation of Eq. (2.5) for the
            quadratic field, and the Kaiser monopole factor (Eq. (3.4), own derivation)
  grad      the adjoint of the estimator with respect to delta(x)

Every function here is pinned by the `-m "not gpu"` tests against something other than
itself (brute force, closed forms, values the paper prints, invariants); the one
exception is listed in its module header as "parity unpinned".
"""
