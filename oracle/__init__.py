"""FP64 CPU oracle for the dense-CRF filtering hot path (TEST INFRASTRUCTURE).

This package is the plain, slow reference that the CUDA path is checked
against.  It is test infrastructure only: the tests, the smoke check and the
CPU-baseline leg of the benchmark may call it; the product path never does.
It shares no code with the CUDA path and imports nothing from it.

Modules
-------
crf           exact definitions: features and kernel (Eq. 3-4), brute-force
              Gaussian sums (Eq. 6 done the O(N^2) way), Psi (Eq. 7), d and D
              (Eq. 11), S_cvx (Eq. 10), the QP objective (Eq. 8), E(x) (Eq. 1)
              and the LP objective (Eq. 18).
permutohedral the permutohedral-lattice filter the paper relies on (Section 3,
              Appendix A), unnormalised, written from the lattice geometry.
qp            Frank-Wolfe on S_cvx (Algorithm 1 with the closed-form step and
              product reuse of Appendix B) and CCCP for the generic DC
              relaxation (Algorithm 2, Section 5.1).
lp            the LP subgradient (Eq. 19-20) by brute force and by the
              divide-and-conquer of Appendix E, simplex projection and the
              projected subgradient loop (Algorithm 3).

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
except the absolute scale of the lattice approximation against the exact
Gaussian sum, which is reported, not pinned (parity unpinned for that ratio).
"""
