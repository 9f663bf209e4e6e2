"""CPU FP64 oracle for the structure-preserving Bethe--Salpeter solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It shares no code with the CUDA path. The modules:

* :mod:`oracle.definition` -- the result Algorithm 1 must reach, written from
  the definitions (Eq. 1, Eq. GMG, Theorem 3, Eq. absp) through the
  Hermitian-definite pencil  S x = (1/lambda) Omega x.
* :mod:`oracle.alg1` -- Algorithm 1 and Algorithm 3 restated step by step in
  the paper's order and notation (M, L, W, T, D, Phi, Y_+), used to check the
  intermediate results of the device pipeline stage by stage.
* :mod:`oracle.alg2` -- Algorithm 2 (real problems, Theorem 5): two Cholesky
  factorizations, the SVD of L2^T L1, and X1, X2 from it.
* :mod:`oracle.sbr` -- the two-stage (band, then tridiagonal) reduction of W:
  the reference the device two-stage reduction is tested against.
* :mod:`oracle.mrrr` -- tridiagonal eigenpairs by a representation tree
  (relatively robust L D L^T representations, child shifts for clusters,
  twisted factorizations): the reference the device tree is tested against.

:mod:`oracle.brute` adds a 50-digit mpmath eigen-decomposition of H for
n <= 4, one of the pins that ties the oracle to something other than itself.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` except the eigenvector phase and the basis inside
a degenerate cluster, which are not unique (parity unpinned by nature; tests
compare phase-free quantities there).
"""
