"""CPU oracle for the matrix-free Riemannian circuit optimiser (test infrastructure).

This package is test infrastructure, not part of the product path.  Only the
test-suite, the smoke check of ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library: it uses
only numpy/scipy and the seeded input generators of ``workloads``.

Everything is complex128 / float64.

* ``model``        Jordan-Wigner Fermi-Hubbard Hamiltonian (dense, and per
                   particle-number sector) and the target ``U = exp(-iHt)``.
* ``dense``        O1: the plain definitions with dense 2^n x 2^n matrices
                   (circuit matrix, cost, first and second derivatives).
* ``statevector``  O2: the paper's matrix-free algorithm (forward pass with
                   caching, backward pass with gate holes, forward-mode +
                   reverse Hessian-vector products) over basis columns.
* ``riemann``      tangent projection, gradient convention, Riemannian
                   Hessian written from its definition, polar retraction,
                   tied-gate sums and the parity pattern.
* ``trust_region`` Riemannian trust region with truncated CG.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force or an independent dense route (see the docstrings).
"""
