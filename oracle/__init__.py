"""FP64 CPU oracle of the paper's discretisation, time integration and misfit.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: it is imported by ``tests/``, by ``__graft_entry__.smoke()`` (to
check one small GPU run) and by ``bench.py``'s CPU-baseline leg, and nowhere
else.  It shares no code with the CUDA path (``paper_2404_17754_gb300``):
the only common module is ``synth`` (seeded input generation, no method
arithmetic).

The oracle is deliberately plain and slow: element matrices are formed
explicitly (stiffness by Gauss quadrature of B^T D B, mass by exact
integration of barycentric monomials), assembled into scipy CSR matrices,
and each Newmark step is solved by a textbook block-Jacobi preconditioned
conjugate gradient in numpy float64.

Modules
-------
fem        element and face matrices, Rayleigh fit, assembly, receivers
newmark    Newmark average-acceleration stepping, block-Jacobi PCG, analysis
misfit     shifted-Green's-function superposition, normal equations,
           truncated eigen pseudo-inverse, ERR, model selection
transfer1d closed-form 1D layered transfer function (used to pin the oracle)
mlp        learned initial guess: features, network, BF16 forward and gradient,
           Adam, extrapolated base guesses, training targets, node sampling
twolevel   first-order (vertex) coarse level of the inner solve: prolongation,
           P^T A P, coarse block Jacobi, the additive two-level preconditioner

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, invariants or brute force (see ``tests/test_oracle_*.py``),
except the paper's printed ERR values, which need data the paper does not
publish (parity unpinned for those numbers only).
"""
