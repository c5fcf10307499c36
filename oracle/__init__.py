"""CPU oracle for the hierarchical Poincare-Steklov (HPS) direct solver with body loads.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy restatement of the
method of Babb, Gillman, Hao and Martinsson, "An accelerated Poisson solver based on
multidomain spectral discretization" (arXiv 1612.02736).  Only the test suite, the
``smoke()`` entry of ``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The GPU library never calls it and shares no code
with it: every table (nodes, differentiation, interpolation), every index set and every
step is computed here independently.

Modules
-------
spectral   reference-element operators: Chebyshev-Lobatto grid, differentiation,
           Gauss-Legendre nodes, barycentric interpolation, L_ce,ge, L_loc, D_ge,c
           (Sec. 3.1-3.4).
leaf       the leaf matrix A and the leaf operators F, S, H, T (Sec. 3, Algorithm 1 leaf
           branch, Eqs. alpine1-alpine4).
tree       uniform box trees, leaf Gauss-node numbering and the merge index sets
           J1, J2, J3 (Sec. 2, Sec. 4, Sec. 5.1).
hps        Algorithm 1 (build), Algorithm 2 (solve, optionally with a flux-jump right
           hand side), the FP64 residual of the global collocation system, and the
           transposed (adjoint) sweeps with the coefficient gradients.
points     node coordinates (leaf Chebyshev nodes, boundary Gaussian nodes) for inputs.
dense      brute force: the global collocation system assembled densely and solved with
           numpy.linalg.solve (for tiny meshes).

Parity status
-------------
Every function is pinned by ``tests/test_oracle_*.py`` against closed forms, brute force or
invariants (polynomial exactness, the dense global solve, DtN identities, flux continuity,
the dot-product identity of the adjoint, heat-equation eigenmodes).  No function here is
"parity unpinned".
"""
