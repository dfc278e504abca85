"""Plain FP64 CPU oracle for the coarse<->fine AMR transfer of
"Fast Higher-Order Interpolation and Restriction in ExaHyPE Avoiding
Non-physical Reflections" (arXiv 2504.15814).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The CUDA product path never calls this package, and this package imports
nothing from the product package.

The oracle works in physical (face-frame) coordinates, one output volume at a
time, following the paper's steps:

* Sec. 3 (operator construction): per fine ghost volume, the nearest coarse
  volume c; derivatives at c from polynomial fits through neighbouring coarse
  centres (here: tensor finite-difference stencils, exact Lagrange derivative
  weights on centred, inward-clamped windows); Taylor's formula about c.
  Restriction: per coarse halo volume, the nearest fine volume and Taylor about
  it on the fine grid (injection where centres coincide, extrapolation
  otherwise).
* Sec. 2 (problem statement): the d-linear tensor-product interpolation and
  averaging restriction P = Px Py Pz, and the same operator assembled into one
  sparse matrix.

Modules
-------
stencils   exact rational 1-D Lagrange derivative weights and window rule
geometry   face-array layout and physical cell centres
operators  operator rows (Taylor-m, d-linear), assembled per item class
transfer   applies the operators to whole buffers (forward and adjoint)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms (textbook finite-difference weights, exact reproduction of
polynomials of the scheme's degree, measured convergence order, row sums,
injection rows, the d-linear tensor-product identity).  The paper prints no
worked numerical example, so no function is pinned to a value printed in the
paper.
"""
