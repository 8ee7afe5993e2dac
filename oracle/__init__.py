"""CPU oracle for the Total-Lagrangian force / tangent / Hessian path (T10
elements, and the ANCF3243 beam and ANCF3443 shell elements in ancf.py).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the paper's hot path computes (Sec. 2 residual and augmented cost,
Sec. 4.1 precomputation, Sec. 4.2 sparsity, Sec. 4.3 internal force, Sec. 4.4
gradient and Hessian, Algorithm 3 Newton step).  Only the test-suite, the
smoke check and the benchmark's CPU-baseline leg may import it.  The CUDA path
(the package next to this one) never imports it, and this package never
imports the CUDA path: the two share no code.

Every function cites the passage of the paper it follows.  Where the paper is
silent (T10 node order, Keast point values, constitutive forms that live in
the companion Part I, the Kelvin-Voigt tangent) the reading taken is stated in
the docstring and listed in the project design notes.

Floating point: float64 throughout; every routine also accepts complex128
arrays so the tangents can be pinned against complex-step derivatives.
"""
