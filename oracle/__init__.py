"""CPU oracle for the stress-velocity Newton (svN) implicit sea-ice step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference arms of ``bench.py`` may import this package.
The CUDA path never calls it and shares no code with it: the two meet only
in the seeded input generators of ``workloads``.

Everything is plain FP64 NumPy/SciPy, written from the paper
(arXiv:2204.10822, "A stress-velocity Newton method for viscous-plastic
sea ice"):

  * ``fem``     -- Q1 discretisation, tau(v), Delta(v), the energy Phi
                   (Eq. "energy"), the residual (Eqs. "Av=F", "A", "F",
                   "sigma"), the standard Newton Jacobian
                   (Eqs. "standardNewton1/2"), the svN Jacobian
                   (Eq. "linearSVNewton" with Eq. "modification") and the
                   dual step (Eq. "tautilde" with Eq. "modification").
  * ``newton``  -- damped Newton (svN / stdN) with a backtracking line search
                   on Phi (Section 5.1) and sparse direct linear solves.
  * ``mg``      -- the pieces of the multigrid-preconditioned FGMRES used by
                   the fast path (Section 5.4): bilinear prolongation,
                   Galerkin coarse operators, block-Jacobi Chebyshev
                   smoothing, dense coarse solve, V-cycle and FGMRES, each in
                   its textbook form.
  * ``transport`` -- explicit first-order upwind finite-volume transport of
                   the cell fields A and H (Eqs. "model:A", "model:H",
                   Sections 3 and 5.1), sub-cycled for the Courant number.
  * ``unet``    -- forward/backward of the small convolutional network that
                   predicts the Newton initial guess (no counterpart in the
                   paper), in plain PyTorch CPU ops.

Parity pins are in ``tests/test_oracle_*.py``.  Functions without an
independent pin say "parity unpinned" in their docstring.
"""
