"""FP64 CPU oracle for the Dual Natural Gradient Descent (D-NGD) step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, calls or links anything from this package.  Only
the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.

The oracle is a plain, slow, obviously-correct NumPy float64 restatement of
what the paper computes (Jnini & Vella, "Dual Natural Gradient Descent for
Scalable Training of Physics-Informed Neural Networks", TMLR 2025):

* ``mlp``       - flat parameter layout of the tanh MLP ansatz (Sec. 2.1).
* ``series``    - truncated bivariate Taylor series (the Taylor-mode AD of
                  Sec. 5, used for the spatial jets and the second directional
                  derivative f_vv of Sec. 3.2).
* ``residual``  - PINN residual map r(theta) with per-class 1/sqrt(N) scaling
                  (Sec. 2.2) and its Jacobian J by per-point reverse mode.
* ``step``      - damped Gauss-Newton step in residual space (Thm. 3.1,
                  Def. 3.1), textbook Cholesky, geodesic acceleration
                  (Def. 3.2, Prop. 3.2) and the acceptance rule of the
                  DenseDualSolve algorithm (App. A.2).
* ``nystrom``   - Nystrom construction of (U, Lambda_hat), the spectral
                  preconditioner (Eq. spec_precond_nystrom, Sec. 3.3.1) and
                  PCG (Alg. PCGStep, App. A.2).
* ``linesearch``- grid line search of the D-NGD workflow (Alg. D-NGD Workflow).
* ``evaluate``  - relative L2 error of u_theta against the manufactured
                  solution on a midpoint grid (the error columns of Sec. 5).

Every function cites the passage it follows.  The oracle shares no code with
the CUDA path; inputs come from the seeded generators in
``paper_2505_21404_gb300.workloads`` (which contain none of the method's
arithmetic) and are passed in as arrays.
"""
