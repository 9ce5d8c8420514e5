"""FP64 CPU oracle for the reactive-blob reaction-diffusion solve.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain definition of what the
GPU library computes, written from the paper (Bhalla, Griffith, Patankar, Donev,
"A Minimally-Resolved Immersed Boundary Model for Reaction-Diffusion Problems").
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import it. The CUDA library never imports, links or calls it, and it shares
no code with the CUDA library.

Contents (every function cites the passage it follows):

* ``kernels``    -- Peskin 3- and 4-point kernels (Sec. III.A, moment conditions
                    Eq. JS_invariance; the formulas are Peskin's, cited there).
* ``operators``  -- 7-point periodic Helmholtz operator A = alpha I - chi L
                    (Sec. III.A, Eq. Helmholtz), averaging J and spreading
                    S = h^-3 J^T (Sec. III.A, Eq. tensor_product), FFT Green's
                    function of A (pseudo-inverse on mean-zero fields when
                    alpha = 0, Appendix A).
* ``direct``     -- exact solutions of the reaction-limited system
                    (Eqs. unsteady_system / steady_state) and the saddle point
                    (Eq. saddle_point) by Schur elimination (Eqs. c_exact,
                    r_schur, plus the solvability condition of Appendix A), and
                    brute-force dense solves for tiny grids.
* ``multigrid``  -- the V-cycle definition the GPU library implements
                    (Sec. III.E: geometric multigrid on the Helmholtz problem);
                    the paper delegates the smoother, transfers and coarse solve
                    to a library, so the choices here are readings (red-black
                    Gauss-Seidel, 8-cell average restriction, trilinear
                    cell-centred prolongation, exact coarsest solve).
* ``outputs``    -- mean concentration, overall rate K, reaction radius a_L,
                    beta_0 (Sec. I.A, Sec. IV.A, Eqs. beta_P_disc, a_phi).
* ``cpu_solver`` -- the paper's iterative method (FGMRES with modified
                    Gram-Schmidt, multigrid V-cycles, Appendix A) written
                    plainly in C + OpenMP (``cpu_solver.c``): the CPU baseline
                    that solves the full benchmark workload on the host cores.
                    Loaded on demand (it needs gcc), not by this package.

Parity status: every function above is pinned by tests in ``tests/`` against
closed forms, exact invariants, brute-force dense solves or printed constants.
"""
from . import kernels, operators, direct, multigrid, outputs  # noqa: F401
