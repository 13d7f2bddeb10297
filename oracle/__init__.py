"""FP64 CPU oracle for the adaptive-multigrid Wilson-Dirac solve (arXiv:0912.2186).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do.  It shares no code with the CUDA path.

It is a plain, slow, obviously-correct restatement in numpy (complex128) of what the
paper computes:

* ``dirac``   -- the Wilson-Dirac operator D(U) of Sec. 2 (the equation for D_xy), the
                 gamma matrices, the free-field closed form, a dense loop-built D.
* ``mg``      -- blocking, block orthonormalisation of the near-null vectors (Sec. 2,
                 the equation defining P), chirality split sigma_3 P = P gamma_5 (Sec. 3),
                 restriction P^dag, prolongation P, the Galerkin coarse operator
                 D^ = P^dag D P (Sec. 2) as a 9-point stencil, its application.
* ``solvers`` -- MR smoother, CGNR coarsest solve, the multigrid cycle with post
                 smoothing only, flexible GCR outer solver (Sec. 3) and the adaptive
                 near-null-vector setup (Sec. 2).
* ``eo_fine`` -- the even-odd (red/black) form of the fine solve of Sec. 3: the Schur complement
                 S = d - H_eo H_oe / d, the prepared right-hand side, the odd-site reconstruction
                 and MG-GCR on S with the whole-lattice cycle as preconditioner.
* ``eo``      -- the even-odd (Schur complement) form of the coarsest-level CG solve:
                 S = A_ee - A_eo A_oo^-1 A_oe, its adjoint, the prepared right-hand side
                 and the reconstruction of the odd sites.

Parity status per function is stated in each module header.  Near-null vectors have
no closed form, so the adaptive setup (``solvers.setup_level``) is pinned as an
algorithm: against a dense restatement of its steps made of library routines on a tiny
lattice, plus the indirect invariants (residual decrease, span, orthonormality).
"""
from . import dirac, eo, eo_fine, mg, solvers  # noqa: F401
