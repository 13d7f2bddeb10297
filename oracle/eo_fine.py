"""Oracle: the even-odd (red/black) form of the fine Wilson solve (Sec. 3, the red/black
preconditioning combined with multigrid).

TEST INFRASTRUCTURE ONLY (see the package header).

With D = d + H, d = 4 + m and H the hopping term of Sec. 2's operator (every hop joins sites of
opposite parity (x + y + z + t) mod 2), the even-odd blocks are D_ee = D_oo = d and D_eo, D_oe
the restrictions of H.  The Schur complement on the even sites is

    S = d - H_eo H_oe / d,

the even-site system S x_e = b_e - H_eo b_o / d, and the odd sites follow from
x_o = (b_o - H_oe x_e) / d.  The residual of the whole system then vanishes on the odd sites and
equals b^_e - S x_e on the even ones.  Since S^-1 is the even-even block of D^-1, the multigrid
cycle K of the whole lattice preconditions S as r_e -> [K(r_e, 0)]_e.

Fields keep the whole-lattice shape (T, Z, Y, X, 12) with zero odd sites.

Pins (tests/test_oracle_eo.py): S and the prepared right-hand side against the blocks of the
brute-force dense D (dense_D) and a dense Schur complement; the reconstructed solution against a
dense solve; S^dag = gamma_5 S gamma_5; the MG-GCR solve of S preconditioned by the cycle against
the dense solution.
"""
from __future__ import annotations

import numpy as np

from . import dirac, solvers


def parity(dims):
    X, Y, Z, T = dims
    if X % 2:
        raise ValueError("the even-odd split needs an even x extent")
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return (x + y + z + t) % 2


def _keep(v, mask):
    return v * mask[..., None]


def hopping(U, psi, m):
    """H psi = D psi - (4 + m) psi (the eight hop terms with the -1/2)."""
    return dirac.apply_D(U, psi, m) - (4.0 + m) * psi


def schur_apply(U, xe, m):
    """S x_e = d x_e - H_eo H_oe x_e / d on the even sites."""
    d = 4.0 + m
    par = parity(dirac_dims(U))
    even, odd = par == 0, par == 1
    xe = _keep(xe, even)
    t = _keep(hopping(U, xe, m), odd)
    return _keep(d * xe - hopping(U, t, m) / d, even)


def prepare(U, b, m):
    """b^_e = b_e - H_eo b_o / d."""
    d = 4.0 + m
    par = parity(dirac_dims(U))
    even, odd = par == 0, par == 1
    return _keep(b - hopping(U, _keep(b, odd), m) / d, even)


def reconstruct(U, b, xe, m):
    """The whole-lattice solution: x_e and x_o = (b_o - H_oe x_e) / d."""
    d = 4.0 + m
    par = parity(dirac_dims(U))
    even, odd = par == 0, par == 1
    xe = _keep(xe, even)
    return xe + _keep((b - hopping(U, xe, m)) / d, odd)


def dirac_dims(U):
    T, Z, Y, X = U.shape[:4]
    return (X, Y, Z, T)


def mg_solve_eo(H, b, tol=1e-10, restart=16, max_iter=1000):
    """MG-GCR on the even-odd system: flexible GCR on S x_e = b^_e with the whole-lattice cycle
    as preconditioner (r_e -> even part of K(r_e)), stopped when |b^_e - S x_e| <= tol |b| (the
    whole system's residual); returns the whole-lattice x and the GCR info."""
    op = H.ops[0]
    U, m = op.U, op.m
    par = parity(dirac_dims(U))
    even = par == 0
    be = prepare(U, b, m)
    bn = float(np.linalg.norm(b))
    scale = bn / max(float(np.linalg.norm(be)), 1e-300)
    xe, info = solvers.fgcr(lambda v: schur_apply(U, v, m),
                            lambda r: _keep(solvers.cycle(H, 0, _keep(r, even)), even),
                            be, tol * scale, restart, max_iter)
    return reconstruct(U, b, xe, m), info
