"""Oracle: the even-odd (Schur complement) form of the coarsest-level CG solve.

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 3 solves the coarsest level by CG on the normal equations.  Every hop of the coarse
9-point stencil joins a site to a site of the other parity (x + y + z + t mod 2, all extents
even), so with the even sites ordered first

    A = [[A_ee, A_eo],
         [A_oe, A_oo]],   A_oo block diagonal (each odd site's own n x n block),

and A x = b is equivalent to

    S x_e = b_e - A_eo A_oo^-1 b_o,        S = A_ee - A_eo A_oo^-1 A_oe,
    x_o   = A_oo^-1 (b_o - A_oe x_e).

CG then runs on the normal equations of S (the CGLS form of solvers.cgnr).  The residual of
the full system at the reconstructed x is that of the Schur system at the even sites and
vanishes at the odd sites, so the stopping test |b - A x| <= tol |b| is |r_e| <= tol |b|.

Vectors here are whole-lattice arrays [T, Z, Y, X, n]; "even part" means the odd sites set to
zero.  S and S^dag are applied from the stencil and the per-site inverses written out
directly (no sigma_3 identity is used), so that the tests can hold them against dense
matrices.

Optionally (cgnr_eo_block_jacobi) the CG runs on the right block-Jacobi preconditioned
operator T = S M, M the inverse of S's diagonal blocks (one per even site), and x_e = M y at
the end; the stopping test is unchanged.

Pinned by tests/test_oracle_eo.py: S against the dense Schur complement formed from the
brute-force matrix of the stencil; S^dag against its conjugate transpose; the reconstructed
solution against a dense solve; the stopping test against the true full-system residual; S's
diagonal blocks against the dense Schur complement's (extent 2 included); the block-Jacobi CG's
solution against a dense solve.
"""
from __future__ import annotations

import numpy as np


def parity(dims):
    """(x + y + z + t) mod 2 as an array [T, Z, Y, X]; every extent must be even."""
    X, Y, Z, T = dims
    if any(L % 2 for L in dims):
        raise ValueError("even-odd split needs even extents")
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return (x + y + z + t) % 2


def odd_block_inverse(A):
    """A_oo^-1: the inverse of every site's own block (only the odd sites' are used)."""
    return np.linalg.inv(A.D[..., 0, :, :])


def _mask(v, keep):
    return v * keep[..., None]


def schur_apply(A, x, inv):
    """S x_e (even part of the result; odd sites zero)."""
    par = parity(A.dims)
    even, odd = par == 0, par == 1
    xe = _mask(x, even)
    t = _mask(A.apply(xe), odd)                     # A_oe x_e
    u = np.matmul(inv, t[..., None])[..., 0]        # A_oo^-1 A_oe x_e at odd sites
    u = _mask(u, odd)
    return _mask(A.apply(xe) - A.apply(u), even)    # A_ee x_e - A_eo u


def schur_apply_dagger(A, y, inv):
    """S^dag y_e = A_ee^dag y_e - A_oe^dag A_oo^-dag A_eo^dag y_e (even part)."""
    par = parity(A.dims)
    even, odd = par == 0, par == 1
    ye = _mask(y, even)
    t = _mask(A.apply_dagger(ye), odd)              # A_eo^dag y_e
    invh = np.conj(np.swapaxes(inv, -1, -2))
    u = _mask(np.matmul(invh, t[..., None])[..., 0], odd)
    return _mask(A.apply_dagger(ye) - A.apply_dagger(u), even)


def prepare(A, b, inv):
    """b_e - A_eo A_oo^-1 b_o (even part)."""
    par = parity(A.dims)
    even, odd = par == 0, par == 1
    u = _mask(np.matmul(inv, _mask(b, odd)[..., None])[..., 0], odd)
    return _mask(b, even) - _mask(A.apply(u), even)


def reconstruct(A, b, xe, inv):
    """The whole-lattice solution: x_e and x_o = A_oo^-1 (b_o - A_oe x_e)."""
    par = parity(A.dims)
    even, odd = par == 0, par == 1
    xe = _mask(xe, even)
    t = _mask(b - A.apply(xe), odd)                 # b_o - A_oe x_e
    xo = _mask(np.matmul(inv, t[..., None])[..., 0], odd)
    return xe + xo


def cgnr_eo(A, b, tol, maxit):
    """CG on the normal equations of the Schur complement; returns (x, iterations) with x the
    whole-lattice solution of A x = b and the stopping test |r_e| <= tol |b|."""
    inv = odd_block_inverse(A)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return np.zeros_like(b), 0
    x = np.zeros_like(b)
    r = prepare(A, b, inv)
    z = schur_apply_dagger(A, r, inv)
    p = z.copy()
    zz = np.vdot(z, z).real
    it = 0
    while it < maxit and float(np.linalg.norm(r)) > tol * bn:
        q = schur_apply(A, p, inv)
        alpha = zz / np.vdot(q, q).real
        x = x + alpha * p
        r = r - alpha * q
        z = schur_apply_dagger(A, r, inv)
        zz_new = np.vdot(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
        it += 1
    return reconstruct(A, b, x, inv), it


def schur_self_blocks(A, inv):
    """The diagonal blocks of S at every even site x: A_xx - sum over the two-hop paths
    x -> y -> x (y odd) of A_{x,y} A_yy^-1 A_{y,x}, read column by column from S applied to
    the unit vectors of one site of each parity class that S cannot mix (sites two hops apart
    in every direction are distinct only on extents >= 4, so the probe is site by site)."""
    par = parity(A.dims)
    T, Z, Y, X = par.shape
    n = A.n
    out = np.zeros((T, Z, Y, X, n, n), dtype=np.complex128)
    for t, z, y, x in zip(*np.nonzero(par == 0)):
        for j in range(n):
            e = np.zeros((T, Z, Y, X, n), dtype=np.complex128)
            e[t, z, y, x, j] = 1.0
            out[t, z, y, x, :, j] = schur_apply(A, e, inv)[t, z, y, x]
    return out


def cgnr_eo_block_jacobi(A, b, tol, maxit):
    """CG on the normal equations of the right block-Jacobi preconditioned Schur complement:
    T = S M with M = the inverse of S's diagonal blocks (per even site), T y = b^_e, x_e = M y;
    the same stopping test |b^_e - S x_e| <= tol |b| as cgnr_eo.  Returns (x, iterations)."""
    inv = odd_block_inverse(A)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return np.zeros_like(b), 0
    par = parity(A.dims)
    even = par == 0
    Mb = np.linalg.inv(np.where(even[..., None, None], schur_self_blocks(A, inv), np.eye(A.n)))
    Mbh = np.conj(np.swapaxes(Mb, -1, -2))

    def Mv(v):
        return _mask(np.matmul(Mb, v[..., None])[..., 0], even)

    def Mhv(v):
        return _mask(np.matmul(Mbh, v[..., None])[..., 0], even)

    y = np.zeros_like(b)
    r = prepare(A, b, inv)
    z = Mhv(schur_apply_dagger(A, r, inv))
    p = z.copy()
    zz = np.vdot(z, z).real
    it = 0
    while it < maxit and float(np.linalg.norm(r)) > tol * bn:
        q = schur_apply(A, Mv(p), inv)
        alpha = zz / np.vdot(q, q).real
        y = y + alpha * p
        r = r - alpha * q
        z = Mhv(schur_apply_dagger(A, r, inv))
        zz_new = np.vdot(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
        it += 1
    return reconstruct(A, b, Mv(y), inv), it
