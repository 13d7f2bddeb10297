"""Seeded synthetic inputs shared by the CPU oracle, the GPU tests and the benchmark.

This module holds input generation only: random SU(3) gauge fields, Gaussian and
point-source right-hand sides, Gaussian starting vectors for the adaptive setup and
random local gauge transformations.  None of the solver's arithmetic lives here.

Conventions (shared by every consumer):

* A lattice has extents ``dims = (X, Y, Z, T)``; direction mu = 0, 1, 2, 3 is
  x, y, z, t.  Arrays are stored with t slowest: a fine field has shape
  ``(T, Z, Y, X, ...)`` and the lexicographic site index is
  ``x + X*(y + Y*(z + Z*t))``.
* A gauge field has shape ``(T, Z, Y, X, 4, 3, 3)`` complex128: ``U[t,z,y,x,mu]`` is
  the 3x3 link U_mu(x) leaving site x in direction +mu.
* A fine spinor has shape ``(T, Z, Y, X, 12)`` complex128 with component index
  ``spin*3 + colour``.

Random fields follow the recipe of the workloads: for every link, a 3x3 matrix A
with independent N(0,1) real and imaginary parts (numpy PCG64, drawn in
[t][z][y][x][mu] order), H = (A + A^dag)/2 - tr(.)/3, U = exp(i eps H) by
eigendecomposition, then re-unitarised to SU(3) (normalise row 0, Gram-Schmidt
row 1 against row 0, row 2 = conj(row0 x row1)).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gauge_field",
    "unit_gauge",
    "gaussian_spinors",
    "point_sources",
    "setup_starts",
    "coarse_starts",
    "random_su3_field",
    "lex_shape",
]


def lex_shape(dims):
    """(X, Y, Z, T) -> numpy shape (T, Z, Y, X)."""
    X, Y, Z, T = dims
    return (T, Z, Y, X)


def _reunitarise(M):
    """Project a batch of near-unitary 3x3 matrices onto SU(3) (rows 0, 1 kept, row 2 rebuilt)."""
    r0 = M[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = M[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _su3_exp(A, eps):
    """exp(i eps H) with H the traceless Hermitian part of A, re-unitarised."""
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1)
    H = H - (tr / 3.0)[..., None, None] * np.eye(3)
    w, Q = np.linalg.eigh(H)
    U = (Q * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(Q, -1, -2))
    return _reunitarise(U)


def gauge_field(dims, eps, seed, chunk_sites=1 << 18):
    """Random SU(3) gauge field U_mu(x) = exp(i eps H_mu(x)), shape (T,Z,Y,X,4,3,3).

    Generated in chunks of sites so that large lattices stay within host memory;
    the random stream is consumed in the same [t][z][y][x][mu] order regardless of
    the chunk size.
    """
    shape = lex_shape(dims)
    V = int(np.prod(shape))
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for s0 in range(0, V, chunk_sites):
        n = min(chunk_sites, V - s0)
        g = rng.standard_normal(size=(n, 4, 3, 3, 2))
        A = g[..., 0] + 1j * g[..., 1]
        out[s0:s0 + n] = _su3_exp(A, eps)
    return out.reshape(shape + (4, 3, 3))


def evolved_gauge(U, eps, seed):
    """A small step of the gauge field, as in a molecular-dynamics update: every link multiplied
    from the left by exp(i eps H) with H the traceless Hermitian part of seeded Gaussian entries
    (drawn in the [t][z][y][x][mu] order), re-unitarised."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(size=U.shape + (2,))
    R = _su3_exp(g[..., 0] + 1j * g[..., 1], eps)
    return _reunitarise(R @ U)


def unit_gauge(dims):
    """The free field U_mu(x) = 1."""
    shape = lex_shape(dims)
    U = np.zeros(shape + (4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def random_su3_field(dims, seed):
    """One random SU(3) matrix per site (a local gauge transformation), shape (T,Z,Y,X,3,3)."""
    shape = lex_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(size=shape + (3, 3, 2))
    A = g[..., 0] + 1j * g[..., 1]
    return _su3_exp(A, 1.0)


def gaussian_spinors(dims, nrhs, seed):
    """nrhs Gaussian fine spinors (re, im ~ N(0,1) iid), shape (nrhs, T,Z,Y,X,12)."""
    shape = lex_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(size=(nrhs,) + shape + (12, 2))
    return g[..., 0] + 1j * g[..., 1]


def point_sources(dims, nrhs=12, site=(0, 0, 0, 0)):
    """Point sources at one site: rhs k is the unit vector on component k (spin*3+colour)."""
    shape = lex_shape(dims)
    b = np.zeros((nrhs,) + shape + (12,), dtype=np.complex128)
    x, y, z, t = site
    for k in range(nrhs):
        b[k, t, z, y, x, k % 12] = 1.0
    return b


def setup_starts(dims, nvec, seed):
    """Gaussian random starting vectors for the adaptive setup, shape (nvec, T,Z,Y,X,12)."""
    return gaussian_spinors(dims, nvec, seed)


def coarse_starts(cdims, ndof, nvec, seed):
    """Gaussian starting vectors on a coarse lattice with ndof complex dof per site,
    shape (nvec, T,Z,Y,X, ndof)."""
    shape = lex_shape(cdims)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(size=(nvec,) + shape + (ndof, 2))
    return g[..., 0] + 1j * g[..., 1]
