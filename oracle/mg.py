"""Oracle: prolongator, restriction and Galerkin coarse operator (Secs. 2 and 3).

TEST INFRASTRUCTURE ONLY (see the package header).

Fields on any level have shape (T, Z, Y, X, n): n = 12 complex dof per site on the
fine lattice (spin*3 + colour) and n = 2N on a coarse lattice built from N near-null
vectors.  On every level the first n/2 dof have chirality +1 (gamma_5 = +1 on the
fine lattice, sigma_3 = +1 on a coarse one) and the last n/2 chirality -1.

* Blocking: the coarse site of x is x_hat = floor(x_mu / b_mu) (Sec. 3: 4^4 blocks on
  the fine lattice).
* Block orthonormalisation (Sec. 2, the equation defining P; chirality split of
  Sec. 3): for each block and chirality s, the N vectors theta_xhat(x) psi^(alpha)_x
  restricted to the s-half of the dof are orthonormalised in the order alpha = 0..N-1
  by modified Gram-Schmidt with one full second pass.  A column whose norm falls
  below 1e-10 of its norm before projection is a rank deficiency (error).
* Coarse dof index: c = s*N + alpha (chirality + first); coarse sites lexicographic.
* Restriction (R = P^dag, Sec. 2):
    phi(xhat, s*N+alpha) = sum_{x in xhat} sum_{d in s} conj(P_alpha(x, d)) psi(x, d)
  Prolongation: psi(x, d) = sum_alpha P_alpha(x, d) phi(xhat(x), s(d)*N + alpha).
* Galerkin operator D^ = P^dag D P (Sec. 2) stored as a 9-point stencil
  D^[xhat, k] (k = 0 self, k = 1 + 2*mu + (0 for +mu, 1 for -mu)), each an n x n
  block:  (D^ phi)(xhat) = sum_k D^[xhat, k] phi(xhat + k).  A hopping term of the
  operator that reads a neighbour in the same block goes to the self slot; one that
  reads a neighbour in another block goes to the slot of its hop direction (so on a
  coarse extent of 2 the +mu and -mu slots stay separate).

Pins (tests/test_oracle_mg.py): P^dag P = I; P P^dag v = v for every setup vector;
sigma_3 P = P gamma_5 (zero cross-chirality blocks); adjointness of restrict and
prolong; the piecewise-constant Laplace prolongator theta/2^d of Sec. 2 for one
constant scalar vector on 4^d blocks; D^ equal to dense P^dag D P on tiny lattices
(D from the loop-built dense matrix, P as an explicit matrix); sigma_3 D^ sigma_3 =
D^dag; the mass shift D^(m) = D^(m0) + (m - m0) I; gauge invariance of D^; the
Petrov-Galerkin projector identities of Sec. 2.
"""
from __future__ import annotations

import numpy as np

from . import cref
from .dirac import AXIS, apply_D, hop as wilson_hop

NSLOT = 9


def slot(mu, sign):
    """Stencil slot of the hop that reads the neighbour xhat + sign*mu."""
    return 1 + 2 * mu + (0 if sign > 0 else 1)


def coarse_dims(dims, block):
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError(f"block {block} does not divide lattice {dims}")
    return tuple(L // b for L, b in zip(dims, block))


def to_blocks(field, block):
    """(T,Z,Y,X,n) -> (Vc, bs, n): coarse site (lexicographic) x site-in-block x dof."""
    T, Z, Y, X, n = field.shape
    bx, by, bz, bt = block
    f = field.reshape(T // bt, bt, Z // bz, bz, Y // by, by, X // bx, bx, n)
    f = f.transpose(0, 2, 4, 6, 1, 3, 5, 7, 8)
    return f.reshape((T // bt) * (Z // bz) * (Y // by) * (X // bx), bt * bz * by * bx, n)


def from_blocks(fb, dims, block):
    """Inverse of to_blocks."""
    X, Y, Z, T = dims
    bx, by, bz, bt = block
    n = fb.shape[-1]
    f = fb.reshape(T // bt, Z // bz, Y // by, X // bx, bt, bz, by, bx, n)
    f = f.transpose(0, 4, 1, 5, 2, 6, 3, 7, 8)
    return f.reshape(T, Z, Y, X, n)


def field_dims(field):
    T, Z, Y, X = field.shape[:4]
    return (X, Y, Z, T)


class RankDeficient(ValueError):
    pass


def block_orthonormalise(vectors, block, rank_tol=1e-10):
    """Orthonormal basis of {theta_xhat(x) psi^(alpha)_x} per block and chirality.

    vectors: (N, T, Z, Y, X, n).  Returns P of the same shape: P[alpha] holds, in
    block xhat and chirality s, the alpha-th orthonormal basis vector of that
    (block, s) sub-space.
    """
    N = vectors.shape[0]
    n = vectors.shape[-1]
    h = n // 2
    dims = field_dims(vectors[0])
    blocks = np.stack([to_blocks(v, block) for v in vectors])  # (N, Vc, bs, n)
    Vc, bs = blocks.shape[1], blocks.shape[2]
    out = np.zeros_like(blocks)
    for s in range(2):
        # columns: (Vc, L, N), L = bs * h
        cols = blocks[:, :, :, s * h:(s + 1) * h].reshape(N, Vc, bs * h).transpose(1, 2, 0).copy()
        for k in range(N):
            v = cols[:, :, k]
            before = np.linalg.norm(v, axis=1)
            for _ in range(2):  # modified Gram-Schmidt, applied twice
                for j in range(k):
                    q = cols[:, :, j]
                    beta = np.sum(np.conj(q) * v, axis=1)
                    v = v - beta[:, None] * q
            after = np.linalg.norm(v, axis=1)
            if np.any(after <= rank_tol * before):
                raise RankDeficient(f"vector {k} is (numerically) in the span of the previous ones")
            cols[:, :, k] = v / after[:, None]
        out[:, :, :, s * h:(s + 1) * h] = cols.transpose(2, 0, 1).reshape(N, Vc, bs, h)
    return np.stack([from_blocks(out[a], dims, block) for a in range(N)])


_BLOCKED = {}


def _blocked(P, block):
    """Per chirality s, the block-restricted columns of P as a (Vc, N, bs*n/2) array
    (cached per array; the cache keeps P alive)."""
    key = (id(P), tuple(block))
    hit = _BLOCKED.get(key)
    if hit is not None and hit[0] is P:
        return hit[1]
    if len(_BLOCKED) > 8:
        _BLOCKED.clear()
    N, n = P.shape[0], P.shape[-1]
    h = n // 2
    Pb = np.stack([to_blocks(p, block) for p in P])  # (N, Vc, bs, n)
    halves = [np.ascontiguousarray(Pb[:, :, :, s * h:(s + 1) * h].reshape(N, Pb.shape[1], -1).transpose(1, 0, 2))
              for s in range(2)]
    _BLOCKED[key] = (P, halves)
    return halves


def restrict(P, psi, block):
    """phi = P^dag psi: (T,Z,Y,X,n) fine -> (Tc,Zc,Yc,Xc,2N) coarse.
    phi(xhat, s*N + alpha) = sum_{x in xhat, d in s} conj(P_alpha(x, d)) psi(x, d)."""
    N = P.shape[0]
    n = psi.shape[-1]
    h = n // 2
    dims = field_dims(psi)
    cd = coarse_dims(dims, block)
    halves = _blocked(P, block)            # [s] -> (Vc, N, bs*h)
    fb = to_blocks(psi, block)             # (Vc, bs, n)
    phi = np.zeros((fb.shape[0], 2 * N), dtype=np.complex128)
    for s in range(2):
        f = fb[:, :, s * h:(s + 1) * h].reshape(fb.shape[0], -1, 1)
        # conj(P)^T f written as conj(P^T conj(f)): the same products and sums, without a
        # conjugated copy of P
        phi[:, s * N:(s + 1) * N] = np.conj(np.matmul(halves[s], np.conj(f)))[..., 0]
    X, Y, Z, T = cd
    return phi.reshape(T, Z, Y, X, 2 * N)


def prolong(P, phi, block):
    """psi = P phi: coarse (Tc,Zc,Yc,Xc,2N) -> fine (T,Z,Y,X,n).
    psi(x, d) = sum_alpha P_alpha(x, d) phi(xhat(x), s(d)*N + alpha)."""
    N = P.shape[0]
    n = P.shape[-1]
    h = n // 2
    dims = field_dims(P[0])
    halves = _blocked(P, block)            # [s] -> (Vc, N, bs*h)
    ph = phi.reshape(-1, 2 * N)
    Vc = ph.shape[0]
    bs = halves[0].shape[2] // h
    fb = np.zeros((Vc, bs, n), dtype=np.complex128)
    for s in range(2):
        v = np.matmul(ph[:, None, s * N:(s + 1) * N], halves[s])[:, 0, :]   # (Vc, bs*h)
        fb[:, :, s * h:(s + 1) * h] = v.reshape(Vc, bs, h)
    return from_blocks(fb, dims, block)


class WilsonOp:
    """The fine operator D(U) with mass m as diagonal plus eight hopping terms."""

    def __init__(self, U, m):
        self.U = U
        self.m = float(m)
        T, Z, Y, X = U.shape[:4]
        self.dims = (X, Y, Z, T)
        self.n = 12

    def diag(self, psi):
        return (4.0 + self.m) * psi

    def hop(self, psi, mu, sign):
        if psi.shape[0] * psi.shape[1] * psi.shape[2] * psi.shape[3] >= 4096:
            return cref.hop(self.U, psi, mu, sign)      # plain C restatement, same arithmetic
        return wilson_hop(self.U, psi, mu, sign)

    def apply(self, psi):
        if psi.shape[0] * psi.shape[1] * psi.shape[2] * psi.shape[3] >= 4096:
            return cref.apply_D(self.U, psi, self.m)
        return apply_D(self.U, psi, self.m)

    def gamma5(self, psi):
        out = psi.copy()
        out[..., 6:] *= -1.0
        return out

    def apply_dagger(self, psi):
        return self.gamma5(self.apply(self.gamma5(psi)))


class StencilOp:
    """A coarse 9-point stencil operator: D[T,Z,Y,X, 9, n, n]."""

    def __init__(self, D):
        self.D = D
        T, Z, Y, X = D.shape[:4]
        self.dims = (X, Y, Z, T)
        self.n = D.shape[-1]

    def diag(self, phi):
        return np.matmul(self.D[..., 0, :, :], phi[..., None])[..., 0]

    def hop(self, phi, mu, sign):
        nb = np.roll(phi, -sign, axis=AXIS[mu])  # phi(xhat + sign*mu)
        return np.matmul(self.D[..., slot(mu, sign), :, :], nb[..., None])[..., 0]

    def apply(self, phi):
        out = self.diag(phi)
        for mu in range(4):
            for sign in (+1, -1):
                out = out + self.hop(phi, mu, sign)
        return out

    def apply_dagger(self, phi):
        """Explicit adjoint: (A^dag phi)(y) = sum_k D[y - k, k]^dag phi(y - k)."""
        Dh = np.conj(np.swapaxes(self.D, -1, -2))
        out = np.matmul(Dh[..., 0, :, :], phi[..., None])[..., 0]
        for mu in range(4):
            for sign in (+1, -1):
                ax = AXIS[mu]
                # term from site y - sign*mu whose slot (mu, sign) points at y
                Dk = np.roll(Dh[..., slot(mu, sign), :, :], sign, axis=ax)
                ph = np.roll(phi, sign, axis=ax)
                out = out + np.matmul(Dk, ph[..., None])[..., 0]
        return out

    def sigma3(self, phi):
        out = phi.copy()
        out[..., self.n // 2:] *= -1.0
        return out

    def shifted(self, dm):
        """D^ + dm * I."""
        D = self.D.copy()
        D[..., 0, :, :] += dm * np.eye(self.n)
        return StencilOp(D)

    def dense(self):
        """Dense matrix of the stencil (tiny lattices only)."""
        X, Y, Z, T = self.dims
        V = X * Y * Z * T
        n = self.n
        A = np.zeros((n * V, n * V), dtype=np.complex128)
        Df = self.D.reshape(V, NSLOT, n, n)
        ext = (X, Y, Z, T)
        for i in range(V):
            c = [i % X, (i // X) % Y, (i // (X * Y)) % Z, i // (X * Y * Z)]
            A[n * i:n * i + n, n * i:n * i + n] += Df[i, 0]
            for mu in range(4):
                for sign in (+1, -1):
                    f = list(c)
                    f[mu] = (f[mu] + sign) % ext[mu]
                    j = f[0] + X * (f[1] + Y * (f[2] + Z * f[3]))
                    A[n * i:n * i + n, n * j:n * j + n] += Df[i, slot(mu, sign)]
        return A


def same_block_mask(dims, block, mu, sign):
    """Boolean (T,Z,Y,X): True where the neighbour x + sign*mu lies in the block of x."""
    L = dims[mu]
    b = block[mu]
    x = np.arange(L)
    same = (x // b) == (((x + sign) % L) // b)
    shape = [1, 1, 1, 1]
    shape[AXIS[mu]] = L
    X, Y, Z, T = dims
    return np.broadcast_to(same.reshape(shape), (T, Z, Y, X))


def galerkin(op, P, block):
    """D^ = P^dag op P as a 9-point stencil (Sec. 2 Galerkin form, R = P^dag).

    For every coarse column c = (s, alpha), the global vector g_c holds the c-th basis
    vector in every block; each hopping term of op applied to g_c is restricted into
    the self slot (neighbour in the same block) or into the slot of its direction.
    """
    N = P.shape[0]
    n = P.shape[-1]
    h = n // 2
    dims = op.dims
    cd = coarse_dims(dims, block)
    X, Y, Z, T = cd
    D = np.zeros((T, Z, Y, X, NSLOT, 2 * N, 2 * N), dtype=np.complex128)
    masks = {(mu, sg): same_block_mask(dims, block, mu, sg)[..., None]
             for mu in range(4) for sg in (+1, -1)}
    for s in range(2):
        for a in range(N):
            c = s * N + a
            g = np.zeros_like(P[a])
            g[..., s * h:(s + 1) * h] = P[a][..., s * h:(s + 1) * h]
            self_term = op.diag(g)
            for mu in range(4):
                for sg in (+1, -1):
                    t = op.hop(g, mu, sg)
                    m = masks[(mu, sg)]
                    self_term = self_term + np.where(m, t, 0)
                    D[..., slot(mu, sg), :, c] = restrict(P, np.where(m, 0, t), block)
            D[..., 0, :, c] = restrict(P, self_term, block)
    return StencilOp(D)


def dense_prolongator(P, block):
    """P as an explicit (n V) x (2N Vc) matrix, built column by column from prolong()."""
    N = P.shape[0]
    dims = field_dims(P[0])
    cd = coarse_dims(dims, block)
    X, Y, Z, T = cd
    Vc = X * Y * Z * T
    cols = []
    for j in range(2 * N * Vc):
        e = np.zeros(2 * N * Vc, dtype=np.complex128)
        e[j] = 1.0
        cols.append(prolong(P, e.reshape(T, Z, Y, X, 2 * N), block).ravel())
    return np.stack(cols, axis=1)
