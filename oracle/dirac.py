"""Oracle: the Wilson-Dirac operator of Sec. 2 (the equation for D_xy(U)).

TEST INFRASTRUCTURE ONLY (see the package header).

Reading of the paper (it prints the index placement in a form that is not gauge
covariant, and fixes neither the gamma basis nor boundary conditions):

  (D psi)(x) = (4 + m) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x)         psi(x + mu)
                            + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]

i.e. the projector signs of the printed equation ((gamma-1)/2 on the forward hop,
-(gamma+1)/2 on the backward hop) with the backward link taken at x - mu.  Periodic
boundaries in all four directions.  Chiral gamma basis:
gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1, 2, 3), gamma_4 = [[0, 1], [1, 0]],
so gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1): spins 0, 1 have
chirality +1, spins 2, 3 chirality -1.

The operator applies the full 4x4 gamma matrices (no spin projection), so it shares
no trick with the GPU stencil.

Pins (tests/test_oracle_dirac.py): Clifford algebra and gamma_5; the free-field
(U = 1) momentum-space closed form by plane waves and by the full dense spectrum;
gamma_5-hermiticity (Sec. 3); gauge covariance under a random SU(3) transform;
linearity in m; an independent dense matrix built by looping over site pairs.
"""
from __future__ import annotations

import numpy as np

# numpy axis of each lattice direction mu in a (T, Z, Y, X, ...) array
AXIS = (3, 2, 1, 0)

_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def gamma_matrices():
    """The four Euclidean gamma matrices in the chiral basis, gamma[mu] for mu = 0..3 (x, y, z, t)."""
    g = []
    for k in range(3):
        G = np.zeros((4, 4), dtype=np.complex128)
        G[0:2, 2:4] = -1j * _SIGMA[k]
        G[2:4, 0:2] = 1j * _SIGMA[k]
        g.append(G)
    G = np.zeros((4, 4), dtype=np.complex128)
    G[0:2, 2:4] = np.eye(2)
    G[2:4, 0:2] = np.eye(2)
    g.append(G)
    return g


def gamma5():
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]


def _spin(M, s):
    """Apply a 4x4 spin matrix to a field of shape (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", M, s)


def _colour(U, s):
    """Apply a field of 3x3 colour matrices to a field of shape (..., 4, 3)."""
    return np.einsum("...ab,...sb->...sa", U, s)


def _colour_dag(U, s):
    """Apply U^dag colour-wise: (U^dag s)_a = sum_b conj(U_ba) s_b."""
    return np.einsum("...ba,...sb->...sa", np.conj(U), s)


def hop(U, psi, mu, sign):
    """One hopping term of D at every site x, reading the neighbour x + sign*mu:

    sign = +1:  -1/2 (1 - gamma_mu) U_mu(x) psi(x + mu)
    sign = -1:  -1/2 (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)

    psi has shape (T, Z, Y, X, 12); so does the result.
    """
    shape = psi.shape
    s = psi.reshape(shape[:4] + (4, 3))
    ax = AXIS[mu]
    G = gamma_matrices()[mu]
    one = np.eye(4)
    Umu = U[..., mu, :, :]
    if sign > 0:
        t = _colour(Umu, np.roll(s, -1, axis=ax))
        out = -0.5 * _spin(one - G, t)
    else:
        t = _colour_dag(np.roll(Umu, 1, axis=ax), np.roll(s, 1, axis=ax))
        out = -0.5 * _spin(one + G, t)
    return out.reshape(shape)


def apply_D(U, psi, m):
    """(D psi)(x) for a fine spinor psi of shape (T, Z, Y, X, 12) (Sec. 2, eq. for D_xy)."""
    out = (4.0 + m) * psi
    for mu in range(4):
        for sign in (+1, -1):
            out = out + hop(U, psi, mu, sign)
    return out


def apply_g5(psi):
    """Multiply each site's spinor by gamma_5 = diag(1, 1, -1, -1) (spin-major components)."""
    out = psi.copy()
    out[..., 6:12] *= -1.0
    return out


def apply_Ddag(U, psi, m):
    """D^dag psi via gamma_5-hermiticity, D^dag = gamma_5 D gamma_5 (Sec. 3)."""
    return apply_g5(apply_D(U, apply_g5(psi), m))


def dense_D(U, m):
    """Dense matrix of D built by looping over site pairs (tiny lattices only).

    Index of (site, spin, colour) is 12*site + 3*spin + colour with the lexicographic
    site index x + X*(y + Y*(z + Z*t)).  Each forward neighbour pair (x, x+mu) gets
    the block -1/2 (1 - gamma_mu) (x) U_mu(x); each backward pair (x, x-mu) the block
    -1/2 (1 + gamma_mu) (x) U_mu(x-mu)^dag; the diagonal gets (4 + m).
    """
    T, Z, Y, X = U.shape[:4]
    ext = (X, Y, Z, T)
    V = X * Y * Z * T
    g = gamma_matrices()
    one = np.eye(4)
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)

    def lex(c):
        return c[0] + X * (c[1] + Y * (c[2] + Z * c[3]))

    for t in range(T):
        for z in range(Z):
            for y in range(Y):
                for x in range(X):
                    c = [x, y, z, t]
                    i = lex(c)
                    D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += (4.0 + m) * np.eye(12)
                    for mu in range(4):
                        f = list(c)
                        f[mu] = (f[mu] + 1) % ext[mu]
                        j = lex(f)
                        blk = np.kron(-0.5 * (one - g[mu]), U[t, z, y, x, mu])
                        D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += blk
                        b = list(c)
                        b[mu] = (b[mu] - 1) % ext[mu]
                        j = lex(b)
                        Ub = U[b[3], b[2], b[1], b[0], mu]
                        blk = np.kron(-0.5 * (one + g[mu]), np.conj(Ub.T))
                        D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += blk
    return D


def free_eigenvalues(dims, m):
    """Closed-form spectrum of the free (U = 1) periodic Wilson operator.

    For momentum p_mu = 2 pi n_mu / L_mu the plane waves give the eigenvalues
    m + sum_mu (1 - cos p_mu) +/- i sqrt(sum_mu sin^2 p_mu), each 6-fold degenerate
    (2 spin states x 3 colours).  Returned sorted as a flat array of 12 V values.
    """
    X, Y, Z, T = dims
    vals = []
    for nt in range(T):
        for nz in range(Z):
            for ny in range(Y):
                for nx in range(X):
                    p = 2 * np.pi * np.array([nx / X, ny / Y, nz / Z, nt / T])
                    re = m + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    vals += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(vals)


def free_plane_wave_factor(p, m):
    """The 4x4 spin matrix M(p) with D e^{ipx} chi = e^{ipx} (M(p) (x) 1_colour) chi for U = 1:
    M(p) = m + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu."""
    g = gamma_matrices()
    M = (m + np.sum(1 - np.cos(p))) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        M = M + 1j * np.sin(p[mu]) * g[mu]
    return M


def gauge_transform(U, Om):
    """U'_mu(x) = Omega(x) U_mu(x) Omega(x + mu)^dag for a site field Omega of shape (T,Z,Y,X,3,3)."""
    out = np.empty_like(U)
    for mu in range(4):
        Op = np.roll(Om, -1, axis=AXIS[mu])
        out[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(Op, -1, -2))
    return out


def transform_spinor(Om, psi):
    """(Omega psi)(x) = Omega(x) psi(x) colour-wise, psi of shape (T,Z,Y,X,12)."""
    s = psi.reshape(psi.shape[:4] + (4, 3))
    return _colour(Om, s).reshape(psi.shape)
