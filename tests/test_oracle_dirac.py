"""Pins of the oracle's Wilson-Dirac operator against what the paper and the
mathematics fix (Sec. 2 eq. for D, Sec. 3 gamma_5-hermiticity), not against itself."""
import numpy as np
import pytest

import synth
from oracle import dirac


def test_gamma_clifford_and_gamma5():
    g = dirac.gamma_matrices()
    for a in range(4):
        assert np.allclose(g[a], np.conj(g[a].T))
        for b in range(4):
            anti = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(anti, 2.0 * np.eye(4) * (a == b))
    # chiral basis: gamma_5 diagonal, spins 0,1 -> +1, spins 2,3 -> -1 (sigma_3 split of Sec. 3)
    assert np.allclose(dirac.gamma5(), np.diag([1, 1, -1, -1]))


def test_synth_gauge_is_su3_and_reproducible():
    dims = (4, 2, 2, 6)
    U = synth.gauge_field(dims, 0.7, 5)
    M = U.reshape(-1, 3, 3)
    assert np.abs(M @ np.conj(np.swapaxes(M, 1, 2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(M) - 1.0).max() < 1e-14
    assert np.array_equal(U, synth.gauge_field(dims, 0.7, 5))
    # chunked generation consumes the stream in the same order
    assert np.array_equal(U, synth.gauge_field(dims, 0.7, 5, chunk_sites=7))


@pytest.mark.parametrize("dims", [(3, 4, 5, 6), (4, 2, 6, 8)])
def test_free_field_plane_waves(dims):
    """U = 1: D e^{ipx} chi = e^{ipx} [m + sum(1-cos p) + i sum gamma sin p] chi (closed form)."""
    rng = np.random.default_rng(1)
    m = 0.137
    U = synth.unit_gauge(dims)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    for _ in range(4):
        n = [rng.integers(0, L) for L in dims]
        p = 2 * np.pi * np.array([n[0] / X, n[1] / Y, n[2] / Z, n[3] / T])
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = (phase[..., None, None] * chi).reshape(x.shape + (12,))
        want = (phase[..., None, None] * (dirac.free_plane_wave_factor(p, m) @ chi)).reshape(psi.shape)
        got = dirac.apply_D(U, psi, m)
        assert np.abs(got - want).max() < 1e-13


def _sorted(v):
    return v[np.lexsort((np.round(v.imag, 9), np.round(v.real, 9)))]


def test_free_field_dense_spectrum():
    """Full spectrum of the loop-built dense D at U = 1 equals the closed form, 6-fold degenerate."""
    dims = (2, 3, 2, 4)
    m = -0.3
    D = dirac.dense_D(synth.unit_gauge(dims), m)
    ev = _sorted(np.linalg.eigvals(D))
    want = _sorted(dirac.free_eigenvalues(dims, m))
    assert np.abs(ev - want).max() < 1e-10


def test_dense_loop_matrix_matches_stencil():
    dims = (2, 2, 4, 2)
    U = synth.gauge_field(dims, 0.6, 3)
    psi = synth.gaussian_spinors(dims, 1, 4)[0]
    D = dirac.dense_D(U, 0.21)
    assert np.abs(D @ psi.ravel() - dirac.apply_D(U, psi, 0.21).ravel()).max() < 1e-13


def test_gamma5_hermiticity():
    """<u, gamma_5 D gamma_5 v> = <D u, v> (Sec. 3)."""
    dims = (4, 4, 2, 6)
    U = synth.gauge_field(dims, 0.7, 8)
    u, v = synth.gaussian_spinors(dims, 2, 9)
    m = -0.4
    lhs = np.vdot(u, dirac.apply_g5(dirac.apply_D(U, dirac.apply_g5(v), m)))
    rhs = np.vdot(dirac.apply_D(U, u, m), v)
    assert abs(lhs - rhs) <= 1e-14 * abs(rhs) * 10


def test_gauge_covariance():
    """D(U') Omega psi = Omega D(U) psi with U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag."""
    dims = (4, 2, 4, 4)
    U = synth.gauge_field(dims, 0.6, 21)
    Om = synth.random_su3_field(dims, 22)
    psi = synth.gaussian_spinors(dims, 1, 23)[0]
    m = 0.05
    Up = dirac.gauge_transform(U, Om)
    lhs = dirac.apply_D(Up, dirac.transform_spinor(Om, psi), m)
    rhs = dirac.transform_spinor(Om, dirac.apply_D(U, psi, m))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_linear_in_mass():
    dims = (2, 4, 2, 4)
    U = synth.gauge_field(dims, 0.4, 2)
    psi = synth.gaussian_spinors(dims, 1, 3)[0]
    d = dirac.apply_D(U, psi, 0.3) - dirac.apply_D(U, psi, -0.2)
    assert np.abs(d - 0.5 * psi).max() < 1e-14


def test_planted_mistakes_are_caught():
    """A wrong link position (the literal index placement of the printed equation) breaks gauge
    covariance, and a flipped backward projector breaks gamma_5-hermiticity: the pins above
    detect both kinds of slip."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.6, 31)
    Om = synth.random_su3_field(dims, 32)
    psi = synth.gaussian_spinors(dims, 1, 33)[0]

    def literal_D(U, psi):  # backward hop with U_mu(x)^dag instead of U_mu(x - mu)^dag
        out = 4.0 * psi
        s = psi.reshape(psi.shape[:4] + (4, 3))
        g = dirac.gamma_matrices()
        for mu in range(4):
            out = out + dirac.hop(U, psi, mu, +1)
            t = np.einsum("...ba,...sb->...sa", np.conj(U[..., mu, :, :]), np.roll(s, 1, axis=dirac.AXIS[mu]))
            out = out - 0.5 * np.einsum("st,...tc->...sc", np.eye(4) + g[mu], t).reshape(psi.shape)
        return out

    Up = dirac.gauge_transform(U, Om)
    lhs = literal_D(Up, dirac.transform_spinor(Om, psi))
    rhs = dirac.transform_spinor(Om, literal_D(U, psi))
    assert np.abs(lhs - rhs).max() > 1e-3


def test_c_restatement_matches_numpy_definition():
    """oracle/c/dirac_ref.c (used for large lattices) against the numpy definition above."""
    from oracle import cref
    dims = (4, 6, 2, 8)
    U = synth.gauge_field(dims, 0.7, 41)
    psi = synth.gaussian_spinors(dims, 1, 42)[0]
    assert np.abs(cref.apply_D(U, psi, -0.31) - dirac.apply_D(U, psi, -0.31)).max() < 1e-13
    for mu in range(4):
        for s in (+1, -1):
            assert np.abs(cref.hop(U, psi, mu, s) - dirac.hop(U, psi, mu, s)).max() < 1e-14
    # and it satisfies the closed form on its own: free-field plane wave on a larger lattice
    dims = (8, 8, 8, 8)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(*(np.arange(L) for L in (T, Z, Y, X)), indexing="ij")
    p = 2 * np.pi * np.array([1 / X, 3 / Y, 2 / Z, 5 / T])
    chi = np.arange(12).reshape(4, 3) + 1j
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    psi = (ph[..., None, None] * chi).reshape(x.shape + (12,))
    want = (ph[..., None, None] * (dirac.free_plane_wave_factor(p, 0.2) @ chi)).reshape(psi.shape)
    assert np.abs(cref.apply_D(synth.unit_gauge(dims), psi, 0.2) - want).max() < 1e-12
