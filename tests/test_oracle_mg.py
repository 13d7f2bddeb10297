"""Pins of the oracle's prolongator, restriction and Galerkin coarse operator
(Sec. 2: P, R = P^dag, D^ = P^dag D P, the projector; Sec. 3: sigma_3 P = P gamma_5)."""
import numpy as np
import pytest

import synth
from oracle import dirac, mg, solvers


def _P(dims, block, N, seed):
    v = synth.setup_starts(dims, N, seed)
    return v, mg.block_orthonormalise(v, block)


@pytest.mark.parametrize("dims,block,N", [((4, 4, 2, 4), (2, 2, 2, 2), 3), ((4, 2, 2, 6), (2, 2, 2, 3), 2)])
def test_orthonormal_and_span(dims, block, N):
    v, P = _P(dims, block, N, 4)
    Pd = mg.dense_prolongator(P, block)
    assert np.abs(np.conj(Pd.T) @ Pd - np.eye(Pd.shape[1])).max() < 1e-13   # P^dag P = I
    for a in range(N):                                                      # v_alpha in span(P)
        back = mg.prolong(P, mg.restrict(P, v[a], block), block)
        assert np.abs(back - v[a]).max() < 1e-12


def test_chirality_split_and_adjointness():
    dims, block, N = (4, 4, 2, 4), (2, 2, 2, 2), 3
    _, P = _P(dims, block, N, 7)
    cd = mg.coarse_dims(dims, block)
    phi = synth.coarse_starts(cd, 2 * N, 1, 8)[0]
    psi = synth.gaussian_spinors(dims, 1, 9)[0]
    # sigma_3 P = P gamma_5
    s3 = phi.copy()
    s3[..., N:] *= -1
    assert np.abs(dirac.apply_g5(mg.prolong(P, phi, block)) - mg.prolong(P, s3, block)).max() < 1e-14
    # <phi, P^dag psi> = <P phi, psi>
    a = np.vdot(phi, mg.restrict(P, psi, block))
    b = np.vdot(mg.prolong(P, phi, block), psi)
    assert abs(a - b) < 1e-12 * abs(b)


def test_laplace_piecewise_constant_prolongator():
    """Sec. 2: one constant vector on 4^d blocks gives P = theta_xhat(x) / 2^d (d = 4)."""
    dims, block = (8, 4, 4, 8), (4, 4, 4, 4)
    v = np.ones((1,) + synth.lex_shape(dims) + (2,), dtype=np.complex128)  # one dof per chirality
    P = mg.block_orthonormalise(v, block)
    assert np.abs(P - 1.0 / 2 ** 4).max() < 1e-15


def test_rank_deficiency_is_reported():
    dims, block = (2, 2, 2, 2), (2, 2, 2, 2)
    v = synth.setup_starts(dims, 2, 3)
    v[1] = 2.0 * v[0]
    with pytest.raises(mg.RankDeficient):
        mg.block_orthonormalise(v, block)


@pytest.mark.parametrize("dims,block,N", [
    ((4, 4, 4, 4), (2, 2, 2, 2), 2),      # coarse extent 2: +mu and -mu reach the same site
    ((4, 2, 2, 6), (2, 2, 2, 2), 2),      # coarse (2,1,1,3): extent 1 keeps hops in-block
])
def test_galerkin_equals_dense_product(dims, block, N):
    """D^ = P^dag D P entrywise: stencil blocks vs explicit dense matrices."""
    U = synth.gauge_field(dims, 0.6, 10)
    m = -0.1
    _, P = _P(dims, block, N, 11)
    Ac = mg.galerkin(mg.WilsonOp(U, m), P, block)
    Pd = mg.dense_prolongator(P, block)
    D = dirac.dense_D(U, m)
    want = np.conj(Pd.T) @ D @ Pd
    assert np.abs(Ac.dense() - want).max() < 1e-12
    # sigma_3 D^ sigma_3 = D^dag (gamma_5-hermiticity carried to the coarse level, Sec. 3)
    n = 2 * N
    s3 = np.tile(np.r_[np.ones(N), -np.ones(N)], Ac.dense().shape[0] // n)
    A = Ac.dense()
    assert np.abs(s3[:, None] * A * s3[None, :] - np.conj(A.T)).max() < 1e-12
    # explicit adjoint used by the coarsest CGNR
    phi = synth.coarse_starts(Ac.dims, n, 1, 3)[0]
    assert np.abs(Ac.apply_dagger(phi).ravel() - np.conj(A.T) @ phi.ravel()).max() < 1e-12
    assert np.abs(Ac.apply(phi).ravel() - A @ phi.ravel()).max() < 1e-12


def test_second_level_galerkin_equals_dense_product():
    dims, block, N = (4, 4, 4, 4), (2, 2, 2, 2), 2
    U = synth.gauge_field(dims, 0.6, 12)
    _, P = _P(dims, block, N, 13)
    A1 = mg.galerkin(mg.WilsonOp(U, 0.02), P, block)
    block2, N2 = (2, 1, 2, 1), 3
    v2 = synth.coarse_starts(A1.dims, 2 * N, N2, 14)
    P2 = mg.block_orthonormalise(v2, block2)
    A2 = mg.galerkin(A1, P2, block2)
    Pd2 = mg.dense_prolongator(P2, block2)
    want = np.conj(Pd2.T) @ A1.dense() @ Pd2
    assert np.abs(A2.dense() - want).max() < 1e-12


def test_mass_shift_and_gauge_invariance():
    dims, block, N = (4, 4, 2, 4), (2, 2, 2, 2), 2
    U = synth.gauge_field(dims, 0.6, 15)
    v, P = _P(dims, block, N, 16)
    A0 = mg.galerkin(mg.WilsonOp(U, 0.1), P, block)
    A1 = mg.galerkin(mg.WilsonOp(U, -0.35), P, block)
    assert np.abs(A0.shifted(-0.45).D - A1.D).max() < 1e-13        # D^(m) = D^(m0) + (m - m0) I
    Om = synth.random_su3_field(dims, 17)
    Ut = dirac.gauge_transform(U, Om)
    vt = np.array([dirac.transform_spinor(Om, x) for x in v])
    Pt = mg.block_orthonormalise(vt, block)
    At = mg.galerkin(mg.WilsonOp(Ut, 0.1), Pt, block)
    assert np.abs(At.D - A0.D).max() < 1e-12                        # D^ is gauge invariant


def test_petrov_galerkin_projector():
    """Sec. 2: the coarse-grid correction projector is idempotent and P^dag projector = 0."""
    dims, block, N = (4, 2, 2, 4), (2, 2, 2, 2), 2
    U = synth.gauge_field(dims, 0.5, 18)
    _, P = _P(dims, block, N, 19)
    D = dirac.dense_D(U, 0.05)
    Pd = mg.dense_prolongator(P, block)
    Dc = np.conj(Pd.T) @ D @ Pd
    proj = np.eye(D.shape[0]) - D @ Pd @ np.linalg.solve(Dc, np.conj(Pd.T))
    assert np.abs(proj @ proj - proj).max() < 1e-11
    assert np.abs(np.conj(Pd.T) @ proj).max() < 1e-11
    # and the cycle's exact coarse correction leaves a residual with zero restriction
    H = solvers.Hierarchy([mg.WilsonOp(U, 0.05), mg.galerkin(mg.WilsonOp(U, 0.05), P, block)], [P], [block],
                          solvers.CycleParams(coarse_tol=1e-14))
    r = synth.gaussian_spinors(dims, 1, 20)[0]
    ec = solvers.cgnr(H.ops[1], mg.restrict(P, r, block), 1e-14, 5000)[0]
    r2 = r - H.ops[0].apply(mg.prolong(P, ec, block))
    assert np.abs(mg.restrict(P, r2, block)).max() < 1e-10
