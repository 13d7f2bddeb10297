"""Pins of the even-odd form of the coarsest solve (oracle/eo.py) against dense linear algebra:
the Schur complement and its adjoint against the blocks of the brute-force matrix of the
stencil, the reconstructed solution against a dense solve, and the stopping test against the
true residual of the whole system."""
import numpy as np
import pytest

import synth
from oracle import dirac, eo, mg, solvers


def random_stencil(dims, n, seed, diag=6.0):
    X, Y, Z, T = dims
    rng = np.random.default_rng(seed)
    D = (rng.standard_normal((T, Z, Y, X, 9, n, n)) + 1j * rng.standard_normal((T, Z, Y, X, 9, n, n))) * 0.3
    D[..., 0, :, :] += diag * np.eye(n)
    return mg.StencilOp(D)


def dense(apply, shape):
    """The matrix of a linear map by applying it to every unit vector."""
    size = int(np.prod(shape))
    M = np.zeros((size, size), complex)
    for j in range(size):
        e = np.zeros(size, complex)
        e[j] = 1.0
        M[:, j] = apply(e.reshape(shape)).ravel()
    return M


def split(A, dims, n):
    par = np.repeat(eo.parity(dims).ravel(), n)
    return par == 0, par == 1


@pytest.mark.parametrize("dims,n", [((4, 2, 2, 4), 4), ((2, 2, 2, 2), 6)])
def test_schur_against_dense_blocks(dims, n):
    A = random_stencil(dims, n, 1)
    shape = A.D.shape[:4] + (n,)
    M = dense(A.apply, shape)
    e, o = split(A, dims, n)
    S = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.inv(M[np.ix_(o, o)]) @ M[np.ix_(o, e)]
    inv = eo.odd_block_inverse(A)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    y = eo.schur_apply(A, x, inv).ravel()
    ref = S @ x.ravel()[e]
    assert np.linalg.norm(y[e] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.all(y[o] == 0)
    yd = eo.schur_apply_dagger(A, x, inv).ravel()
    refd = S.conj().T @ x.ravel()[e]
    assert np.linalg.norm(yd[e] - refd) <= 1e-12 * np.linalg.norm(refd)
    assert np.all(yd[o] == 0)


def test_sigma3_identity_of_a_gamma5_hermitian_stencil():
    """For a stencil with sigma_3 A sigma_3 = A^dag (the coarse operator's Sec. 3 property) the
    Schur complement keeps it: S^dag = sigma_3 S sigma_3 (the form the kernels use)."""
    dims, n = (2, 2, 2, 4), 4
    A0 = random_stencil(dims, n, 3)
    s3 = np.diag([1.0] * (n // 2) + [-1.0] * (n // 2))
    # symmetrise: B = (A + sigma_3 A^dag sigma_3) / 2 satisfies sigma_3 B sigma_3 = B^dag
    shape = A0.D.shape[:4] + (n,)
    M = dense(A0.apply, shape)
    S3 = np.kron(np.eye(int(np.prod(shape[:4]))), s3)
    Mb = 0.5 * (M + S3 @ M.conj().T @ S3)
    # back to stencil form: read the blocks of Mb
    X, Y, Z, T = dims
    V = X * Y * Z * T
    D = np.zeros_like(A0.D)
    v = np.arange(V)
    crd = [v % X, (v // X) % Y, (v // (X * Y)) % Z, v // (X * Y * Z)]
    for k in range(9):
        c = [a.copy() for a in crd]
        if k > 0:
            mu, sg = (k - 1) // 2, (1 if (k - 1) % 2 == 0 else -1)
            c[mu] = (c[mu] + sg) % (X, Y, Z, T)[mu]
        nb = c[0] + X * (c[1] + Y * (c[2] + Z * c[3]))
        for s in range(V):
            D.reshape(V, 9, n, n)[s, k] = Mb[s * n:(s + 1) * n, nb[s] * n:(nb[s] + 1) * n]
    # on a lattice with extent 2 the +mu and -mu neighbours coincide: their two slots then
    # hold the same block twice; halve them so the stencil reproduces Mb
    for mu, L in enumerate((X, Y, Z, T)):
        if L == 2:
            D.reshape(V, 9, n, n)[:, 1 + 2 * mu] *= 0.5
            D.reshape(V, 9, n, n)[:, 2 + 2 * mu] *= 0.5
    B = mg.StencilOp(D)
    assert np.allclose(dense(B.apply, shape), Mb, atol=1e-13)
    inv = eo.odd_block_inverse(B)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    lhs = eo.schur_apply_dagger(B, x, inv)
    rhs = B.sigma3(eo.schur_apply(B, B.sigma3(x), inv))
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)


def test_cgnr_eo_solution_and_stopping_test():
    dims, n = (4, 2, 2, 4), 4
    A = random_stencil(dims, n, 5, diag=4.0)
    shape = A.D.shape[:4] + (n,)
    M = dense(A.apply, shape)
    rng = np.random.default_rng(6)
    b = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    x, it = eo.cgnr_eo(A, b, 1e-13, 500)
    xr = np.linalg.solve(M, b.ravel())
    assert np.linalg.norm(x.ravel() - xr) <= 1e-11 * np.linalg.norm(xr)
    assert 0 < it < 500
    # loose tolerance: the full-system residual at the reconstructed x meets the test
    for tol in (1e-2, 1e-5):
        x, it = eo.cgnr_eo(A, b, tol, 500)
        assert np.linalg.norm(b - A.apply(x)) <= tol * np.linalg.norm(b) * (1 + 1e-9)


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        eo.parity((3, 2, 2, 2))


def test_two_level_solve_with_even_odd_coarsest():
    """The MG-GCR solve with the even-odd coarsest CG: same solution as the plain CGNR
    hierarchy (dense solve reference) and an equal iteration count at a tight coarse tolerance."""
    import synth
    from oracle import dirac, solvers
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.4, 3)
    op = mg.WilsonOp(U, 0.1)
    starts = synth.setup_starts(dims, 4, 4)
    v = np.array([solvers._normalise(solvers.mr(op.apply, np.zeros_like(s), s, 10)) for s in starts])
    b = synth.gaussian_spinors(dims, 1, 5)[0]
    its = []
    for flag in (False, True):
        H = solvers.hierarchy_from_vectors(op, [(2, 2, 2, 2)], [v], solvers.CycleParams(coarse_tol=1e-10,
                                                                                       coarse_eo=flag))
        x, info = solvers.mg_solve(H, b, 1e-10, 16)
        assert np.linalg.norm(b - dirac.apply_D(U, x, 0.1)) <= 1.01e-10 * np.linalg.norm(b)
        its.append(info.iters)
    assert abs(its[0] - its[1]) <= 1


# ---- the even-odd (red/black) form of the fine Wilson solve (oracle/eo_fine.py) ----
from oracle import eo_fine  # noqa: E402


def _fine_blocks(dims, U, m):
    """Dense D from the loop-built matrix, split by site parity (dof index = site * 12 + k)."""
    D = dirac.dense_D(U, m)
    par = np.repeat(eo_fine.parity(dims).ravel(), 12)
    e, o = np.nonzero(par == 0)[0], np.nonzero(par == 1)[0]
    return D, e, o


def test_fine_schur_against_dense_blocks():
    dims, m = (4, 2, 2, 4), -0.3
    U = synth.gauge_field(dims, 0.6, 120)
    D, e, o = _fine_blocks(dims, U, m)
    S = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    x = synth.gaussian_spinors(dims, 1, 121)[0]
    xe = x.ravel().copy()
    xe[o] = 0
    got = eo_fine.schur_apply(U, xe.reshape(x.shape), m).ravel()
    assert np.abs(got[o]).max() == 0
    assert np.abs(got[e] - S @ xe[e]).max() < 1e-13 * np.abs(S @ xe[e]).max()
    # the odd-odd block is the scalar d = 4 + m (no hop stays on one parity)
    assert np.abs(D[np.ix_(o, o)] - (4 + m) * np.eye(len(o))).max() < 1e-15
    # S^dag = gamma_5 S gamma_5
    g5 = np.where(np.arange(len(D)) % 12 < 6, 1.0, -1.0)[e]
    assert np.abs(np.conj(S.T) - g5[:, None] * S * g5[None, :]).max() < 1e-13


def test_fine_prepare_and_reconstruct_against_dense_solve():
    dims, m = (4, 2, 2, 4), -0.3
    U = synth.gauge_field(dims, 0.6, 122)
    D, e, o = _fine_blocks(dims, U, m)
    b = synth.gaussian_spinors(dims, 1, 123)[0]
    bv = b.ravel()
    S = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    bh = eo_fine.prepare(U, b, m).ravel()
    want_bh = bv[e] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], bv[o])
    assert np.abs(bh[e] - want_bh).max() < 1e-13 * np.abs(want_bh).max() and np.abs(bh[o]).max() == 0
    xe = np.zeros_like(bv)
    xe[e] = np.linalg.solve(S, bh[e])
    x = eo_fine.reconstruct(U, b, xe.reshape(b.shape), m).ravel()
    want = np.linalg.solve(D, bv)
    assert np.abs(x - want).max() < 1e-11 * np.abs(want).max()


def test_fine_even_odd_mg_solve():
    """MG-GCR on the even-odd system (the whole-lattice cycle on (r_e, 0) as preconditioner)
    reaches the whole system's 1e-10 residual and the dense solution."""
    dims, block, N = (4, 4, 2, 4), (2, 2, 2, 2), 3
    U = synth.gauge_field(dims, 0.5, 124)
    op = mg.WilsonOp(U, 0.02)
    P = mg.block_orthonormalise(synth.setup_starts(dims, N, 125), block)
    H = solvers.Hierarchy([op, mg.galerkin(op, P, block)], [P], [block], solvers.CycleParams(coarse_tol=1e-10))
    b = synth.gaussian_spinors(dims, 1, 126)[0]
    x, info = eo_fine.mg_solve_eo(H, b, 1e-10)
    assert np.linalg.norm(b - dirac.apply_D(U, x, 0.02)) <= 1.01e-10 * np.linalg.norm(b)
    want = np.linalg.solve(dirac.dense_D(U, 0.02), b.ravel())
    assert np.abs(x.ravel() - want).max() < 1e-8 * np.abs(want).max()


def test_block_jacobi_schur_cg():
    """Right block-Jacobi preconditioning of the coarsest CG: S's diagonal blocks against the
    dense Schur complement (extent 2 included, where two hops return by either slot) and the
    preconditioned CG's solution against a dense solve."""
    for dims, seed in (((4, 4, 2, 2), 130), ((2, 2, 2, 4), 131)):
        n = 4
        A = random_stencil(dims, n, seed)
        inv = eo.odd_block_inverse(A)
        Sd = eo.schur_self_blocks(A, inv)
        par = eo.parity(dims).ravel()
        Ad = A.dense()
        e = np.nonzero(np.repeat(par, n) == 0)[0]
        o = np.nonzero(np.repeat(par, n) == 1)[0]
        S = Ad[np.ix_(e, e)] - Ad[np.ix_(e, o)] @ np.linalg.solve(Ad[np.ix_(o, o)], Ad[np.ix_(o, e)])
        ev_sites = np.nonzero(par == 0)[0]
        flat = Sd.reshape(-1, n, n)
        for i, site in enumerate(ev_sites):
            blk = S[i * n:(i + 1) * n, i * n:(i + 1) * n]
            assert np.abs(flat[site] - blk).max() < 1e-12 * np.abs(blk).max()
        b = (np.random.default_rng(seed).standard_normal(A.D.shape[:4] + (n,)) + 0j)
        x, it = eo.cgnr_eo_block_jacobi(A, b, 1e-12, 5000)
        want = np.linalg.solve(Ad, b.ravel())
        assert np.abs(x.ravel() - want).max() < 1e-9 * np.abs(want).max()
