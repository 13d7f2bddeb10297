"""Pins of the oracle's smoother, coarsest solve, outer GCR and MG-GCR (Sec. 3)
against dense linear algebra and closed-form special cases."""
import numpy as np
import pytest

import synth
from oracle import dirac, mg, solvers


def _tiny():
    dims, block, N = (4, 4, 2, 4), (2, 2, 2, 2), 3
    U = synth.gauge_field(dims, 0.5, 40)
    op = mg.WilsonOp(U, 0.02)
    v = synth.setup_starts(dims, N, 41)
    P = mg.block_orthonormalise(v, block)
    return dims, block, op, P, mg.galerkin(op, P, block)


def test_mr_identity_and_monotone():
    b = synth.gaussian_spinors((2, 2, 2, 2), 1, 1)[0]
    x = solvers.mr(lambda v: v, b, np.zeros_like(b), 1)       # A = I: exact after one step
    assert np.abs(x - b).max() < 1e-15
    dims, block, op, P, _ = _tiny()
    b = synth.gaussian_spinors(dims, 1, 2)[0]
    res = [solvers.norm(b - op.apply(solvers.mr(op.apply, b, np.zeros_like(b), k))) for k in range(8)]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(7))


def test_cgnr_against_dense_solve():
    *_, Ac = _tiny()
    b = synth.coarse_starts(Ac.dims, Ac.n, 1, 3)[0]
    x, it = solvers.cgnr(Ac, b, 1e-13, 10000)
    want = np.linalg.solve(Ac.dense(), b.ravel())
    assert np.abs(x.ravel() - want).max() < 1e-10 * np.abs(want).max()


def test_fgcr_exact_preconditioner_one_iteration():
    dims, block, op, P, _ = _tiny()
    D = dirac.dense_D(op.U, op.m)
    Dinv = np.linalg.inv(D)
    b = synth.gaussian_spinors(dims, 1, 5)[0]
    x, info = solvers.fgcr(op.apply, lambda r: (Dinv @ r.ravel()).reshape(r.shape), b, 1e-10)
    assert info.iters == 1 and info.true_resid < 1e-12


def test_fgcr_unpreconditioned_matches_lu():
    dims, block, op, P, _ = _tiny()
    b = synth.gaussian_spinors(dims, 1, 6)[0]
    x, info = solvers.fgcr(op.apply, lambda r: r, b, 1e-11, restart=16, max_iter=2000)
    h = info.history
    restart_ends = set(range(15, len(h), 16))
    assert all(h[i + 1] <= h[i] * (1 + 1e-10) for i in range(len(h) - 1) if i not in restart_ends)
    want = np.linalg.solve(dirac.dense_D(op.U, op.m), b.ravel())
    assert np.abs(x.ravel() - want).max() < 1e-9 * np.abs(want).max()


def test_mg_gcr_matches_lu_and_beats_unpreconditioned():
    dims, block, op, P, Ac = _tiny()
    H = solvers.Hierarchy([op, Ac], [P], [block], solvers.CycleParams(coarse_tol=1e-10))
    b = synth.gaussian_spinors(dims, 1, 7)[0]
    x, info = solvers.mg_solve(H, b, 1e-10)
    assert info.true_resid <= 1e-10
    want = np.linalg.solve(dirac.dense_D(op.U, op.m), b.ravel())
    assert np.abs(x.ravel() - want).max() < 1e-8 * np.abs(want).max()
    _, plain = solvers.fgcr(op.apply, lambda r: r, b, 1e-10, 16, 5000)
    assert info.iters < plain.iters


def test_three_level_cycle_converges():
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.5, 50)
    op = mg.WilsonOp(U, 0.05)
    blocks = [(2, 2, 2, 2), (2, 2, 1, 2)]
    v1 = synth.setup_starts(dims, 3, 51)
    P1 = mg.block_orthonormalise(v1, blocks[0])
    A1 = mg.galerkin(op, P1, blocks[0])
    v2 = synth.coarse_starts(A1.dims, A1.n, 4, 52)
    H = solvers.hierarchy_from_vectors(op, blocks, [v1, v2], solvers.CycleParams(coarse_tol=1e-10))
    assert H.nlevels == 3 and np.abs(H.ops[1].D - A1.D).max() == 0
    b = synth.gaussian_spinors(dims, 1, 53)[0]
    x, info = solvers.mg_solve(H, b, 1e-10)
    assert info.true_resid <= 1e-10
    assert solvers.norm(b - dirac.apply_D(U, x, 0.05)) <= 1e-10 * solvers.norm(b) * 1.01


def test_setup_homogeneous_cycle_kills_vectors_in_span():
    """Why the setup improves vectors by inverse iteration: a vector already in span(P),
    passed through the cycle on the homogeneous equation with an exact coarse solve,
    comes back as exactly zero (the coarse correction reproduces it)."""
    dims, block, op, P, Ac = _tiny()
    H = solvers.Hierarchy([op, Ac], [P], [block], solvers.CycleParams(coarse_tol=1e-14))
    cd = mg.coarse_dims(dims, block)
    v = mg.prolong(P, synth.coarse_starts(cd, Ac.n, 1, 60)[0], block)
    e = solvers.cycle(H, 0, -op.apply(v))
    assert solvers.norm(v + e) < 1e-10 * solvers.norm(v)


def test_setup_passes_lower_the_rayleigh_quotient():
    """Setup parity is unpinned at the vector level; its indirect pin: the mean
    |A psi_k| / |psi_k| decreases from pass to pass, and the final vectors lie in span(P)."""
    dims, block = (4, 4, 4, 8), (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.5, 61)
    op = mg.WilsonOp(U, 0.0)
    starts = synth.setup_starts(dims, 4, 62)
    hist = []
    P, Ac, psi = solvers.setup_level(op, block, starts, passes=4, relax=10,
                                     params=solvers.CycleParams(coarse_tol=1e-8), history=hist)
    assert all(hist[i + 1] < hist[i] for i in range(len(hist) - 1)), hist
    for v in psi:
        assert solvers.norm(mg.prolong(P, mg.restrict(P, v, block), block) - v) < 1e-12


# ---- the cycle against dense closed forms (Sec. 3: coarse correction, then post-smoothing) ----
def _lstsq_step(A, r, e):
    """One minimal-residual step as a least-squares problem: the multiple of the residual
    rho = r - A e that, added to e, minimises |r - A e'| (numpy's least-squares routine)."""
    rho = r - A @ e
    alpha = np.linalg.lstsq((A @ rho)[:, None], rho, rcond=None)[0][0]
    return e + alpha * rho


def _dense_two_level(r, D, Pd, nu):
    """K(r) = nu minimal-residual steps on D e = r from the exact coarse correction
    Pd (Pd^dag D Pd)^-1 Pd^dag r (no pre-smoothing)."""
    Dc = np.conj(Pd.T) @ D @ Pd
    e = Pd @ np.linalg.solve(Dc, np.conj(Pd.T) @ r)
    for _ in range(nu):
        e = _lstsq_step(D, r, e)
    return e


def _exact_coarse(A, b):
    return np.linalg.solve(A.dense(), b.ravel()).reshape(b.shape)


@pytest.mark.parametrize("nu", [0, 1, 2, 4])
def test_two_level_cycle_equals_dense_formula(nu):
    """The oracle cycle with an exact coarsest solve equals the dense closed form: nu = 0 is the
    coarse-grid correction alone, nu >= 1 adds exactly nu post-smoothing steps after it.  A cycle
    that smoothed before the correction, or took a different number of steps, fails."""
    dims, block, op, P, Ac = _tiny()
    D = dirac.dense_D(op.U, op.m)
    Pd = mg.dense_prolongator(P, block)
    H = solvers.Hierarchy([op, Ac], [P], [block], solvers.CycleParams(nu=nu))
    H.coarse_solver = _exact_coarse
    r = synth.gaussian_spinors(dims, 1, 90)[0]
    got = solvers.cycle(H, 0, r).ravel()
    want = _dense_two_level(r.ravel(), D, Pd, nu)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    if nu == 1:  # the smoothing step really is after the correction: pre-smoothing differs
        pre = _lstsq_step(D, r.ravel(), np.zeros_like(want))
        pre = pre + Pd @ np.linalg.solve(np.conj(Pd.T) @ D @ Pd, np.conj(Pd.T) @ (r.ravel() - D @ pre))
        assert np.abs(pre - want).max() > 1e-3 * np.abs(want).max()


@pytest.mark.parametrize("gamma", [1, 2])
def test_three_level_cycle_equals_dense_formula(gamma):
    """Three levels, exact coarsest solve: the middle level repeats {restrict the residual of the
    current correction, coarse correction, nu smoothing steps on A_1} gamma times (gamma = 2 is
    the W-cycle of Sec. 3), the fine level once; every operator and prolongator is a dense matrix."""
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.5, 91)
    op = mg.WilsonOp(U, 0.1)
    blocks = [(2, 2, 2, 2), (2, 2, 1, 2)]
    v1 = synth.setup_starts(dims, 3, 92)
    P0 = mg.block_orthonormalise(v1, blocks[0])
    A1 = mg.galerkin(op, P0, blocks[0])
    v2 = synth.coarse_starts(A1.dims, A1.n, 4, 93)
    nu = 2
    H = solvers.hierarchy_from_vectors(op, blocks, [v1, v2], solvers.CycleParams(nu=nu, gamma=gamma))
    H.coarse_solver = _exact_coarse
    D = dirac.dense_D(U, 0.1)
    P0d = mg.dense_prolongator(H.P[0], blocks[0])
    P1d = mg.dense_prolongator(H.P[1], blocks[1])
    A1d = np.conj(P0d.T) @ D @ P0d
    A2d = np.conj(P1d.T) @ A1d @ P1d

    def K1(r1):
        e = np.zeros_like(r1)
        for _ in range(gamma):
            e = e + P1d @ np.linalg.solve(A2d, np.conj(P1d.T) @ (r1 - A1d @ e))
            for _ in range(nu):
                e = _lstsq_step(A1d, r1, e)
        return e

    r = synth.gaussian_spinors(dims, 1, 94)[0]
    e = P0d @ K1(np.conj(P0d.T) @ r.ravel())
    for _ in range(nu):
        e = _lstsq_step(D, r.ravel(), e)
    got = solvers.cycle(H, 0, r).ravel()
    assert np.abs(got - e).max() < 1e-10 * np.abs(e).max()


def _dense_block_basis(psi, dims, block, nvec):
    """Per (block, chirality), the orthonormal basis Gram-Schmidt gives for the vectors in
    order: numpy's QR with the diagonal of R made real positive (that QR is unique).  Returned
    as N fields (T, Z, Y, X, 12), and as the dense prolongator (columns per block, chirality, k)."""
    X, Y, Z, T = dims
    t, z, y, x = np.indices((T, Z, Y, X))
    bid = ((t // block[3]) * (Z // block[2]) + z // block[2]) * (Y // block[1]) + y // block[1]
    bid = (bid * (X // block[0]) + x // block[0]).ravel()
    nb = bid.max() + 1
    V = X * Y * Z * T
    P = np.zeros((nvec, V, 12), dtype=np.complex128)
    cols = []
    flat = psi.reshape(nvec, V, 12)
    for b in range(nb):
        sites = np.nonzero(bid == b)[0]
        for s in range(2):
            M = flat[:, sites, 6 * s:6 * s + 6].reshape(nvec, -1).T
            Q, R = np.linalg.qr(M)
            ph = np.diag(R) / np.abs(np.diag(R))
            Q = Q * ph[None, :]
            for k in range(nvec):
                P[k, sites, 6 * s:6 * s + 6] = Q[:, k].reshape(len(sites), 6)
                col = np.zeros((V, 12), dtype=np.complex128)
                col[sites, 6 * s:6 * s + 6] = Q[:, k].reshape(len(sites), 6)
                cols.append(col.ravel())
    return P.reshape(psi.shape), np.stack(cols, axis=1)


def test_adaptive_setup_equals_dense_restatement():
    """The oracle's fixed-N adaptive setup (Sec. 2: relax D psi = 0 from random starts, build a
    trial hierarchy, use it to solve again, repeat) against a dense restatement made of library
    routines: `relax` least-squares MR steps on D psi = 0, normalisation, Gram-Schmidt as QR per
    block and chirality, then per later pass psi_k <- K(psi_k) with the dense two-level cycle of
    the current basis (exact coarse solve, nu post-smoothing steps), normalised, and the basis
    rebuilt once per pass.  A different relax count, a basis rebuilt per vector, or a vector
    left unnormalised fails."""
    dims, block, N, passes, relax, nu = (4, 4, 2, 4), (2, 2, 2, 2), 3, 3, 5, 4
    U = synth.gauge_field(dims, 0.5, 95)
    m = 0.05
    op = mg.WilsonOp(U, m)
    starts = synth.setup_starts(dims, N, 96)
    P, Ac, psi = solvers.setup_level(op, block, starts, passes=passes, relax=relax,
                                     params=solvers.CycleParams(nu=nu),
                                     coarse_solver_factory=lambda A: _exact_coarse)
    D = dirac.dense_D(U, m)
    w = []
    for s in starts:
        e = s.ravel().copy()
        for _ in range(relax):
            e = _lstsq_step(D, np.zeros_like(e), e)
        w.append(e / np.linalg.norm(e))
    w = np.array(w)
    for _ in range(passes - 1):
        _, Pd = _dense_block_basis(w.reshape(psi.shape), dims, block, N)
        w = np.array([_dense_two_level(v, D, Pd, nu) for v in w])
        w = w / np.linalg.norm(w, axis=1)[:, None]
    Pw, _ = _dense_block_basis(w.reshape(psi.shape), dims, block, N)
    assert np.abs(psi.reshape(N, -1) - w).max() < 1e-10
    assert np.abs(P - Pw).max() < 1e-10
