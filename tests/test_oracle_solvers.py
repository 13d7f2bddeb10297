"""Pins of the oracle's smoother, coarsest solve, outer GCR and MG-GCR (Sec. 3)
against dense linear algebra and closed-form special cases."""
import numpy as np

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
