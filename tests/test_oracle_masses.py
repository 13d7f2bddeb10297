"""Pins of the oracle's mass search (workload definition lambda_min(D^dag D) = r m^2)."""
import numpy as np

import synth
from oracle import dirac, masses, mg, solvers


def _hier(U, m, dims, block=(2, 2, 2, 2), N=2):
    op = mg.WilsonOp(U, m)
    P = mg.block_orthonormalise(synth.setup_starts(dims, N, 3), block)
    return solvers.Hierarchy([op, mg.galerkin(op, P, block)], [P], [block])


def test_free_field_ratio_is_one():
    """U = 1: lambda_min(D^dag D) = m^2 (the p = 0 plane wave), i.e. ratio 1."""
    dims, m = (4, 4, 4, 4), 0.3
    H = masses.shifted_hierarchy(_hier(synth.unit_gauge(dims), m, dims), m)
    lam, _ = masses.lambda_min(H, synth.gaussian_spinors(dims, 1, 1)[0])
    assert abs(lam / m ** 2 - 1.0) < 1e-6


def test_lanczos_matches_dense_smallest_eigenvalue():
    dims, m = (4, 2, 2, 4), -0.2
    U = synth.gauge_field(dims, 0.5, 4)
    D = dirac.dense_D(U, m)
    want = np.linalg.eigvalsh(np.conj(D.T) @ D).min()
    H = masses.shifted_hierarchy(_hier(U, m, dims), m)
    lam, v = masses.lambda_min(H, synth.gaussian_spinors(dims, 1, 2)[0])
    assert abs(lam - want) < 1e-6 * want


def test_sparse_coarse_matrix_matches_stencil():
    dims = (4, 4, 2, 4)
    H = _hier(synth.gauge_field(dims, 0.5, 5), 0.1, dims)
    A = H.ops[1]
    phi = synth.coarse_starts(A.dims, A.n, 1, 6)[0]
    assert np.abs(masses.stencil_sparse(A) @ phi.ravel() - A.apply(phi).ravel()).max() < 1e-13
