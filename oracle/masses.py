"""Oracle: Wilson masses at which lambda_min(D(m)^dag D(m)) is a given fraction r of its
free-field value.

TEST INFRASTRUCTURE ONLY (see the package header).

The workloads are specified by the ratio r = lambda_min(D^dag D) / lambda_min^free, where
the free periodic operator at mass m has lambda_min^free = m^2 (its p = 0 mode has
eigenvalue m, from the closed form in oracle/dirac.py).  lambda_min(D^dag D) is the
largest eigenvalue of (D^dag D)^-1 = D^-1 gamma_5 D^-1 gamma_5 (gamma_5-hermiticity,
Sec. 3), found by Lanczos (scipy's ARPACK eigsh) with each D^-1 an oracle MG-GCR solve
whose coarsest level is solved by a sparse LU factorisation (an exact coarse solve; the
mass search only needs accurate D^-1, not the paper's CGNR).  The mass is located from the
heavy side (m above the critical mass) with the model sqrt(lambda_min) = s (m - m_c),
refitted from the two evaluations closest to the target (a secant step on
sqrt(lambda_min)), until the ratio is within `rtol` of r.  The hierarchy is built once near
the first target and moved to other masses by the exact coarse shift
D^(m) = D^(m0) + (m - m0) I (P^dag P = 1).

Pinned by tests/test_oracle_masses.py: on the free field lambda_min = m^2 (ratio 1), and on
a tiny lattice the Lanczos value agrees with the dense smallest eigenvalue of D^dag D.
"""
from __future__ import annotations

import json
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from . import mg, solvers


def _g5(v):
    out = v.copy()
    out[..., 6:] *= -1.0
    return out


def stencil_sparse(A):
    """The coarse stencil operator as a scipy CSC matrix (rows site*n + i, columns nb*n + j)."""
    X, Y, Z, T = A.dims
    V, n = X * Y * Z * T, A.n
    Df = A.D.reshape(V, mg.NSLOT, n, n)
    v = np.arange(V)
    crd = [v % X, (v // X) % Y, (v // (X * Y)) % Z, v // (X * Y * Z)]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rows, cols, vals = [], [], []
    for k in range(mg.NSLOT):
        c = [a.copy() for a in crd]
        if k > 0:
            mu, sg = (k - 1) // 2, (1 if (k - 1) % 2 == 0 else -1)
            c[mu] = (c[mu] + sg) % (X, Y, Z, T)[mu]
        nb = c[0] + X * (c[1] + Y * (c[2] + Z * c[3]))
        rows.append((v[:, None, None] * n + ii[None]).ravel())
        cols.append((nb[:, None, None] * n + jj[None]).ravel())
        vals.append(Df[:, k].ravel())
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(V * n, V * n))


def direct_coarse_solver(A):
    """Exact coarsest solve by sparse LU (used by the mass search only)."""
    lu = sla.splu(stencil_sparse(A))
    return lambda _A, b: lu.solve(b.ravel()).reshape(b.shape)


def shifted_hierarchy(H, m):
    """The hierarchy H (built at some mass m0) moved to mass m by the exact diagonal shift."""
    op0 = H.ops[0]
    dm = m - op0.m
    ops = [mg.WilsonOp(op0.U, m)] + [A.shifted(dm) for A in H.ops[1:]]
    Hm = solvers.Hierarchy(ops, H.P, H.blocks, H.params)
    Hm.coarse_solver = direct_coarse_solver(ops[-1])
    return Hm


def lambda_min(H, v0, tol=1e-10, eig_tol=1e-3, log=None):
    """Smallest eigenvalue of D^dag D (D = H.ops[0]) and its eigenvector, by Lanczos on
    (D^dag D)^-1 applied with MG-GCR solves."""
    shape = v0.shape
    nsolve = [0]

    def matvec(x):
        v = x.reshape(shape)
        y, _ = solvers.mg_solve(H, _g5(v), tol)
        w, _ = solvers.mg_solve(H, _g5(y), tol)
        nsolve[0] += 2
        return w.ravel()

    n = v0.size
    Op = sla.LinearOperator((n, n), matvec=matvec, dtype=np.complex128)
    vals, vecs = sla.eigsh(Op, k=1, which="LA", v0=v0.ravel(), tol=eig_tol, ncv=12)
    lam = 1.0 / float(vals[0])
    if log:
        log(f"    Lanczos: lambda_min = {lam:.6e} ({nsolve[0]} MG solves)")
    return lam, vecs[:, 0].reshape(shape)


def find_masses(U, ratios, block=(4, 4, 4, 4), nvec=24, m_start=0.0, m_step=0.2, seed=7, rtol=0.05,
                setup_passes=5, log=print, max_evals=12):
    """Masses m (heavier than critical) with lambda_min(D^dag D) = r m^2 for each r in ratios."""
    from synth import gaussian_spinors, setup_starts

    T, Z, Y, X = U.shape[:4]
    dims = (X, Y, Z, T)
    v = gaussian_spinors(dims, 1, seed + 100)[0]
    evals = []  # (m, lambda)
    H = None

    def build(m):
        t = time.time()
        op = mg.WilsonOp(U, m)
        starts = setup_starts(dims, nvec, seed)
        P, Ac, _ = solvers.setup_level(op, block, starts, passes=setup_passes,
                                       coarse_solver_factory=direct_coarse_solver)
        log(f"  setup at m = {m:.6f}: {time.time() - t:.1f} s")
        return solvers.Hierarchy([op, Ac], [P], [block])

    def evaluate(m):
        nonlocal v
        t = time.time()
        lam, v = lambda_min(shifted_hierarchy(H, m), v, log=log)
        evals.append((m, lam))
        log(f"  m = {m:.6f}: lambda_min = {lam:.6e}, ratio = {lam / m ** 2:.4e} ({time.time() - t:.1f} s)")
        return lam

    H = build(m_start)
    evaluate(m_start)
    evaluate(m_start - m_step)
    out = {}
    for r in sorted(ratios, reverse=True):
        for _ in range(max_evals):
            close = [e for e in evals if abs(e[1] / e[0] ** 2 - r) <= rtol * r]
            if close:
                out[r] = close[0][0]
                break
            (m1, l1), (m2, l2) = sorted(evals, key=lambda e: abs(np.log(e[1] / e[0] ** 2 / r)))[:2]
            s = (np.sqrt(l1) - np.sqrt(l2)) / (m1 - m2)
            mc = m1 - np.sqrt(l1) / s
            # sqrt(r) |m| = s (m - m_c) on the heavy side of m_c
            cands = [c for c in (s * mc / (s - np.sqrt(r)), s * mc / (s + np.sqrt(r))) if c > mc]
            evaluate(min(cands, key=lambda c: abs(c - m1)))
        else:
            raise RuntimeError(f"mass search for ratio {r} did not converge: {evals}")
    return out, evals


# ---- staged search (one process builds the hierarchy, evaluations and the per-ratio secant
# searches run in parallel processes sharing it through files) ----

def build_hierarchy(U, m, block=(4, 4, 4, 4), nvec=24, seed=7, setup_passes=3, log=print):
    """Adaptive 2-level hierarchy at mass m for the search's MG solves (its quality only affects
    the solves' speed, not the eigenvalues); setup passes use the oracle's CGNR coarse solve."""
    from synth import setup_starts

    T, Z, Y, X = U.shape[:4]
    dims = (X, Y, Z, T)
    t = time.time()
    op = mg.WilsonOp(U, m)
    P, Ac, _ = solvers.setup_level(op, block, setup_starts(dims, nvec, seed), passes=setup_passes,
                                   params=solvers.CycleParams(coarse_tol=1e-4))
    log(f"  setup at m = {m:.6f}: {time.time() - t:.1f} s")
    return solvers.Hierarchy([op, Ac], [P], [block])


def save_hierarchy(path, H):
    np.savez(path, P=H.P[0], D=H.ops[1].D, m=H.ops[0].m, block=np.array(H.blocks[0]))


def load_hierarchy(path, U):
    z = np.load(path)
    op = mg.WilsonOp(U, float(z["m"]))
    return solvers.Hierarchy([op, mg.StencilOp(z["D"])], [z["P"]], [tuple(int(b) for b in z["block"])])


def evaluate(H, m, v0, solve_tol=1e-5, eig_tol=1e-2, log=print):
    """(lambda_min(D(m)^dag D(m)), its eigenvector) with H moved to mass m.  The ratio is needed
    to 5 %: MG solves to a relative residual of 1e-5 put the eigenvalue within ~1e-3 of its
    exact value (solution error <= 1e-5 times the condition number of D, ~1e2 here)."""
    t = time.time()
    lam, v = lambda_min(shifted_hierarchy(H, m), v0, tol=solve_tol, eig_tol=eig_tol, log=log)
    log(f"  m = {m:.6f}: lambda_min = {lam:.6e}, ratio = {lam / m ** 2:.4e} ({time.time() - t:.1f} s)")
    return lam, v


def next_mass(evals, r):
    """Secant step on sqrt(lambda_min) = s (m - m_c) through the two evaluations nearest ratio r,
    heavy side of m_c."""
    (m1, l1), (m2, l2) = sorted(evals, key=lambda e: abs(np.log(e[1] / e[0] ** 2 / r)))[:2]
    s = (np.sqrt(l1) - np.sqrt(l2)) / (m1 - m2)
    mc = m1 - np.sqrt(l1) / s
    cands = [c for c in (s * mc / (s - np.sqrt(r)), s * mc / (s + np.sqrt(r))) if c > mc]
    return min(cands, key=lambda c: abs(c - m1))


def search_ratio(H, r, evals, v0, rtol=0.05, max_evals=8, log=print, on_eval=None):
    """Mass with lambda_min = r m^2 within rtol, starting from evals [(m, lambda)]."""
    evals = list(evals)
    v = v0
    for _ in range(max_evals):
        close = [e for e in evals if abs(e[1] / e[0] ** 2 - r) <= rtol * r]
        if close:
            return close[0][0], evals
        m = next_mass(evals, r)
        lam, v = evaluate(H, m, v, log=log)
        evals.append((m, lam))
        if on_eval:
            on_eval(m, lam)
    raise RuntimeError(f"mass search for ratio {r} did not converge: {evals}")


def main(dims, eps, gauge_seed, ratios, out_path, **kw):
    from synth import gauge_field

    U = gauge_field(dims, eps, gauge_seed)
    t = time.time()
    masses, evals = find_masses(U, ratios, **kw)
    rec = {
        "dims": list(dims), "eps": eps, "gauge_seed": gauge_seed,
        "definition": "lambda_min(D^dag D) = ratio * m^2 (free-field lambda_min at mass m)",
        "masses": {f"{r:.0e}": m for r, m in masses.items()},
        "evaluations": [[m, lam, lam / m ** 2] for m, lam in evals],
        "oracle_seconds": time.time() - t,
    }
    with open(out_path, "w") as f:
        json.dump(rec, f, indent=1)
    return rec
