"""Oracle: Wilson masses at which lambda_min(D(m)^dag D(m)) is a given fraction r of its
free-field value.

TEST INFRASTRUCTURE ONLY (see the package header).

The workloads are specified by the ratio r = lambda_min(D^dag D) / lambda_min^free, where
the free periodic operator at mass m has lambda_min^free = m^2 (its p = 0 mode has
eigenvalue m, from the closed form in oracle/dirac.py).  lambda_min(D^dag D) is found by
inverse iteration, v <- (D^dag D)^-1 v = D^-1 gamma_5 D^-1 gamma_5 v (gamma_5-hermiticity,
Sec. 3), with each D^-1 an oracle MG-GCR solve; the mass is then located from the heavy
side (m above the critical mass) with the model sqrt(lambda_min) = s (m - m_c), refitted
from the two most recent evaluations (a secant step on sqrt(lambda_min)), until the ratio
is within `rtol` of r.  The hierarchy is built once near the target and moved to other
masses by the exact coarse shift D^(m) = D^(m0) + (m - m0) I (P^dag P = 1).

Pinned by tests/test_oracle_masses.py: on the free field the finder reproduces
lambda_min = m^2 (ratio 1), and on a tiny lattice inverse iteration agrees with the dense
smallest eigenvalue of D^dag D.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import mg, solvers


def _g5(v):
    out = v.copy()
    out[..., 6:] *= -1.0
    return out


def shifted_hierarchy(H, m):
    """The hierarchy H (built at some mass m0) moved to mass m by the exact diagonal shift."""
    op0 = H.ops[0]
    dm = m - op0.m
    ops = [mg.WilsonOp(op0.U, m)] + [A.shifted(dm) for A in H.ops[1:]]
    return solvers.Hierarchy(ops, H.P, H.blocks, H.params)


def lambda_min(H, v0, tol=1e-8, rel=1e-4, max_steps=12, log=None):
    """Smallest eigenvalue of D^dag D (D = H.ops[0]) by inverse iteration with MG-GCR solves.
    Returns (lambda, eigenvector estimate)."""
    D = H.ops[0]
    v = v0 / solvers.norm(v0)
    lam_old = np.inf
    lam = np.inf
    for step in range(max_steps):
        y, _ = solvers.mg_solve(H, _g5(v), tol)
        w, _ = solvers.mg_solve(H, _g5(y), tol)
        v = w / solvers.norm(w)
        Dv = D.apply(v)
        lam = float(np.vdot(Dv, Dv).real)
        if log:
            log(f"    inverse iteration {step}: lambda = {lam:.6e}")
        if abs(lam_old - lam) <= rel * lam:
            break
        lam_old = lam
    return lam, v


def find_masses(U, ratios, block=(4, 4, 4, 4), nvec=24, m_start=0.0, m_step=0.2, seed=7, rtol=0.05,
                setup_passes=5, coarse_tol=1e-6, log=print, max_evals=12):
    """Masses m (heavier than critical) with lambda_min(D^dag D) = r m^2 for each r in ratios."""
    from synth import gaussian_spinors, setup_starts

    T, Z, Y, X = U.shape[:4]
    dims = (X, Y, Z, T)
    params = solvers.CycleParams(coarse_tol=coarse_tol)
    v = gaussian_spinors(dims, 1, seed + 100)[0]
    evals = []  # (m, lambda)
    H = None

    def build(m):
        t = time.time()
        op = mg.WilsonOp(U, m)
        starts = setup_starts(dims, nvec, seed)
        Hn = solvers.adaptive_setup(op, [block], [starts], passes=setup_passes, params=params)
        log(f"  setup at m = {m:.6f}: {time.time() - t:.1f} s")
        return Hn

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
    rebuilt = False
    out = {}
    for r in sorted(ratios, reverse=True):
        for _ in range(max_evals):
            (m1, l1), (m2, l2) = sorted(evals, key=lambda e: abs(e[1] / e[0] ** 2 - r) / r)[:2]
            s = (np.sqrt(l1) - np.sqrt(l2)) / (m1 - m2)
            mc = m1 - np.sqrt(l1) / s
            # sqrt(r) |m| = s (m - m_c), m on the heavy side of m_c
            cands = [s * mc / (s - np.sqrt(r)), s * mc / (s + np.sqrt(r))]
            cands = [c for c in cands if c > mc]
            m = min(cands, key=lambda c: abs(c - m1))
            close = [e for e in evals if abs(e[1] / e[0] ** 2 - r) <= rtol * r]
            if close:
                out[r] = close[0][0]
                break
            if not rebuilt and r == max(ratios):
                pass
            if not rebuilt and abs(m - mc) < 0.05:
                H = build(m)
                rebuilt = True
            evaluate(m)
        else:
            raise RuntimeError(f"mass search for ratio {r} did not converge: {evals}")
    return out, evals


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
