"""Oracle: smoother, coarsest solve, multigrid cycle, outer GCR and adaptive setup.

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 3 fixes the outline: a multigrid cycle with post-smoothing only (4 steps), a
Krylov GCR outer solver on the finest level, and CG on the normal equations as a
complete solve on the coarsest level.  Sec. 2 fixes the adaptive setup outline
(relax D psi = 0 from random starts, build a trial hierarchy, use it to improve
the vectors, repeat).  The details the paper leaves open are read as follows:

* MR(A, b, x0, nu): r = b - A x0; nu times: q = A r; alpha = <q,r>/<q,q>;
  x += alpha r; r -= alpha q  (stops early if q = 0).  <a,b> = sum conj(a) b.
* CGNR(A, b, tol, maxit) on A^dag A x = A^dag b (CGLS form): x = 0, r = b, z = A^dag r,
  p = z; loop: q = A p; alpha = |z|^2/|q|^2; x += alpha p; r -= alpha q;
  z' = A^dag r; beta = |z'|^2/|z|^2; p = z' + beta p; stop when |r| <= tol |b|.
  Optionally (CycleParams.coarse_eo) the same CG on the even-odd Schur complement of the
  coarsest operator (oracle/eo.py), with the same stopping test on the whole system.
* Cycle K_l(r): at the coarsest level CGNR(A_l, r); otherwise e = 0 and gamma times
  { r_c = P^dag (r - A e); e += P K_{l+1}(r_c); e = MR(A, r, e, nu) }.
  gamma = 1 is the V-cycle, gamma = 2 at intermediate levels the W-cycle.
* FGCR(m): x = 0, r = b; per cycle of m: z_k = K(r), w_k = A z_k, modified
  Gram-Schmidt of w_k against w_j (z_k updated alongside), normalise, alpha =
  <w_k, r>, x += alpha z_k, r -= alpha w_k; break on |r| <= tol |b|; then the true
  residual r = b - A x decides whether to restart.  "Iterations" counts K calls
  (Table 1's fine-grid iteration count).
* Adaptive setup (fixed N): pass 1 relaxes each random start with `relax` MR steps
  on A psi = 0 and normalises; every later pass uses the trial hierarchy built
  from the current vectors to solve again: psi_k <- K(psi_k) (one cycle as an
  approximate solve of A psi_new = psi_k, i.e. inverse iteration), normalised; P
  and D^ are rebuilt after each pass.  (Applying the cycle to the homogeneous
  equation instead, psi_k + K(-A psi_k), returns zero for a vector that already
  lies in span(P) when the coarse solve is exact, so a fixed set cannot be
  improved that way.)  Three levels: finish level 1, then the same procedure on
  A_2 = D^ with its own starts and a 2-level cycle.

Pins (tests/test_oracle_solvers.py): MR residual non-increasing and one-step exact
for A = I; CGNR against a dense solve; FGCR with the exact inverse as
preconditioner converges in one iteration, residual norms non-increasing, solution
against dense LU; the full MG-GCR solution against dense LU on a tiny lattice; the
cycle (2 levels with nu = 0, 1, 2, 4; 3 levels, V and W) against its dense closed form
with an exact coarsest solve (the Petrov-Galerkin correction P (P^dag D P)^-1 P^dag r,
then nu minimal-residual steps each solved as a one-column least-squares problem); the
adaptive setup against a dense restatement built from library routines (least-squares
relaxation steps, Gram-Schmidt as the QR factorisation with a positive diagonal, the
dense cycle), which a different relax count, smoothing count or per-vector rebuild of
the basis fails.  Near-null vectors have no closed form: the setup is pinned as an
algorithm, not by its result.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import eo, mg


def dot(a, b):
    return np.vdot(a, b)


def norm(a):
    return float(np.linalg.norm(a))


def mr(apply, b, x0, nu):
    """Minimal-residual smoother (nu steps)."""
    x = x0.copy()
    r = b - apply(x)
    for _ in range(nu):
        q = apply(r)
        qq = dot(q, q).real
        if qq == 0.0:
            break
        alpha = dot(q, r) / qq
        x = x + alpha * r
        r = r - alpha * q
    return x


def cgnr(op, b, tol, maxit):
    """CG on the normal equations A^dag A x = A^dag b. Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = norm(b)
    if bn == 0.0:
        return x, 0
    z = op.apply_dagger(r)
    p = z.copy()
    zz = dot(z, z).real
    it = 0
    while it < maxit and norm(r) > tol * bn:
        q = op.apply(p)
        alpha = zz / dot(q, q).real
        x = x + alpha * p
        r = r - alpha * q
        z = op.apply_dagger(r)
        zz_new = dot(z, z).real
        beta = zz_new / zz
        zz = zz_new
        p = z + beta * p
        it += 1
    return x, it


@dataclass
class CycleParams:
    nu: int = 4                 # post-smoothing MR steps (Sec. 3: 4 post smoothing iterations)
    gamma: int = 1              # 1 = V-cycle, 2 = W-cycle at intermediate levels
    coarse_tol: float = 1e-8    # CGNR relative tolerance on the coarsest level
    coarse_maxit: int = 5000
    coarse_eo: bool = False     # CGNR on the even-odd Schur complement (oracle/eo.py) instead


@dataclass
class Hierarchy:
    ops: list                   # A_0 (fine), A_1, ... ; A_{l+1} = P_l^dag A_l P_l
    P: list                     # P_0, P_1, ... (orthonormalised block vectors)
    blocks: list                # block shape used to coarsen level l
    params: CycleParams = field(default_factory=CycleParams)
    coarse_iters: list = field(default_factory=list)
    coarse_solver: object = None   # optional callable(A, b) replacing CGNR on the coarsest level

    @property
    def nlevels(self):
        return len(self.ops)


def cycle(H, level, r):
    """K_level(r): the multigrid preconditioner (post-smoothing only)."""
    p = H.params
    A = H.ops[level]
    if level == H.nlevels - 1:
        if H.coarse_solver is not None:
            return H.coarse_solver(A, r)
        solve = eo.cgnr_eo if p.coarse_eo else cgnr
        x, it = solve(A, r, p.coarse_tol, p.coarse_maxit)
        H.coarse_iters.append(it)
        return x
    P, blk = H.P[level], H.blocks[level]
    e = np.zeros_like(r)
    reps = 1 if level == 0 else p.gamma
    for rep in range(reps):
        rr = r if rep == 0 else r - A.apply(e)
        rc = mg.restrict(P, rr, blk)
        ec = cycle(H, level + 1, rc)
        e = e + mg.prolong(P, ec, blk)
        e = mr(A.apply, r, e, p.nu)
    return e


@dataclass
class SolveInfo:
    iters: int = 0
    restarts: int = 0
    true_resid: float = np.inf
    history: list = field(default_factory=list)


def fgcr(apply, precond, b, tol=1e-10, restart=16, max_iter=1000):
    """Flexible GCR(restart) with right preconditioner precond. Returns (x, SolveInfo)."""
    info = SolveInfo()
    bn = norm(b)
    x = np.zeros_like(b)
    if bn == 0.0:
        info.true_resid = 0.0
        return x, info
    r = b.copy()
    while info.iters < max_iter:
        Z, W = [], []
        for k in range(restart):
            z = precond(r)
            w = apply(z)
            info.iters += 1
            for j in range(k):
                beta = dot(W[j], w)
                w = w - beta * W[j]
                z = z - beta * Z[j]
            nw = norm(w)
            w = w / nw
            z = z / nw
            alpha = dot(w, r)
            x = x + alpha * z
            r = r - alpha * w
            Z.append(z)
            W.append(w)
            info.history.append(norm(r) / bn)
            if norm(r) <= tol * bn or info.iters >= max_iter:
                break
        r = b - apply(x)
        info.true_resid = norm(r) / bn
        if info.true_resid <= tol:
            break
        info.restarts += 1
    return x, info


def mg_solve(H, b, tol=1e-10, restart=16, max_iter=1000):
    """MG-GCR: flexible GCR on the finest level preconditioned by the cycle."""
    A = H.ops[0]
    return fgcr(A.apply, lambda r: cycle(H, 0, r), b, tol, restart, max_iter)


def _normalise(v):
    return v / norm(v)


def setup_level(op, block, starts, passes=5, relax=20, params=None, history=None, coarse_solver_factory=None):
    """Adaptive near-null vectors for one level (2-level cycle on op).

    Returns (P, coarse StencilOp, final vectors).  `history`, if a list, receives per
    pass the mean of |op psi_k| / |psi_k| over k before P is rebuilt.
    """
    params = params or CycleParams()
    psi = np.array([_normalise(mr(op.apply, np.zeros_like(s), s, relax)) for s in starts])

    def record():
        if history is not None:
            history.append(float(np.mean([norm(op.apply(v)) / norm(v) for v in psi])))

    record()
    P = mg.block_orthonormalise(psi, block)
    Ac = mg.galerkin(op, P, block)
    for _ in range(passes - 1):
        H = Hierarchy([op, Ac], [P], [block], params)
        if coarse_solver_factory is not None:
            H.coarse_solver = coarse_solver_factory(Ac)
        new = []
        for v in psi:
            new.append(_normalise(cycle(H, 0, v)))
        psi = np.array(new)
        record()
        P = mg.block_orthonormalise(psi, block)
        Ac = mg.galerkin(op, P, block)
    return P, Ac, psi


def adaptive_setup(op, blocks, starts_per_level, passes=5, relax=20, params=None):
    """Build a hierarchy with len(blocks)+1 levels, level by level (Sec. 2 adaptive setup)."""
    params = params or CycleParams()
    ops, Ps = [op], []
    cur = op
    for blk, starts in zip(blocks, starts_per_level):
        P, Ac, _ = setup_level(cur, blk, starts, passes, relax, params)
        Ps.append(P)
        ops.append(Ac)
        cur = Ac
    return Hierarchy(ops, Ps, list(blocks), params)


def hierarchy_from_vectors(op, blocks, vectors_per_level, params=None):
    """Hierarchy from given (already final) near-null vectors, one set per level."""
    params = params or CycleParams()
    ops, Ps = [op], []
    cur = op
    for blk, vecs in zip(blocks, vectors_per_level):
        P = mg.block_orthonormalise(vecs, blk)
        Ac = mg.galerkin(cur, P, blk)
        Ps.append(P)
        ops.append(Ac)
        cur = Ac
    return Hierarchy(ops, Ps, list(blocks), params)
