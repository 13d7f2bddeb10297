"""GPU-against-oracle parity of the adaptive setup (Sec. 2), the multigrid cycle and its
smoother (Sec. 3), and of the transfer and Galerkin kernels at the instantiations the 16^3x32
workload runs (N = 24, 12 right-hand sides), through the C ABI.

* Setup: both sides run the same fixed-N adaptive setup in FP64 from the same starts with a
  tight coarsest solve; the near-null spaces must agree per (block, chirality) up to a largest
  principal angle below 1e-6, and the MG-GCR iteration counts of the two hierarchies within 1.
* Cycle: one application of K (2 levels, V; 3 levels, V and W) on a hierarchy built from the
  oracle's vectors, element by element against the oracle's cycle with an exact coarsest solve.
* Smoother: nu MR steps (the FP32 dslash with fused sums) against the oracle's MR.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import cref, dirac, mg, solvers
from tests.gpu_util import TOL, coarse_buf, dev, host, native_fine, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_2186_b300 import build, wmg
    build.build()
    return wmg


def max_block_angle_sine(Pa, Pb, block):
    """Largest sin(principal angle) between the spans of Pa and Pb over all (block, chirality):
    |(1 - B B^dag) A|_2 for the orthonormal block bases A of Pa and B of Pb."""
    N = Pa.shape[0]
    A = np.stack([mg.to_blocks(p, block) for p in Pa])  # (N, Vc, bs, 12)
    B = np.stack([mg.to_blocks(p, block) for p in Pb])
    worst = 0.0
    for s in range(2):
        a = A[..., 6 * s:6 * s + 6].reshape(N, A.shape[1], -1).transpose(1, 2, 0)
        b = B[..., 6 * s:6 * s + 6].reshape(N, B.shape[1], -1).transpose(1, 2, 0)
        resid = a - b @ (np.conj(b).transpose(0, 2, 1) @ a)
        worst = max(worst, float(np.linalg.norm(resid, ord=2, axis=(1, 2)).max()))
    return worst


def oracle_resid(U, m, b, x):
    return np.linalg.norm(b - cref.apply_D(U, x, m)) / np.linalg.norm(b)


def test_setup_matches_oracle_setup(W):
    """The 8^4 workload (epsilon 0.4, m = 0.05, N = 8, 4^4 blocks, 5 passes, 20 relaxation steps,
    MR nu = 4) in FP64 from shared starts, coarsest solves to 1e-12 on both sides (the even-odd
    CG on the GPU and in the oracle)."""
    dims, eps, m, N, block = (8, 8, 8, 8), 0.4, 0.05, 8, (4, 4, 4, 4)
    U = synth.gauge_field(dims, eps, 11)
    starts = synth.setup_starts(dims, N, 12)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    p = W.default_params(nvec=[N], prec_sloppy=W.PREC_DOUBLE, coarse_tol=1e-12, coarse_maxit=20000, setup_relax=20)
    ctx.setup(p, starts)
    Pg = ctx.export_nullvecs(0, N).reshape((N,) + starts.shape[1:])
    op = mg.WilsonOp(U, m)
    prm = solvers.CycleParams(coarse_tol=1e-12, coarse_maxit=20000, coarse_eo=True)
    Po, Ao, _ = solvers.setup_level(op, block, starts, passes=p.setup_passes, relax=p.setup_relax, params=prm)
    sine = max_block_angle_sine(Pg, Po, block)
    assert sine < 1e-6, sine
    b = synth.gaussian_spinors(dims, 1, 13)
    x = dev(np.zeros_like(b))
    _, info = ctx.solve(dev(b), x, 1)
    H = solvers.Hierarchy([op, Ao], [Po], [block], prm)
    xo, io = solvers.mg_solve(H, b[0], 1e-10, 16)
    assert abs(info[0]["iters"] - io.iters) <= 1, (info[0]["iters"], io.iters)
    assert oracle_resid(U, m, b[0], host(x)[0]) <= 1.05e-10


def _exact(A, b):
    return np.linalg.solve(A.dense(), b.ravel()).reshape(b.shape)


def _hierarchy(W, dims, eps, m, blocks, nvecs, prec, seed, **kw):
    """The same hierarchy on both sides: the oracle's starts, imported into the GPU context (which
    orthonormalises them and builds its coarse operators) and built by the oracle."""
    U = synth.gauge_field(dims, eps, seed)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    p = W.default_params(nlevels=len(blocks) + 1, block=blocks, nvec=nvecs, prec_sloppy=prec, **kw)
    v0 = synth.setup_starts(dims, nvecs[0], seed + 1)
    ctx.import_nullvecs(0, v0, p)
    vecs = [v0]
    if len(blocks) == 2:
        A1 = mg.galerkin(mg.WilsonOp(U, m), mg.block_orthonormalise(v0, blocks[0]), blocks[0])
        v1 = synth.coarse_starts(A1.dims, A1.n, nvecs[1], seed + 2)
        ctx.import_nullvecs(1, v1.reshape(nvecs[1], -1, A1.n))
        vecs.append(v1)
    op = mg.WilsonOp(U, m)
    gamma = kw.get("cycle_gamma", 1)
    H = solvers.hierarchy_from_vectors(op, blocks, vecs, solvers.CycleParams(nu=4, gamma=gamma))
    H.coarse_solver = _exact
    return ctx, U, H


@pytest.mark.parametrize("case", [
    dict(dims=(8, 8, 8, 8), eps=0.4, m=0.05, blocks=[(4, 4, 4, 4)], nvecs=[8], gamma=1),
    dict(dims=(8, 8, 8, 16), eps=0.5, m=0.0, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[4, 6], gamma=1),
    dict(dims=(8, 8, 8, 16), eps=0.5, m=0.0, blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[4, 6], gamma=2),
], ids=["2lvl-V", "3lvl-V", "3lvl-W"])
def test_cycle_matches_oracle(W, case):
    """One FP64 cycle application K(r) on 3 right-hand sides, element by element against the
    oracle's cycle (exact coarsest solve; the GPU's coarsest CG runs to 1e-13): relative to the
    largest entry within 1e-9."""
    ctx, U, H = _hierarchy(W, case["dims"], case["eps"], case["m"], case["blocks"], case["nvecs"], 0, 60,
                           coarse_tol=1e-13, coarse_maxit=50000, cycle_gamma=case["gamma"])
    nrhs = 3
    r = synth.gaussian_spinors(case["dims"], nrhs, 61)
    V = ctx.V
    rin, eout = native_fine(V, nrhs, 0), native_fine(V, nrhs, 0)
    ctx.pack(0, dev(r), rin, nrhs)
    ctx.apply_cycle(0, rin, eout, nrhs)
    canon = dev(np.zeros_like(r))
    ctx.unpack(0, eout, canon, nrhs)
    got = host(canon)
    want = np.stack([solvers.cycle(H, 0, r[k]) for k in range(nrhs)])
    err = rel_err(got, want)
    assert err < 1e-9, err


def test_cycle_single_precision_matches_oracle(W):
    """The FP32 cycle (FP32 operators, mma.sync FP16 coarse stencil off: coarse_tc = 0, coarsest CG
    to 1e-6) against the oracle's FP64 cycle with an exact coarsest solve, relative to the largest
    entry: within 1e-4 (FP32 rounding through a 1e-6 coarse solve and 4 smoothing steps)."""
    case = dict(dims=(8, 8, 8, 8), eps=0.4, m=0.05, blocks=[(4, 4, 4, 4)], nvecs=[8])
    ctx, U, H = _hierarchy(W, case["dims"], case["eps"], case["m"], case["blocks"], case["nvecs"], 1, 62,
                           coarse_tol=1e-6, coarse_maxit=50000, coarse_tc=0)
    nrhs = 3
    r = synth.gaussian_spinors(case["dims"], nrhs, 63)
    V = ctx.V
    rin, eout = native_fine(V, nrhs, 1), native_fine(V, nrhs, 1)
    ctx.pack(1, dev(r), rin, nrhs)
    ctx.apply_cycle(1, rin, eout, nrhs)
    canon = dev(np.zeros_like(r))
    ctx.unpack(1, eout, canon, nrhs)
    want = np.stack([solvers.cycle(H, 0, r[k]) for k in range(nrhs)])
    err = rel_err(host(canon), want)
    assert err < 1e-4, err


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(6, 4, 4, 10), (8, 8, 8, 16)])
def test_smoother_matches_oracle_mr(W, prec, dims, fused, monkeypatch):
    """nu = 4 MR steps on D x = b from a random guess, 12 right-hand sides (the FP32 dslash with
    fused <q, r>, |q|^2 sums over 4 site blocks per CTA; fused = 1: each later step fused with the
    previous step's update, WMG_MR_FUSE=1); V = 960 leaves a ragged last CTA."""
    m = -0.4
    U = synth.gauge_field(dims, 0.6, 64)
    monkeypatch.setenv("WMG_MR_FUSE", str(fused))
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    nrhs = 12
    b = synth.gaussian_spinors(dims, nrhs, 65)
    x0 = synth.gaussian_spinors(dims, nrhs, 66)
    bn, xn = native_fine(ctx.V, nrhs, prec), native_fine(ctx.V, nrhs, prec)
    ctx.pack(prec, dev(b), bn, nrhs)
    ctx.pack(prec, dev(x0), xn, nrhs)
    ctx.smooth(prec, bn, xn, nrhs, 4)
    canon = dev(np.zeros_like(b))
    ctx.unpack(prec, xn, canon, nrhs)
    got = host(canon)
    want = np.stack([solvers.mr(lambda v: dirac.apply_D(U, v, m), b[k], x0[k], 4) for k in range(nrhs)])
    assert rel_err(got, want) < TOL[prec]


def test_galerkin_and_transfers_at_workload_instantiation(W):
    """N = 24 on 4^4 blocks, 12 right-hand sides, FP32: the fused Galerkin kernel's coarse operator,
    restrict and prolong (the kernel instantiations of the 16^3x32 workload) on 8^3x16 against the
    oracle at 1e-5."""
    dims, blocks, N, m, nrhs = (8, 8, 8, 16), [(4, 4, 4, 4)], 24, -0.3, 12
    U = synth.gauge_field(dims, 0.6, 70)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    p = W.default_params(nvec=[N], block=blocks, prec_sloppy=W.PREC_SINGLE)
    v = synth.setup_starts(dims, N, 71)
    ctx.import_nullvecs(0, v, p)
    P = mg.block_orthonormalise(v, blocks[0])
    A = mg.galerkin(mg.WilsonOp(U, m), P, blocks[0])
    Ag = ctx.export_coarse(0)
    assert rel_err(Ag, A.D.reshape(Ag.shape)) < TOL[1]
    _transfers_against_oracle(ctx, P, blocks[0], dims, A.dims, 2 * N, nrhs, 72)


def _transfers_against_oracle(ctx, P, block, dims, cdims, n, nrhs, seed):
    V = ctx.V
    psi = synth.gaussian_spinors(dims, nrhs, seed)
    fin = native_fine(V, nrhs, 1)
    ctx.pack(1, dev(psi), fin, nrhs)
    nc = int(np.prod(cdims))
    co = coarse_buf(nc * n, nrhs, 1)
    ctx.restrict(0, 1, fin, co, nrhs)
    want = np.stack([mg.restrict(P, psi[r], block) for r in range(nrhs)])
    assert rel_err(host(co), want.reshape(nrhs, -1)) < TOL[1]
    phi = synth.coarse_starts(cdims, n, nrhs, seed + 1)
    fout = native_fine(V, nrhs, 1)
    ctx.prolong(0, 1, dev(phi.reshape(-1).astype(np.complex64)), fout, nrhs)
    canon = dev(np.zeros_like(psi))
    ctx.unpack(1, fout, canon, nrhs)
    want = np.stack([mg.prolong(P, phi[r], block) for r in range(nrhs)])
    assert rel_err(host(canon), want) < TOL[1]


WORKLOAD = dict(dims=(16, 16, 16, 32), eps=0.6, gauge_seed=11, N=24, block=(4, 4, 4, 4), nrhs=12,
                masses=os.path.join(ROOT, "tests", "golden", "masses_16x16x16x32_eps0.6.json"))


@pytest.mark.slow
def test_workload_transfers_and_smoother_full_size(W):
    """At the full 16^3x32 size in the launch configuration of the benchmark (N = 24, 12 rhs,
    FP32): restrict and prolong on the oracle's block-orthonormal vectors, and the 4-step MR
    smoother, element by element against the oracle at 1e-5."""
    w = WORKLOAD
    dims, N, blk, nrhs = w["dims"], w["N"], w["block"], w["nrhs"]
    U = synth.gauge_field(dims, w["eps"], w["gauge_seed"])
    m = -1.5
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    v = synth.setup_starts(dims, N, 80)
    ctx.import_nullvecs(0, v, W.default_params(nvec=[N], block=[blk], prec_sloppy=W.PREC_SINGLE))
    P = mg.block_orthonormalise(v, blk)
    _transfers_against_oracle(ctx, P, blk, dims, mg.coarse_dims(dims, blk), 2 * N, nrhs, 81)
    b = synth.gaussian_spinors(dims, nrhs, 82)
    x0 = synth.gaussian_spinors(dims, nrhs, 83)
    bn, xn = native_fine(ctx.V, nrhs, 1), native_fine(ctx.V, nrhs, 1)
    ctx.pack(1, dev(b), bn, nrhs)
    ctx.pack(1, dev(x0), xn, nrhs)
    ctx.smooth(1, bn, xn, nrhs, 4)
    canon = dev(np.zeros_like(b))
    ctx.unpack(1, xn, canon, nrhs)
    want = np.stack([solvers.mr(lambda q: cref.apply_D(U, q, m), b[k], x0[k], 4) for k in range(nrhs)])
    assert rel_err(host(canon), want) < TOL[1]


@pytest.mark.slow
def test_workload_job_true_residuals(W):
    """The benchmark's job at full size: adaptive setup (device starts, N = 24, 5 passes) at the
    lightest of the oracle's three masses, then the 12 point sources at each mass; every solution's
    true residual |b - D x| / |b| computed with the oracle's C operator is <= 1e-10."""
    w = WORKLOAD
    dims = w["dims"]
    with open(w["masses"]) as f:
        masses = sorted(json.load(f)["masses"].values(), reverse=True)
    U = synth.gauge_field(dims, w["eps"], w["gauge_seed"])
    b = synth.point_sources(dims, w["nrhs"])
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(masses[-1])
    ctx.setup(W.default_params(nvec=[w["N"]], block=[w["block"]], prec_sloppy=W.PREC_SINGLE))
    worst, its = 0.0, []
    for m in masses:
        ctx.set_mass(m)
        x = dev(np.zeros_like(b))
        st, info = ctx.solve(dev(b), x, w["nrhs"])
        xs = host(x)
        its.append(float(np.mean([i["iters"] for i in info])))
        for r in range(w["nrhs"]):
            assert info[r]["converged"]
            worst = max(worst, oracle_resid(U, m, b[r], xs[r]))
    print(f"16^3x32 job: mean outer iterations per mass {its}, largest oracle residual {worst:.3e}")
    assert worst <= 1.05e-10


def test_w_cycle_three_level_solve(W):
    """The W-cycle (cycle_gamma = 2 at the middle level, Sec. 3's cycle) in a 3-level FP32 solve:
    every solution meets the 1e-10 true residual with the oracle's operator."""
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 84)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(0.0)
    p = W.default_params(nlevels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 8], prec_sloppy=1, cycle_gamma=2)
    ctx.setup(p, synth.setup_starts(dims, 6, 85))
    b = synth.gaussian_spinors(dims, 3, 86)
    x = dev(np.zeros_like(b))
    _, info = ctx.solve(dev(b), x, 3)
    xs = host(x)
    for r in range(3):
        assert info[r]["converged"]
        assert oracle_resid(U, 0.0, b[r], xs[r]) <= 1.05e-10
