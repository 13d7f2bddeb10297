"""GPU MG-GCR solves (Sec. 3) through the C ABI, checked by the FP64 oracle: every solution
has |b - D x| / |b| <= 1e-10 with D applied by the oracle; the solve is independent of the
other right-hand sides of its batch; the hierarchy built from oracle vectors gives the
oracle's iteration count."""
import numpy as np
import pytest

import synth
from oracle import dirac, mg, solvers
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_2186_b300 import build, wmg
    build.build()
    return wmg


def oracle_resid(U, m, b, x):
    return np.linalg.norm(b - dirac.apply_D(U, x, m)) / np.linalg.norm(b)


CFG1 = dict(dims=(8, 8, 8, 8), eps=0.4, m=0.05, N=8)


def _ctx(W, cfg, prec, seed=11, setup=True, **kw):
    U = synth.gauge_field(cfg["dims"], cfg["eps"], seed)
    ctx = W.Context(cfg["dims"])
    ctx.load_gauge(U)
    ctx.set_mass(cfg["m"])
    p = W.default_params(nvec=[cfg["N"]], prec_sloppy=prec, **kw)
    if setup:
        ctx.setup(p, synth.setup_starts(cfg["dims"], cfg["N"], seed + 1))
    return ctx, U, p


@pytest.mark.parametrize("prec", [0, 1])
def test_mg_solve_true_residual(W, prec):
    ctx, U, p = _ctx(W, CFG1, prec)
    b = synth.gaussian_spinors(CFG1["dims"], 2, 13)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 2)
    xs = host(x)
    for r in range(2):
        assert info[r]["converged"] and info[r]["true_resid"] <= 1e-10
        assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10
        assert info[r]["iters"] < 60


def test_host_solve_and_plain_solver(W):
    ctx, U, p = _ctx(W, CFG1, 1)
    b = synth.gaussian_spinors(CFG1["dims"], 1, 14)
    x = np.zeros_like(b)
    st, info = ctx.solve(b, x, 1)
    assert oracle_resid(U, CFG1["m"], b[0], x[0]) <= 1.05e-10
    xp = dev(np.zeros_like(b))
    st, pinfo = ctx.solve(dev(b), xp, 1, plain=True)
    assert oracle_resid(U, CFG1["m"], b[0], host(xp)[0]) <= 1.05e-10
    assert pinfo[0]["iters"] > 2 * info[0]["iters"]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_independence(W, prec):
    """Each right-hand side gives bit-identical results alone and inside a batch."""
    ctx, U, p = _ctx(W, CFG1, prec)
    b = synth.gaussian_spinors(CFG1["dims"], 3, 15)
    b[2] *= 1e-3                      # very different scales in one batch
    xb = dev(np.zeros_like(b))
    _, ib = ctx.solve(dev(b), xb, 3)
    xb = host(xb)
    for r in (0, 1, 2):
        x1 = dev(np.zeros_like(b[r:r + 1]))
        _, i1 = ctx.solve(dev(b[r:r + 1]), x1, 1)
        assert np.array_equal(host(x1)[0], xb[r])
        assert i1[0]["iters"] == ib[r]["iters"]


def test_iterations_match_oracle_with_shared_vectors(W):
    """FP64 hierarchy from the oracle's own near-null vectors: same iteration count (+-1)."""
    cfg = dict(dims=(8, 8, 8, 8), eps=0.5, m=-0.2, N=6)
    ctx, U, p = _ctx(W, cfg, 0, seed=21, setup=False, coarse_tol=1e-8)
    v = synth.setup_starts(cfg["dims"], cfg["N"], 22)
    op = mg.WilsonOp(U, cfg["m"])
    v = np.array([solvers._normalise(solvers.mr(op.apply, np.zeros_like(s), s, 20)) for s in v])
    ctx.import_nullvecs(0, v.reshape(cfg["N"], -1, 12), p)
    H = solvers.hierarchy_from_vectors(op, [(4, 4, 4, 4)], [v], solvers.CycleParams(coarse_tol=1e-8))
    b = synth.gaussian_spinors(cfg["dims"], 1, 23)
    xo, io = solvers.mg_solve(H, b[0], 1e-10, 16)
    x = dev(np.zeros_like(b))
    _, info = ctx.solve(dev(b), x, 1)
    assert abs(info[0]["iters"] - io.iters) <= 1
    assert oracle_resid(U, cfg["m"], b[0], host(x)[0]) <= 1.05e-10


def test_three_level_solve(W):
    cfg = dict(dims=(8, 8, 8, 16), eps=0.5, m=0.0)
    U = synth.gauge_field(cfg["dims"], cfg["eps"], 31)
    ctx = W.Context(cfg["dims"])
    ctx.load_gauge(U)
    ctx.set_mass(cfg["m"])
    p = W.default_params(nlevels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 8], prec_sloppy=1)
    ctx.setup(p, synth.setup_starts(cfg["dims"], 6, 32))
    b = synth.gaussian_spinors(cfg["dims"], 2, 33)
    x = dev(np.zeros_like(b))
    _, info = ctx.solve(dev(b), x, 2)
    xs = host(x)
    for r in range(2):
        assert oracle_resid(U, cfg["m"], b[r], xs[r]) <= 1.05e-10


def test_tcgen05_coarse_solve(W):
    """The mixed-precision solve with the coarse stencil on tcgen05 tensor cores (plain coarsest
    CGNR: the even-odd passes use the mma.sync stencil)."""
    ctx, U, p = _ctx(W, CFG1, 1, coarse_tc=2, coarse_eo=0)
    b = synth.gaussian_spinors(CFG1["dims"], 3, 16)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 3)
    xs = host(x)
    for r in range(3):
        assert info[r]["converged"]
        assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10


def test_half_nullvec_solve(W):
    """FP16 null vectors in the cycle: every solution still meets the FP64 true residual 1e-10."""
    ctx, U, p = _ctx(W, CFG1, 1, prec_nullvec=2)
    b = synth.gaussian_spinors(CFG1["dims"], 3, 17)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 3)
    xs = host(x)
    for r in range(3):
        assert info[r]["converged"]
        assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10


def test_half_storage_three_level_solve(W):
    """The reduced-precision configuration on a small lattice: 3 levels, FP16 smoother storage,
    FP16 null vectors, tensor-core coarse stencils, 12 Gaussian right-hand sides; every solution
    meets the FP64 true residual 1e-10 (oracle D) and the batch result equals the single solve."""
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.7, 35)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(-0.05)
    p = W.default_params(nlevels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[8, 8], prec_sloppy=1,
                         prec_smoother=2, prec_nullvec=2, coarse_tc=1)
    ctx.setup(p, synth.setup_starts(dims, 8, 36))
    b = synth.gaussian_spinors(dims, 12, 37)
    x = dev(np.zeros_like(b))
    _, info = ctx.solve(dev(b), x, 12)
    xs = host(x)
    for r in range(12):
        assert info[r]["converged"]
        assert oracle_resid(U, -0.05, b[r], xs[r]) <= 1.05e-10
    x1 = dev(np.zeros_like(b[5:6]))
    _, i1 = ctx.solve(dev(b[5:6]), x1, 1)
    assert np.array_equal(host(x1)[0], xs[5]) and i1[0]["iters"] == info[5]["iters"]


def _big_solve(W, dims, eps, mass, params, nrhs, seed):
    from oracle import cref
    U = synth.gauge_field(dims, eps, seed)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(mass)
    ctx.setup(params)
    ctx.bytes_after_setup = ctx.device_bytes()
    b = synth.gaussian_spinors(dims, nrhs, seed + 1)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, nrhs)
    xs = host(x)
    res = []
    for r in range(nrhs):
        assert info[r]["converged"]
        res.append(np.linalg.norm(b[r] - cref.apply_D(U, xs[r], mass)) / np.linalg.norm(b[r]))
    return ctx, info, res


@pytest.mark.slow
def test_24x24x24x48_three_level_half_storage(W):
    """The 24^3x48 workload at full size: epsilon = 0.7, 3 levels (4^4 then 2^4 blocks, N = 24 and
    32), FP16 per-site-norm smoother storage, tensor-core coarse stencils, 12 Gaussian right-hand
    sides in one batch; every true residual (oracle C operator) <= 1e-10."""
    p = W.default_params(nlevels=3, block=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[24, 32], prec_sloppy=1,
                         prec_smoother=2, coarse_tc=1)
    ctx, info, res = _big_solve(W, (24, 24, 24, 48), 0.7, -1.2, p, 12, 31)
    assert max(res) <= 1.05e-10
    ctx.close()


@pytest.mark.slow
def test_48x48x48x96_memory_and_residual(W):
    """The 48^3x96 workload at full size: 3 levels (N = 24 / 32), FP16 null vectors in the cycle,
    FP32 12-real links, 4 right-hand sides; every true residual (oracle C operator) <= 1e-10, and
    the context's device footprint is reported: after the setup (links, FP16 fine null vectors,
    coarse operators, level-2 transfer) and after the solve (plus FP64 solution and residual and
    the FP32 flexible-GCR basis of 2 x 16 vectors per right-hand side); it fits one B300."""
    p = W.default_params(nlevels=3, block=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[24, 32], prec_sloppy=1,
                         prec_nullvec=2, prec_smoother=2, coarse_tc=1)
    ctx, info, res = _big_solve(W, (48, 48, 48, 96), 0.7, -1.2, p, 4, 51)
    assert max(res) <= 1.05e-10
    gb_setup, gb = ctx.bytes_after_setup / 1e9, ctx.device_bytes() / 1e9
    print(f"48^3x96 context device footprint: {gb_setup:.1f} GB after the setup, {gb:.1f} GB after the "
          f"4-rhs solve; iterations {[i['iters'] for i in info]}; max true residual {max(res):.2e}")
    assert gb < 250
    ctx.close()


def test_autotuned_coarse_stencil(W):
    """coarse_tc = 3: the setup times the CUDA-core, mma.sync and tcgen05 stencils of the coarse
    level and keeps the fastest; the solve with that choice meets the 1e-10 true residual."""
    ctx, U, p = _ctx(W, CFG1, 1, coarse_tc=3)
    impl, ms = ctx.coarse_impl(1)
    assert impl in (0, 1, 2) and all(t > 0 for t in ms)
    assert ms[impl] == min(ms)
    b = synth.gaussian_spinors(CFG1["dims"], 2, 18)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 2)
    xs = host(x)
    for r in range(2):
        assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10


def test_persistent_coarse_cgnr(W):
    """coarse_persistent = 1 (with the plain CGNR, coarse_eo = 0): the coarsest CGNR as one
    cooperative kernel; every solution meets the 1e-10 true residual, and a right-hand side's
    result is the same alone and in its batch."""
    ctx, U, p = _ctx(W, CFG1, 1, coarse_persistent=1, coarse_eo=0)
    b = synth.gaussian_spinors(CFG1["dims"], 3, 19)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 3)
    xs = host(x)
    for r in range(3):
        assert info[r]["converged"]
        assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10
    x1 = dev(np.zeros_like(b[1:2]))
    _, i1 = ctx.solve(dev(b[1:2]), x1, 1)
    assert np.array_equal(host(x1)[0], xs[1]) and i1[0]["iters"] == info[1]["iters"]


@pytest.mark.parametrize("prec", [0, 1])
def test_even_odd_coarsest_solve(W, prec):
    """coarse_eo = 1 (default) and 0 on the same hierarchy: both meet the 1e-10 true residual
    (oracle D) with iteration counts within 2 of each other; the even-odd batch result equals the
    single solve."""
    its = {}
    for flag in (1, 0):
        ctx, U, p = _ctx(W, CFG1, prec, coarse_eo=flag)
        b = synth.gaussian_spinors(CFG1["dims"], 3, 24)
        x = dev(np.zeros_like(b))
        st, info = ctx.solve(dev(b), x, 3)
        xs = host(x)
        for r in range(3):
            assert info[r]["converged"]
            assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10
        its[flag] = [i["iters"] for i in info]
        if flag:
            x1 = dev(np.zeros_like(b[2:3]))
            _, i1 = ctx.solve(dev(b[2:3]), x1, 1)
            assert np.array_equal(host(x1)[0], xs[2]) and i1[0]["iters"] == info[2]["iters"]
    assert all(abs(a - b) <= 2 for a, b in zip(its[0], its[1]))


def test_cgnr_fine_baseline(W):
    """The unpreconditioned baseline: FP64 CG on the fine normal equations meets the 1e-10 true
    residual with the oracle's operator, takes the oracle CGNR's iteration count to within 2 % (+2),
    and many more iterations than MG-GCR."""
    ctx, U, p = _ctx(W, CFG1, 0)
    b = synth.gaussian_spinors(CFG1["dims"], 2, 19)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve_cgnr(dev(b), x, 2)
    xs = host(x)
    op = mg.WilsonOp(U, CFG1["m"])
    for r in range(2):
        assert info[r]["converged"]
        assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10
    _, it_o = solvers.cgnr(op, b[0], 1e-10, 100000)
    assert abs(info[0]["iters"] - it_o) <= 2 + 0.02 * it_o, (info[0]["iters"], it_o)
    xm = dev(np.zeros_like(b))
    _, im = ctx.solve(dev(b), xm, 2)
    assert info[0]["iters"] > 5 * im[0]["iters"]


def test_gauge_update_keeps_subspace_and_refresh(W):
    """Setup amortisation across gauge updates: after a small step of the field (links times
    exp(0.02 i H)), the kept subspace with rebuilt coarse operators still solves to 1e-10 (oracle
    operator of the new field), the coarse operator equals the oracle's Galerkin product of the
    new field with the kept vectors (FP64, 1e-12), and one refresh pass brings the iteration count
    to within 10 % (+2) of a full setup on the new field, at a fraction of its cost."""
    import time
    cfg = dict(dims=(8, 8, 8, 16), eps=0.5, m=-0.3, N=8)
    dims, m = cfg["dims"], cfg["m"]
    U = synth.gauge_field(dims, cfg["eps"], 41)
    U2 = synth.evolved_gauge(U, 0.02, 42)
    b = synth.gaussian_spinors(dims, 3, 43)
    # operator-level: oracle vectors, FP64, new field's Galerkin product
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    p64 = W.default_params(nvec=[cfg["N"]], prec_sloppy=0)
    v = synth.setup_starts(dims, cfg["N"], 44)
    ctx.import_nullvecs(0, v, p64)
    ctx.update_gauge(U2)
    A2 = mg.galerkin(mg.WilsonOp(U2, m), mg.block_orthonormalise(v, (4, 4, 4, 4)), (4, 4, 4, 4))
    Ag = ctx.export_coarse(0)
    assert np.abs(Ag - A2.D.reshape(Ag.shape)).max() < 1e-12 * np.abs(A2.D).max()
    ctx.close()

    def solve(ctx):
        x = dev(np.zeros_like(b))
        st, info = ctx.solve(dev(b), x, 3)
        xs = host(x)
        for r in range(3):
            assert info[r]["converged"]
            assert oracle_resid(U2, m, b[r], xs[r]) <= 1.05e-10
        return float(np.mean([i["iters"] for i in info]))

    p = W.default_params(nvec=[cfg["N"]], prec_sloppy=1)
    full = W.Context(dims)
    full.load_gauge(U2)
    full.set_mass(m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full.setup(p)
    t_full = time.perf_counter() - t0
    it_full = solve(full)
    kept = W.Context(dims)
    kept.load_gauge(U)
    kept.set_mass(m)
    kept.setup(p)
    kept.update_gauge(U2)
    it_kept = solve(kept)
    t0 = time.perf_counter()
    kept.refresh_setup(1)
    t_ref = time.perf_counter() - t0
    it_ref = solve(kept)
    print(f"iterations: full setup {it_full}, kept subspace {it_kept}, after one refresh pass {it_ref}; "
          f"setup {t_full:.3f} s, refresh {t_ref:.3f} s")
    assert it_ref <= 1.1 * it_full + 2
    assert t_ref < t_full


@pytest.mark.parametrize("prec", [0, 1])
def test_fine_even_odd_solve(W, prec):
    """fine_eo = 1 (red/black preconditioning of the fine solve): every solution meets the 1e-10
    true residual of the whole system with the oracle's operator, in a number of iterations close
    to the whole-lattice solve's, and a right-hand side's result is the same alone and in its batch."""
    its = {}
    for flag in (0, 1):
        ctx, U, p = _ctx(W, CFG1, prec, fine_eo=flag)
        b = synth.gaussian_spinors(CFG1["dims"], 3, 27)
        x = dev(np.zeros_like(b))
        st, info = ctx.solve(dev(b), x, 3)
        xs = host(x)
        for r in range(3):
            assert info[r]["converged"]
            assert oracle_resid(U, CFG1["m"], b[r], xs[r]) <= 1.05e-10
        its[flag] = [i["iters"] for i in info]
        if flag:
            x1 = dev(np.zeros_like(b[1:2]))
            _, i1 = ctx.solve(dev(b[1:2]), x1, 1)
            assert np.array_equal(host(x1)[0], xs[1]) and i1[0]["iters"] == info[1]["iters"]
    print(f"outer iterations whole lattice {its[0]}, red/black {its[1]}")
    assert all(b <= 1.3 * a + 2 for a, b in zip(its[0], its[1]))


def test_coarse_cg_graph_and_host_loop_identical(W, monkeypatch):
    """The coarsest CG as a CUDA graph with a WHILE node and as the host-driven loop (a context
    created with WMG_NO_GRAPHS=1, the form the instrumented benchmark step and the ncu launch lists
    use) launch the same kernels in the same order, programmatic launches included: the solutions
    are bit-identical and meet the 1e-10 true residual (oracle D)."""
    b = synth.gaussian_spinors(CFG1["dims"], 3, 31)
    xs, its = {}, {}
    for flag in ("0", "1"):
        monkeypatch.setenv("WMG_NO_GRAPHS", flag)
        ctx, U, p = _ctx(W, CFG1, 1, fine_eo=1)
        x = dev(np.zeros_like(b))
        st, info = ctx.solve(dev(b), x, 3)
        xs[flag] = host(x)
        its[flag] = [i["iters"] for i in info]
        for r in range(3):
            assert info[r]["converged"]
            assert oracle_resid(U, CFG1["m"], b[r], xs[flag][r]) <= 1.05e-10
        ctx.close()
    assert its["0"] == its["1"]
    assert np.array_equal(xs["0"], xs["1"])


@pytest.mark.parametrize("gamma", [1, 2])
def test_three_level_red_black_solve(W, gamma):
    """3 levels (V- and W-cycle) with the red/black fine solve and the FP32 smoother, where the cycle
    reads the half-lattice residual (restriction from the even sites, the smoother's first residual
    with b on the even sites) and its smoother defers the solution updates: every solution meets
    the 1e-10 true residual (oracle D) in about as many outer iterations as the whole-lattice
    solve, and a right-hand side's result is the same alone and in its batch."""
    dims, m = (8, 8, 8, 16), 0.0
    U = synth.gauge_field(dims, 0.5, 91)
    b = synth.gaussian_spinors(dims, 3, 92)
    its = {}
    for eo in (0, 1):
        ctx = W.Context(dims)
        ctx.load_gauge(U)
        ctx.set_mass(m)
        p = W.default_params(nlevels=3, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[6, 8], prec_sloppy=1,
                             cycle_gamma=gamma, fine_eo=eo)
        ctx.setup(p, synth.setup_starts(dims, 6, 93))
        x = dev(np.zeros_like(b))
        _, info = ctx.solve(dev(b), x, 3)
        xs = host(x)
        for r in range(3):
            assert info[r]["converged"]
            assert oracle_resid(U, m, b[r], xs[r]) <= 1.05e-10
        its[eo] = [i["iters"] for i in info]
        if eo:
            x1 = dev(np.zeros_like(b[2:3]))
            _, i1 = ctx.solve(dev(b[2:3]), x1, 1)
            assert np.array_equal(host(x1)[0], xs[2]) and i1[0]["iters"] == info[2]["iters"]
        ctx.close()
    print(f"outer iterations whole lattice {its[0]}, red/black {its[1]}")
    assert all(e <= 1.3 * w + 2 for w, e in zip(its[0], its[1]))
