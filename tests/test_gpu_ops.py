"""GPU parity of the operator-level kernels against the FP64 oracle, through the C ABI:
packing, the Wilson operator (Sec. 2 eq. for D), block orthonormalisation and P / P^dag
(Sec. 2), the Galerkin coarse operator and its adjoint sigma_3 D^ sigma_3 (Sec. 3)."""
import numpy as np
import pytest

import synth
from oracle import dirac, mg
from tests.gpu_util import TOL, coarse_buf, dev, host, native_fine, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_2186_b300 import build, wmg
    build.build()
    return wmg


@pytest.mark.parametrize("prec", [0, 1])
def test_pack_roundtrip(W, prec):
    dims = (6, 4, 4, 6)
    ctx = W.Context(dims)
    b = synth.gaussian_spinors(dims, 3, 1)
    nat = native_fine(ctx.V, 3, prec)
    out = dev(np.zeros_like(b))
    ctx.pack(prec, dev(b), nat, 3)
    ctx.unpack(prec, nat, out, 3)
    got = host(out)
    if prec == 0:
        assert np.array_equal(got, b)
    else:
        assert rel_err(got, b) < 1e-7


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(6, 4, 4, 6), (4, 6, 2, 10), (8, 8, 8, 8)])
def test_dslash_parity(W, prec, dims):
    """V = 576 and 480 are not multiples of the 128-site CTA (ragged tail)."""
    U = synth.gauge_field(dims, 0.6, 3)
    m = -0.27
    nrhs = 3
    b = synth.gaussian_spinors(dims, nrhs, 4)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    xin, xout = native_fine(ctx.V, nrhs, prec), native_fine(ctx.V, nrhs, prec)
    ctx.pack(prec, dev(b), xin, nrhs)
    ctx.apply_D(prec, xin, xout, nrhs)
    canon = dev(np.zeros_like(b))
    ctx.unpack(prec, xout, canon, nrhs)
    got = host(canon)
    want = np.stack([dirac.apply_D(U, b[r], m) for r in range(nrhs)])
    assert rel_err(got, want) < TOL[prec]


def _hier(W, dims, blocks, nvecs, prec, seed=10, m=-0.1, eps=0.6, tc=1, **kw):
    U = synth.gauge_field(dims, eps, seed)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    p = W.default_params(nlevels=len(blocks) + 1, block=blocks, nvec=nvecs, prec_sloppy=prec, coarse_tc=tc, **kw)
    v0 = synth.setup_starts(dims, nvecs[0], seed + 1)
    ctx.import_nullvecs(0, v0, p)
    op = mg.WilsonOp(U, m)
    P0 = mg.block_orthonormalise(v0, blocks[0])
    A1 = mg.galerkin(op, P0, blocks[0])
    out = dict(ctx=ctx, U=U, op=op, P=[P0], A=[op, A1], v=[v0])
    if len(blocks) == 2:
        v1 = synth.coarse_starts(A1.dims, A1.n, nvecs[1], seed + 2)
        ctx.import_nullvecs(1, v1.reshape(nvecs[1], -1, A1.n))
        P1 = mg.block_orthonormalise(v1, blocks[1])
        out["P"].append(P1)
        out["A"].append(mg.galerkin(A1, P1, blocks[1]))
        out["v"].append(v1)
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_two_level_operator_parity(W, prec):
    dims, blocks, nv = (8, 8, 8, 12), [(4, 4, 4, 4)], [4]
    h = _hier(W, dims, blocks, nv, prec)
    ctx, P0, A1 = h["ctx"], h["P"][0], h["A"][1]
    # P after block Gram-Schmidt (always FP64 on the device)
    Pg = ctx.export_nullvecs(0, nv[0])
    assert rel_err(Pg, P0.reshape(nv[0], -1, 12)) < 1e-12
    # Galerkin operator
    Ag = ctx.export_coarse(0)
    assert rel_err(Ag, A1.D.reshape(Ag.shape)) < TOL[prec]
    # restrict / prolong / coarse apply on 5 right-hand sides
    nrhs = 5
    psi = synth.gaussian_spinors(dims, nrhs, 30)
    V = ctx.V
    nc, n = A1.D.reshape(-1, 9, A1.n, A1.n).shape[0], A1.n
    fin = native_fine(V, nrhs, prec)
    ctx.pack(prec, dev(psi), fin, nrhs)
    co = coarse_buf(nc * n, nrhs, prec)
    ctx.restrict(0, prec, fin, co, nrhs)
    want = np.stack([mg.restrict(P0, psi[r], blocks[0]) for r in range(nrhs)])
    assert rel_err(host(co), want.reshape(nrhs, -1)) < TOL[prec]
    phi = synth.coarse_starts(A1.dims, n, nrhs, 31)
    fout = native_fine(V, nrhs, prec)
    ctx.prolong(0, prec, dev(phi.reshape(-1).astype(np.complex128 if prec == 0 else np.complex64)), fout, nrhs)
    canon = dev(np.zeros_like(psi))
    ctx.unpack(prec, fout, canon, nrhs)
    want = np.stack([mg.prolong(P0, phi[r], blocks[0]) for r in range(nrhs)])
    assert rel_err(host(canon), want) < TOL[prec]
    cdt = np.complex128 if prec == 0 else np.complex64
    for dag in (False, True):
        out = coarse_buf(nc * n, nrhs, prec)
        ctx.apply_coarse(1, prec, dev(phi.reshape(-1).astype(cdt)), out, nrhs, dagger=dag)
        f = A1.apply_dagger if dag else A1.apply
        want = np.stack([f(phi[r]) for r in range(nrhs)])
        assert rel_err(host(out), want.reshape(nrhs, -1)) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_three_level_operator_parity(W, prec):
    dims, blocks, nv = (8, 8, 8, 8), [(2, 2, 2, 2), (2, 2, 2, 2)], [3, 5]
    h = _hier(W, dims, blocks, nv, prec, seed=40)
    ctx, A1, A2, P1 = h["ctx"], h["A"][1], h["A"][2], h["P"][1]
    assert rel_err(ctx.export_nullvecs(1, nv[1]), P1.reshape(nv[1], -1, A1.n)) < 1e-12
    Ag = ctx.export_coarse(1)
    assert rel_err(Ag, A2.D.reshape(Ag.shape)) < TOL[prec]
    nrhs = 3
    cdt = np.complex128 if prec == 0 else np.complex64
    phi1 = synth.coarse_starts(A1.dims, A1.n, nrhs, 41)
    out2 = coarse_buf(A2.D.reshape(-1, 9, A2.n, A2.n).shape[0] * A2.n, nrhs, prec)
    ctx.restrict(1, prec, dev(phi1.reshape(-1).astype(cdt)), out2, nrhs)
    want = np.stack([mg.restrict(P1, phi1[r], blocks[1]) for r in range(nrhs)])
    assert rel_err(host(out2), want.reshape(nrhs, -1)) < TOL[prec]
    phi2 = synth.coarse_starts(A2.dims, A2.n, nrhs, 42)
    out1 = coarse_buf(phi1.size // nrhs, nrhs, prec)
    ctx.prolong(1, prec, dev(phi2.reshape(-1).astype(cdt)), out1, nrhs)
    want = np.stack([mg.prolong(P1, phi2[r], blocks[1]) for r in range(nrhs)])
    assert rel_err(host(out1), want.reshape(nrhs, -1)) < TOL[prec]
    out = coarse_buf(phi2.size // nrhs, nrhs, prec)
    ctx.apply_coarse(2, prec, dev(phi2.reshape(-1).astype(cdt)), out, nrhs)
    want = np.stack([A2.apply(phi2[r]) for r in range(nrhs)])
    assert rel_err(host(out), want.reshape(nrhs, -1)) < TOL[prec]


def test_mass_shift_on_coarse_levels(W):
    """set_mass after the setup shifts D^ by (m - m_setup) I (exact since P^dag P = 1)."""
    dims, blocks, nv = (8, 8, 8, 12), [(4, 4, 4, 4)], [4]
    h = _hier(W, dims, blocks, nv, 0, m=-0.1)
    ctx, A1 = h["ctx"], h["A"][1]
    ctx.set_mass(0.35)
    phi = synth.coarse_starts(A1.dims, A1.n, 2, 50)
    out = coarse_buf(phi.size // 2, 2, 0)
    ctx.apply_coarse(1, 0, dev(phi.reshape(-1)), out, 2)
    want = np.stack([A1.shifted(0.45).apply(phi[r]) for r in range(2)])
    assert rel_err(host(out), want.reshape(2, -1)) < 1e-12


@pytest.mark.parametrize("tc", [1, 2])
@pytest.mark.parametrize("dims,block,N", [((8, 8, 8, 8), (2, 2, 2, 2), 8), ((8, 8, 8, 12), (4, 4, 4, 4), 24),
                                          ((8, 8, 8, 8), (2, 2, 2, 2), 32)])
def test_tensor_core_coarse_apply(W, dims, block, N, tc):
    """FP16 tensor-core coarse stencil (2N = 16, 48, 64; tc 1 = mma.sync, 2 = tcgen05 with a TMEM
    accumulator) against the oracle, FP16 tolerance 2e-3."""
    h = _hier(W, dims, [block], [N], 1, tc=tc)
    ctx, A1 = h["ctx"], h["A"][1]
    nrhs = 13                                    # two chunks of the 16-rhs kernel, ragged
    phi = synth.coarse_starts(A1.dims, A1.n, nrhs, 60)
    for dag in (False, True):
        out = coarse_buf(phi.size // nrhs, nrhs, 1)
        ctx.apply_coarse(1, 2, dev(phi.reshape(-1).astype(np.complex64)), out, nrhs, dagger=dag)
        f = A1.apply_dagger if dag else A1.apply
        want = np.stack([f(phi[r]) for r in range(nrhs)])
        got = host(out).reshape(want.shape)
        for r in range(nrhs):                    # per right-hand side (each has its own FP16 scale)
            assert rel_err(got[r], want[r]) < 2e-3


@pytest.mark.parametrize("dims,block,N", [((8, 8, 8, 12), (4, 4, 4, 4), 24), ((6, 4, 4, 6), (2, 2, 2, 2), 8)])
def test_half_nullvec_transfers(W, dims, block, N):
    """FP16 null vectors (prec_nullvec = HALF) in restrict / prolong with FP32 vectors, against the
    FP64 oracle at the FP16 storage tolerance 2e-3, per right-hand side; 7 rhs = a ragged chunk."""
    h = _hier(W, dims, [block], [N], 1, prec_nullvec=2)
    ctx, P0, A1 = h["ctx"], h["P"][0], h["A"][1]
    nrhs = 7
    psi = synth.gaussian_spinors(dims, nrhs, 40)
    nc, n = A1.D.reshape(-1, 9, A1.n, A1.n).shape[0], A1.n
    fin = native_fine(ctx.V, nrhs, 1)
    ctx.pack(1, dev(psi), fin, nrhs)
    co = coarse_buf(nc * n, nrhs, 1)
    ctx.restrict(0, 2, fin, co, nrhs)
    got = host(co).reshape(nrhs, -1)
    for r in range(nrhs):
        assert rel_err(got[r], mg.restrict(P0, psi[r], block)) < 2e-3
    phi = synth.coarse_starts(A1.dims, n, nrhs, 41)
    fout = native_fine(ctx.V, nrhs, 1)
    ctx.prolong(0, 2, dev(phi.reshape(-1).astype(np.complex64)), fout, nrhs)
    canon = dev(np.zeros_like(psi))
    ctx.unpack(1, fout, canon, nrhs)
    got = host(canon)
    for r in range(nrhs):
        assert rel_err(got[r], mg.prolong(P0, phi[r], block)) < 2e-3


@pytest.mark.parametrize("dims", [(6, 4, 4, 6), (8, 8, 8, 8)])
def test_dslash_half_storage_parity(W, dims):
    """The smoother's FP16 storage (per-site norm, FP32 arithmetic): D applied to an FP16-rounded
    input and rounded to FP16 again, against the FP64 oracle at 2e-3 per right-hand side; a
    per-rhs amplitude spread of 1e6 checks that the per-site scaling keeps small fields exact."""
    U = synth.gauge_field(dims, 0.6, 5)
    m = -0.27
    nrhs = 3
    b = synth.gaussian_spinors(dims, nrhs, 6)
    b[1] *= 1e-6
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    xin, xout = native_fine(ctx.V, nrhs, 1), native_fine(ctx.V, nrhs, 1)
    ctx.pack(1, dev(b), xin, nrhs)
    ctx.apply_D(2, xin, xout, nrhs)
    canon = dev(np.zeros_like(b))
    ctx.unpack(1, xout, canon, nrhs)
    got = host(canon)
    for r in range(nrhs):
        assert rel_err(got[r], dirac.apply_D(U, b[r], m)) < 2e-3


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dims,block,N", [((8, 8, 8, 8), (2, 2, 2, 2), 8), ((8, 8, 8, 16), (4, 4, 4, 4), 24)])
def test_coarse_schur_apply(W, prec, dims, block, N):
    """The even-odd Schur complement S = A_ee - A_eo A_oo^-1 A_oe of the coarse operator and
    S^dag (the operator of the coarsest CG with coarse_eo) against the oracle, which forms S^dag
    from the explicit adjoint rather than through sigma_3: FP64 1e-12, FP32 1e-5, the FP16
    tensor-core stencil 2e-3 per right-hand side; odd-site outputs exactly zero; 13 right-hand
    sides (ragged chunks); at the setup mass and after a mass shift."""
    from oracle import eo
    hp = 0 if prec == 0 else 1
    h = _hier(W, dims, [block], [N], hp, tc=1)
    ctx, A1 = h["ctx"], h["A"][1]
    nrhs = 13
    phi = synth.coarse_starts(A1.dims, A1.n, nrhs, 70)
    odd = eo.parity(A1.dims) == 1
    tol = {0: 1e-12, 1: 1e-5, 2: 2e-3}[prec]
    cdt = np.complex128 if prec == 0 else np.complex64
    for shift in (0.0, 0.23):
        ctx.set_mass(-0.1 + shift)
        As = A1.shifted(shift)
        inv = eo.odd_block_inverse(As)
        for dag in (False, True):
            out = coarse_buf(phi.size // nrhs, nrhs, 0 if prec == 0 else 1)
            ctx.apply_coarse_schur(1, prec, dev(phi.reshape(-1).astype(cdt)), out, nrhs, dagger=dag)
            f = eo.schur_apply_dagger if dag else eo.schur_apply
            want = np.stack([f(As, phi[r], inv) for r in range(nrhs)])
            got = host(out).reshape(want.shape)
            for r in range(nrhs):
                assert rel_err(got[r], want[r]) < tol
                assert np.all(got[r][odd] == 0)


@pytest.mark.parametrize("reals", [8, 18])
@pytest.mark.parametrize("dims", [(6, 4, 4, 6), (8, 8, 8, 8)])
def test_dslash_link_forms_parity(W, dims, reals):
    """8-real FP32 links (Table 2's "8 floats") and uncompressed 18-real FP32 links: the FP32
    operator against the oracle at 1e-5 and the FP16-storage path at 2e-3 (V = 576 leaves a ragged
    last CTA)."""
    U = synth.gauge_field(dims, 0.6, 3)
    m, nrhs = -0.27, 3
    b = synth.gaussian_spinors(dims, nrhs, 4)
    ctx = W.Context(dims)
    ctx.set_gauge_compression(reals)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    want = np.stack([dirac.apply_D(U, b[r], m) for r in range(nrhs)])
    for prec, tol in ((1, TOL[1]), (2, 2e-3)):
        xin, xout = native_fine(ctx.V, nrhs, 1), native_fine(ctx.V, nrhs, 1)
        ctx.pack(1, dev(b), xin, nrhs)
        ctx.apply_D(prec, xin, xout, nrhs)
        canon = dev(np.zeros_like(b))
        ctx.unpack(1, xout, canon, nrhs)
        assert rel_err(host(canon), want) < tol, prec


@pytest.mark.parametrize("reals", [8, 18])
def test_link_forms_solve_and_free_field(W, reals):
    """A mixed-precision MG-GCR solve (whole-lattice and red/black) with 8- or 18-real FP32 links
    meets the 1e-10 true residual (oracle D); on the free field, which the 8-real form cannot
    represent, the 8-real operator keeps 12-real links; the 18-real one represents it exactly."""
    dims, m = (8, 8, 8, 8), 0.05
    U = synth.gauge_field(dims, 0.4, 11)
    ctx = W.Context(dims)
    ctx.set_gauge_compression(reals)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    ctx.setup(W.default_params(nvec=[8], prec_sloppy=1), synth.setup_starts(dims, 8, 12))
    b = synth.gaussian_spinors(dims, 2, 13)
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 2)
    xs = host(x)
    for r in range(2):
        assert info[r]["converged"]
        assert np.linalg.norm(b[r] - dirac.apply_D(U, xs[r], m)) / np.linalg.norm(b[r]) <= 1.05e-10
    ctx.setup(W.default_params(nvec=[8], prec_sloppy=1, fine_eo=1), synth.setup_starts(dims, 8, 12))
    x = dev(np.zeros_like(b))
    st, info = ctx.solve(dev(b), x, 2)
    xs = host(x)
    for r in range(2):
        assert info[r]["converged"]
        assert np.linalg.norm(b[r] - dirac.apply_D(U, xs[r], m)) / np.linalg.norm(b[r]) <= 1.05e-10
    ctx.load_gauge(synth.unit_gauge(dims))
    xin, xout = native_fine(ctx.V, 1, 1), native_fine(ctx.V, 1, 1)
    ctx.pack(1, dev(b[:1]), xin, 1)
    ctx.apply_D(1, xin, xout, 1)
    canon = dev(np.zeros_like(b[:1]))
    ctx.unpack(1, xout, canon, 1)
    want = dirac.apply_D(synth.unit_gauge(dims), b[0], m)
    assert rel_err(host(canon)[0], want) < TOL[1]


@pytest.mark.parametrize("prec,reals", [(0, 12), (1, 12), (1, 8), (1, 18)])
@pytest.mark.parametrize("dims", [(6, 4, 4, 6), (8, 8, 8, 8)])
def test_fine_schur_parity(W, prec, reals, dims):
    """The red/black Schur complement S = d - H_eo H_oe / d of the fine operator against the oracle
    (V / 2 = 288 leaves a ragged last CTA), FP32 with each link form; odd sites of the result are
    zero."""
    from oracle import eo_fine
    U = synth.gauge_field(dims, 0.6, 5)
    m, nrhs = -0.3, 3
    x = synth.gaussian_spinors(dims, nrhs, 6)
    ctx = W.Context(dims)
    ctx.set_gauge_compression(reals)
    ctx.load_gauge(U)
    ctx.set_mass(m)
    xin, xout = native_fine(ctx.V, nrhs, prec), native_fine(ctx.V, nrhs, prec)
    ctx.pack(prec, dev(x), xin, nrhs)
    ctx.apply_D_eo(prec, xin, xout, nrhs)
    canon = dev(np.zeros_like(x))
    ctx.unpack(prec, xout, canon, nrhs)
    even = eo_fine.parity(dims) == 0
    want = np.stack([eo_fine.schur_apply(U, x[r] * even[..., None], m) for r in range(nrhs)])
    assert rel_err(host(canon), want) < TOL[prec]
