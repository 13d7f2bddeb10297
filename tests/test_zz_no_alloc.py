"""The allocation-free residual entry point (wmg_residual_noalloc) against the ordinary
operator entry point wmg_apply_D and against the FP64 oracle's operator.

wmg_residual_noalloc serves callers that cannot allocate device memory during a call (an
application that owns all device memory through its own arena, or one that cannot accept
the device-wide synchronisation of cudaMalloc / cudaFree); its scratch is a fixed static
device array.  This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import synth
from oracle import dirac
from tests.gpu_util import TOL, dev, host, native_fine, rel_err

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
def test_residual_noalloc_matches_apply_D(W, prec):
    dims = (6, 4, 4, 6)                     # V = 576: a ragged last CTA
    U = synth.gauge_field(dims, 0.6, 71)
    ctx = W.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(-0.3)
    nrhs = 3
    V = ctx.V
    for call, seed in enumerate((72, 73)):  # two calls in a row share the static scratch
        xs = synth.gaussian_spinors(dims, nrhs, seed)
        bs = synth.gaussian_spinors(dims, nrhs, seed + 10)
        x, b = native_fine(V, nrhs, prec), native_fine(V, nrhs, prec)
        ctx.pack(prec, dev(xs), x, nrhs)
        ctx.pack(prec, dev(bs), b, nrhs)
        r = native_fine(V, nrhs, prec)
        n2 = torch.full((nrhs,), -1.0, dtype=torch.float64, device="cuda")
        ctx.residual_noalloc(prec, b, x, r, n2, nrhs)
        Dx = native_fine(V, nrhs, prec)
        ctx.apply_D(prec, x, Dx, nrhs)
        torch.cuda.synchronize()
        want = (b - Dx).view(nrhs, -1)
        assert rel_err(r.view(nrhs, -1).cpu().numpy(), want.cpu().numpy()) < TOL[prec], call
        want_n2 = (want.abs() ** 2).sum(dim=1).double().cpu().numpy()
        assert np.abs(n2.cpu().numpy() - want_n2).max() < TOL[prec] * want_n2.max() * 10, call
        # the oracle: r = b - D x with the FP64 definition of D (inputs as rounded on the device)
        xc, bc, rc = (dev(np.zeros_like(xs)) for _ in range(3))
        ctx.unpack(prec, x, xc, nrhs)
        ctx.unpack(prec, b, bc, nrhs)
        ctx.unpack(prec, r, rc, nrhs)
        xh, bh = host(xc), host(bc)
        ro = np.stack([bh[k] - dirac.apply_D(U, xh[k], -0.3) for k in range(nrhs)])
        assert rel_err(host(rc), ro) < TOL[prec], call
        n2o = np.array([np.vdot(ro[k], ro[k]).real for k in range(nrhs)])
        assert np.abs(n2.cpu().numpy() - n2o).max() < TOL[prec] * n2o.max() * 10, call


def test_residual_noalloc_rejects_oversize(W):
    ctx = W.Context((4, 4, 4, 4))
    ctx.load_gauge(synth.unit_gauge((4, 4, 4, 4)))
    x = native_fine(256, 65, 1)
    r = native_fine(256, 65, 1)
    n2 = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(W.WmgError) as e:
        ctx.residual_noalloc(1, x, x.clone(), r, n2, 65)
    assert e.value.status == W.EINVAL and "static" in str(e.value)
