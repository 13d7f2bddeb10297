"""The continuous-batching server (wmg_server_*): resident fields of different lattice sizes,
requests with different masses and right-hand-side counts, admission into free slots while
other work is running, and each result identical alone and in the mix."""
import threading
import time

import numpy as np
import pytest

import synth
from oracle import dirac

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_2186_b300 import build, wmg
    build.build()
    return wmg


FIELDS = [dict(dims=(8, 8, 8, 8), eps=0.4, seed=11, m_setup=0.05, masses=(0.05, 0.1)),
          dict(dims=(8, 8, 8, 16), eps=0.5, seed=12, m_setup=-0.3, masses=(-0.3, -0.2))]


def _server(W, nslots=6):
    srv = W.Server(hbm_budget_bytes=64 << 30)
    Us = []
    for f in FIELDS:
        U = synth.gauge_field(f["dims"], f["eps"], f["seed"])
        ctx = W.Context(f["dims"])
        ctx.load_gauge(U)
        ctx.set_mass(f["m_setup"])
        ctx.setup(W.default_params(nvec=[8], prec_sloppy=1))
        srv.add_field(ctx, nslots)
        Us.append(U)
    return srv, Us


def _requests(n=10, seed=5):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        fi = int(rng.integers(0, len(FIELDS)))
        f = FIELDS[fi]
        m = float(f["masses"][int(rng.integers(0, 2))])
        nrhs = int(rng.integers(1, 4))
        b = synth.gaussian_spinors(f["dims"], nrhs, 100 + i)
        reqs.append((fi, m, b))
    return reqs


def test_alone_vs_mix_identical_and_correct(W):
    reqs = _requests()
    srv, Us = _server(W)
    alone = []
    for fi, m, b in reqs:               # one request at a time: nothing else in the batch
        x = np.zeros_like(b)
        st, info, lat = srv.wait(srv.submit(fi, m, b, x))
        assert st == W.OK
        alone.append(x)
    mix = [np.zeros_like(b) for _, _, b in reqs]
    tickets = []

    def producer():                      # staggered arrivals while earlier requests are solving
        rng = np.random.default_rng(9)
        for (fi, m, b), x in zip(reqs, mix):
            tickets.append(srv.submit(fi, m, b, x))
            time.sleep(float(rng.exponential(0.005)))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    lats = []
    for t in tickets:
        st, info, lat = srv.wait(t)
        assert st == W.OK and all(i["converged"] for i in info)
        lats.append(lat)
    srv.close()
    for (fi, m, b), xa, xm in zip(reqs, alone, mix):
        assert np.array_equal(xa, xm)    # bit-identical alone and in the mix
        for r in range(b.shape[0]):
            res = np.linalg.norm(b[r] - dirac.apply_D(Us[fi], xm[r], m)) / np.linalg.norm(b[r])
            assert res <= 1.05e-10
    assert len(lats) == len(reqs) and min(lats) > 0


def test_budget_admission(W):
    f = FIELDS[0]
    ctx = W.Context(f["dims"])
    ctx.load_gauge(synth.gauge_field(f["dims"], f["eps"], f["seed"]))
    ctx.setup(W.default_params(nvec=[8], prec_sloppy=1))
    srv = W.Server(hbm_budget_bytes=1 << 20)
    with pytest.raises(W.WmgError) as e:
        srv.add_field(ctx, 4)
    assert e.value.status == W.ENOMEM
    srv.close()
