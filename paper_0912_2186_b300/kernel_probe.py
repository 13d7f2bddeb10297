"""Runs the hot kernels of the solve on the 16^3x32 workload inside an NVTX range "probe", for
profiling (ncu --nvtx --nvtx-include "probe/") and quick timing.

    python -m paper_0912_2186_b300.kernel_probe [--nrhs 12] [--reps 2] [--time]

The hierarchy is built once (adaptive setup, 4^4 blocks, N = 24, FP32 cycle) before the range;
inside it each of the fine dslash (FP32, fused MR reductions off), restrict, prolong, the
tensor-core coarse stencil and the even-odd Schur complement of the coarse operator (two
parity-restricted tensor-core stencil passes and the odd-site block inverses) runs `reps` times
on nrhs right-hand sides.  --time prints CUDA-event
times per call of 50 back-to-back calls; for kernels shorter than the host's per-call cost
(Python and ctypes, some 10 us) that time is the host's, not the kernel's.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--mass", type=float, default=-1.1)
    ap.add_argument("--time", action="store_true")
    a = ap.parse_args(argv)
    import torch

    import synth
    from paper_0912_2186_b300 import build, wmg
    build.build()
    dims = (16, 16, 16, 32)
    V = 16 * 16 * 16 * 32
    U = synth.gauge_field(dims, 0.6, 11)
    ctx = wmg.Context(dims)
    ctx.load_gauge(U)
    ctx.set_mass(a.mass)
    ctx.setup(wmg.default_params(nvec=[24], prec_sloppy=wmg.PREC_SINGLE))
    nc, n = ctx.level_info(1)
    nr = a.nrhs
    g = torch.Generator(device="cuda").manual_seed(7)
    fi = torch.randn(nr * 12 * V, dtype=torch.complex64, device="cuda", generator=g)
    fo = torch.zeros_like(fi)
    ci = torch.randn(nr * nc * n, dtype=torch.complex64, device="cuda", generator=g)
    co = torch.zeros_like(ci)
    ops = {
        "dslash": lambda: ctx.apply_D(wmg.PREC_SINGLE, fi, fo, nr),
        "restrict": lambda: ctx.restrict(0, wmg.PREC_SINGLE, fi, co, nr),
        "prolong": lambda: ctx.prolong(0, wmg.PREC_SINGLE, ci, fo, nr),
        "coarse": lambda: ctx.apply_coarse(1, wmg.PREC_HALF, ci, co, nr),
        "schur": lambda: ctx.apply_coarse_schur(1, wmg.PREC_HALF, ci, co, nr),
    }
    for f in ops.values():
        f()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("probe")
    for f in ops.values():
        for _ in range(a.reps):
            f()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if a.time:
        res = {}
        for k, f in ops.items():
            reps = 50
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f()
            e1.record()
            torch.cuda.synchronize()
            res[k + "_us_per_call"] = e0.elapsed_time(e1) * 1e3 / reps
        print(json.dumps(res))
    ctx.close()
    print("ok")


if __name__ == "__main__":
    main()
