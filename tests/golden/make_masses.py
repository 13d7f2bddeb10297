"""Writes tests/golden/masses_*.json with the FP64 oracle only (oracle.masses).

The masses define the 16^3x32 workload: lambda_min(D^dag D) = r m^2 for r = 1e-3, 1e-4, 1e-5.
Single process:
    python tests/golden/make_masses.py 16,16,16,32 0.6 11 [out.json]
Staged (the evaluations and the three searches run as parallel processes sharing a stage
directory; each stage writes its results there):
    python tests/golden/make_masses.py --stage setup  --m 1.42- ...   (see --help)
"""
import argparse
import glob
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import masses  # noqa: E402
from synth import gauge_field, gaussian_spinors  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
RATIOS = [1e-3, 1e-4, 1e-5]


def default_out(dims, eps):
    return os.path.join(HERE, f"masses_{'x'.join(map(str, dims))}_eps{eps}.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("dims")
    ap.add_argument("eps", type=float)
    ap.add_argument("seed", type=int)
    ap.add_argument("out", nargs="?", default=None)
    ap.add_argument("--stage", choices=["all", "setup", "eval", "search", "merge"], default="all")
    ap.add_argument("--dir", default=os.path.join(HERE, ".masses_stage"), help="stage directory")
    ap.add_argument("--m", type=float, help="mass of the setup / of an evaluation")
    ap.add_argument("--ratio", type=float, help="target ratio of a search")
    ap.add_argument("--rtol", type=float, default=0.05, help="accepted relative error of the ratio (search)")
    a = ap.parse_args()
    dims = tuple(int(v) for v in a.dims.split(","))
    out = a.out or default_out(dims, a.eps)
    if a.stage == "all":
        rec = masses.main(dims, a.eps, a.seed, RATIOS, out, m_start=float(os.environ.get("M_START", "0.0")),
                          m_step=float(os.environ.get("M_STEP", "0.2")))
        print(rec["masses"])
        return
    os.makedirs(a.dir, exist_ok=True)
    U = gauge_field(dims, a.eps, a.seed)
    hfile = os.path.join(a.dir, "hierarchy.npz")
    log = lambda s: print(s, flush=True)  # noqa: E731
    if a.stage == "setup":
        masses.save_hierarchy(hfile, masses.build_hierarchy(U, a.m, log=log))
        return
    if a.stage == "merge":
        found = {}
        for f in sorted(glob.glob(os.path.join(a.dir, "found_*.json"))):
            with open(f) as fh:
                found.update(json.load(fh))
        evals = []
        for f in sorted(glob.glob(os.path.join(a.dir, "eval_*.json"))):
            with open(f) as fh:
                evals.append(json.load(fh))
        ratios_found = {}
        for k, m in found.items():
            lam = [e["lambda"] for e in evals if e["m"] == m]
            ratios_found[k] = lam[0] / m ** 2 if lam else None
        rec = {"dims": list(dims), "eps": a.eps, "gauge_seed": a.seed,
               "definition": "lambda_min(D^dag D) = ratio * m^2 (free-field lambda_min at mass m)",
               "masses": {k: found[k] for k in sorted(found, key=float, reverse=True)},
               "ratio_at_mass": {k: ratios_found[k] for k in sorted(found, key=float, reverse=True)},
               "evaluations": sorted([[e["m"], e["lambda"], e["lambda"] / e["m"] ** 2] for e in evals]),
               "method": "oracle MG-GCR solves (tol 1e-5) inside Lanczos on (D^dag D)^-1 (eig tol 1e-2); "
                         "secant on sqrt(lambda_min); the ratio reached at each mass is in ratio_at_mass"}
        with open(out, "w") as fh:
            json.dump(rec, fh, indent=1)
        print(rec["masses"])
        return
    H = masses.load_hierarchy(hfile, U)
    v0 = gaussian_spinors(dims, 1, a.seed + 100)[0]

    def save_eval(m, lam):
        with open(os.path.join(a.dir, f"eval_{m:.8f}.json"), "w") as fh:
            json.dump({"m": m, "lambda": lam}, fh)

    if a.stage == "eval":
        lam, _ = masses.evaluate(H, a.m, v0, log=log)
        save_eval(a.m, lam)
        return
    # search one ratio from every evaluation so far
    evals = []
    for f in glob.glob(os.path.join(a.dir, "eval_*.json")):
        with open(f) as fh:
            e = json.load(fh)
        evals.append((e["m"], e["lambda"]))
    t = time.time()
    m, _ = masses.search_ratio(H, a.ratio, evals, v0, rtol=a.rtol, log=log, on_eval=save_eval)
    with open(os.path.join(a.dir, f"found_{a.ratio:.0e}.json"), "w") as fh:
        json.dump({f"{a.ratio:.0e}": m}, fh)
    log(f"ratio {a.ratio:.0e}: m = {m:.6f} ({time.time() - t:.0f} s)")


if __name__ == "__main__":
    main()
