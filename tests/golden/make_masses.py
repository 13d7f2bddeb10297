"""Writes tests/golden/masses_*.json with the FP64 oracle only (oracle.masses).

Usage: python tests/golden/make_masses.py 16,16,16,32 0.6 11 [out.json]
The masses define the 16^3x32 workload: lambda_min(D^dag D) = r m^2 for r = 1e-3, 1e-4, 1e-5.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import masses  # noqa: E402

if __name__ == "__main__":
    dims = tuple(int(a) for a in sys.argv[1].split(","))
    eps = float(sys.argv[2])
    seed = int(sys.argv[3])
    out = sys.argv[4] if len(sys.argv) > 4 else os.path.join(
        os.path.dirname(os.path.abspath(__file__)), f"masses_{'x'.join(map(str, dims))}_eps{eps}.json")
    rec = masses.main(dims, eps, seed, [1e-3, 1e-4, 1e-5], out, m_start=float(os.environ.get("M_START", "0.0")),
                      m_step=float(os.environ.get("M_STEP", "0.2")))
    print(rec["masses"])
