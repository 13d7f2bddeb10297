"""ctypes access to oracle/c/dirac_ref.c, the plain C restatement of Sec. 2's Wilson operator.

TEST INFRASTRUCTURE ONLY.  Built by build() (gcc -O2 -fopenmp) into oracle/c/libdirac_ref.so.
Pinned by tests/test_oracle_dirac.py against the numpy definition in oracle/dirac.py and the
closed forms there.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c")
SRC = os.path.join(HERE, "dirac_ref.c")
LIB = os.path.join(HERE, "libdirac_ref.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", SRC, "-o", LIB])
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        # numpy's BLAS pool and this OpenMP pool share the cores: do not let idle threads spin
        os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
        L = ctypes.CDLL(LIB)
        vp = ctypes.c_void_p
        L.dirac_ref_apply.argtypes = [vp, vp, vp, vp, ctypes.c_double]
        L.dirac_ref_hop.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib = L
    return _lib


def _dims(U):
    T, Z, Y, X = U.shape[:4]
    return np.array([X, Y, Z, T], dtype=np.int32)


def apply_D(U, psi, m):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    d = _dims(U)
    lib().dirac_ref_apply(U.ctypes.data, psi.ctypes.data, out.ctypes.data, d.ctypes.data, float(m))
    return out


def hop(U, psi, mu, sign):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    d = _dims(U)
    lib().dirac_ref_hop(U.ctypes.data, psi.ctypes.data, out.ctypes.data, d.ctypes.data, int(mu), int(sign), 0)
    return out
