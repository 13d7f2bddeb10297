"""Thin ctypes binding of libwmg's C ABI (include/wmg.h): argument marshalling only.

Every step of the solve runs in the CUDA kernels of libwmg.so.  Device buffers are passed as
torch CUDA tensors (their data pointers); host buffers as numpy arrays.  The library must be
built (``paper_0912_2186_b300.build.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwmg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wmg.h")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ERANK, ETIMEOUT, ESTATE = range(8)
PREC_DOUBLE, PREC_SINGLE, PREC_HALF = 0, 1, 2
MAX_LEVELS = 3


class WmgError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(what)
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("nlevels", ctypes.c_int),
        ("block", (ctypes.c_int * 4) * (MAX_LEVELS - 1)),
        ("nvec", ctypes.c_int * (MAX_LEVELS - 1)),
        ("setup_passes", ctypes.c_int),
        ("setup_relax", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("gcr_restart", ctypes.c_int),
        ("cycle_gamma", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("coarse_tol", ctypes.c_double),
        ("coarse_maxit", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("prec_sloppy", ctypes.c_int),
        ("coarse_tc", ctypes.c_int),
        ("reliable_delta", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("prec_nullvec", ctypes.c_int),
        ("prec_smoother", ctypes.c_int),
        ("coarse_persistent", ctypes.c_int),
        ("coarse_eo", ctypes.c_int),
        ("fine_eo", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("pad_", ctypes.c_int),
        ("true_resid", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


_lib = None


def load():
    """Load libwmg.so (fails loudly if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libwmg.so not built ({LIB_PATH}); run paper_0912_2186_b300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "wmg_default_params": (None, [P(Params)]),
        "wmg_strerror": (ctypes.c_char_p, [i]),
        "wmg_last_error": (ctypes.c_char_p, [vp]),
        "wmg_create": (i, [P(vp), P(ctypes.c_int * 4), vp]),
        "wmg_destroy": (i, [vp]),
        "wmg_load_gauge": (i, [vp, vp]),
        "wmg_load_gauge_dev": (i, [vp, vp]),
        "wmg_set_mass": (i, [vp, d]),
        "wmg_set_gauge_compression": (i, [vp, i]),
        "wmg_setup": (i, [vp, P(Params), vp]),
        "wmg_import_nullvecs": (i, [vp, P(Params), i, vp]),
        "wmg_update_gauge": (i, [vp, vp]),
        "wmg_update_gauge_dev": (i, [vp, vp]),
        "wmg_refresh_setup": (i, [vp, i]),
        "wmg_export_nullvecs": (i, [vp, i, vp]),
        "wmg_export_coarse": (i, [vp, i, vp]),
        "wmg_level_info": (i, [vp, i, P(i), P(i)]),
        "wmg_device_bytes": (i, [vp, P(ctypes.c_size_t)]),
        "wmg_coarse_impl": (i, [vp, i, P(i), P(ctypes.c_float)]),
        "wmg_solve": (i, [vp, vp, vp, i, P(Info)]),
        "wmg_solve_dev": (i, [vp, vp, vp, i, P(Info)]),
        "wmg_solve_plain_dev": (i, [vp, vp, vp, i, P(Info)]),
        "wmg_solve_cgnr_dev": (i, [vp, vp, vp, i, i, P(Info)]),
        "wmg_pack_spinor": (i, [vp, i, vp, vp, i]),
        "wmg_unpack_spinor": (i, [vp, i, vp, vp, i]),
        "wmg_apply_D": (i, [vp, i, vp, vp, i]),
        "wmg_apply_cycle": (i, [vp, i, vp, vp, i]),
        "wmg_apply_D_eo": (i, [vp, i, vp, vp, i]),
        "wmg_smooth": (i, [vp, i, vp, vp, i, i]),
        "wmg_restrict": (i, [vp, i, i, vp, vp, i]),
        "wmg_prolong": (i, [vp, i, i, vp, vp, i]),
        "wmg_apply_coarse": (i, [vp, i, i, i, vp, vp, i]),
        "wmg_apply_coarse_schur": (i, [vp, i, i, i, vp, vp, i]),
        "wmg_residual_noalloc": (i, [vp, i, vp, vp, vp, vp, i]),
        "wmg_server_create": (i, [P(vp), ctypes.c_size_t]),
        "wmg_server_add_field": (i, [vp, vp, i, P(i)]),
        "wmg_server_submit": (i, [vp, i, d, vp, vp, i, P(ctypes.c_longlong)]),
        "wmg_server_poll": (i, [vp, ctypes.c_longlong, P(i)]),
        "wmg_server_wait": (i, [vp, ctypes.c_longlong, P(Info), P(d)]),
        "wmg_server_destroy": (i, [vp]),
        "wmg_profile_enable": (i, [vp, i]),
        "wmg_launch_count": (i, [P(ctypes.c_longlong)]),
        "wmg_probe_alu_peaks": (i, [P(d), P(d)]),
        "wmg_profile_get": (i, [vp, i, P(d), P(ctypes.c_longlong), P(d), P(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_symbols(header=HEADER):
    """Names of the functions include/wmg.h declares."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(wmg_[a-z_0-9]+)\s*\(", txt)))


def default_params(**kw):
    p = Params()
    load().wmg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "block":
            for l, blk in enumerate(v):
                for j in range(4):
                    p.block[l][j] = blk[j]
        elif k == "nvec":
            for l, n in enumerate(v):
                p.nvec[l] = n
        else:
            setattr(p, k, v)
    return p


def probe_alu_peaks():
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().wmg_probe_alu_peaks(ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise RuntimeError(f"wmg_probe_alu_peaks: status {st}")
    return {"fp32_tflops": a.value, "fp64_tflops": b.value}


def launch_count():
    n = ctypes.c_longlong()
    load().wmg_launch_count(ctypes.byref(n))
    return n.value


def _ptr(x):
    """Device pointer of a torch tensor or host pointer of a numpy array (contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous()
    return ctypes.c_void_p(x.data_ptr())


class Context:
    """One lattice (dims = (X, Y, Z, T)) with its gauge field and multigrid hierarchy."""

    def __init__(self, dims, stream=None):
        self.lib = load()
        self.dims = tuple(int(a) for a in dims)
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        self._check(self.lib.wmg_create(ctypes.byref(h), ctypes.byref(arr), ctypes.c_void_p(stream or 0)), None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.wmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, h=True, allow=()):
        if st == OK or st in allow:
            return st
        msg = self.lib.wmg_strerror(st).decode()
        if h and getattr(self, "h", None):
            msg += ": " + (self.lib.wmg_last_error(self.h) or b"").decode()
        raise WmgError(st, msg)

    @property
    def V(self):
        X, Y, Z, T = self.dims
        return X * Y * Z * T

    # --- state ---
    def load_gauge(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            return self._check(self.lib.wmg_load_gauge(self.h, _ptr(U)))
        return self._check(self.lib.wmg_load_gauge_dev(self.h, _ptr(U)))

    def set_gauge_compression(self, reals):
        """18, 12 (default) or 8 reals per link in the FP32 fine operator."""
        return self._check(self.lib.wmg_set_gauge_compression(self.h, int(reals)))

    def set_mass(self, m):
        return self._check(self.lib.wmg_set_mass(self.h, float(m)))

    def setup(self, params, starts=None):
        s = None if starts is None else np.ascontiguousarray(starts, dtype=np.complex128)
        return self._check(self.lib.wmg_setup(self.h, ctypes.byref(params), _ptr(s) if s is not None else None))

    def update_gauge(self, U):
        """New gauge field, same near-null subspace: only the coarse operators are rebuilt."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            return self._check(self.lib.wmg_update_gauge(self.h, _ptr(U)))
        return self._check(self.lib.wmg_update_gauge_dev(self.h, _ptr(U)))

    def refresh_setup(self, passes=1):
        """`passes` improvement passes of the adaptive setup from the current subspace."""
        return self._check(self.lib.wmg_refresh_setup(self.h, int(passes)))

    def import_nullvecs(self, level, vecs, params=None):
        v = np.ascontiguousarray(vecs, dtype=np.complex128)
        p = ctypes.byref(params) if params is not None else None
        return self._check(self.lib.wmg_import_nullvecs(self.h, p, int(level), _ptr(v)))

    def coarse_impl(self, level):
        """(implementation of the FP32 cycle's stencil on `level`, autotuner ms per impl)."""
        impl, ms = ctypes.c_int(), (ctypes.c_float * 3)()
        self._check(self.lib.wmg_coarse_impl(self.h, int(level), ctypes.byref(impl), ms))
        return impl.value, list(ms)

    def device_bytes(self):
        """Device bytes this context holds now (fields, operators, workspaces)."""
        n = ctypes.c_size_t()
        self._check(self.lib.wmg_device_bytes(self.h, ctypes.byref(n)))
        return n.value

    def level_info(self, level):
        ns, nd = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wmg_level_info(self.h, int(level), ctypes.byref(ns), ctypes.byref(nd)))
        return ns.value, nd.value

    def export_nullvecs(self, level, nvec):
        ns, nd = self.level_info(level)
        out = np.empty((nvec, ns, nd), dtype=np.complex128)
        self._check(self.lib.wmg_export_nullvecs(self.h, int(level), _ptr(out)))
        return out

    def export_coarse(self, level):
        ns, nd = self.level_info(level + 1)
        out = np.empty((ns, 9, nd, nd), dtype=np.complex128)
        self._check(self.lib.wmg_export_coarse(self.h, int(level), _ptr(out)))
        return out

    # --- solves ---
    def solve(self, b, x, nrhs, plain=False):
        """b, x: canonical complex128 fine spinors (torch CUDA tensors or numpy host arrays)."""
        info = (Info * nrhs)()
        if isinstance(b, np.ndarray):
            assert not plain
            st = self.lib.wmg_solve(self.h, _ptr(b), _ptr(x), int(nrhs), info)
        else:
            f = self.lib.wmg_solve_plain_dev if plain else self.lib.wmg_solve_dev
            st = f(self.h, _ptr(b), _ptr(x), int(nrhs), info)
        self._check(st, allow=(ENOCONV,))
        return st, [i.as_dict() for i in info]

    def solve_cgnr(self, b, x, nrhs, maxit=100000):
        """Unpreconditioned FP64 CG on the normal equations (baseline); b, x canonical CUDA tensors."""
        info = (Info * nrhs)()
        st = self.lib.wmg_solve_cgnr_dev(self.h, _ptr(b), _ptr(x), int(nrhs), int(maxit), info)
        self._check(st, allow=(ENOCONV,))
        return st, [i.as_dict() for i in info]

    # --- operator-level entry points (device tensors) ---
    def pack(self, prec, canon, native, nrhs):
        return self._check(self.lib.wmg_pack_spinor(self.h, prec, _ptr(canon), _ptr(native), int(nrhs)))

    def unpack(self, prec, native, canon, nrhs):
        return self._check(self.lib.wmg_unpack_spinor(self.h, prec, _ptr(native), _ptr(canon), int(nrhs)))

    def apply_D(self, prec, inp, out, nrhs):
        return self._check(self.lib.wmg_apply_D(self.h, prec, _ptr(inp), _ptr(out), int(nrhs)))

    def apply_D_eo(self, prec, inp, out, nrhs):
        """out = S in on the even sites: the red/black Schur complement of the fine operator."""
        return self._check(self.lib.wmg_apply_D_eo(self.h, prec, _ptr(inp), _ptr(out), int(nrhs)))

    def apply_cycle(self, prec, inp, out, nrhs):
        """out = K(in): one multigrid cycle of the fine level (native fine spinors)."""
        return self._check(self.lib.wmg_apply_cycle(self.h, prec, _ptr(inp), _ptr(out), int(nrhs)))

    def smooth(self, prec, b, x, nrhs, nu):
        """x <- nu MR steps on D x = b from the initial guess x (native fine spinors, in place)."""
        return self._check(self.lib.wmg_smooth(self.h, prec, _ptr(b), _ptr(x), int(nrhs), int(nu)))

    def restrict(self, level, prec, fine, coarse, nrhs):
        return self._check(self.lib.wmg_restrict(self.h, int(level), prec, _ptr(fine), _ptr(coarse), int(nrhs)))

    def prolong(self, level, prec, coarse, fine, nrhs):
        return self._check(self.lib.wmg_prolong(self.h, int(level), prec, _ptr(coarse), _ptr(fine), int(nrhs)))

    def residual_noalloc(self, prec, b, x, r, norm2, nrhs):
        """r = b - D x and norm2[k] = |r_k|^2 without any device allocation (static scratch)."""
        return self._check(self.lib.wmg_residual_noalloc(self.h, prec, _ptr(b), _ptr(x), _ptr(r), _ptr(norm2),
                                                         int(nrhs)))

    PROF_CLASSES = ("dslash_sloppy", "dslash_fp64", "coarse", "restrict", "prolong", "blas", "setup", "cgnr",
                    "blas_coarse")

    def profile(self, on=True):
        return self._check(self.lib.wmg_profile_enable(self.h, int(bool(on))))

    def profile_get(self):
        out = {}
        for k, name in enumerate(self.PROF_CLASSES):
            ms, n, b, u = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.wmg_profile_get(self.h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                                 ctypes.byref(u)))
            out[name] = {"ms": ms.value, "launches": n.value, "bytes": b.value, "units": u.value}
        return out

    def apply_coarse(self, level, prec, inp, out, nrhs, dagger=False):
        return self._check(self.lib.wmg_apply_coarse(self.h, int(level), prec, int(bool(dagger)), _ptr(inp),
                                                     _ptr(out), int(nrhs)))

    def apply_coarse_schur(self, level, prec, inp, out, nrhs, dagger=False):
        return self._check(self.lib.wmg_apply_coarse_schur(self.h, int(level), prec, int(bool(dagger)), _ptr(inp),
                                                           _ptr(out), int(nrhs)))


class Server:
    """Continuous-batching solve server over resident fields (contexts handed over with add_field)."""

    def __init__(self, hbm_budget_bytes=200 << 30):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.wmg_server_create(ctypes.byref(h), ctypes.c_size_t(int(hbm_budget_bytes)))
        if st != OK:
            raise WmgError(st, "wmg_server_create")
        self.h = h
        self.fields = []
        self.pending = {}

    def add_field(self, ctx, nslots):
        fid = ctypes.c_int()
        st = self.lib.wmg_server_add_field(self.h, ctx.h, int(nslots), ctypes.byref(fid))
        if st != OK:
            raise WmgError(st, self.lib.wmg_strerror(st).decode() + ": " + (self.lib.wmg_last_error(ctx.h) or b"").decode())
        self.fields.append(ctx)           # keep the context alive while served
        return fid.value

    def submit(self, field, mass, b, x):
        """b, x: canonical host arrays (nrhs, T, Z, Y, X, 12) complex128, kept alive until wait()."""
        assert b.flags["C_CONTIGUOUS"] and x.flags["C_CONTIGUOUS"] and b.dtype == np.complex128
        t = ctypes.c_longlong()
        st = self.lib.wmg_server_submit(self.h, int(field), float(mass), _ptr(b), _ptr(x), int(b.shape[0]),
                                        ctypes.byref(t))
        if st != OK:
            raise WmgError(st, "wmg_server_submit")
        self.pending[t.value] = (b, x)
        return t.value

    def poll(self, ticket):
        d = ctypes.c_int()
        self.lib.wmg_server_poll(self.h, ctypes.c_longlong(ticket), ctypes.byref(d))
        return bool(d.value)

    def wait(self, ticket):
        b, x = self.pending.pop(ticket)
        info = (Info * b.shape[0])()
        lat = ctypes.c_double()
        st = self.lib.wmg_server_wait(self.h, ctypes.c_longlong(ticket), info, ctypes.byref(lat))
        return st, [i.as_dict() for i in info], lat.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.wmg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

