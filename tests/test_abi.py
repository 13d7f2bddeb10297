"""Host-side checks of the C ABI boundary (no GPU needed): the library loads and exports every
function include/wmg.h declares; argument checks that fail before any device work."""
import ctypes
import os
import subprocess
import tempfile

import pytest

from paper_0912_2186_b300 import build, wmg


@pytest.fixture(scope="module")
def lib():
    build.build()
    return wmg.load()


def test_every_declared_symbol_is_exported(lib):
    names = wmg.declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_default_params_and_strerror(lib):
    p = wmg.default_params()
    assert p.nlevels == 2 and p.nu_post == 4 and p.tol == 1e-10
    assert tuple(p.block[0]) == (4, 4, 4, 4)
    assert p.prec_nullvec == 1 and p.prec_smoother == 1 and p.coarse_persistent == 0 and p.coarse_eo == 1
    assert p.fine_eo == 0 and p.setup_relax == 100 and p.setup_passes == 5 and p.coarse_tol == 0.1
    assert lib.wmg_strerror(wmg.ENOCONV) == b"solver did not converge"


def test_binding_structs_match_the_header():
    """Every field of the ctypes structs sits at the offset the C compiler gives it from wmg.h."""
    fields = [f for f, _ in wmg.Params._fields_] + ["info." + f for f, _ in wmg.Info._fields_]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wmg.h"', "int main(void) {",
             'printf("%zu %zu\\n", sizeof(wmg_params), sizeof(wmg_info));']
    for f in fields:
        if f.startswith("info."):
            lines.append(f'printf("%zu\\n", offsetof(wmg_info, {f[5:]}));')
        else:
            lines.append(f'printf("%zu\\n", offsetof(wmg_params, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(src, "w").write("\n".join(lines))
        inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
        subprocess.check_call(["gcc", "-I", inc, src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes, offs = [int(v) for v in out[:2]], [int(v) for v in out[2:]]
    assert sizes == [ctypes.sizeof(wmg.Params), ctypes.sizeof(wmg.Info)]
    want = [getattr(wmg.Params, f).offset for f, _ in wmg.Params._fields_] + \
           [getattr(wmg.Info, f).offset for f, _ in wmg.Info._fields_]
    assert offs == want


def test_invalid_arguments_rejected_without_device_work(lib):
    h = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(8, 8, 1, 8)
    assert lib.wmg_create(ctypes.byref(h), ctypes.byref(bad), None) == wmg.EINVAL
    assert lib.wmg_destroy(None) == wmg.EINVAL
    assert lib.wmg_set_mass(None, 0.1) == wmg.EINVAL
    assert lib.wmg_apply_D(None, 0, None, None, 1) == wmg.EINVAL


def test_server_host_side_argument_checks(lib):
    h = ctypes.c_void_p()
    assert lib.wmg_server_create(ctypes.byref(h), 1 << 30) == wmg.OK
    t = ctypes.c_longlong()
    fid = ctypes.c_int()
    assert lib.wmg_server_add_field(h, None, 4, ctypes.byref(fid)) == wmg.EINVAL
    assert lib.wmg_server_submit(h, 0, 0.1, None, None, 1, ctypes.byref(t)) == wmg.EINVAL
    d = ctypes.c_int()
    assert lib.wmg_server_poll(h, 12345, ctypes.byref(d)) == wmg.EINVAL
    assert lib.wmg_server_destroy(h) == wmg.OK
