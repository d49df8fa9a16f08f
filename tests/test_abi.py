"""C-ABI checks that need no GPU: the library loads, exports every entry
point that ``include/clbm.h`` declares, and rejects invalid arguments before
touching the device."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def clbm():
    from paper_1908_05396_gb300 import build
    build.build()
    from paper_1908_05396_gb300 import clbm as c
    c.lib()
    return c


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*|void)\s+(clbm_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(clbm):
    names = _declared()
    assert {"clbm_create", "clbm_step", "clbm_fields", "clbm_residual", "clbm_destroy"} <= names
    L = clbm.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


def _create(clbm, **kw):
    d = clbm.Domain()
    d.nx, d.ny, d.nz = kw.get("dims", (4, 4, 4))
    for i, f in enumerate(kw.get("face", (0,) * 6)):
        d.face[i] = f
    d.in_place = kw.get("in_place", 0)
    h = ctypes.c_void_p()
    U = kw.get("U")
    Uc = (ctypes.c_double * 3)(*U) if U is not None else None
    rc = clbm.lib().clbm_create(ctypes.byref(d), kw.get("K", 0.1), kw.get("n", 1.0), Uc, None,
                                kw.get("dtype", 0), ctypes.byref(h))
    return rc, clbm.lib().clbm_last_error(None).decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(dims=(0, 4, 4)), "dimensions"),
    (dict(K=-1.0), "K must"),
    (dict(K=float("nan")), "K must"),
    (dict(n=0.0), "n must"),
    (dict(n=3.5), "n must"),
    (dict(dtype=7), "dtype"),
    (dict(face=(0, 1, 0, 0, 0, 0)), "periodic"),
    (dict(face=(0, 0, 1, 2, 0, 0)), "without U_lid"),
    (dict(face=(0, 0, 1, 2, 0, 0), U=(0.4, 0, 0)), "< 0.3"),
    (dict(face=(0, 0, 1, 2, 0, 0), U=(0, 0.05, 0)), "tangential"),
    (dict(face=(0, 0, 5, 1, 0, 0)), "face kind"),
    (dict(dims=(1400, 1400, 1400), dtype=2), "too large"),   # fits HBM in FP16, not int32
    (dict(dims=(1290, 1290, 1290), dtype=1), "too large"),
    (dict(dims=(1, 1, 65536)), "65535"),      # one launch grid row per z plane
    (dict(dims=(1, 65536, 1)), "65535"),
])
def test_create_rejects_bad_arguments(clbm, kw, frag):
    rc, msg = _create(clbm, **kw)
    assert rc == clbm.ERR_ARG
    assert frag in msg


def test_in_place_rejects_the_f16r_form(clbm):
    rc, msg = _create(clbm, dtype=3, in_place=1)
    assert rc == clbm.ERR_UNSUPPORTED and "in-place" in msg


def test_null_handle_calls_fail_cleanly(clbm):
    L = clbm.lib()
    out = ctypes.c_double()
    assert L.clbm_step(None, 1) == clbm.ERR_ARG
    assert L.clbm_residual(None, ctypes.byref(out)) == clbm.ERR_ARG
    assert L.clbm_destroy(None) == clbm.OK


def test_set_allocator_needs_both_functions(clbm):
    L = clbm.lib()
    alloc = clbm._ALLOC_FN(lambda n, d, s, u: 0)
    free = clbm._FREE_FN(lambda p, n, d, s, u: None)
    null_a, null_f = clbm._ALLOC_FN(), clbm._FREE_FN()
    assert L.clbm_set_allocator(alloc, null_f, None) == clbm.ERR_ARG
    assert L.clbm_set_allocator(null_a, free, None) == clbm.ERR_ARG
    assert L.clbm_set_allocator(null_a, null_f, None) == clbm.OK
    with pytest.raises(ValueError):
        clbm.set_allocator(lambda n, d, s: 0, None)


@pytest.mark.parametrize("dims,dtype,code,frag", [
    ((1, 1, 65536), "f32", "ERR_ARG", "65535"),
    ((0, 4, 4), "f32", "ERR_ARG", "dimensions"),
    ((8, 8, 8), "f16r", "ERR_UNSUPPORTED", "F16R"),
    ((8, 8, 8), 9, "ERR_ARG", "dtype"),
])
def test_noalloc_rejects_bad_arguments(clbm, dims, dtype, code, frag):
    # Argument checks of clbm_step_noalloc run before any device access; the
    # buffer addresses are never dereferenced here.
    rc = clbm.step_noalloc(*dims, face=(0,) * 6, K=0.1, n=1.0, U_lid=None, body_force=None,
                           dtype=dtype, src=4096, dst=8192, u_prev=12288, stats=16384)
    assert rc == getattr(clbm, code)
    assert frag in clbm.last_error()
