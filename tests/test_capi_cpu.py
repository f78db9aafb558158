"""C-ABI checks that need no GPU: the library builds, loads, exports every entry
point declared in include/frg.h, and rejects invalid parameters before it
touches the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1510_07799_gb300 import build as cuda_build
from paper_1510_07799_gb300 import frg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return frg.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "frg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|long|const char)\s*\*?\s*(frg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", frg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (frg_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)  # resolvable through the dynamic loader
    assert set(frg.EXPORTED) <= set(names)


def test_library_is_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", frg.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def _params(**kw):
    d = dict(U=1.0, T=0.05, eps_d=-0.5, Delta=1.0, N_f=16, Lambda0=1e3, Lambda_f=1e-3,
             rtol=1e-8, atol=1e-10, h0=-0.01, max_steps=1000, precision=0, channel_mask=0xF, cutoff=0)
    d.update(kw)
    return frg._Params(**d)


@pytest.mark.parametrize("bad", [dict(N_f=15), dict(N_f=0), dict(N_f=258), dict(T=0.0),
                                 dict(T=-1.0), dict(Delta=0.0), dict(rtol=0.0),
                                 dict(Lambda_f=2e3), dict(Lambda_f=0.0), dict(h0=0.5),
                                 dict(precision=7), dict(channel_mask=0x100), dict(channel_mask=0xF | 0x20 | 0x40),
                                 dict(channel_mask=-1), dict(cutoff=2),
                                 dict(U=float("nan"))])
def test_init_rejects_invalid_parameters_without_device(lib, bad):
    arr = (frg._Params * 1)(_params(**bad))
    h = C.c_void_p(123)
    rc = lib.frg_init(arr, 1, None, C.byref(h))
    assert rc == frg.EINVAL and not h.value


def test_init_rejects_mixed_precision_batch(lib):
    arr = (frg._Params * 2)(_params(), _params(precision=1))
    h = C.c_void_p()
    assert lib.frg_init(arr, 2, None, C.byref(h)) == frg.EINVAL
    assert lib.frg_init(arr, 0, None, C.byref(h)) == frg.EINVAL
    assert lib.frg_init(None, 1, None, C.byref(h)) == frg.EINVAL


def test_null_context_calls_fail_cleanly(lib):
    assert lib.frg_rhs(None, 0, 1.0, None, None, None, None) == frg.EINVAL
    assert lib.frg_flow(None, None) == frg.EINVAL
    assert lib.frg_advance(None, 1, None) == frg.EINVAL
    assert b"null context" in lib.frg_last_error(None)
    assert lib.frg_autotune(None, None) == frg.EINVAL
    assert lib.frg_selftest_wait(None, 10.0) == frg.EINVAL
    assert lib.frg_rhs_host_async(None, 0, 1.0, None, None, None, None) == frg.EINVAL
    assert lib.frg_sync(None) == frg.EINVAL
    lib.frg_destroy(None)
