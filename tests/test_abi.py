"""C ABI: the library builds, loads and exports every entry point the header
declares; argument checks run on the host (no GPU needed)."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "tdgemm.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tdgemm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_5765_gb300 import build
    build.build()
    from paper_1110_5765_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1110_5765_gb300 import _lib
    syms = declared_symbols()
    assert len(syms) >= 12
    assert sorted(_lib.EXPORTS) == syms
    for s in syms:
        assert hasattr(lib, s), s


def test_version(lib):
    assert b"sm_103a" in lib.tdgemm_version()


def _plan(lib, **kw):
    a = dict(tA=b"N", tB=b"N", M=64, N=64, K=64, lda=64, ldb=64, ldc=64, L=64, W=2, dtype=0,
             form=1, target=math.nan, bits=8, flags=0)
    a.update(kw)
    h = ctypes.c_void_p()
    st = lib.tdgemm_plan(ctypes.byref(h), a["tA"], a["tB"], a["M"], a["N"], a["K"], a["lda"],
                         a["ldb"], a["ldc"], a["L"], a["W"], a["dtype"], a["form"], a["target"],
                         a["bits"], a["flags"])
    return st, h


@pytest.mark.parametrize("bad,err", [
    (dict(M=0), "M, N, K"),
    (dict(lda=10), "lda"),
    (dict(ldb=10), "ldb"),
    (dict(ldc=10), "ldc"),
    (dict(L=20), "multiple of 16"),
    (dict(L=2048), "multiple of 16"),
    (dict(W=5), "W must"),
    (dict(tA=b"X"), "trans"),
    (dict(bits=0, target=math.nan), "finite"),
    (dict(bits=0, target=30.0, W=1), "W >= 2"),
    (dict(bits=30), "bits"),
    (dict(form=0, W=2), "W must be 1"),
    (dict(form=3, W=1, dtype=1), "fp32"),
    (dict(form=3, W=1, L=96), "L % 64"),
    (dict(form=4, W=1, L=64, bits=0, target=0.0), "L % 128"),
    (dict(form=3, W=1, L=128, bits=13), "gamma"),
    (dict(form=7), "bad form"),
])
def test_argument_checks_fail_before_any_device_work(lib, bad, err):
    st, h = _plan(lib, **bad)
    assert st in (1, 4)            # TDG_EINVAL / TDG_EUNSUPPORTED
    assert h.value is None
    assert err in lib.tdgemm_last_error().decode()


def test_null_plan_calls_are_rejected(lib):
    assert lib.tdgemm_quantize_pack(None, None, None, None) == 1
    assert lib.tdgemm_gemm(None, None, 1.0, 0.0, None) == 1
    assert lib.tdgemm_unpack(None, None, None, None) == 1
    assert lib.tdgemm_set_manual(None, 10, 1.0, 1.0) == 1
    assert lib.tdgemm_set_kernel_control(None, 2, 0.5) == 1
    assert lib.tdgemm_kernel_mask(None, None, 0) == 1
    assert lib.tdgemm_quantize_pack_a(None, None, None) == 1
    assert lib.tdgemm_run(None, None, None, None, 1.0, 0.0, None) == 1
    assert lib.tdgemm_run_host(None, None, None, None, 1.0, 0.0, None) == 1
    assert lib.tdgemm_run_host_async(None, None, None, None, 1.0, 0.0, None) == 1
    assert lib.tdgemm_plan_destroy(None) == 0
    assert lib.tdgemm_set_wait_test(None, 0) == 1
    assert lib.tdgemm_set_speedup(None, 2, 1.5) == 1


def test_fma_probe_argument_checks(lib):
    """The FMA-pipe probe rejects a bad dtype, a non-positive iteration count
    and a NULL output before touching the device."""
    fl = ctypes.c_double()
    assert lib.tdgemm_fma_probe(5, 10, ctypes.byref(fl), None) == 1
    assert lib.tdgemm_fma_probe(0, 0, ctypes.byref(fl), None) == 1
    assert lib.tdgemm_fma_probe(0, 10, None, None) == 1
