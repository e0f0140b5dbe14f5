"""tdgemm_run_static, the entry point that allocates nothing (its workspace is a
static device array), against the plan-based entry point, through the C ABI.

It serves callers that may not allocate device memory where they call (stream
capture, device-owning allocators).  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FORM = {"sym": 1, "asym": 2}
DT = {"f32": (0, np.float32, torch.float32), "f64": (1, np.float64, torch.float64)}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5765_gb300 import build
    build.build()
    from paper_1110_5765_gb300 import _lib
    return _lib.load()


def run_static(lib, A, B, *, L, W, dtype, form, bits, C=None, alpha=1.0, beta=0.0):
    code, npt, tt = DT[dtype]
    M, K = A.shape
    N = B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.zeros((M, N), dtype=tt, device="cuda") if C is None else C
    st = lib.tdgemm_run_static(b"N", b"N", M, N, K, K, N, N, L, W, code, FORM[form], bits,
                               dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), alpha, beta,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, dC


def run_plan(A, B, *, L, W, dtype, form, bits):
    import paper_1110_5765_gb300 as tdg
    M, K = A.shape
    N = B.shape[1]
    p = tdg.Plan(M, N, K, L=L, W=W, dtype=dtype, form=form, bits=bits)
    C = p.run(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    torch.cuda.synchronize()
    out = C.cpu().numpy()
    p.close()
    return out


CASES = [
    dict(shape=(300, 257, 190), L=64, W=2, dtype="f32", form="sym", bits=7, seed=1),
    dict(shape=(130, 512, 300), L=128, W=3, dtype="f64", form="asym", bits=9, seed=2),
]


def test_static_entry_matches_plan_entry_on_two_calls_in_a_row(lib):
    """Two different products back to back through the static scratch (the
    second must not see the first's leftovers); each equals the plan-based
    result bit for bit, the tolerance the other GPU tests use for these forms."""
    for case in CASES:
        M, K, N = case["shape"]
        _, npt, _ = DT[case["dtype"]]
        A = synth.laplace((M, K), 10 + case["seed"], npt)
        B = synth.laplace((K, N), 20 + case["seed"], npt)
        kw = {k: case[k] for k in ("L", "W", "dtype", "form", "bits")}
        st, C = run_static(lib, A, B, **kw)
        assert st == 0, lib.tdgemm_last_error().decode()
        ref = run_plan(A, B, **kw)
        assert np.all(np.isfinite(ref)) and np.count_nonzero(ref) > ref.size // 2
        assert np.array_equal(C.cpu().numpy().view(np.uint8), ref.view(np.uint8))


def test_static_entry_rejects_products_beyond_its_scratch(lib):
    """A product whose workspace exceeds the static array fails with TDG_EINVAL
    and a message naming the limit, before any device work."""
    M = N = K = 4096
    dummy = torch.zeros(1, device="cuda")
    p = dummy.data_ptr()
    st = lib.tdgemm_run_static(b"N", b"N", M, N, K, K, N, N, 128, 2, 0, 1, 6, p, p, p, 1.0, 0.0,
                               None)
    assert st == 1
    msg = lib.tdgemm_last_error().decode()
    assert "static scratch holds" in msg
