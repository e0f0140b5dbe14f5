"""tdgemm_run_static, the entry point that allocates nothing (its workspace is a
static device array), through the C ABI: against the plan-based entry point
and against the CPU oracle.

It serves callers that may not allocate device memory where they call: a
framework whose allocator owns the whole device, a plug-in handed only the
buffers it computes on, a service that must not allocate on first use.  This
file is collected last so that a run stopping at the first failure has already
run every other test."""
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


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def _stored(X, trans):
    """The matrix as the caller stores it for trans 'N' / 'T' (row-major)."""
    return np.ascontiguousarray(X.T if trans == "T" else X)


def run_static(lib, A, B, *, L, W, dtype, form, bits, tA="N", tB="N", C_in=None, alpha=1.0,
               beta=0.0):
    """A = op(A) (M x K), B = op(B) (K x N); stored transposed where asked."""
    code, npt, tt = DT[dtype]
    M, K = A.shape
    N = B.shape[1]
    As, Bs = _stored(A, tA), _stored(B, tB)
    dA = torch.from_numpy(As).cuda()
    dB = torch.from_numpy(Bs).cuda()
    dC = (torch.zeros((M, N), dtype=tt, device="cuda") if C_in is None
          else torch.from_numpy(np.ascontiguousarray(C_in)).cuda())
    st = lib.tdgemm_run_static(tA.encode(), tB.encode(), M, N, K, As.shape[1], Bs.shape[1], N,
                               L, W, code, FORM[form], bits, dA.data_ptr(), dB.data_ptr(),
                               dC.data_ptr(), alpha, beta,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, dC.cpu().numpy()


def run_plan(A, B, *, L, W, dtype, form, bits, tA="N", tB="N", C_in=None, alpha=1.0, beta=0.0):
    import paper_1110_5765_gb300 as tdg
    M, K = A.shape
    N = B.shape[1]
    _, _, tt = DT[dtype]
    p = tdg.Plan(M, N, K, L=L, W=W, dtype=dtype, form=form, bits=bits, transA=tA, transB=tB)
    C = None if C_in is None else torch.from_numpy(np.ascontiguousarray(C_in)).cuda()
    C = p.run(torch.from_numpy(_stored(A, tA)).cuda(), torch.from_numpy(_stored(B, tB)).cuda(),
              C=C, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    out = C.cpu().numpy()
    p.close()
    return out


CASES = [
    dict(shape=(300, 257, 190), L=64, W=2, dtype="f32", form="sym", bits=7, seed=1),
    dict(shape=(130, 512, 300), L=128, W=3, dtype="f64", form="asym", bits=9, seed=2),
    # operands stored transposed, and an alpha / beta epilogue over a given C
    dict(shape=(200, 300, 170), L=64, W=2, dtype="f32", form="asym", bits=6, seed=3,
         tA="T", tB="T"),
    dict(shape=(257, 129, 260), L=64, W=4, dtype="f64", form="sym", bits=8, seed=4,
         tA="T", tB="N", alpha=0.75, beta=-1.5),
]


def _case_inputs(case):
    M, K, N = case["shape"]
    _, npt, _ = DT[case["dtype"]]
    A = synth.laplace((M, K), 10 + case["seed"], npt)
    B = synth.laplace((K, N), 20 + case["seed"], npt)
    C_in = synth.gaussian((M, N), 30 + case["seed"]).astype(npt) if case.get("beta") else None
    return A, B, C_in


def test_static_entry_matches_plan_entry_and_oracle_on_calls_in_a_row(lib, orc):
    """Products back to back through the static scratch (each must not see the
    previous one's leftovers): every result equals the plan-based result and
    the CPU oracle's bit for bit, the tolerance the other GPU tests use for the
    CUDA-core forms."""
    for case in CASES:
        A, B, C_in = _case_inputs(case)
        kw = {k: case[k] for k in ("L", "W", "dtype", "form", "bits")}
        ep = dict(tA=case.get("tA", "N"), tB=case.get("tB", "N"), C_in=C_in,
                  alpha=case.get("alpha", 1.0), beta=case.get("beta", 0.0))
        st, C = run_static(lib, A, B, **kw, **ep)
        assert st == 0, lib.tdgemm_last_error().decode()
        ref = run_plan(A, B, **kw, **ep)
        assert np.all(np.isfinite(ref)) and np.count_nonzero(ref) > ref.size // 2
        assert np.array_equal(C.view(np.uint8), ref.view(np.uint8)), case
        orc_C = orc.tdgemm(A, B, **kw, alpha=ep["alpha"], beta=ep["beta"], C_in=C_in).C
        assert np.array_equal(C.view(np.uint8), orc_C.view(np.uint8)), case


def test_static_entry_twice_with_the_same_arguments(lib):
    """The same call twice in a row gives the same bits (what the first call
    leaves in the shared array does not leak into the second)."""
    case = CASES[0]
    A, B, _ = _case_inputs(case)
    kw = {k: case[k] for k in ("L", "W", "dtype", "form", "bits")}
    st1, C1 = run_static(lib, A, B, **kw)
    st2, C2 = run_static(lib, A, B, **kw)
    assert st1 == 0 and st2 == 0, lib.tdgemm_last_error().decode()
    assert np.array_equal(C1.view(np.uint8), C2.view(np.uint8))


def test_static_entry_rejects_products_beyond_its_scratch(lib):
    """A product whose workspace exceeds the static array fails with TDG_EINVAL
    and a message naming the limit, before any device work; so do sizes beyond
    2^31."""
    M = N = K = 4096
    dummy = torch.zeros(1, device="cuda")
    p = dummy.data_ptr()
    st = lib.tdgemm_run_static(b"N", b"N", M, N, K, K, N, N, 128, 2, 0, 1, 6, p, p, p, 1.0, 0.0,
                               None)
    assert st == 1
    assert "static scratch holds" in lib.tdgemm_last_error().decode()
    big = (1 << 31) + 1
    st = lib.tdgemm_run_static(b"N", b"N", big, 16, 16, 16, 16, 16, 16, 2, 0, 2, 6, p, p, p,
                               1.0, 0.0, None)
    assert st == 1
    assert "2^31" in lib.tdgemm_last_error().decode()
