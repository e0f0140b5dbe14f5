"""The device-side failure path, made to happen on purpose without a fault:
every wait in the kernels is bounded, and when its limit passes the kernel
records TDG_ETIMEOUT, lets the copies it issued land, frees its tensor memory
and returns.  The test makes the CUDA-core GEMM's first wait for operand tiles
wait on a barrier that nothing completes (tdgemm_set_wait_test) with a 1 ms
limit, reads the status on the host, and checks that the same plan then runs
normally (needs a GB300)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tdg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5765_gb300 import build
    build.build()
    import paper_1110_5765_gb300 as t
    return t


TDG_ETIMEOUT = 6


@pytest.mark.parametrize("dtype,form,W,bits", [("f32", "sym", 2, 7), ("f64", "asym", 3, 8),
                                               ("f32", "plain", 1, 0), ("f32", "asym", 2, 6)])
def test_wait_expiry_reports_timeout_and_plan_recovers(tdg, orc, dtype, form, W, bits):
    npt = np.float32 if dtype == "f32" else np.float64
    M, K, N = 300, 384, 260
    A = synth.laplace((M, K), 71, npt)
    B = synth.laplace((K, N), 72, npt)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    p = tdg.Plan(M, N, K, L=128, W=W, dtype=dtype, form=form, bits=bits)
    C = torch.zeros((M, N), dtype=dA.dtype, device="cuda")
    p.set_wait_test(1_000_000)                      # 1 ms on a barrier nothing completes
    p.run(dA, dB, C)
    torch.cuda.synchronize()
    assert p.info()["device_status"] == TDG_ETIMEOUT
    # the context stays usable and the plan computes again once the test is off
    p.set_wait_test(0)
    p.run(dA, dB, C)
    torch.cuda.synchronize()
    assert p.info()["device_status"] == 0
    kw = dict(L=128, W=W, dtype=dtype, form=form, bits=bits)
    ref = orc.tdgemm(A, B, **kw).C
    assert np.array_equal(C.cpu().numpy().view(np.uint8), ref.view(np.uint8))
    p.close()


def test_wait_test_argument_checks(tdg):
    p = tdg.Plan(64, 64, 128, L=128, W=1, dtype="f32", form="tc_int", bits=8)
    with pytest.raises(tdg.TDGemmError):
        p.set_wait_test(1000)                       # tensor-core form: not covered
    p.close()
    p = tdg.Plan(64, 64, 64, L=64, W=2, dtype="f32", form="sym", bits=6)
    with pytest.raises(tdg.TDGemmError):
        p.set_wait_test(-1)
    with pytest.raises(tdg.TDGemmError):
        p.set_wait_test(2_000_000_000)
    p.close()
