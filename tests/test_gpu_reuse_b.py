"""tdgemm_quantize_pack_a: a product repeated with the same right operand
reuses B's statistics, companders and packed form.  Through the C ABI, the
result equals a full pack of the same A and B bit for bit."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NP = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def tdg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5765_gb300 import build
    build.build()
    import paper_1110_5765_gb300 as t
    return t


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


CASES = [
    dict(form="sym", dtype="f32", L=128, W=2, bits=6, transB="N"),
    dict(form="sym", dtype="f32", L=128, W=2, bits=6, transB="T"),
    dict(form="asym", dtype="f64", L=64, W=3, bits=9, transB="N"),
    dict(form="plain", dtype="f32", L=128, W=1, bits=0, transB="T"),
    dict(form="tc_int", dtype="f32", L=128, W=1, bits=8, transB="N"),
    dict(form="tc_fp8", dtype="f32", L=128, W=1, bits=0, transB="N"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['form']}-{c['dtype']}-B{c['transB']}")
def test_reused_b_equals_full_pack(tdg, orc, case):
    dt = case["dtype"]
    M, K, N = 300, 384, 260
    A1 = synth.laplace((M, K), 1201, NP[dt])
    A2 = synth.gaussian((M, K), 1202, NP[dt])
    B = synth.laplace((K, N), 1203, NP[dt])
    Bs = np.ascontiguousarray(B.T) if case["transB"] == "T" else B
    kw = dict(L=case["L"], W=case["W"], dtype=dt, form=case["form"], bits=case["bits"],
              transB=case["transB"], rep_noise=None)
    tt = torch.float64 if dt == "f64" else torch.float32
    p = tdg.Plan(M, N, K, **kw)
    dB = dev(Bs)
    C1 = torch.zeros((M, N), dtype=tt, device="cuda")
    C2 = torch.zeros((M, N), dtype=tt, device="cuda")
    p.quantize_pack(dev(A1), dB)
    p.gemm(C1)
    p.quantize_pack(dev(A2))              # B reused
    p.gemm(C2)
    torch.cuda.synchronize()
    assert p.info()["device_status"] == 0
    q = tdg.Plan(M, N, K, **kw)
    R2 = q.run(dev(A2), dB)
    torch.cuda.synchronize()
    assert same_bits(C2.cpu().numpy(), R2.cpu().numpy())
    assert not same_bits(C1.cpu().numpy(), C2.cpu().numpy())
    if case["form"] in ("sym", "asym"):
        ref = orc.tdgemm(A2, B, L=case["L"], W=case["W"], dtype=dt, form=case["form"],
                         bits=case["bits"])
        assert same_bits(C2.cpu().numpy(), ref.C)
    p.close()
    q.close()


def test_reuse_refused_where_b_depends_on_a(tdg):
    from paper_1110_5765_gb300._lib import TDGemmError
    A = dev(synth.uniform((256, 256), 1211, np.float32))
    B = dev(synth.uniform((256, 256), 1212, np.float32))
    p = tdg.Plan(256, 256, 256, L=128, W=2, dtype="f32", form="sym", target_snr_db=20.0)
    p.quantize_pack(A, B)
    with pytest.raises(TDGemmError) as e:
        p.quantize_pack(A)
    assert e.value.status == 1                      # TDG_EINVAL: target mode
    p.close()
    q = tdg.Plan(256, 256, 256, L=128, W=2, dtype="f32", form="sym", bits=6, rep_noise=None)
    with pytest.raises(TDGemmError) as e:
        q.quantize_pack(A)
    assert e.value.status == 8                      # TDG_ESTATE: nothing packed yet
    q.quantize_pack(A, B)
    q.set_kernel_control("fraction", 0.5)
    with pytest.raises(TDGemmError) as e:
        q.quantize_pack(A)
    assert e.value.status == 8                      # control changed: pack B again
    q.close()
