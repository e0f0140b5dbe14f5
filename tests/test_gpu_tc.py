"""Tensor-core forms (tcgen05) against the CPU oracle (needs a GB300)."""
import math

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_tc(tdg, A, B, *, form, L=128, bits=0, target=math.nan, transA="N", transB="N"):
    M, K = A.shape
    N = B.shape[1]
    As = dev(A.T if transA == "T" else A)
    Bs = dev(B.T if transB == "T" else B)
    p = tdg.Plan(M, N, K, L=L, W=1, dtype="f32", form=form, bits=bits, target_snr_db=target,
                 transA=transA, transB=transB)
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    p.run(As, Bs, C)
    torch.cuda.synchronize()
    info = p.info()
    p.close()
    assert info["device_status"] == 0, info
    return C.cpu().numpy(), info


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


@pytest.mark.parametrize("shape", [(128, 128, 256), (256, 384, 200), (130, 300, 270),
                                   (1, 64, 1), (300, 1000, 129)])
@pytest.mark.parametrize("L", [64, 128])
def test_tc_int_8bit_bitexact(tdg, orc, shape, L):
    """8-bit companded integers on tensor cores: every per-slab fp32 sum is an
    exact integer, so C equals the oracle's exact-integer product bit for bit."""
    M, K, N = shape
    A = synth.laplace((M, K), 11 + M, np.float32)
    B = synth.laplace((K, N), 12 + N, np.float32)
    ref = orc.tc_int_gemm(A, B, L=L, bits=8)
    C, info = run_tc(tdg, A, B, form="tc_int", L=L, bits=8)
    assert info["gamma_a"] == 127 and info["carrier"] == 16
    assert same_bits(C, ref.C)


@pytest.mark.parametrize("transA,transB", [("T", "N"), ("N", "T")])
def test_tc_int_transposes(tdg, orc, transA, transB):
    A = synth.gaussian((200, 256), 21, np.float32)
    B = synth.gaussian((256, 300), 22, np.float32)
    ref = orc.tc_int_gemm(A, B, L=128, bits=8)
    C, _ = run_tc(tdg, A, B, form="tc_int", bits=8, transA=transA, transB=transB)
    assert same_bits(C, ref.C)


def test_tc_int_widest_exact_companders(tdg, orc):
    """Target mode: the largest companders with L gamma_A gamma_B < 2^24 (split
    per eq. 26) — still exact, 40 dB on Laplacian inputs."""
    A = synth.laplace((256, 512), 31, np.float32)
    B = synth.laplace((512, 256), 32, np.float32)
    ref = orc.tc_int_gemm(A, B, L=128, bits=0)
    C, info = run_tc(tdg, A, B, form="tc_int", target=40.0)
    assert (info["gamma_a"], info["gamma_b"]) == (ref.plan.gA, ref.plan.gB)
    assert same_bits(C, ref.C)
    snr = orc.snr_db(C, orc.exact_gemm(A, B))
    assert snr > 40.0


def test_tc_fp8_matches_oracle(tdg, orc):
    """E4M3 codes: the tensor core's fp32 accumulation order is its own, so the
    check is elementwise within the rounding of fp32 sums plus SNR within 0.1 dB."""
    A = synth.laplace((256, 512), 41, np.float32)
    B = synth.laplace((512, 320), 42, np.float32)
    ref = orc.tc_fp8_gemm(A, B, L=128)
    C, info = run_tc(tdg, A, B, form="tc_fp8")
    assert info["carrier"] == 8
    # bound: per slab, fp32 summation error <= L * 2^-23 * sum|a~ b~|, scaled
    cA = np.repeat(np.repeat(ref.cA.astype(np.float32), 128, 0), 128, 1)[:256, :512]
    cB = np.repeat(np.repeat(ref.cB.astype(np.float32), 128, 0), 128, 1)[:512, :320]
    Aq = np.abs(orc.e4m3((A * cA).astype(np.float64)))
    Bq = np.abs(orc.e4m3((B * cB).astype(np.float64)))
    bound = np.zeros((256, 320))
    for l in range(4):
        scale = np.repeat(np.repeat(np.outer(ref.sA[:, l], ref.sB[l, :]), 128, 0), 128, 1)
        bound += (Aq[:, l * 128:(l + 1) * 128] @ Bq[l * 128:(l + 1) * 128]) * scale[:256, :320]
    bound = bound * 128 * 2.0**-23 + 4 * 2.0**-24 * np.abs(ref.C)
    assert np.all(np.abs(C.astype(np.float64) - ref.C) <= bound + 1e-30)
    ex = orc.exact_gemm(A, B)
    assert abs(orc.snr_db(C, ex) - orc.snr_db(ref.C, ex)) < 0.1


def test_tc_precision_size_sampled(tdg, orc):
    """8192^3 Laplacian, L = 128, the precision-form workload: two sampled
    128 x 128 tiles over the full K, bit-exact for the integer form."""
    n = 8192
    A = synth.laplace((n, n), 51, np.float32)
    B = synth.laplace((n, n), 52, np.float32)
    C, info = run_tc(tdg, A, B, form="tc_int", target=40.0)
    for (ti, tj) in synth.sample_tiles(64, 64, 2, seed=53):
        rows, cols = (ti * 128, ti * 128 + 128), (tj * 128, tj * 128 + 128)
        ref = orc.tc_int_gemm(A, B, L=128, bits=0, rows=rows, cols=cols)
        assert same_bits(C[rows[0]:rows[1], cols[0]:cols[1]], ref.C), (ti, tj)
