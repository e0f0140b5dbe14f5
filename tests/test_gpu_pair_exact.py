"""Pair-exact companders (TDG_PAIR_EXACT: eq. 26 per subblock product) on the
GPU against the oracle, through the C ABI: C bit-identical, the plan equal to
the separable planner's, and the SNR above the separable product's on blocks
of unlike peak-to-RMS ratios."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


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


def run_px(tdg, A, B, *, L, W, dtype, bits=0, target=math.nan, alpha=1.0, beta=0.0, Cin=None,
           pair_exact=True):
    M, K = A.shape
    N = B.shape[1]
    p = tdg.Plan(M, N, K, L=L, W=W, dtype=dtype, form="sym", bits=bits, target_snr_db=target,
                 pair_exact=pair_exact)
    C = dev(Cin) if Cin is not None else torch.zeros((M, N), dtype=TT[dtype], device="cuda")
    p.run(dev(A), dev(B), C, alpha, beta)
    torch.cuda.synchronize()
    info = p.info()
    assert info["device_status"] == 0, info
    p.close()
    return C.cpu().numpy(), info


CASES = [
    dict(dtype="f32", L=128, W=2, bits=7, shape=(300, 400, 260)),
    dict(dtype="f32", L=128, W=4, bits=4, shape=(256, 384, 128)),
    dict(dtype="f64", L=64, W=2, bits=12, shape=(150, 200, 130)),
    dict(dtype="f64", L=64, W=4, bits=9, shape=(128, 256, 192)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dtype']}-W{c['W']}-b{c['bits']}")
def test_fixed_bits_matches_oracle(tdg, orc, case):
    M, K, N = case["shape"]
    T = NP[case["dtype"]]
    A = synth.blockwise_crest((M, K), 1401, case["L"], T)
    B = synth.blockwise_crest((K, N), 1402, case["L"], T)
    kw = dict(L=case["L"], W=case["W"], dtype=case["dtype"])
    plan = orc.tdgemm(A, B, form="sym", bits=case["bits"], **kw).plan
    ref = orc.tdgemm_pair_exact(A, B, plan=plan, alpha=0.5, beta=2.0,
                                C_in=synth.gaussian((M, N), 1403, T), **kw)
    C, info = run_px(tdg, A, B, bits=case["bits"], alpha=0.5, beta=2.0,
                     Cin=synth.gaussian((M, N), 1403, T), **kw)
    assert (info["q"], info["r_max"]) == (plan.q, plan.R)
    assert same_bits(C, ref)


def test_target_mode_matches_oracle(tdg, orc):
    """20 dB target with the package's representation-noise table: the same plan
    as the separable planner and C equal to the oracle's pair-exact product.
    Beyond the error-free region the representation noise of the shared R_max
    dominates, so the SNR stays that of the separable product (within 0.5 dB)."""
    L, M, K, N = 128, 384, 1024, 256
    A = synth.blockwise_crest((M, K), 1411, L, np.float32, kmax=11)
    B = synth.blockwise_crest((K, N), 1412, L, np.float32, kmax=11)
    st = orc.load_s_table()
    sep = orc.tdgemm(A, B, L=L, W=2, dtype="f32", form="sym", target_db=20.0, s_table=st)
    assert sep.plan.W == 2
    ref = orc.tdgemm_pair_exact(A, B, L=L, W=2, dtype="f32", plan=sep.plan)
    C, info = run_px(tdg, A, B, L=L, W=2, dtype="f32", target=20.0)
    assert (info["W_used"], info["q"], info["r_max"]) == (2, sep.plan.q, sep.plan.R)
    assert same_bits(C, ref)
    Csep, _ = run_px(tdg, A, B, L=L, W=2, dtype="f32", target=20.0, pair_exact=False)
    exact = orc.exact_gemm(A, B)
    assert abs(orc.snr_db(C, exact) - orc.snr_db(Csep, exact)) < 0.5


def test_beats_separable_inside_headroom(tdg, orc):
    """fp64, 10 bits, W = 2 (inside the error-free region, only quantization
    noise): on blocks of unlike peak-to-RMS ratios the per-pair split lowers
    the noise at the same R_max."""
    L, M, K, N = 64, 256, 512, 256
    A = synth.blockwise_crest((M, K), 51, L, np.float64, kmax=11)
    B = synth.blockwise_crest((K, N), 52, L, np.float64, kmax=11)
    C, info = run_px(tdg, A, B, L=L, W=2, dtype="f64", bits=10)
    Csep, _ = run_px(tdg, A, B, L=L, W=2, dtype="f64", bits=10, pair_exact=False)
    assert info["w_ef"] >= 2
    exact = orc.exact_gemm(A, B)
    assert orc.snr_db(C, exact) > orc.snr_db(Csep, exact) + 0.1


def test_argument_checks(tdg):
    from paper_1110_5765_gb300._lib import TDGemmError
    bad = [dict(form="asym", L=128, W=2, bits=6, dtype="f32"),
           dict(form="sym", L=64, W=2, bits=6, dtype="f32"),
           dict(form="sym", L=128, W=3, bits=6, dtype="f32"),
           dict(form="sym", L=128, W=4, target_snr_db=20.0, dtype="f32"),
           dict(form="sym", L=128, W=2, bits=6, dtype="f32", transA="T")]
    for kw in bad:
        with pytest.raises(TDGemmError) as e:
            tdg.Plan(256, 256, 256, pair_exact=True, **kw)
        assert e.value.status == 1, kw
