"""Sec. 6 control over inner kernels on the GPU against the oracle, through the
C ABI: the mask of accelerated L x L output blocks is identical, and C is
bit-identical (packed product where the mask is set, conventional product
elsewhere)."""
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


def inputs(shape_mkn, L, dtype, seed):
    """Blocks of different ranges and peak-to-RMS ratios, so the inner
    kernels' predicted SNRs spread over many dB (the situation Sec. 6 targets)."""
    M, K, N = shape_mkn
    T = NP[dtype]
    A = synth.blockwise_crest((M, K), seed, L, T)
    B = synth.blockwise_crest((K, N), seed + 1, L, T)
    return A, B


def run_ctrl(tdg, A, B, *, L, W, dtype, bits=0, target=math.nan, ctrl, rms=False,
             alpha=1.0, beta=0.0, Cin=None, dense=None, speedup=None):
    M, K = A.shape
    N = B.shape[1]
    p = tdg.Plan(M, N, K, L=L, W=W, dtype=dtype, form="sym", bits=bits, target_snr_db=target,
                 rep_noise=None, noise_rms=rms, speedup=speedup)
    if dense is not None:
        for w, arr in dense.items():
            p.set_rep_noise(w, arr, 0)
    p.set_kernel_control(*ctrl)
    C = dev(Cin) if Cin is not None else torch.zeros((M, N), dtype=TT[dtype], device="cuda")
    p.run(dev(A), dev(B), C, alpha, beta)
    torch.cuda.synchronize()
    info = p.info()
    assert info["device_status"] == 0, info
    mask = p.kernel_mask()
    out = C.cpu().numpy()
    p.close()
    return out, mask, info


CASES = [
    # (M, K, N), L, W, dtype, bits: ragged edges on every axis, several tiles
    ((500, 300, 600), 128, 2, "f32", 6),
    ((200, 256, 190), 64, 3, "f64", 9),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[3])
@pytest.mark.parametrize("frac", [0.0, 0.3, 0.7, 1.0])
def test_fraction_mode_matches_oracle(tdg, orc, case, frac):
    shape, L, W, dtype, bits = case
    A, B = inputs(shape, L, dtype, 700 + bits)
    ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form="sym", bits=bits,
                     kernel_control=("fraction", frac))
    C, mask, _ = run_ctrl(tdg, A, B, L=L, W=W, dtype=dtype, bits=bits, ctrl=("fraction", frac))
    want = ref.plan.extra["kernel_mask"]
    assert int(mask.sum()) == math.ceil(frac * mask.size)
    assert np.array_equal(mask.astype(bool), want)
    assert same_bits(C, ref.C)
    if frac == 0.0:
        assert same_bits(C, orc.gemm_plain(A, B, dtype))


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[3])
def test_snr_mode_matches_oracle(tdg, orc, case):
    """Thresholds half-way between neighbouring predicted kernel SNRs (so no
    kernel sits on a threshold), at the low end, middle and top."""
    shape, L, W, dtype, bits = case
    A, B = inputs(shape, L, dtype, 800 + bits)
    stA, stB = orc.block_stats(A, L), orc.block_stats(B, L)
    pl = orc.plan_fixed(bits, L, W, dtype, "sym", orc.aggregates(stA, stB, L), None)
    db = np.sort(10.0 * np.log10(orc.kernel_ratios(stA, stB, L, pl.gA, pl.gB, 0.0).ravel()))
    for k in (1, db.size // 2, db.size - 1):
        thr = 0.5 * (db[k - 1] + db[k])
        ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form="sym", bits=bits,
                         kernel_control=("snr", thr))
        C, mask, _ = run_ctrl(tdg, A, B, L=L, W=W, dtype=dtype, bits=bits, ctrl=("snr", thr))
        assert int(mask.sum()) == db.size - k
        assert np.array_equal(mask.astype(bool), ref.plan.extra["kernel_mask"])
        assert same_bits(C, ref.C)


@pytest.mark.parametrize("rms", [False, True])
def test_target_mode_with_control_and_epilogue(tdg, orc, rms):
    """Distortion-target plan with a representation-noise table (s > 0 in the
    kernel model), alpha/beta epilogue on both kinds of inner kernel."""
    dtype, L, W = "f32", 128, 3
    A, B = inputs((384, 512, 400), L, dtype, 901)
    dense, tabs = {}, {}
    for w in (2, 3):
        d, arr = {}, np.full(192, -1.0)
        for t in range(0, orc.T_MAX[dtype] + 1):
            R = orc.r_level(t)
            s = 1e-3 * R * (w - 1) if R >= L else 0.0
            d[str(t)] = {"s": s}
            arr[t] = s
        tabs[orc.STable.key(dtype, "sym", w, L)] = d
        dense[w] = arr
    st = orc.STable(tabs)
    Cin = synth.gaussian((384, 400), 902, np.float32)
    ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form="sym", target_db=20.0, s_table=st,
                     noise_rms=rms, alpha=0.5, beta=-2.0, C_in=Cin,
                     kernel_control=("fraction", 0.5))
    C, mask, info = run_ctrl(tdg, A, B, L=L, W=W, dtype=dtype, target=20.0, rms=rms,
                             ctrl=("fraction", 0.5), alpha=0.5, beta=-2.0, Cin=Cin, dense=dense)
    assert info["W_used"] == ref.plan.W
    if ref.plan.W > 1:
        assert np.array_equal(mask.astype(bool), ref.plan.extra["kernel_mask"])
    else:
        assert not mask.any()
    assert same_bits(C, ref.C)


@pytest.mark.parametrize("trans", ["NT", "TN", "TT"])
def test_transposed_operands(tdg, orc, trans):
    """Stored transposes: the conventional-product tiles read op(A) / op(B)
    from the caller's buffers where the layout allows (A stored 'T', B stored
    'N') and from the plan's copies otherwise; mask and C unchanged."""
    tA, tB = trans[0], trans[1]
    dtype, L = "f32", 128
    A, B = inputs((384, 256, 300), L, dtype, 970)
    M, K = A.shape
    N = B.shape[1]
    As = np.ascontiguousarray(A.T) if tA == "T" else A
    Bs = np.ascontiguousarray(B.T) if tB == "T" else B
    ref = orc.tdgemm(A, B, L=L, W=2, dtype=dtype, form="sym", bits=6,
                     kernel_control=("fraction", 0.4))
    p = tdg.Plan(M, N, K, L=L, W=2, dtype=dtype, form="sym", bits=6, rep_noise=None,
                 transA=tA, transB=tB)
    p.set_kernel_control("fraction", 0.4)
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    p.run(dev(As), dev(Bs), C)
    torch.cuda.synchronize()
    assert p.info()["device_status"] == 0
    assert np.array_equal(p.kernel_mask().astype(bool), ref.plan.extra["kernel_mask"])
    assert same_bits(C.cpu().numpy(), ref.C)
    p.close()


def test_fallback_plan_accelerates_nothing(tdg, orc):
    """A target no packing can meet: the planner falls back to W = 1, the mask
    is empty and C is the conventional product."""
    A, B = inputs((256, 384, 300), 128, "f32", 960)
    ref = orc.tdgemm(A, B, L=128, W=2, dtype="f32", form="sym", target_db=90.0,
                     kernel_control=("fraction", 0.5))
    assert ref.plan.W == 1
    C, mask, info = run_ctrl(tdg, A, B, L=128, W=2, dtype="f32", target=90.0,
                             ctrl=("fraction", 0.5))
    assert info["W_used"] == 1 and not mask.any()
    assert same_bits(C, ref.C)
    assert same_bits(C, orc.gemm_plain(A, B, "f32"))


def test_control_off_again_and_argument_checks(tdg, orc):
    """Turning control off restores the plain plan's result; invalid settings
    fail with TDG_EINVAL before any device work; the mask before a pack fails
    with TDG_ESTATE."""
    from paper_1110_5765_gb300._lib import TDGemmError
    dtype, L = "f32", 128
    A, B = inputs((256, 256, 256), L, dtype, 950)
    p = tdg.Plan(256, 256, 256, L=L, W=2, dtype=dtype, form="sym", bits=6, rep_noise=None)
    with pytest.raises(TDGemmError) as e:
        p.kernel_mask()
    assert e.value.status == 8
    p.set_kernel_control("fraction", 0.5)
    C1 = p.run(dev(A), dev(B))
    p.set_kernel_control(None)
    C2 = p.run(dev(A), dev(B))
    torch.cuda.synchronize()
    ref = orc.tdgemm(A, B, L=L, W=2, dtype=dtype, form="sym", bits=6)
    ref_c = orc.tdgemm(A, B, L=L, W=2, dtype=dtype, form="sym", bits=6,
                       kernel_control=("fraction", 0.5))
    assert same_bits(C1.cpu().numpy(), ref_c.C)
    assert same_bits(C2.cpu().numpy(), ref.C)
    for bad in (("fraction", 1.5), ("fraction", -0.1), ("snr", math.nan)):
        with pytest.raises(TDGemmError) as e:
            p.set_kernel_control(*bad)
        assert e.value.status == 1
    p.close()
    for kw in (dict(form="asym", L=128), dict(form="sym", L=64),
               dict(form="sym", L=128, keep_packed=True)):
        q = tdg.Plan(256, 256, 256, W=2, dtype="f32", bits=6, rep_noise=None, **kw)
        with pytest.raises(TDGemmError) as e:
            q.set_kernel_control("fraction", 0.5)
        assert e.value.status == 1
        q.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[3])
@pytest.mark.parametrize("F", [1.0, 1.25, 1.5, 3.0])
def test_throughput_mode_matches_oracle(tdg, orc, case, F):
    """Sec. 6 (ii): a throughput target F (x the conventional product) through
    the measured F_W (here 1.7): the device computes the kernel count from
    the packing the planner chose; mask and C bit-identical to the oracle."""
    shape, L, W, dtype, bits = case
    A, B = inputs(shape, L, dtype, 750 + bits)
    ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form="sym", bits=bits,
                     kernel_control=("throughput", F, {W: 1.7}))
    C, mask, _ = run_ctrl(tdg, A, B, L=L, W=W, dtype=dtype, bits=bits, ctrl=("throughput", F),
                          speedup={f"{dtype}/sym/W{W}/L{L}": {"F": 1.7}})
    T = mask.size
    assert int(mask.sum()) == orc.kernels_for_throughput(T, F, 1.7)
    assert np.array_equal(mask.astype(bool), ref.plan.extra["kernel_mask"])
    assert same_bits(C, ref.C)


def test_throughput_mode_uses_the_planned_packing(tdg, orc):
    """Distortion-target plan (W chosen on the device among 3 and 2) with
    different F_W per packing: the count follows the F_W of the chosen W."""
    dtype, L, W = "f32", 128, 3
    A, B = inputs((384, 512, 400), L, dtype, 911)
    dense, tabs = {}, {}
    for w in (2, 3):
        d, arr = {}, np.full(192, -1.0)
        for t in range(0, orc.T_MAX[dtype] + 1):
            R = orc.r_level(t)
            s = 1e-3 * R * (w - 1) if R >= L else 0.0
            d[str(t)] = {"s": s}
            arr[t] = s
        tabs[orc.STable.key(dtype, "sym", w, L)] = d
        dense[w] = arr
    st = orc.STable(tabs)
    fw = {2: 1.55, 3: 2.2}
    seen = set()
    for target, F in ((15.0, 1.4), (25.0, 1.3)):       # the planner packs W = 3, then W = 2
        ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form="sym", target_db=target, s_table=st,
                         kernel_control=("throughput", F, fw))
        seen.add(ref.plan.W)
        C, mask, info = run_ctrl(tdg, A, B, L=L, W=W, dtype=dtype, target=target, rms=True,
                                 ctrl=("throughput", F), dense=dense,
                                 speedup={f"{dtype}/sym/W{w}/L{L}": {"F": v} for w, v in fw.items()})
        assert info["W_used"] == ref.plan.W >= 2
        assert int(mask.sum()) == orc.kernels_for_throughput(mask.size, F, fw[ref.plan.W])
        assert np.array_equal(mask.astype(bool), ref.plan.extra["kernel_mask"])
        assert same_bits(C, ref.C)
    assert seen == {2, 3}


def test_throughput_mode_argument_checks(tdg):
    from paper_1110_5765_gb300._lib import TDGemmError
    p = tdg.Plan(256, 256, 256, L=128, W=2, dtype="f32", form="sym", bits=6, rep_noise=None,
                 speedup=None)
    with pytest.raises(TDGemmError) as e:
        p.set_kernel_control("throughput", 1.3)     # no F_W given
    assert e.value.status == 1
    p.set_speedup(2, 1.6)
    with pytest.raises(TDGemmError) as e:
        p.set_kernel_control("throughput", 0.9)     # below the conventional product
    assert e.value.status == 1
    p.set_kernel_control("throughput", 1.3)
    with pytest.raises(TDGemmError):
        p.set_speedup(5, 1.5)
    with pytest.raises(TDGemmError):
        p.set_speedup(2, -1.0)
    p.close()
