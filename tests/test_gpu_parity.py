"""GPU path against the CPU oracle, through the C ABI (needs a GB300)."""
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


NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def stored(X, trans):
    """the stored matrix whose op() is X"""
    return np.ascontiguousarray(X.T) if trans == "T" else np.ascontiguousarray(X)


def run_gpu(tdg, A, B, *, L, W, dtype, form, transA="N", transB="N", bits=0, target=math.nan,
            manual=None, keep_packed=False, alpha=1.0, beta=0.0, Cin=None, rep=None,
            allow_fallback=True, expect_status=0):
    M, K = A.shape
    N = B.shape[1]
    As, Bs = dev(stored(A, transA)), dev(stored(B, transB))
    p = tdg.Plan(M, N, K, L=L, W=W, dtype=dtype, form=form, bits=bits, target_snr_db=target,
                 transA=transA, transB=transB, keep_packed=keep_packed,
                 allow_fallback=allow_fallback, rep_noise=rep)
    if manual is not None:
        p.set_manual(*manual)
    C = dev(Cin) if Cin is not None else torch.zeros((M, N), dtype=TT[dtype], device="cuda")
    p.run(As, Bs, C, alpha, beta)
    torch.cuda.synchronize()
    out = {"C": C.cpu().numpy(), "info": p.info(), "plan": p}
    assert out["info"]["device_status"] == expect_status, out["info"]
    if keep_packed:
        nK = -(-K // L)
        r = torch.zeros((M, N, nK), dtype=torch.int64, device="cuda")
        C2 = torch.zeros((M, N), dtype=TT[dtype], device="cuda")
        p.unpack(r, C2)
        torch.cuda.synchronize()
        out["rint"] = r.cpu().numpy()
        out["C_unfused"] = C2.cpu().numpy()
    return out


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))


# ------------------------------------------------- 256^3 fp64, 8 bits, W = 2
@pytest.mark.parametrize("form", ["sym", "asym"])
def test_256_fp64_8bit_w2_bitexact(tdg, orc, form):
    """256^3 fp64 Gaussian, L = 64, 8-bit companding, W = 2: integers and C
    bit-identical to the oracle; plan identical."""
    A = synth.gaussian((256, 256), 1111)
    B = synth.gaussian((256, 256), 1112)
    ref = orc.tdgemm(A, B, L=64, W=2, dtype="f64", form=form, bits=8, want_rint=True)
    g = run_gpu(tdg, A, B, L=64, W=2, dtype="f64", form=form, bits=8, keep_packed=True)
    i = g["info"]
    assert (i["W_used"], i["q"], i["gamma_a"], i["gamma_b"], i["r_max"], i["w_ef"]) == \
        (ref.plan.W, ref.plan.q, ref.plan.gA, ref.plan.gB, ref.plan.R, ref.plan.Wef)
    assert np.array_equal(g["rint"], ref.rint)
    assert same_bits(g["C"], ref.C)
    assert same_bits(g["C_unfused"], ref.C)
    assert abs(i["pred_snr_db"] - ref.plan.pred_snr_db) < 1e-9
    assert i["device_status"] == 0


# ------------------------------------------------------------------ tiny ragged shapes
def _largest_R(orc, W, dtype, L):
    best = 0
    for R in range(L, 1 << 24, L):
        if orc.w_ef(R, orc.q_for(R), dtype) >= W:
            best = R
        elif best and R > 4 * best:
            break
    return best


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", ["sym", "asym"])
@pytest.mark.parametrize("W", [1, 2, 3, 4])
def test_tiny_ragged_manual(tdg, orc, dtype, form, W):
    """Sizes {1, W, L-1, L+1, 2L} on every axis (L = 16), integer inputs,
    c = 1: C and the per-slab integers bit-identical to the oracle (inside
    the error-free region they are also the brute-force products)."""
    L = 16
    Rlim = max(_largest_R(orc, max(W, 2), dtype, L), 4 * L)
    g_ = max(1, int(math.isqrt(Rlim // L)))
    gA, gB = g_, max(1, (Rlim // L) // g_)
    q = orc.q_for(L * gA * gB)
    T = NP[dtype]
    for M in sorted({1, W, L - 1, L + 1, 2 * L}):
        for K in sorted({1, W, L - 1, L + 1, 2 * L}):
            for N in (1, L + 1):
                A = synth.int_uniform((M, K), 100 + M * 7 + K, gA).astype(T)
                B = synth.int_uniform((K, N), 200 + K * 5 + N, gB).astype(T)
                ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form=form, manual=(q, 1.0, 1.0),
                                 want_rint=True)
                g = run_gpu(tdg, A, B, L=L, W=W, dtype=dtype, form=form, bits=8,
                            manual=(q, 1.0, 1.0), keep_packed=True)
                assert same_bits(g["C"], ref.C), (M, K, N)
                assert np.array_equal(g["rint"], ref.rint), (M, K, N)


# ------------------------------------------------------------------ beyond headroom
@pytest.mark.parametrize("dtype,W,gam", [("f32", 2, (60, 60)), ("f32", 3, (20, 20)),
                                         ("f64", 3, (300, 300)), ("f64", 4, (80, 80))])
@pytest.mark.parametrize("form", ["sym", "asym"])
def test_beyond_headroom_bit_identical(tdg, orc, dtype, W, gam, form):
    """Past Prop. 1's limit the result depends on the order of every rounding;
    the fixed fma order makes GPU and oracle agree bit for bit anyway."""
    T = NP[dtype]
    A = synth.uniform((200, 300), 7, T)
    B = synth.uniform((300, 150), 8, T)
    L = 64
    gA, gB = gam
    q = orc.q_for(L * gA * gB)
    assert orc.w_ef(L * gA * gB, q, dtype) < W
    ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form=form, manual=(q, float(gA), float(gB)),
                     want_rint=True)
    g = run_gpu(tdg, A, B, L=L, W=W, dtype=dtype, form=form, bits=8,
                manual=(q, float(gA), float(gB)), keep_packed=True)
    assert np.array_equal(g["rint"], ref.rint)
    assert same_bits(g["C"], ref.C)


# ------------------------------------------------------------------ transposes, alpha/beta
@pytest.mark.parametrize("transA,transB", [("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("form", ["plain", "sym", "asym"])
def test_transposes(tdg, orc, transA, transB, form):
    A = synth.laplace((130, 200), 11, np.float32)
    B = synth.laplace((200, 70), 12, np.float32)
    W = 1 if form == "plain" else 2
    ref = orc.tdgemm(A, B, L=64, W=W, dtype="f32", form=form, bits=6)
    g = run_gpu(tdg, A, B, L=64, W=W, dtype="f32", form=form, bits=6, transA=transA,
                transB=transB)
    assert same_bits(g["C"], ref.C)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", ["plain", "sym", "asym"])
def test_alpha_beta(tdg, orc, dtype, form):
    T = NP[dtype]
    A = synth.gaussian((100, 90), 21, T)
    B = synth.gaussian((90, 110), 22, T)
    Cin = synth.gaussian((100, 110), 23, T)
    W = 1 if form == "plain" else 2
    ref = orc.tdgemm(A, B, L=32, W=W, dtype=dtype, form=form, bits=7, alpha=0.75, beta=-1.5,
                     C_in=Cin)
    g = run_gpu(tdg, A, B, L=32, W=W, dtype=dtype, form=form, bits=7, alpha=0.75, beta=-1.5,
                Cin=Cin)
    assert same_bits(g["C"], ref.C)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_plain_equals_oracle_fma_chain(tdg, orc, dtype):
    T = NP[dtype]
    A = synth.gaussian((257, 300), 31, T)
    B = synth.gaussian((300, 129), 32, T)
    g = run_gpu(tdg, A, B, L=128, W=1, dtype=dtype, form="plain")
    assert same_bits(g["C"], orc.gemm_plain(A, B, dtype))


# ------------------------------------------------------------------ planner (target mode)
def _synthetic_table(orc, dtype, form, L, Wmax):
    """A made-up s(R) table (not a measurement) fed to both planners, so the
    planner logic is compared on identical inputs."""
    tabs, dense = {}, {}
    for W in range(2, Wmax + 1):
        d, arr = {}, np.full(192, -1.0)
        for t in range(0, orc.T_MAX[dtype] + 1):
            R = orc.r_level(t)
            s = 1e-3 * R * (W - 1) if R >= L else 0.0
            d[str(t)] = {"s": s}
            arr[t] = s
        tabs[orc.STable.key(dtype, form, W, L)] = d
        dense[W] = arr
    return orc.STable(tabs), dense


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", ["sym", "asym"])
@pytest.mark.parametrize("target", [10.0, 30.0, 60.0])
@pytest.mark.parametrize("rms", [False, True])
def test_target_mode_matches_oracle(tdg, orc, dtype, form, target, rms):
    T = NP[dtype]
    L = 64
    A = 3.0 * synth.uniform((192, 256), 41, T)
    B = synth.laplace((256, 160), 42, T)
    st, dense = _synthetic_table(orc, dtype, form, L, 3)
    ref = orc.tdgemm(A, B, L=L, W=3, dtype=dtype, form=form, target_db=target, s_table=st,
                     noise_rms=rms)
    M, K = A.shape
    N = B.shape[1]
    p = tdg.Plan(M, N, K, L=L, W=3, dtype=dtype, form=form, target_snr_db=target, rep_noise=None,
                 noise_rms=rms)
    for W in (2, 3):
        p.set_rep_noise(W, dense[W], 0)
    C = torch.zeros((M, N), dtype=TT[dtype], device="cuda")
    p.run(dev(A), dev(B), C)
    i = p.info()
    assert i["device_status"] == 0, i
    assert i["W_used"] == ref.plan.W
    if ref.plan.W > 1:
        assert (i["q"], i["gamma_a"], i["gamma_b"], i["level"]) == \
            (ref.plan.q, ref.plan.gA, ref.plan.gB, ref.plan.t)
        assert abs(i["pred_snr_db"] - ref.plan.pred_snr_db) < 1e-6
    assert same_bits(C.cpu().numpy(), ref.C)


def test_unreachable_without_fallback(tdg, orc):
    A = synth.gaussian((64, 64), 51, np.float32)
    B = synth.gaussian((64, 64), 52, np.float32)
    g = run_gpu(tdg, A, B, L=64, W=2, dtype="f32", form="sym", target=90.0,
                allow_fallback=False, rep=None, expect_status=5)
    assert g["info"]["device_status"] == 5       # TDG_EUNREACHABLE
    g = run_gpu(tdg, A, B, L=64, W=2, dtype="f32", form="sym", target=90.0, rep=None)
    assert g["info"]["W_used"] == 1 and g["info"]["device_status"] == 0
    assert same_bits(g["C"], orc.gemm_plain(A, B, "f32"))


def test_nonfinite_input_flagged(tdg):
    A = synth.gaussian((64, 64), 61, np.float32)
    A[3, 5] = np.nan
    B = synth.gaussian((64, 64), 62, np.float32)
    g = run_gpu(tdg, A, B, L=64, W=2, dtype="f32", form="sym", bits=6, expect_status=7)
    assert g["info"]["device_status"] == 7       # TDG_ENONFINITE


def test_snr_reduction(tdg):
    C = synth.gaussian((300, 200), 71, np.float32)
    R = synth.gaussian((300, 200), 72, np.float64)
    s = tdg.snr_sums(dev(C), dev(R))
    err = C.astype(np.float64) - R
    assert math.isclose(s[0], float(np.sum(R * R)), rel_tol=1e-12)
    assert math.isclose(s[1], float(np.sum(err * err)), rel_tol=1e-12)
    assert math.isclose(s[2], float(np.sum(err)), rel_tol=1e-9, abs_tol=1e-9)


# ------------------------------------------------------------------ full size, sampled
@pytest.mark.parametrize("form", ["sym", "asym"])
def test_distortion_sweep_size_sampled_tiles(tdg, orc, form):
    """4096^3 fp32 uniform, L = 128, W = 2, fixed 6-bit companders (the launch
    shape of the benchmark): three sampled 128 x 128 output tiles over the full
    K equal the oracle's bit for bit."""
    n = 4096
    A = synth.uniform((n, n), 81, np.float32)
    B = synth.uniform((n, n), 82, np.float32)
    g = run_gpu(tdg, A, B, L=128, W=2, dtype="f32", form=form, bits=6)
    for (ti, tj) in synth.sample_tiles(32, 32, 3, seed=83):
        rows, cols = (ti * 128, ti * 128 + 128), (tj * 128, tj * 128 + 128)
        ref = orc.tdgemm(A, B, L=128, W=2, dtype="f32", form=form, bits=6, rows=rows, cols=cols)
        assert same_bits(g["C"][rows[0]:rows[1], cols[0]:cols[1]], ref.C), (ti, tj)


def test_benchmark_configuration_sampled_tiles(tdg, orc):
    """The benchmark's own configuration and inputs (4096^3 fp32 uniform[-1,1]
    drawn from the benchmark's seeds 1112 / 1113, L = 128, symmetric W = 2,
    20 dB target, the built-in s-table): the device planner's choice equals the
    oracle's on the full matrices and three sampled 128 x 128 output tiles over
    the full K equal the oracle's bit for bit."""
    n = 4096
    A = synth.uniform((n, n), 1112, np.float32)
    B = synth.uniform((n, n), 1113, np.float32)
    # the plan exactly as the benchmark makes it (built-in s-table)
    p = tdg.Plan(n, n, n, L=128, W=2, dtype="f32", form="sym", target_snr_db=20.0)
    C = p.run(dev(A), dev(B))
    torch.cuda.synchronize()
    info = p.info()
    p.close()
    assert info["device_status"] == 0, info
    g = {"C": C.cpu().numpy()}
    st = orc.load_s_table()
    for (ti, tj) in synth.sample_tiles(32, 32, 3, seed=1114):
        rows, cols = (ti * 128, ti * 128 + 128), (tj * 128, tj * 128 + 128)
        ref = orc.tdgemm(A, B, L=128, W=2, dtype="f32", form="sym", target_db=20.0,
                         s_table=st, rows=rows, cols=cols)
        assert (info["W_used"], info["q"], info["gamma_a"], info["gamma_b"]) == \
            (ref.plan.W, ref.plan.q, ref.plan.gA, ref.plan.gB)
        assert abs(info["pred_snr_db"] - ref.plan.pred_snr_db) < 1e-6
        assert same_bits(g["C"][rows[0]:rows[1], cols[0]:cols[1]], ref.C), (ti, tj)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", ["sym", "asym"])
@pytest.mark.parametrize("W", [1, 2, 3, 4])
def test_fixed_bits_per_block_companders(tdg, orc, dtype, form, W):
    """Per-block companders that differ block to block (Laplacian rows scaled
    per block), ragged sizes, every W: bit-identical to the oracle."""
    T = NP[dtype]
    A = synth.laplace((200, 300), 91, T) * np.repeat(np.linspace(0.5, 4, 4), 64)[:200, None].astype(T)
    B = synth.laplace((300, 150), 92, T)
    ref = orc.tdgemm(A, B, L=64, W=W, dtype=dtype, form=form, bits=6)
    g = run_gpu(tdg, A, B, L=64, W=W, dtype=dtype, form=form, bits=6)
    assert same_bits(g["C"], ref.C)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", ["sym", "asym"])
def test_few_tiles_many_slabs(tdg, orc, dtype, form):
    """Few output tiles over many slabs (the plan splits the slabs of each tile
    over several CTAs and sums them in order in a second kernel): C equals the
    oracle bit for bit, including alpha / beta, beyond the error-free region."""
    T = NP[dtype]
    M, K, N = 200, 4096 + 70, 250
    A = synth.laplace((M, K), 1301, T)
    B = synth.gaussian((K, N), 1302, T)
    Cin = synth.gaussian((M, N), 1303, T)
    W = 2 if dtype == "f32" else 3
    ref = orc.tdgemm(A, B, L=128, W=W, dtype=dtype, form=form, bits=7, alpha=0.75, beta=-1.5,
                     C_in=Cin)
    g = run_gpu(tdg, A, B, L=128, W=W, dtype=dtype, form=form, bits=7, alpha=0.75, beta=-1.5,
                Cin=Cin)
    assert same_bits(g["C"], ref.C)


# ------------------------------------------------------------------ all-zero blocks
def _run_target(tdg, orc, A, B, *, L, W, dtype, form, target):
    """Target mode on both sides with the same made-up s(R) table."""
    st, dense = _synthetic_table(orc, dtype, form, L, W)
    ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form=form, target_db=target, s_table=st)
    M, K = A.shape
    N = B.shape[1]
    p = tdg.Plan(M, N, K, L=L, W=W, dtype=dtype, form=form, target_snr_db=target, rep_noise=None)
    for w in range(2, W + 1):
        p.set_rep_noise(w, dense[w], 0)
    C = torch.zeros((M, N), dtype=TT[dtype], device="cuda")
    p.run(dev(A), dev(B), C)
    i = p.info()
    assert i["device_status"] == 0, i
    assert i["W_used"] == ref.plan.W
    if ref.plan.W > 1:
        assert (i["q"], i["gamma_a"], i["gamma_b"], i["level"]) == \
            (ref.plan.q, ref.plan.gA, ref.plan.gB, ref.plan.t)
        if math.isinf(ref.plan.pred_snr_db):
            assert i["pred_snr_db"] == ref.plan.pred_snr_db
        else:
            assert abs(i["pred_snr_db"] - ref.plan.pred_snr_db) < 1e-6
    return C.cpu().numpy(), ref


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("form", ["sym", "asym"])
@pytest.mark.parametrize("mode", ["bits", "target"])
def test_zero_blocks(tdg, orc, dtype, form, mode):
    """All-zero blocks (c = s = 0): a slab of A zero in every row block and a
    zero column panel of B, ragged M, K, N; fixed bits at W = 2 and 3, and
    target mode: C (and the plan) bit-identical to the oracle, the zero panel
    exactly 0."""
    L = 64
    T = NP[dtype]
    A = synth.gaussian((3 * L + 5, 5 * L + 9), 1401, T)
    B = synth.laplace((5 * L + 9, 2 * L + 7), 1402, T)
    A[:, 2 * L:3 * L] = 0
    B[:, L:2 * L] = 0
    if mode == "bits":
        for W in (2, 3):
            ref = orc.tdgemm(A, B, L=L, W=W, dtype=dtype, form=form, bits=7)
            g = run_gpu(tdg, A, B, L=L, W=W, dtype=dtype, form=form, bits=7)
            assert same_bits(g["C"], ref.C), W
            assert np.all(g["C"][:, L:2 * L] == 0)
    else:
        C, ref = _run_target(tdg, orc, A, B, L=L, W=3, dtype=dtype, form=form, target=20.0)
        assert ref.plan.W >= 2
        assert same_bits(C, ref.C)
        assert np.all(C[:, L:2 * L] == 0)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_zero_operand_target_mode(tdg, orc, dtype):
    """A = 0: the model's noise and signal vanish (predicted SNR infinite), so
    both planners keep the requested W at the lowest R_max level; C = 0."""
    L = 64
    A = np.zeros((2 * L + 3, 3 * L), NP[dtype])
    B = synth.gaussian((3 * L, 2 * L), 1403, NP[dtype])
    C, ref = _run_target(tdg, orc, A, B, L=L, W=3, dtype=dtype, form="sym", target=30.0)
    assert ref.plan.W == 3 and math.isinf(ref.plan.pred_snr_db)
    assert same_bits(C, ref.C) and np.all(C == 0)
