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


def _fp8_bound(orc, A, B, ref, rows, cols, L=128):
    """Elementwise bound on |C_gpu - C_oracle| for the E4M3 form over an output
    window.  Both sides compute, per slab l, a sum of L exact products
    a~ b~ (E4M3 products are exact in fp32), round it to fp32 (the oracle
    once, the tensor core along its own accumulation order: at most L
    roundings of 2^-24 relative to a partial sum no larger than
    sum |a~ b~|), and then run the same fma chain over the slabs, whose nK
    roundings differ by at most 2^-23 of its running magnitude.  So
    |dC| <= (L + nK) 2^-23 sum_l (s_A s_B)_l sum_k |a~ b~|."""
    r0, r1 = rows
    c0, c1 = cols
    K = A.shape[1]
    nK = -(-K // L)
    cA = np.repeat(ref.cA.astype(np.float32), L, 1)[:, :K]       # per (row block, k)
    cB = np.repeat(ref.cB.astype(np.float32), L, 0)[:K]          # per (k, column block)
    ib = np.arange(r0, r1) // L
    jb = np.arange(c0, c1) // L
    Aq = np.abs(orc.e4m3((A[r0:r1] * cA[ib]).astype(np.float64)))
    Bq = np.abs(orc.e4m3((B[:, c0:c1] * cB[:, jb]).astype(np.float64)))
    tot = np.zeros((r1 - r0, c1 - c0))
    for l in range(nK):
        k0, k1 = l * L, min(K, (l + 1) * L)
        scale = np.outer(ref.sA[ib, l], ref.sB[l, jb])
        tot += (Aq[:, k0:k1] @ Bq[k0:k1]) * scale
    return (L + nK) * 2.0**-23 * tot


def test_tc_fp8_multi_tile_persistent_full_c(tdg, orc):
    """E4M3 and the integer form at 4000 x 400 x 3900: 256 output tile pairs
    over at most 76 clusters, so every cluster walks several tiles and the
    double-buffered accumulators' phases wrap many times (ragged M, N and a
    16-wide last slab).  Integer form bit-exact over all of C; E4M3 within the
    fp32 accumulation bound everywhere and whole-C SNR within 0.1 dB of the
    oracle's."""
    M, K, N = 4000, 400, 3900
    A = synth.laplace((M, K), 61, np.float32)
    B = synth.laplace((K, N), 62, np.float32)
    ex = orc.exact_gemm(A, B)
    ref_i = orc.tc_int_gemm(A, B, L=128, bits=8)
    C, _ = run_tc(tdg, A, B, form="tc_int", bits=8)
    assert same_bits(C, ref_i.C)
    ref = orc.tc_fp8_gemm(A, B, L=128)
    C, info = run_tc(tdg, A, B, form="tc_fp8")
    assert info["carrier"] == 8
    bound = _fp8_bound(orc, A, B, ref, (0, M), (0, N))
    assert np.all(np.abs(C.astype(np.float64) - ref.C) <= bound + 1e-30)
    assert abs(orc.snr_db(C, ex) - orc.snr_db(ref.C, ex)) < 0.1


def test_tc_fp8_precision_size_sampled(tdg, orc):
    """E4M3 at the precision-form workload, 8192^3 Laplacian(b = 1), L = 128:
    13.5 tile pairs per cluster and 64 slabs per tile.  Three sampled 128 x 128
    tiles over the full K (one in the last row and column of tiles) within the
    fp32 accumulation bound, and their SNR within 0.1 dB of the oracle's."""
    n = 8192
    A = synth.laplace((n, n), 51, np.float32)
    B = synth.laplace((n, n), 52, np.float32)
    C, info = run_tc(tdg, A, B, form="tc_fp8")
    tiles = synth.sample_tiles(64, 64, 2, seed=54) + [(63, 63)]
    got, want, exact = [], [], []
    for (ti, tj) in tiles:
        rows, cols = (ti * 128, ti * 128 + 128), (tj * 128, tj * 128 + 128)
        ref = orc.tc_fp8_gemm(A, B, L=128, rows=rows, cols=cols)
        g = C[rows[0]:rows[1], cols[0]:cols[1]]
        bound = _fp8_bound(orc, A, B, ref, rows, cols)
        assert np.all(np.abs(g.astype(np.float64) - ref.C) <= bound + 1e-30), (ti, tj)
        got.append(g)
        want.append(ref.C)
        exact.append(orc.exact_gemm(A, B, rows, cols))
    ex = np.concatenate([e.ravel() for e in exact])
    sg = orc.snr_db(np.concatenate([x.ravel() for x in got]), ex)
    so = orc.snr_db(np.concatenate([x.ravel() for x in want]), ex)
    assert abs(sg - so) < 0.1, (sg, so)


def _fma32(a, b, c):
    """fp32 fma(a, b, c) with one rounding, elementwise (exact rationals)."""
    from fractions import Fraction
    a, b, c = (np.asarray(x, np.float32) for x in (a, b, c))
    out = np.empty(a.shape, np.float32)
    fa, fb, fc = a.ravel(), b.ravel(), c.ravel()
    o = out.ravel()
    for i in range(fa.size):
        v = Fraction(float(fa[i])) * Fraction(float(fb[i])) + Fraction(float(fc[i]))
        o[i] = np.float32(float(v)) if v == 0 else _round32(v)
    return out


def _round32(v):
    """Round a rational to the nearest fp32, ties to even (no overflow here)."""
    from fractions import Fraction
    import math
    sign = -1 if v < 0 else 1
    v = abs(v)
    e = math.floor(math.log2(v.numerator) - math.log2(v.denominator))
    while Fraction(2) ** e > v:
        e -= 1
    while Fraction(2) ** (e + 1) <= v:
        e += 1
    q = max(e, -126) - 23                      # quantum of the binade (subnormals below 2^-126)
    m = v / Fraction(2) ** q
    n = m.numerator // m.denominator
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return np.float32(sign * float(Fraction(n) * Fraction(2) ** q))


@pytest.mark.parametrize("L", [64, 128])
def test_tc_int_output_paths_alpha_beta_ldc(tdg, orc, L):
    """The three ways C leaves the tensor-core kernel: TMA stores (beta = 0,
    16-byte aligned rows), plain stores with beta != 0 (C read back), and
    plain stores where a row pitch of N + 1 floats rules the TMA map out.
    Each equals alpha * C_oracle (one fp32 rounding) or fma(alpha, C_oracle,
    beta * C_in) bit for bit; 300 rows and 260 columns leave ragged edge tiles."""
    M, K, N = 300, 256, 260
    A = synth.laplace((M, K), 71, np.float32)
    B = synth.laplace((K, N), 72, np.float32)
    ref = orc.tc_int_gemm(A, B, L=L, bits=8).C.astype(np.float32)
    alpha = np.float32(0.75)
    cases = [(0.0, N), (-1.5, N), (0.0, N + 1)]
    for beta, ldc in cases:
        p = tdg.Plan(M, N, K, L=L, W=1, dtype="f32", form="tc_int", bits=8, ldc=ldc)
        Cin = synth.gaussian((M, ldc), 73, np.float32)
        Cfull = dev(Cin)
        C = Cfull[:, :N]
        p.run(dev(A), dev(B), C, float(alpha), beta)
        torch.cuda.synchronize()
        assert p.info()["device_status"] == 0
        p.close()
        got = Cfull.cpu().numpy()
        if beta == 0.0:
            want = (alpha * ref).astype(np.float32)
        else:
            want = _fma32(np.full_like(ref, alpha), ref, (np.float32(beta) * Cin[:, :N]).astype(np.float32))
        assert same_bits(got[:, :N], want), (beta, ldc)
        if ldc > N:
            assert same_bits(got[:, N:], Cin[:, N:]), "padding column written"


@pytest.mark.parametrize("form,bits,target", [("tc_int", 8, math.nan), ("tc_int", 0, 40.0),
                                              ("tc_fp8", 0, math.nan)])
def test_tc_zero_blocks(tdg, orc, form, bits, target):
    """All-zero blocks (c = s = 0) on the tensor-core forms: a slab of A zero
    in every row block and a zero column panel of B, ragged M, K, N (both
    the k-contiguous A and the x-contiguous B path of the code kernels): the
    integer form bit-exact, E4M3 within the fp32-summation bound; the zero
    panel exactly 0."""
    L = 128
    A = synth.laplace((300, 5 * L + 40), 1411, np.float32)
    B = synth.gaussian((5 * L + 40, 2 * L + 30), 1412, np.float32)
    A[:, 2 * L:3 * L] = 0
    B[:, L:2 * L] = 0
    if form == "tc_int":
        ref = orc.tc_int_gemm(A, B, L=L, bits=bits)
        C, info = run_tc(tdg, A, B, form=form, bits=bits, target=target)
        assert (info["gamma_a"], info["gamma_b"]) == (ref.plan.gA, ref.plan.gB)
        assert same_bits(C, ref.C)
    else:
        ref = orc.tc_fp8_gemm(A, B, L=L)
        C, _ = run_tc(tdg, A, B, form=form)
        bound = _fp8_bound(orc, A, B, ref, (0, A.shape[0]), (0, B.shape[1]), L)
        assert np.all(np.abs(C.astype(np.float64) - ref.C) <= bound + 1e-30)
    assert np.all(C[:, L:2 * L] == 0)
