"""tdgemm_run_host (host buffers in, host buffer out) against the device path
(needs a GB300).  Pinned C takes the in-place path (the GEMM writes C over the
CPU-GPU link), pageable C and beta != 0 the staged copy back; every path must
give the device path's bits."""
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


CASES = {
    "sym_f32_w2": dict(M=300, N=260, K=270, form="sym", W=2, dtype="f32", target_snr_db=20.0),
    "asym_f32_w2": dict(M=256, N=384, K=512, form="asym", W=2, dtype="f32", target_snr_db=20.0),
    "sym_f64_w3": dict(M=200, N=136, K=300, form="sym", W=3, dtype="f64", target_snr_db=40.0),
    "plain_f32": dict(M=130, N=300, K=270, form="plain", W=1, dtype="f32"),
    "tc_int8": dict(M=130, N=300, K=270, form="tc_int", W=1, dtype="f32", bits=8),
}


def host(x, pinned):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("name", list(CASES))
def test_run_host_matches_device(tdg, name, pinned):
    kw = dict(CASES[name])
    M, N, K = kw.pop("M"), kw.pop("N"), kw.pop("K")
    dt = np.float64 if kw["dtype"] == "f64" else np.float32
    A = synth.uniform((M, K), 700 + M, dt)
    B = synth.uniform((K, N), 701 + N, dt)
    C0 = synth.uniform((M, N), 702, dt)
    p = tdg.Plan(M, N, K, L=64, **kw)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ref = p.run(Ad, Bd).cpu().numpy()
    Cin = torch.from_numpy(C0).cuda()
    ref2 = p.run(Ad, Bd, Cin, alpha=0.5, beta=-1.25).cpu().numpy()
    torch.cuda.synchronize()

    Ah, Bh = host(A, pinned), host(B, pinned)
    Ch = host(np.zeros((M, N), dt), pinned)
    p.run_host(Ah, Bh, Ch)
    assert np.array_equal(Ch.numpy().view(np.uint8), ref.view(np.uint8))
    Ch2 = host(C0, pinned)
    p.run_host(Ah, Bh, Ch2, alpha=0.5, beta=-1.25)
    assert np.array_equal(Ch2.numpy().view(np.uint8), ref2.view(np.uint8))
    assert p.info()["device_status"] == 0
    p.close()


@pytest.mark.parametrize("name", list(CASES))
def test_run_host_async_pipeline_matches_device(tdg, name):
    """Five pipelined calls on one plan and stream, inputs alternating between
    three pinned sets and C between fresh buffers (beta = 0) and C_in with
    alpha, beta: the copies of a call overlap the previous call's computation
    through the plan's two staging sets; every C equals the device path's bits
    after one synchronisation at the end."""
    kw = dict(CASES[name])
    M, N, K = kw.pop("M"), kw.pop("N"), kw.pop("K")
    dt = np.float64 if kw["dtype"] == "f64" else np.float32
    p = tdg.Plan(M, N, K, L=64, **kw)
    sets = [(synth.uniform((M, K), 710 + i, dt), synth.uniform((K, N), 720 + i, dt)) for i in range(3)]
    C0 = synth.uniform((M, N), 730, dt)
    calls = [(0, 1.0, 0.0), (1, 0.5, -1.25), (2, 1.0, 0.0), (0, 0.75, 0.5), (1, 1.0, 0.0)]
    refs = []
    for i, alpha, beta in calls:
        A, B = sets[i]
        Cin = torch.from_numpy(C0).cuda()
        refs.append(p.run(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cin, alpha, beta)
                    .cpu().numpy().copy())
    torch.cuda.synchronize()
    hsets = [(host(A, True), host(B, True)) for A, B in sets]
    outs = []
    stream = torch.cuda.Stream()
    for i, alpha, beta in calls:
        Ch = host(C0 if beta != 0.0 else np.zeros((M, N), dt), True)
        p.run_host_async(hsets[i][0], hsets[i][1], Ch, alpha, beta, stream=stream)
        outs.append(Ch)
    stream.synchronize()
    for k, (Ch, ref) in enumerate(zip(outs, refs)):
        assert np.array_equal(Ch.numpy().view(np.uint8), ref.view(np.uint8)), k
    assert p.info()["device_status"] == 0
    p.close()


def test_run_host_async_rejects_pageable(tdg):
    p = tdg.Plan(64, 64, 64, L=64, W=1, dtype="f32", form="plain")
    A = torch.zeros((64, 64))
    with pytest.raises(ValueError):
        p.run_host_async(A, A, A)
    from paper_1110_5765_gb300 import _lib
    L = _lib.load()
    assert L.tdgemm_run_host_async(p._h, A.data_ptr(), A.data_ptr(), A.data_ptr(), 1.0, 0.0, None) == 1
    p.close()
