"""Differentiation form: TDGemmFn forward/backward through the companded and
packed kernels (needs a GB300)."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5765_gb300 import build
    build.build()
    from paper_1110_5765_gb300 import autograd
    yield autograd
    for p in autograd._plans.values():
        assert p.info()["device_status"] == 0
    autograd.clear_plan_cache()


def snr(x, ref):
    x, ref = x.double(), ref.double()
    return 10 * math.log10(float((ref * ref).sum()) / float(((x - ref) ** 2).sum()))


OPTS = dict(L=128, W=2, form="sym", bits=8)


def test_backward_products_use_trans_flags_and_match_oracle(ag, orc):
    """dA = dC B^T and dB = A^T dC are the library's companded products of the
    transposed operands: bit-identical to the oracle on op() of the inputs."""
    A = torch.from_numpy(synth.gaussian((192, 256), 1, np.float32)).cuda().requires_grad_()
    B = torch.from_numpy(synth.gaussian((256, 160), 2, np.float32)).cuda().requires_grad_()
    G = torch.from_numpy(synth.gaussian((192, 160), 3, np.float32)).cuda()
    C = ag.tdg_matmul(A, B, **OPTS)
    C.backward(G)
    An, Bn, Gn = A.detach().cpu().numpy(), B.detach().cpu().numpy(), G.cpu().numpy()
    kw = dict(L=128, W=2, dtype="f32", form="sym", bits=8)
    assert np.array_equal(C.detach().cpu().numpy(), orc.tdgemm(An, Bn, **kw).C)
    assert np.array_equal(A.grad.cpu().numpy(), orc.tdgemm(Gn, Bn.T.copy(), **kw).C)
    assert np.array_equal(B.grad.cpu().numpy(), orc.tdgemm(An.T.copy(), Gn, **kw).C)


def test_gradients_against_fp64_and_finite_differences(ag):
    """Straight-through gradients: against the exact fp64 gradient (SNR) and
    against central finite differences of the smooth (unquantized) loss at 16
    sampled weights.  fp64 packing, 8-bit companders, W = 2: inside the
    error-free region, so only quantization noise (eq. 19) remains."""
    X = torch.from_numpy(synth.gaussian((512, 128), 11, np.float64)).cuda()
    Wt = torch.from_numpy(synth.gaussian((128, 256), 12, np.float64) / math.sqrt(128)).cuda()
    Y = torch.from_numpy(synth.gaussian((512, 256), 13, np.float64)).cuda()
    Wq = Wt.clone().requires_grad_()
    loss = ((torch.tanh(ag.tdg_matmul(X, Wq, dtype="f64", **OPTS)) - Y) ** 2).sum() / 2
    loss.backward()
    W64 = Wt.double().requires_grad_()
    l64 = ((torch.tanh(X.double() @ W64) - Y.double()) ** 2).sum() / 2
    l64.backward()
    s = snr(Wq.grad, W64.grad)
    assert s > 25.0, s

    def smooth(Wm):
        return float((((torch.tanh(X.double() @ Wm) - Y.double()) ** 2).sum() / 2).item())

    rng = np.random.default_rng(14)
    h = 1e-6
    diffs, refs = [], []
    for _ in range(16):
        i, j = int(rng.integers(128)), int(rng.integers(256))
        Wp, Wm = Wt.double().clone(), Wt.double().clone()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (smooth(Wp) - smooth(Wm)) / (2 * h)
        diffs.append(float(Wq.grad[i, j]) - fd)
        refs.append(fd)
    rel = math.sqrt(sum(d * d for d in diffs) / sum(r * r for r in refs))
    assert rel < 10 ** (-20 / 20), rel          # within the companding noise of ~25+ dB


def test_mlp_training_50_steps(ag):
    """Synthetic teacher MLP 128-1024-1024-10 (tanh), batch 4096, cross-entropy,
    SGD lr 0.1, 50 steps, every GEMM (forward and both adjoints) through
    TDGemmFn: the loss falls like fp32 training does."""
    sizes = [128, 1024, 1024, 10]
    teacher = [torch.from_numpy(w).cuda() for w in synth.mlp_teacher(sizes, 4)]
    X = torch.from_numpy(synth.mlp_inputs(4096, 128, 5)).cuda()
    with torch.no_grad():
        h = X
        for k, w in enumerate(teacher):
            h = h @ w
            if k < 2:
                h = torch.tanh(h)
        labels = h.argmax(1)
    init = [torch.from_numpy(w).cuda() for w in synth.mlp_teacher(sizes, 6)]
    opts = dict(L=128, W=2, form="sym", target_snr_db=20.0)

    def train(use_tdg):
        ws = [w.clone().requires_grad_() for w in init]
        losses = []
        for _ in range(50):
            h = X
            for k, w in enumerate(ws):
                h = ag.tdg_matmul(h, w, **opts) if use_tdg else h @ w
                if k < 2:
                    h = torch.tanh(h)
            loss = torch.nn.functional.cross_entropy(h, labels)
            for w in ws:
                w.grad = None
            loss.backward()
            with torch.no_grad():
                for w in ws:
                    w -= 0.1 * w.grad
            losses.append(float(loss.detach()))
        return losses

    ref = train(False)
    got = train(True)
    assert got[-1] < 0.8 * got[0]
    assert abs(got[-1] - ref[-1]) < 0.05 * ref[0]


@pytest.mark.parametrize("target", [20.0, 30.0])
def test_mlp_128_1024_1024_10_gradients_every_layer(ag, target):
    """The 128-1024-1024-10 MLP (tanh, batch 4096, synthetic teacher
    labels, cross-entropy) at the student's initial weights: every layer's dW
    from the companded-and-packed forward and adjoint products (fp32, sym,
    W = 2, distortion target ``target``) against
      (a) the exact fp64 gradient of the same loss, whole matrix (SNR), and
      (b) central finite differences (h = 1e-6, fp64) of the smooth
          (unquantized) loss at 16 sampled weights per layer, which first
          agree with the fp64 autograd gradient (pinning the reference).
    Straight-through: the gradient error is the companding noise of the
    products on the path, so it is bounded by the target less the depth of
    the chain (forward through up to three products, back through up to
    three)."""
    sizes = [128, 1024, 1024, 10]
    teacher = [torch.from_numpy(w).cuda().double() for w in synth.mlp_teacher(sizes, 4)]
    X32 = torch.from_numpy(synth.mlp_inputs(4096, 128, 5)).cuda()
    X64 = X32.double()
    with torch.no_grad():
        h = X64
        for k, w in enumerate(teacher):
            h = h @ w
            if k < 2:
                h = torch.tanh(h)
        labels = h.argmax(1)
    init = [torch.from_numpy(w).cuda() for w in synth.mlp_teacher(sizes, 6)]
    opts = dict(L=128, W=2, form="sym", target_snr_db=target)

    def loss_of(ws, X, mm):
        h = X
        for k, w in enumerate(ws):
            h = mm(h, w)
            if k < 2:
                h = torch.tanh(h)
        return torch.nn.functional.cross_entropy(h, labels)

    ws = [w.clone().requires_grad_() for w in init]
    loss_of(ws, X32, lambda a, b: ag.tdg_matmul(a, b, **opts)).backward()
    w64 = [w.double().clone().requires_grad_() for w in init]
    loss_of(w64, X64, lambda a, b: a @ b).backward()

    rng = np.random.default_rng(7)
    h = 1e-6
    for k in range(3):
        g, g64 = ws[k].grad.double(), w64[k].grad
        s = snr(g, g64)
        assert s > target - 12.0, (k, s)
        fds, got, ex = [], [], []
        for _ in range(16):
            i, j = int(rng.integers(sizes[k])), int(rng.integers(sizes[k + 1]))
            vals = []
            for d in (h, -h):
                wd = [w.detach().double().clone() for w in init]
                wd[k][i, j] += d
                with torch.no_grad():
                    vals.append(float(loss_of(wd, X64, lambda a, b: a @ b)))
            fds.append((vals[0] - vals[1]) / (2 * h))
            got.append(float(g[i, j]))
            ex.append(float(g64[i, j]))
        fds, got, ex = np.array(fds), np.array(got), np.array(ex)
        ref_scale = math.sqrt(float(np.mean(fds * fds)))
        assert np.sqrt(np.mean((ex - fds) ** 2)) < 1e-4 * ref_scale, k
        rel = math.sqrt(float(np.mean((got - fds) ** 2))) / ref_scale
        assert rel < 10 ** (-(target - 14.0) / 20), (k, rel)
