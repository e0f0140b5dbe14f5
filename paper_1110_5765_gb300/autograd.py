"""Differentiation form: the companded-and-packed product behind
``torch.autograd.Function``.

forward:   C  = op(A) op(B)              through tdgemm (steps a-d)
backward:  dA = dC op(B)^T,  dB = op(A)^T dC
           through the same companded/packed kernels, with the transposes
           expressed as the trans flags of the C ABI (no copies).
The quantizer is straight-through: its derivative is taken as the identity,
so the backward products see the incoming gradient and the saved (unquantized)
inputs; each backward product is companded and packed on its own, with
companders and packing chosen from its own block statistics (Sec. 5, Sec. 6).
Inside CUDA-graph capture the two adjoints of one product run on two streams.

Plans (device workspace) are cached per shape, layout and options.
"""
from __future__ import annotations

import torch

from .api import Plan

_plans: dict = {}


def _op_layout(X: torch.Tensor):
    """(trans, ld, stored tensor) such that op(stored) == X without copying."""
    r, c = X.shape
    s0, s1 = X.stride()
    if s1 == 1 and s0 >= c:
        return "N", s0, X
    if s0 == 1 and s1 >= r:
        return "T", s1, X.t()
    X = X.contiguous()
    return "N", c, X


_side: dict = {}


def _side_stream(device) -> "torch.cuda.Stream":
    key = torch.device(device).index
    st = _side.get(key)
    if st is None:
        st = torch.cuda.Stream(device=device)
        _side[key] = st
    return st


def _plan_for(M, N, K, tA, tB, lda, ldb, opts) -> Plan:
    key = (M, N, K, tA, tB, lda, ldb, tuple(sorted(opts.items())))
    p = _plans.get(key)
    if p is None:
        p = Plan(M, N, K, transA=tA, transB=tB, lda=lda, ldb=ldb, **opts)
        _plans[key] = p
    return p


def clear_plan_cache():
    for p in _plans.values():
        p.close()
    _plans.clear()


def product(A: torch.Tensor, B: torch.Tensor, opts: dict) -> torch.Tensor:
    """C = A B through the library; A, B may be transposed views."""
    tA, lda, As = _op_layout(A)
    tB, ldb, Bs = _op_layout(B)
    M, K = A.shape
    N = B.shape[1]
    p = _plan_for(M, N, K, tA, tB, lda, ldb, opts)
    C = torch.empty((M, N), dtype=A.dtype, device=A.device)
    p.run(As, Bs, C)
    return C


class TDGemmFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, opts):
        ctx.save_for_backward(A, B)
        ctx.opts = opts
        return product(A, B, opts)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous()
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        # two streams only inside CUDA-graph capture: replayed graphs carry no
        # host cost, while in eager mode the extra stream bookkeeping costs
        # more host time than the overlap saves on the device
        if not (need_a and need_b) or not torch.cuda.is_current_stream_capturing():
            dA = product(dC, B.t(), ctx.opts) if need_a else None
            dB = product(A.t(), dC, ctx.opts) if need_b else None
            return dA, dB, None
        # the two adjoints are independent: dB on a side stream, so one
        # product's latency-bound steps (statistics, fp64 planner, packing)
        # overlap the other's
        cur = torch.cuda.current_stream(dC.device)
        side = _side_stream(dC.device)
        side.wait_stream(cur)
        dA = product(dC, B.t(), ctx.opts)
        with torch.cuda.stream(side):
            dB = product(A.t(), dC, ctx.opts)
        cur.wait_stream(side)
        A.record_stream(side)
        dC.record_stream(side)
        dB.record_stream(cur)
        return dA, dB, None


def tdg_matmul(A: torch.Tensor, B: torch.Tensor, **opts) -> torch.Tensor:
    """Differentiable companded-and-packed A @ B.  ``opts`` are Plan options
    (L, W, dtype, form, target_snr_db / bits, ...)."""
    if "dtype" not in opts:
        opts["dtype"] = "f64" if A.dtype == torch.float64 else "f32"
    return TDGemmFn.apply(A, B, opts)
