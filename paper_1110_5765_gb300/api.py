"""PyTorch-facing wrapper of the tdgemm C ABI (marshalling only).

A ``Plan`` is created for fixed shapes and parameters and can be run many
times; it owns the device workspace.  Tensors are passed by pointer with
their leading dimensions; a tensor whose last dimension is contiguous is
used as stored ('N'), one whose first dimension is contiguous is passed as
the transpose of its storage ('T').
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np
import torch

from . import _lib
from ._lib import (DTYPES, FORMS, TDG_ALLOW_FALLBACK, TDG_KEEP_PACKED, TDG_NOISE_UNIFORM,
                   TDG_PAIR_EXACT, Info, check)

_TORCH_DT = {"f32": torch.float32, "f64": torch.float64}
_DT_OF = {torch.float32: "f32", torch.float64: "f64"}
S_TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "s_table.json")
F_TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "f_table.json")
MAX_LEVELS = 192

_table_cache: dict | None = None


def load_rep_noise(path: str = S_TABLE_PATH) -> dict:
    """The package's measured representation-noise table (Sec. 4.B), keyed
    ``"{dtype}/{form}/W{W}/L{L}" -> {level: {"s": ...}}``; empty if absent."""
    global _table_cache
    if path == S_TABLE_PATH and _table_cache is not None:
        return _table_cache
    tabs = {}
    if os.path.exists(path):
        with open(path) as f:
            tabs = json.load(f)["tables"]
    if path == S_TABLE_PATH:
        _table_cache = tabs
    return tabs


def load_speedups(path: str = F_TABLE_PATH) -> dict:
    """The package's measured throughput-scaling table F_W (Sec. 5.B), keyed
    ``"{dtype}/{form}/W{W}/L{L}" -> {"F": ...}``; empty if absent."""
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)["tables"]


def rep_noise_table(dtype: str, form: str, W: int, L: int, tables: dict | None = None):
    """Levels and s values for one (dtype, form, W, L), as a dense array over
    levels [0, MAX_LEVELS) with -1 where nothing was measured; None if absent."""
    tables = load_rep_noise() if tables is None else tables
    d = tables.get(f"{dtype}/{form}/W{W}/L{L}")
    if not d:
        return None
    arr = np.full(MAX_LEVELS, -1.0)
    for t, v in d.items():
        t = int(t)
        if 0 <= t < MAX_LEVELS:
            arr[t] = float(v["s"])
    return arr


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _layout(X: torch.Tensor):
    """(trans, ld, base tensor) for a 2-D op(X) tensor."""
    if X.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    r, c = X.shape
    s0, s1 = X.stride()
    if s1 == 1 and (s0 >= c or r == 1):
        return "N", max(s0, c), X
    if s0 == 1 and (s1 >= r or c == 1):
        return "T", max(s1, r), X
    Xc = X.contiguous()
    return "N", c, Xc


class Plan:
    """A tdgemm plan: C = alpha op(A) op(B) + beta C for fixed shapes.

    form: 'plain' | 'sym' | 'asym' | 'tc_int' | 'tc_fp8'
    Parameters follow the paper: block size L, packing W, and either a
    distortion target (dB) or fixed bits.  ``noise_rms=False`` plans with the
    representation noise as calibrated on uniform integers, unscaled
    (TDG_NOISE_UNIFORM); the default scales it by the blocks' crest factors.
    """

    def __init__(self, M: int, N: int, K: int, *, L: int = 128, W: int = 2, dtype: str = "f32",
                 form: str = "sym", target_snr_db: float = math.nan, bits: int = 0,
                 transA: str = "N", transB: str = "N", lda: int | None = None,
                 ldb: int | None = None, ldc: int | None = None, allow_fallback: bool = True,
                 keep_packed: bool = False, rep_noise: str | dict | None = "package",
                 noise_rms: bool = True, pair_exact: bool = False,
                 speedup: str | dict | None = "package"):
        self._L = _lib.load()
        self.M, self.N, self.K = int(M), int(N), int(K)
        self.L, self.W, self.dtype, self.form = int(L), int(W), dtype, form
        self.transA, self.transB = transA, transB
        self.lda = lda if lda is not None else (self.K if transA == "N" else self.M)
        self.ldb = ldb if ldb is not None else (self.N if transB == "N" else self.K)
        self.ldc = ldc if ldc is not None else self.N
        flags = ((TDG_ALLOW_FALLBACK if allow_fallback else 0) | (TDG_KEEP_PACKED if keep_packed else 0)
                 | (0 if noise_rms else TDG_NOISE_UNIFORM) | (TDG_PAIR_EXACT if pair_exact else 0))
        h = ctypes.c_void_p()
        check(self._L.tdgemm_plan(ctypes.byref(h), transA.encode(), transB.encode(), self.M,
                                  self.N, self.K, self.lda, self.ldb, self.ldc, self.L, self.W,
                                  DTYPES[dtype], FORMS[form], float(target_snr_db), int(bits),
                                  flags))
        self._h = h
        if form in ("sym", "asym") and bits == 0 and rep_noise is not None:
            tables = load_rep_noise() if rep_noise == "package" else rep_noise
            for w in range(2, self.W + 1):
                arr = rep_noise_table(dtype, form, w, self.L, tables)
                if arr is not None:
                    self.set_rep_noise(w, arr, 0)
        if form == "sym" and speedup is not None:
            ftab = load_speedups() if speedup == "package" else speedup
            for w in range(2, self.W + 1):
                d = ftab.get(f"{dtype}/{form}/W{w}/L{self.L}")
                if d:
                    self.set_speedup(w, float(d["F"]))

    # -- configuration
    def set_rep_noise(self, W: int, s, t0: int = 0):
        a = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
        check(self._L.tdgemm_set_rep_noise(self._h, int(W),
                                           a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           int(t0), int(a.size)))

    def set_manual(self, q: int, c_a: float = 1.0, c_b: float = 1.0):
        check(self._L.tdgemm_set_manual(self._h, int(q), float(c_a), float(c_b)))

    def set_speedup(self, W: int, speedup: float):
        """F_W of Sec. 5.B for packing W (throughput control)."""
        check(self._L.tdgemm_set_speedup(self._h, int(W), float(speedup)))

    _KCTRL = {None: 0, "off": 0, "snr": 1, "fraction": 2, "throughput": 3}

    def set_kernel_control(self, mode: str | None, value: float = 0.0):
        """Sec. 6 control over inner kernels: mode 'snr' accelerates the L x L
        output blocks whose predicted SNR (dB) reaches ``value``, 'fraction'
        the ``ceil(value * nM * nN)`` blocks of highest predicted SNR,
        'throughput' the fewest of highest predicted SNR whose predicted
        acceleration over the conventional product reaches ``value`` (through
        the measured F_W); the others are computed with the conventional
        product.  None turns it off."""
        check(self._L.tdgemm_set_kernel_control(self._h, self._KCTRL[mode], float(value)))

    def set_wait_test(self, limit_ns: int):
        """Test of the bounded device waits: > 0 makes the next GEMMs' first
        wait for operand tiles run out after ``limit_ns`` and report
        TDG_ETIMEOUT in ``info()['device_status']``; 0 turns it off."""
        check(self._L.tdgemm_set_wait_test(self._h, int(limit_ns)))

    def kernel_mask(self) -> np.ndarray:
        """(nM, nN) uint8 mask of the inner kernels the last pack accelerated."""
        nM = -(-self.M // self.L)
        nN = -(-self.N // self.L)
        out = np.zeros(nM * nN, dtype=np.uint8)
        check(self._L.tdgemm_kernel_mask(self._h, out.ctypes.data, out.size))
        return out.reshape(nM, nN)

    # -- steps
    def _check_operand(self, X: torch.Tensor, trans: str, ld: int, what: str):
        if not X.is_cuda:
            raise ValueError(f"{what} must be a CUDA tensor")
        want = torch.float32 if self.form.startswith("tc") else _TORCH_DT[self.dtype]
        if X.dtype != want:
            raise ValueError(f"{what} must be {want}")

    def quantize_pack(self, A: torch.Tensor, B: torch.Tensor | None = None, stream=None):
        """A, B: the STORED matrices matching the plan's trans flags and lds.
        B = None reuses the B of the previous call (fixed-bit, manual, plain
        and E4M3 plans; the caller keeps that B unchanged)."""
        self._check_operand(A, self.transA, self.lda, "A")
        if B is None:
            self._keep = (A, self._keep[1] if getattr(self, "_keep", None) else None)
            check(self._L.tdgemm_quantize_pack_a(self._h, A.data_ptr(), _stream_ptr(stream)))
            return
        self._check_operand(B, self.transB, self.ldb, "B")
        self._keep = (A, B)
        check(self._L.tdgemm_quantize_pack(self._h, A.data_ptr(), B.data_ptr(), _stream_ptr(stream)))

    def gemm(self, C: torch.Tensor, alpha: float = 1.0, beta: float = 0.0, stream=None):
        check(self._L.tdgemm_gemm(self._h, C.data_ptr(), float(alpha), float(beta),
                                  _stream_ptr(stream)))
        return C

    def run(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None,
            alpha: float = 1.0, beta: float = 0.0, stream=None) -> torch.Tensor:
        if C is None:
            dt = torch.float32 if self.form.startswith("tc") else _TORCH_DT[self.dtype]
            C = torch.empty((self.M, self.ldc), dtype=dt, device=A.device)[:, :self.N]
        self._check_operand(A, self.transA, self.lda, "A")
        self._check_operand(B, self.transB, self.ldb, "B")
        check(self._L.tdgemm_run(self._h, A.data_ptr(), B.data_ptr(), C.data_ptr(), float(alpha),
                                 float(beta), _stream_ptr(stream)))
        return C

    def run_host(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, alpha: float = 1.0,
                 beta: float = 0.0, stream=None) -> torch.Tensor:
        """Host tensors (pinned for asynchronous copies); synchronises."""
        for X in (A, B, C):
            if X.is_cuda or not X.is_contiguous():
                raise ValueError("run_host takes contiguous host tensors")
        check(self._L.tdgemm_run_host(self._h, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                      float(alpha), float(beta), _stream_ptr(stream)))
        return C

    def run_host_async(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor,
                       alpha: float = 1.0, beta: float = 0.0, stream=None) -> torch.Tensor:
        """Pinned host tensors; queues the copies on the plan's copy stream and the
        computation on `stream`, without synchronising: the copies of one call
        overlap the computation of the previous one.  C is final (and A, B may
        be reused) once `stream` has finished."""
        for X in (A, B, C):
            if X.is_cuda or not X.is_contiguous() or not X.is_pinned():
                raise ValueError("run_host_async takes contiguous pinned host tensors")
        check(self._L.tdgemm_run_host_async(self._h, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                                            float(alpha), float(beta), _stream_ptr(stream)))
        return C

    def unpack(self, rint_out: torch.Tensor | None = None, C: torch.Tensor | None = None,
               stream=None):
        check(self._L.tdgemm_unpack(self._h, rint_out.data_ptr() if rint_out is not None else None,
                                    C.data_ptr() if C is not None else None, _stream_ptr(stream)))

    def info(self) -> dict:
        inf = Info()
        check(self._L.tdgemm_plan_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in Info._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._L.tdgemm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tdgemm(A: torch.Tensor, B: torch.Tensor, *, alpha: float = 1.0, beta: float = 0.0,
           C: torch.Tensor | None = None, **plan_kw) -> torch.Tensor:
    """One-shot C = alpha op(A) op(B) + beta C; op() is read from the strides."""
    tA, lda, A = _layout(A)
    tB, ldb, B = _layout(B)
    M, K = A.shape
    N = B.shape[1]
    dtype = plan_kw.pop("dtype", _DT_OF.get(A.dtype, "f32"))
    with Plan(M, N, K, transA=tA, transB=tB, lda=lda, ldb=ldb, dtype=dtype, **plan_kw) as p:
        out = p.run(A.t() if tA == "T" else A, B.t() if tB == "T" else B, C, alpha, beta)
        torch.cuda.current_stream().synchronize()
    return out


def fma_probe(dtype: str, iters: int, stream=None) -> float:
    """Queue one launch of independent FMA chains on every SM (FP32 pipe
    through fma.rn.f32x2, or FP64); returns the flops it performs.  Time it
    with CUDA events around the call."""
    L = _lib.load()
    fl = ctypes.c_double()
    check(L.tdgemm_fma_probe(DTYPES[dtype], int(iters), ctypes.byref(fl), _stream_ptr(stream)))
    return fl.value


def snr_sums(C: torch.Tensor, ref: torch.Tensor, stream=None) -> tuple[float, float, float]:
    """(sum ref^2, sum (C-ref)^2, sum (C-ref)) in fp64, computed on the device."""
    L = _lib.load()
    if ref.dtype != torch.float64:
        raise ValueError("ref must be fp64")
    out = torch.zeros(3, dtype=torch.float64, device=C.device)
    check(L.tdgemm_snr(C.data_ptr(), C.stride(0), DTYPES[_DT_OF[C.dtype]], ref.data_ptr(),
                       ref.stride(0), C.shape[0], C.shape[1], out.data_ptr(), _stream_ptr(stream)))
    s = out.cpu().tolist()
    return s[0], s[1], s[2]


def snr_db(C: torch.Tensor, ref: torch.Tensor) -> float:
    """Eq. 20 measured over all of C against an fp64 reference."""
    sig, noise, _ = snr_sums(C, ref)
    return math.inf if noise == 0 else 10.0 * math.log10(sig / noise)
