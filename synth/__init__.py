"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This module only draws random numbers and lays them out; it holds none of the
companding, packing or GEMM arithmetic.  Every generator takes an explicit seed
and uses NumPy's PCG64 bit generator, so the same seed gives the same bits on
x86 and Arm hosts.

Input families follow the workloads of the paper:
  * iid zero-mean Gaussian, Laplacian (b=1) and uniform[-1,1] matrices — the
    zero-mean iid sources of the noise model (Sec. 4.C) and the distortion sweep;
  * uniform integer matrices with max|A| and max|B| set, c_A = c_B = 1 — the
    representation-noise measurement protocol of Sec. 4.B;
  * uniform matrices whose per-L x L-block range max_e is drawn from
    {4, 5, ..., 2048} — the generic experiments of Sec. 7;
  * eigenface-shaped pixel matrices (uniform integers 0..255, per-row mean
    removed) standing in for the face database of Sec. 8.A;
  * Gaussian MLP inputs and N(0, 1/fan_in) teacher weights standing in for the
    music-feature dataset of Sec. 8.B.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "gaussian",
    "laplace",
    "uniform",
    "iid",
    "int_uniform",
    "blockwise_range_uniform",
    "blockwise_crest",
    "eigenface_pixels",
    "mlp_teacher",
    "mlp_inputs",
    "sample_tiles",
    "calibration_pair",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed`` (the only source of randomness here)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _cast(x: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(x.astype(dtype, copy=False))


def gaussian(shape, seed: int, dtype=np.float64, sigma: float = 1.0) -> np.ndarray:
    """iid N(0, sigma^2) samples drawn in float64, then cast to ``dtype``."""
    return _cast(rng(seed).standard_normal(shape) * sigma, dtype)


def laplace(shape, seed: int, dtype=np.float64, b: float = 1.0) -> np.ndarray:
    """iid zero-mean Laplacian samples with scale ``b``."""
    return _cast(rng(seed).laplace(0.0, b, shape), dtype)


def uniform(shape, seed: int, dtype=np.float64, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """iid uniform samples on [lo, hi)."""
    return _cast(rng(seed).uniform(lo, hi, shape), dtype)


def iid(kind: str, shape, seed: int, dtype=np.float64) -> np.ndarray:
    """One of the three zero-mean iid families of the distortion sweep."""
    if kind == "gaussian":
        return gaussian(shape, seed, dtype)
    if kind == "laplace":
        return laplace(shape, seed, dtype)
    if kind == "uniform":
        return uniform(shape, seed, dtype)
    raise ValueError(f"unknown source kind {kind!r}")


def int_uniform(shape, seed: int, vmax: int, dtype=np.float64) -> np.ndarray:
    """Uniform integers in {-vmax, ..., vmax} stored as floating point."""
    return _cast(rng(seed).integers(-int(vmax), int(vmax) + 1, size=shape), dtype)


def blockwise_range_uniform(shape, seed: int, L: int, dtype=np.float64,
                            emin: int = 4, emax: int = 2048) -> np.ndarray:
    """Uniform values on [-max_e, max_e] where max_e is drawn per L x L block from
    the integers {emin, ..., emax}."""
    g = rng(seed)
    rows, cols = shape
    nbr, nbc = -(-rows // L), -(-cols // L)
    me = g.integers(emin, emax + 1, size=(nbr, nbc)).astype(np.float64)
    x = g.uniform(-1.0, 1.0, size=shape)
    scale = np.repeat(np.repeat(me, L, axis=0), L, axis=1)[:rows, :cols]
    return _cast(x * scale, dtype)


def blockwise_crest(shape, seed: int, L: int, dtype=np.float64, kmax: int = 11,
                    emin: int = 1, emax: int = 4096) -> np.ndarray:
    """Per L x L block: sign(u) |u|^k * e with u uniform on [-1, 1], an odd
    exponent k drawn from {1, 3, ..., kmax} and an integer range e drawn from
    {emin, ..., emax}.  Larger k gives a larger peak-to-RMS ratio, so blocks
    differ in both scale and shape."""
    g = rng(seed)
    rows, cols = shape
    nbr, nbc = -(-rows // L), -(-cols // L)
    k = 2 * g.integers(0, (kmax - 1) // 2 + 1, size=(nbr, nbc)) + 1
    me = g.integers(emin, emax + 1, size=(nbr, nbc)).astype(np.float64)
    u = g.uniform(-1.0, 1.0, size=shape)
    kk = np.repeat(np.repeat(k, L, axis=0), L, axis=1)[:rows, :cols]
    scale = np.repeat(np.repeat(me, L, axis=0), L, axis=1)[:rows, :cols]
    return _cast(np.sign(u) * np.abs(u) ** kk * scale, dtype)


def eigenface_pixels(pixels: int, images: int, seed: int, dtype=np.float32) -> np.ndarray:
    """``pixels x images`` matrix of uniform integers 0..255 with each row's mean
    (the mean image) removed, the pre-processing of the face-recognition study."""
    x = rng(seed).integers(0, 256, size=(pixels, images)).astype(np.float64)
    x -= x.mean(axis=1, keepdims=True)
    return _cast(x, dtype)


def mlp_teacher(sizes, seed: int, dtype=np.float32):
    """Teacher MLP weights W_i (fan_in x fan_out) ~ N(0, 1/fan_in), zero biases."""
    g = rng(seed)
    ws = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        ws.append(_cast(g.standard_normal((fi, fo)) / np.sqrt(fi), dtype))
    return ws


def mlp_inputs(batch: int, dim: int, seed: int, dtype=np.float32) -> np.ndarray:
    """iid N(0,1) feature vectors, one per row."""
    return gaussian((batch, dim), seed, dtype)


def sample_tiles(n_row_tiles: int, n_col_tiles: int, count: int, seed: int):
    """``count`` distinct (i, j) output-tile indices drawn without replacement."""
    g = rng(seed)
    total = n_row_tiles * n_col_tiles
    pick = g.choice(total, size=min(count, total), replace=False)
    return [(int(p) // n_col_tiles, int(p) % n_col_tiles) for p in sorted(pick)]


def _key_seed(key) -> int:
    import zlib
    return zlib.crc32(repr(tuple(key)).encode("ascii")) & 0x7FFFFFFF


def calibration_pair(L: int, gamma_a: int, gamma_b: int, key):
    """One instantiation of the representation-noise measurement inputs
    (Sec. 4.B): L x L integer matrices uniform on {-gamma_a..gamma_a} and
    {-gamma_b..gamma_b}; ``key`` (a tuple of plain values) fixes the seeds."""
    s = _key_seed(key)
    A = int_uniform((L, L), s, gamma_a, np.float64)
    B = int_uniform((L, L), s ^ 0x5A5A5A5, gamma_b, np.float64)
    return A, B
