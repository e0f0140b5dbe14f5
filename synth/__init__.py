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
    "faces_2dpca",
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


def faces_2dpca(persons: int, per_person: int, size: int, seed: int,
                person_amp: float = 13.0, image_amp: float = 16.0,
                noise: float = 20.0) -> np.ndarray:
    """Synthetic face images for the 2DPCA recognition study, shape
    (persons, per_person, size, size), integer pixel values 0..255.

    Every image is 128 + gain * (common + person_p) + variation + noise: a
    component shared by all persons and one per person, each a sum of random
    low-frequency 2-D cosines (amplitudes ~ N(0, 40^2) and ~ N(0, person_amp^2)
    per mode), an image gain from U[0.8, 1.2], an image-specific cosine field
    (~ N(0, image_amp^2) per mode) and pixel noise N(0, noise^2), clipped and
    rounded.  The defaults give a nearest-neighbour recognition rate near the
    paper's 78 % with 5 training and 6 test images per person and d = 10."""
    g = rng(seed)
    yy, xx = np.mgrid[0:size, 0:size] / float(size)

    def field(nmodes: int, amp: float) -> np.ndarray:
        f = np.zeros((size, size))
        for _ in range(nmodes):
            fx, fy = g.uniform(0.5, 6.0, 2)
            ph = g.uniform(0.0, 2.0 * np.pi, 2)
            a = g.normal() * amp
            f += a * np.cos(2 * np.pi * fx * xx + ph[0]) * np.cos(2 * np.pi * fy * yy + ph[1])
        return f

    common = field(16, 40.0)
    out = np.empty((persons, per_person, size, size))
    for p in range(persons):
        base = common + field(8, person_amp)
        for k in range(per_person):
            gain = g.uniform(0.8, 1.2)
            im = 128.0 + gain * base + field(16, image_amp) + g.normal(0.0, noise, (size, size))
            out[p, k] = np.clip(np.rint(im), 0, 255)
    return out


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
