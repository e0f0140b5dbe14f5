"""tdgemm: companded-and-packed GEMM (Anastasia & Andreopoulos) on one GB300.

The computation runs in the CUDA library under ``csrc/`` behind the C ABI of
``include/tdgemm.h``; this package only marshals PyTorch tensors into it.

    from paper_1110_5765_gb300 import Plan, tdgemm, snr_db
"""
from .api import (Plan, fma_probe, load_rep_noise, rep_noise_table, snr_db,  # noqa: F401
                  snr_sums, tdgemm)
from ._lib import TDGemmError  # noqa: F401

__all__ = ["Plan", "tdgemm", "snr_db", "snr_sums", "TDGemmError", "rep_noise_table",
           "load_rep_noise", "fma_probe"]
