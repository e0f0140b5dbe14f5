"""tdgemm: companded-and-packed GEMM (Anastasia & Andreopoulos) on one GB300.

The computation runs in the CUDA library under ``csrc/`` behind the C ABI of
``include/tdgemm.h``; this package only marshals PyTorch tensors into it.

    from paper_1110_5765_gb300 import Plan, tdgemm, snr_db
"""
from .api import Plan, tdgemm, snr_db, snr_sums, rep_noise_table, load_rep_noise  # noqa: F401
from ._lib import TDGemmError  # noqa: F401

__all__ = ["Plan", "tdgemm", "snr_db", "snr_sums", "TDGemmError", "rep_noise_table",
           "load_rep_noise"]
