"""Representation-noise calibration of the library on the GPU (Sec. 4.B, eq. 18).

    python -m paper_1110_5765_gb300.calibrate [--L 64 128] [--out ...s_table.json]

Writes the s(R_max, W) table the planner uses beyond the error-free packing
region.  It is measured on this library's own kernels, in manual mode:
for every working type, packing form, W in {2, 3, 4}, block size L and
candidate level t (R_t = floor(2^(t div 4) (4 + t mod 4) / 4) >= L):
  z = 2^-q with the smallest q meeting eq. 15 for R_t,
  Gamma_A = min(22, R_t // L) (the paper keeps max|A| = 22), Gamma_B = R_t // (L Gamma_A),
  five instantiations of L x L integer matrices uniform on +-Gamma, c_A = c_B = 1,
  error = unpacked product - exact integer product;
  s = root-mean-square error, m = mean error, over all outputs of the five.
The PAPER measured this offline on its target machine; this is the same
measurement for GB300, done once and shipped as data.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1110_5765_gb300.api import Plan, S_TABLE_PATH  # noqa: E402

U_SAFE = 50
GAMMA_A_CAL = 22
INSTANCES = 5
T_MAX = {"f32": 4 * 24, "f64": 4 * 40}
NP_T = {"f32": np.float32, "f64": np.float64}


def r_level(t: int) -> int:
    return ((4 + (t & 3)) << (t >> 2)) >> 2


def q_for(R: int) -> int:
    return (2 * R + U_SAFE - 1).bit_length()


def levels(L: int, dtype: str):
    t = 0
    while r_level(t) < L:
        t += 1
    return range(t, T_MAX[dtype] + 1)


def calibrate_one(dtype: str, form: str, W: int, L: int, ts=None) -> dict:
    T = NP_T[dtype]
    out = {}
    with Plan(L, L, L, L=L, W=W, dtype=dtype, form=form, bits=8, rep_noise=None) as p:
        C = torch.empty((L, L), dtype=torch.float64 if dtype == "f64" else torch.float32,
                        device="cuda")
        for t in (ts if ts is not None else levels(L, dtype)):
            R = r_level(t)
            q = q_for(R)
            gA = min(GAMMA_A_CAL, R // L)
            gB = R // (L * gA)
            p.set_manual(q, 1.0, 1.0)
            errs = []
            for inst in range(INSTANCES):
                A, B = synth.calibration_pair(L, gA, gB, (dtype, form, W, L, t, inst))
                p.run(torch.from_numpy(A.astype(T)).cuda(), torch.from_numpy(B.astype(T)).cuda(), C)
                got = C.cpu().numpy().astype(np.float64)
                exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
                errs.append((got - exact).ravel())
            e = np.concatenate(errs)
            s = math.sqrt(math.fsum((e * e).tolist()) / e.size)
            m = math.fsum(e.tolist()) / e.size
            out[str(t)] = {"R": R, "q": q, "gA": gA, "gB": gB, "s": s, "m": m}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[64, 128])
    ap.add_argument("--out", default=S_TABLE_PATH)
    args = ap.parse_args(argv)
    tables = {}
    for L in args.L:
        for dtype in ("f32", "f64"):
            for form in ("sym", "asym"):
                for W in (2, 3, 4):
                    key = f"{dtype}/{form}/W{W}/L{L}"
                    tables[key] = calibrate_one(dtype, form, W, L)
                    print(key, len(tables[key]), flush=True)
    doc = {"what": "representation-noise RMSE s(R_max, W) measured on the GB300 kernels",
           "protocol": "Sec. 4.B: c_A=c_B=1, integer inputs, max|A|=22, five instantiations",
           "levels": "R_t = floor(2^(t//4) (4 + t%4) / 4); z = 2^-q, smallest q with 2^q >= 2 R_t + 50",
           "device": torch.cuda.get_device_name(0),
           "tables": tables}
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=0, sort_keys=True)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
