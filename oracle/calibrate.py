"""Representation-noise calibration on the oracle's arithmetic (Sec. 4.B, eq. 18).

TEST INFRASTRUCTURE ONLY: writes ``oracle/s_table.json``, the s(R_max, W) table
the oracle's planner reads.  It calls nothing but ``oracle`` and ``synth``.

Protocol (Sec. 4.B, adapted to a ladder of R_max levels):
  for every working type, packing form, W in {2,3,4} and block size L,
  for every level t with R_t = floor(2^(t//4) (4 + t%4) / 4) >= L:
    z = 2^-q with the smallest q meeting eq. 15 for R_t,
    Gamma_A = min(22, R_t // L)   (the paper keeps max|A| = 22),
    Gamma_B = R_t // (L Gamma_A)  (the paper sweeps max|B|),
    five instantiations of L x L integer matrices, uniform on +-Gamma,
    c_A = c_B = 1 (no companding loss), packed product unpacked and compared
    with the exact integer product;
    m = mean error, s = root-mean-square error over all outputs of all five
    instantiations (the RMSE of eq. 18; the reading is stated in the design notes).

Usage:  python -m oracle.calibrate [--L 64 128] [--out oracle/s_table.json]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
from oracle import oracle as orc  # noqa: E402

FORMS = ("sym", "asym")
WS = (2, 3, 4)
DTYPES = ("f32", "f64")
INSTANCES = 5
GAMMA_A_CAL = 22


def level_range(L: int, dtype: str):
    t = 0
    while orc.r_level(t) < L:
        t += 1
    return range(t, orc.T_MAX[dtype] + 1)


def calibrate_one(dtype: str, form: str, W: int, L: int, ts=None) -> dict:
    T = orc.NP_T[dtype]
    out = {}
    for t in (ts if ts is not None else level_range(L, dtype)):
        R = orc.r_level(t)
        q = orc.q_for(R)
        gA = min(GAMMA_A_CAL, R // L)
        gB = R // (L * gA)
        errs = []
        for inst in range(INSTANCES):
            A, B = synth.calibration_pair(L, gA, gB, (dtype, form, W, L, t, inst))
            res = orc.tdgemm(A.astype(T), B.astype(T), L=L, W=W, dtype=dtype, form=form,
                             manual=(q, 1.0, 1.0))
            exact = A.astype(np.int64) @ B.astype(np.int64)
            errs.append((res.C.astype(np.float64) - exact.astype(np.float64)).ravel())
        e = np.concatenate(errs)
        s = math.sqrt(math.fsum((e * e).tolist()) / e.size)
        m = math.fsum(e.tolist()) / e.size
        out[str(t)] = {"R": R, "q": q, "gA": gA, "gB": gB, "s": s, "m": m}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[64, 128])
    ap.add_argument("--out", default=os.path.join(orc.HERE, "s_table.json"))
    args = ap.parse_args(argv)
    tables = {}
    for L in args.L:
        for dtype in DTYPES:
            for form in FORMS:
                for W in WS:
                    key = orc.STable.key(dtype, form, W, L)
                    tables[key] = calibrate_one(dtype, form, W, L)
                    print(key, len(tables[key]), flush=True)
    doc = {
        "what": "representation-noise RMSE s(R_max, W) on the oracle's arithmetic",
        "protocol": "Sec. 4.B: c_A=c_B=1, integer inputs, max|A|=22, five instantiations",
        "levels": "R_t = floor(2^(t//4) (4 + t%4) / 4); z = 2^-q, smallest q with 2^q >= 2 R_t + 50",
        "tables": tables,
    }
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=0, sort_keys=True)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
