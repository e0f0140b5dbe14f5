"""Benchmark of the companded-and-packed GEMM on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-forms]

One step is one pass of the whole path — block statistics, device planner,
companding + packing of A and B, packed GEMM with fused unpack/de-companding —
on the distortion-sweep workload: M = N = K = 4096, fp32 inputs iid
uniform[-1, 1], block L = 128, symmetric packing W = 2, distortion target
20 dB.  Inputs are resident in HBM when timing starts; L2 is flushed between
steps (a 256 MB write outside the per-step events).  ``value`` is effective
GFLOP/s = 2 M N K per step over the device time of the steps, summed over all
ranks (each rank runs its own independent product: weak scaling).

The JSON line also carries:
  e2e          the same metric through tdgemm_run_host_async (pinned host
               buffers, every step's host-to-device and device-to-host copies
               inside the timing; the copies of one step overlap the
               computation of the previous one)
  roofline     the packed GEMM kernel against the FP32 FMA peak
  cpu_baseline the CPU oracle on a bounded sample (rank 0, N = 1 only)
  forms        every other form at the same size with its measured SNR
  clocks       SM clocks sampled by nvidia-smi during the timed steps
``--impl reference`` times the CPU oracle itself on host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "effective GFLOP/s (2MNK/t) vs output SNR dB, packed & TC forms vs plain FP64/FP32 GEMM"
N_SIZE = 4096
L_BLOCK = 128
W_PACK = 2
TARGET_DB = 20.0
SEED_A, SEED_B = 1112, 1113
WORKLOAD = ("distortion sweep point: C = A B, M = N = K = 4096, fp32 inputs iid uniform[-1,1], "
            "block L = 128, per-block adaptive companding, symmetric packing W = 2, "
            "target 20 dB")
FP32_LANES_PER_SM = 128


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU, weak scaling)
# ---------------------------------------------------------------------------
def dist_setup(ngpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != ngpus:
        raise SystemExit(f"--gpus {ngpus} but WORLD_SIZE={world}")
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (the job finishes when the last rank does)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, steps: int, flops_per_step: float, t_max: float) -> float:
    """Effective GFLOP/s of the whole job: every rank runs its own product
    (weak scaling), so the work is world x steps x 2MNK over the slowest rank's
    time."""
    return world * steps * flops_per_step / t_max / 1e9


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------
def _oracle_tile_flops() -> float:
    return 2.0 * L_BLOCK * L_BLOCK * N_SIZE


def _oracle_tile(A, B, ti, tj, st):
    """One output tile through the whole oracle path (statistics, planning,
    companding, packing, packed product, unpacking) on the 128-row panel of A
    and the 128-column panel of B it depends on (full K)."""
    from oracle import oracle as orc
    Ap = np.ascontiguousarray(A[ti * L_BLOCK:(ti + 1) * L_BLOCK])
    Bp = np.ascontiguousarray(B[:, tj * L_BLOCK:(tj + 1) * L_BLOCK])
    orc.tdgemm(Ap, Bp, L=L_BLOCK, W=W_PACK, dtype="f32", form="sym", target_db=TARGET_DB,
               s_table=st)


_WORKER = {}


def _oracle_worker_init(seed_a, seed_b):
    """Process-pool worker: the benchmark's inputs regenerated from their seeds
    (nothing is shared with the GPU process) and the oracle loaded."""
    from oracle import oracle as orc
    orc.build()
    _WORKER["A"] = synth.uniform((N_SIZE, N_SIZE), seed_a, np.float32)
    _WORKER["B"] = synth.uniform((N_SIZE, N_SIZE), seed_b, np.float32)
    _WORKER["st"] = orc.load_s_table()


def _oracle_worker_tile(tile):
    _oracle_tile(_WORKER["A"], _WORKER["B"], tile[0], tile[1], _WORKER["st"])
    return 1


def oracle_sample(A, B, budget_s: float = 20.0, max_tiles: int = 64) -> dict:
    """The CPU oracle, as it stands, on one host core: sampled output tiles of
    the workload (``_oracle_tile``), taken until ``budget_s`` seconds have
    passed (at least one)."""
    from oracle import oracle as orc
    st = orc.load_s_table()
    tiles = synth.sample_tiles(N_SIZE // L_BLOCK, N_SIZE // L_BLOCK, max_tiles, seed=99)
    t0 = time.perf_counter()
    done = 0
    for (ti, tj) in tiles:
        _oracle_tile(A, B, ti, tj, st)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": _oracle_tile_flops() * done / t / 1e9, "unit": "GFLOP/s", "cores": 1,
            "kind": "oracle", "tiles": done, "seconds": t,
            "sample": (f"{done} output tile(s) of 128 x 128, each the whole companded-and-"
                       "packed path on its 128 x 4096 panel of A and 4096 x 128 panel of B "
                       "(single-threaded C + NumPy oracle)")}


class OraclePool:
    """The oracle on every host core: one spawned process per core (started
    before or apart from any GPU work, so nothing forked shares the CUDA
    context), each holding the benchmark's inputs regenerated from their
    seeds, computing whole sampled output tiles independently."""

    def __init__(self, procs: int | None = None, seed_a: int = SEED_A, seed_b: int = SEED_B):
        import multiprocessing as mp
        self.procs = max(1, procs or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_worker_init,
                                                 initargs=(seed_a, seed_b))
        # every worker initialised and warm before any timing (bounded: a pool
        # that cannot start is reported by the caller, not waited for)
        try:
            self.pool.map_async(_oracle_worker_tile, [(0, 0)] * self.procs,
                                chunksize=1).get(timeout=300)
        except Exception:
            self.close()
            raise

    def run(self, n_tiles: int, seed: int = 99) -> dict:
        nt = N_SIZE // L_BLOCK
        tiles = synth.sample_tiles(nt, nt, min(n_tiles, nt * nt), seed=seed)
        t0 = time.perf_counter()
        done = sum(self.pool.imap_unordered(_oracle_worker_tile, tiles, chunksize=1))
        t = time.perf_counter() - t0
        return {"value": _oracle_tile_flops() * done / t / 1e9, "unit": "GFLOP/s",
                "cores": self.procs, "kind": "oracle", "tiles": done, "seconds": t,
                "sample": (f"{done} output tiles of 128 x 128 on {self.procs} processes (one "
                           "per host core), each tile the whole companded-and-packed path on "
                           "its 128 x 4096 panel of A and 4096 x 128 panel of B (C + NumPy "
                           "oracle)")}

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline_all_cores(A, B, budget_s: float = 20.0) -> dict:
    """The oracle on all host cores (tiles spread over one process per core)
    with the single-core figure beside it; about ``budget_s`` of CPU work."""
    single = oracle_sample(A, B, budget_s=min(5.0, budget_s / 4), max_tiles=16)
    per_tile = single["seconds"] / max(1, single["tiles"])
    try:
        pool = OraclePool()
    except Exception as e:             # no process pool here: the single-core figure alone
        single["single_core"] = {"value": single["value"], "unit": "GFLOP/s",
                                 "tiles": single["tiles"], "pool_error": str(e)[:120]}
        return single
    try:
        # about budget_s of wall time spread over the cores, a few tiles each at least
        n = max(2 * pool.procs, int(budget_s * pool.procs / max(per_tile, 1e-3) / 2))
        multi = pool.run(n)
    finally:
        pool.close()
    multi["single_core"] = {"value": single["value"], "unit": "GFLOP/s", "tiles": single["tiles"]}
    return multi


def run_reference(args):
    """--impl reference: the CPU oracle timed on all host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.run(pool.procs, seed=7)
        # the whole run stays within about three minutes whatever K and W are:
        # tiles per step from the measured per-tile time of the warm-up
        probe = pool.run(pool.procs, seed=8)
        per_tile = probe["seconds"] / max(1, probe["tiles"])
        per_step_budget = max(0.2, 150.0 / max(1, args.steps))
        n = max(1, int(per_step_budget / max(per_tile, 1e-4)))
        vals, secs = [], 0.0
        r = probe
        for k in range(args.steps):
            r = pool.run(n, seed=100 + k)
            vals.append(r["value"])
            secs += r["seconds"]
    finally:
        pool.close()
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def launches_per_step(plan) -> int:
    """Kernels this library queues per tdgemm_run for a target-mode symmetric
    fp32 plan with fallback, inputs 'N'/'N': block statistics of A and B (one
    launch), planner (per-slab aggregates; every candidate level, the last CTA
    deciding the plan), companders and de-companding factors, the packs of A
    and B for W = 2 (one launch), plain copy of A for the W = 1 fallback (B is
    used in place), the packed GEMM for W = 2 in both rounding variants of
    eq. 10 (the add-subtract one when the planned q allows it, the rintf one
    otherwise) and the plain GEMM for the fallback (kernels not chosen by the
    planner exit at entry).  Counted from the ncu launch list of one step."""
    return 1 + 2 + 2 + 1 + 1 + 3


def run_gpu(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_1110_5765_gb300 import build as b
    if rank == 0:
        b.build()
    barrier(world)
    import paper_1110_5765_gb300 as tdg

    M = N = K = N_SIZE
    A_h = synth.uniform((M, K), SEED_A + 17 * rank, np.float32)
    B_h = synth.uniform((K, N), SEED_B + 17 * rank, np.float32)
    A = torch.from_numpy(A_h).cuda()
    B = torch.from_numpy(B_h).cuda()
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    plan = tdg.Plan(M, N, K, L=L_BLOCK, W=W_PACK, dtype="f32", form="sym",
                    target_snr_db=TARGET_DB)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.run(A, B, C)
    torch.cuda.synchronize()
    info = plan.info()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1, e2 = ev[i]
        e0.record(stream)
        plan.quantize_pack(A, B)
        e1.record(stream)
        plan.gemm(C)
        e2.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    gemm_ms = [b_.elapsed_time(c) for _, b_, c in ev]
    t_steps = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_steps, world)
    flops_step = 2.0 * M * N * K
    value = whole_job_value(world, args.steps, flops_step, t_max)

    # ---- SNR of the timed configuration against the fp64 product
    ref = torch.matmul(A.double(), B.double())
    snr = tdg.snr_db(C, ref)
    del ref

    # ---- roofline of the packed GEMM kernel (FP32 FMA pipe)
    pk, src = peaks()
    probe = fma_peaks(tdg, torch)
    W_used = max(1, info["W_used"])
    P = -(-L_BLOCK // W_used)
    Kp = (K // L_BLOCK) * P if W_used > 1 else K
    gemm_flops = 2.0 * M * N * Kp                        # algorithmic: 2 M N K / W
    gemm_s = statistics.mean(gemm_ms) / 1e3
    sms = probe["sms"]
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12   # TFLOP/s
    achieved = gemm_flops / gemm_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": gemm_traffic(W_used),
                "kernel": f"packed_gemm_kernel<float, {'SYM' if W_used > 1 else 'PLAIN'}, W={W_used}> (FP32 FMA pipe)",
                "peak_source": (f"{sms} SMs x 128 FP32 lanes x 2 flop x {pk['sm_max_mhz']:.0f} MHz "
                                "(unit counts and maximum SM clock)"),
                "peak_probe": probe["f32_tflops"],
                "frac_of_probe": achieved / probe["f32_tflops"],
                "probe_source": "tdgemm_fma_probe: fma.rn.f32x2 chains on every SM, CUDA events",
                "work_per_launch": f"2 M N K / W flops = {gemm_flops:.3e}"}

    # ---- end to end through the pipelined host-buffer entry point: pinned
    # inputs alternating between two sets and C between two buffers; each step
    # copies its A and B in (the plan's copy stream) and writes C back over the
    # CPU-GPU link, the copies of step k + 1 running during step k's computation
    A2_h = synth.uniform((M, K), SEED_A + 17 * rank + 1, np.float32)
    B2_h = synth.uniform((K, N), SEED_B + 17 * rank + 1, np.float32)
    host_in = [(torch.from_numpy(A_h).pin_memory(), torch.from_numpy(B_h).pin_memory()),
               (torch.from_numpy(A2_h).pin_memory(), torch.from_numpy(B2_h).pin_memory())]
    host_out = [torch.empty((M, N), dtype=torch.float32).pin_memory() for _ in range(2)]
    for i in range(2):
        plan.run_host_async(host_in[i][0], host_in[i][1], host_out[i], stream=stream)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 50))
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for k in range(e2e_steps):
        plan.run_host_async(host_in[k % 2][0], host_in[k % 2][1], host_out[k % 2], stream=stream)
    s1.record(stream)
    torch.cuda.synchronize()
    e2e_t = max_over_ranks(s0.elapsed_time(s1) / 1e3, world)
    e2e = {"value": world * e2e_steps * flops_step / e2e_t / 1e9, "unit": "GFLOP/s",
           "h2d_bytes_per_step": A_h.nbytes + B_h.nbytes,
           "d2h_bytes_per_step": host_out[0].numel() * 4, "steps": e2e_steps,
           "api": "tdgemm_run_host_async (pinned host buffers; the copies of step k + 1 overlap "
                  "step k's computation through two device staging sets)"}

    forms = {}
    if args.forms and rank == 0:
        forms = measure_forms(tdg, torch, A, B)

    cpu = None
    if rank == 0 and world == 1 and args.cpu_baseline:
        cpu = cpu_baseline_all_cores(A_h, B_h, budget_s=20.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded PCG64 uniform[-1,1])",
                "config": {"workload": WORKLOAD, "M": M, "N": N, "K": K, "L": L_BLOCK,
                           "W": W_PACK, "form": "sym", "target_snr_db": TARGET_DB,
                           "l2": "flushed between steps (256 MB write outside step events)",
                           "W_used": info["W_used"], "q": info["q"],
                           "gamma_a": info["gamma_a"], "gamma_b": info["gamma_b"],
                           "pred_snr_db": info["pred_snr_db"], "snr_db": snr,
                           "parallelism": f"replicas x{world}"},
                "gpu_launches": launches_per_step(plan) * args.steps,
                "wall_s": wall,
                "gemm_ms": statistics.mean(gemm_ms),
                "pack_ms": statistics.mean([a.elapsed_time(b_) for a, b_, _ in ev]),
                "roofline": roofline, "e2e": e2e, "clocks": clocks,
                "peaks_source": src}
        if cpu is not None:
            line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                        "single_core")}
        line["fma_peaks"] = {"f32_tflops": probe["f32_tflops"], "f64_tflops": probe["f64_tflops"],
                             "sms": sms}
        if forms:
            line["forms"] = forms
            # compact per-form rooflines, printed last so the end of the line shows them
            line["rooflines"] = rooflines(forms, {"f32_tflops": probe["f32_tflops"],
                                                  "f64_tflops": probe["f64_tflops"],
                                                  "bf16_tflops": pk["bf16_tflops"]})
        print(json.dumps(line))
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# sources that define the packed GEMM kernel: the DRAM traffic recorded from an
# ncu capture is reported only while they are unchanged since the capture
GEMM_SOURCES = ("tdg_gemm.cuh", "tdg_gemm_tiles.h", "tdg_gemm_f32.cu", "tdg_common.cuh",
                "tdg_internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "packed_gemm_f32_sym_w2_4096_traffic.md")


def gemm_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1110_5765_gb300", "csrc")
    for name in GEMM_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def gemm_traffic(W_used):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of the timed
    packed GEMM (4096^3 sym W = 2) from the committed ncu summary, or None when
    the kernel sources changed since that capture (or W differs)."""
    try:
        with open(TRAFFIC_FILE) as f:
            text = f.read()
    except OSError:
        return None
    vals = dict(re.findall(r"^(traffic_bytes_per_launch|sources_sha256|W): *(\S+)", text, re.M))
    if W_used != int(vals.get("W", 0)) or vals.get("sources_sha256") != gemm_sources_sha256():
        return None
    return float(vals["traffic_bytes_per_launch"])


def _time(fn, torch, reps=3):
    fn()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(reps):
        fn()
    s1.record()
    torch.cuda.synchronize()
    return s0.elapsed_time(s1) / 1e3 / reps


def fma_peaks(tdg, torch) -> dict:
    """FP32 / FP64 FMA-pipe peaks measured on this GPU (tdgemm_fma_probe:
    independent fma.rn.f32x2 / fma.rn.f64 chains on every SM, no memory),
    best of three CUDA-event-timed launches, and the SM count from the
    device's properties."""
    out = {"sms": torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count}
    for dt, iters in (("f32", 20000), ("f64", 400)):
        tdg.fma_probe(dt, max(1, iters // 10))
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fl = tdg.fma_probe(dt, iters)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) / 1e3))
        out[f"{dt}_tflops"] = best / 1e12
    return out


def _time_split(p, A, B, C, torch, reps=3):
    """Whole path and GEMM step (tdgemm_gemm alone) per call, CUDA events on
    the launching stream, after one warm-up call."""
    p.run(A, B, C)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(reps)]
    for e0, e1, e2 in ev:
        e0.record()
        p.quantize_pack(A, B)
        e1.record()
        p.gemm(C)
        e2.record()
    torch.cuda.synchronize()
    t = statistics.mean(a.elapsed_time(c) for a, _, c in ev) / 1e3
    tg = statistics.mean(b.elapsed_time(c) for _, b, c in ev) / 1e3
    return t, tg


def kernel_work(form: str, W: int, M: int, N: int, K: int, L: int) -> float:
    """Algorithmic flops of the GEMM kernel of one call: 2 per fused
    multiply-add the packed (or plain, or tensor-core) main loop performs:
    sym M x N x nK ceil(L/W), asym nM ceil(L/W) x N x K, plain and tensor-core
    forms M x N x K."""
    nM, nK = -(-M // L), -(-K // L)
    P = -(-L // W)
    if form == "sym" and W > 1:
        return 2.0 * M * N * nK * P
    if form == "asym" and W > 1:
        return 2.0 * nM * P * N * K
    return 2.0 * M * N * K


def roofline_entry(rec: dict, form: str, dtype: str, M: int, N: int, K: int, pk: dict) -> dict:
    """Compact per-form roofline: whole-path effective TFLOP/s, SNR, W used,
    the GEMM kernel's algorithmic TFLOP/s and its fraction of the pipe it runs
    on (FP32 / FP64 FMA probe, tensor pipe: measured bf16 burst, x2 for E4M3)."""
    W = int(rec.get("W_used", 1) or 1)
    fam = form if W > 1 or form.startswith("tc") else "plain"
    if form == "tc_fp8":
        peak, src = 2.0 * pk["bf16_tflops"], "tc8"
    elif form == "tc_int":
        peak, src = pk["bf16_tflops"], "tc16"
    else:
        peak, src = pk[f"{dtype}_tflops"], dtype
    e = {"T": round(rec["gflops"] / 1e3, 2), "dB": round(rec["snr_db"], 1), "W": W}
    if "gemm_ms" in rec:
        kt = kernel_work(fam, W, M, N, K, L_BLOCK) / (rec["gemm_ms"] / 1e3) / 1e12
        e.update({"kT": round(kt, 2), "f": round(kt / peak, 3), "pk": src})
    return e


ROOFLINE_FORMS = [
    # (key in forms, form, dtype, size)
    ("cublas_f32", "cublas", "f32", 4096), ("cublas_f64", "cublas", "f64", 4096),
    ("plain_f32", "plain", "f32", 4096), ("plain_f64", "plain", "f64", 4096),
    ("sym_f32_W2_20dB", "sym", "f32", 4096), ("asym_f32_W2_20dB", "asym", "f32", 4096),
    ("sym_f32_W2_40dB", "sym", "f32", 4096), ("asym_f32_W2_40dB", "asym", "f32", 4096),
    ("sym_f64_W2_40dB", "sym", "f64", 4096), ("sym_f64_W3_40dB", "sym", "f64", 4096),
    ("asym_f64_W2_40dB", "asym", "f64", 4096), ("asym_f64_W3_40dB", "asym", "f64", 4096),
    ("tc_int_40dB", "tc_int", "f32", 4096), ("tc_fp8", "tc_fp8", "f32", 4096),
    ("p8192_cublas_f32", "cublas", "f32", 8192),
    ("p8192_sym_f32_W2_40dB", "sym", "f32", 8192), ("p8192_sym_f64_W3_40dB", "sym", "f64", 8192),
    ("p8192_asym_f64_W3_40dB", "asym", "f64", 8192),
    ("p8192_tc_int_40dB", "tc_int", "f32", 8192), ("p8192_tc_fp8", "tc_fp8", "f32", 8192),
]


def rooflines(forms: dict, pk: dict) -> dict:
    """Per-form rooflines of every form beside the conventional products
    (4096^3 uniform, 8192^3 Laplacian; 40 dB targets, 20 dB where fp32 packing
    engages)."""
    out = {"_": ("T: whole-path effective TFLOP/s (2MNK/t); dB: SNR vs fp64; W: packing used; "
                 "kT: GEMM kernel algorithmic TFLOP/s (2 per FMA it performs); f = kT / peak; "
                 f"pk: f32 = {pk['f32_tflops']:.1f}, f64 = {pk['f64_tflops']:.2f} TFLOP/s "
                 "(FMA probe, measured), tc16 = measured bf16 burst "
                 f"{pk['bf16_tflops']:.0f}, tc8 = 2 x that")}
    for key, form, dtype, n in ROOFLINE_FORMS:
        rec = forms.get(key)
        if not rec or "gflops" not in rec:
            continue
        if form == "cublas":
            rec = dict(rec, gemm_ms=rec["ms"], W_used=1)
            form = "plain"
        out[key.replace("p8192_", "8k_")] = roofline_entry(rec, form, dtype, n, n, n, pk)
    return out


def measure_forms(tdg, torch, A32, B32) -> dict:
    """Every form at 4096^3 beside plain fp32/fp64 GEMM on the same GPU:
    effective GFLOP/s (whole path) and SNR against the fp64 product."""
    n = N_SIZE
    flops = 2.0 * n ** 3
    out = {}
    ref = torch.matmul(A32.double(), B32.double())
    A64, B64 = A32.double(), B32.double()
    torch.backends.cuda.matmul.allow_tf32 = False
    C32 = torch.empty_like(A32)
    C64 = torch.empty_like(A64)

    def rec(name, t, C, extra=None):
        d = {"gflops": flops / t / 1e9, "ms": t * 1e3, "snr_db": tdg.snr_db(C, ref)}
        if extra:
            d.update(extra)
        out[name] = d

    rec("cublas_f32", _time(lambda: torch.matmul(A32, B32, out=C32), torch), C32)
    rec("cublas_f64", _time(lambda: torch.matmul(A64, B64, out=C64), torch, reps=1), C64)
    cases = [
        ("plain_f32", dict(dtype="f32", form="plain", W=1, bits=0), A32, B32),
        ("plain_f64", dict(dtype="f64", form="plain", W=1, bits=0), A64, B64),
        ("sym_f32_W2_20dB", dict(dtype="f32", form="sym", W=2, target_snr_db=20.0), A32, B32),
        ("asym_f32_W2_20dB", dict(dtype="f32", form="asym", W=2, target_snr_db=20.0), A32, B32),
        ("sym_f32_W2_20dB_pair_exact", dict(dtype="f32", form="sym", W=2, target_snr_db=20.0,
                                            pair_exact=True), A32, B32),
        ("sym_f32_W2_40dB", dict(dtype="f32", form="sym", W=2, target_snr_db=40.0), A32, B32),
        ("asym_f32_W2_40dB", dict(dtype="f32", form="asym", W=2, target_snr_db=40.0), A32, B32),
        ("sym_f64_W2_40dB", dict(dtype="f64", form="sym", W=2, target_snr_db=40.0), A64, B64),
        ("sym_f64_W3_40dB", dict(dtype="f64", form="sym", W=3, target_snr_db=40.0), A64, B64),
        ("asym_f64_W2_40dB", dict(dtype="f64", form="asym", W=2, target_snr_db=40.0), A64, B64),
        ("asym_f64_W3_40dB", dict(dtype="f64", form="asym", W=3, target_snr_db=40.0), A64, B64),
        ("sym_f64_W4_20dB", dict(dtype="f64", form="sym", W=4, target_snr_db=20.0), A64, B64),
        ("tc_int_8bit", dict(dtype="f32", form="tc_int", W=1, bits=8), A32, B32),
        ("tc_int_40dB", dict(dtype="f32", form="tc_int", W=1, target_snr_db=40.0), A32, B32),
        ("tc_fp8", dict(dtype="f32", form="tc_fp8", W=1, bits=0), A32, B32),
    ]
    out.update(measure_precision_form(tdg, torch))
    out.update(measure_eigenface(tdg, torch))
    for name, kw, A, B in cases:
        try:
            p = tdg.Plan(n, n, n, L=L_BLOCK, **kw)
            C = C64 if kw["dtype"] == "f64" and not kw["form"].startswith("tc") else C32
            reps = 1 if kw["dtype"] == "f64" else 3
            t, tg = _time_split(p, A, B, C, torch, reps=reps)
            info = p.info()
            rec(name, t, C, {"W_used": info["W_used"], "pred_snr_db": info["pred_snr_db"],
                             "gemm_ms": tg * 1e3})
            p.close()
        except Exception as e:     # a form not built yet is reported, not hidden
            out[name] = {"error": str(e)[:200]}
    return out


def profile_case(form: str, n: int):
    """A small case for ncu captures: three runs of one plan, no timing."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    A = torch.from_numpy(synth.uniform((n, n), 1, np.float32)).cuda()
    B = torch.from_numpy(synth.uniform((n, n), 2, np.float32)).cuda()
    if form.startswith("tc"):
        p = tdg.Plan(n, n, n, L=L_BLOCK, W=1, dtype="f32", form=form,
                     bits=8 if form == "tc_int" else 0)
    elif form == "plain":
        p = tdg.Plan(n, n, n, L=L_BLOCK, W=1, dtype="f32", form="plain")
    elif form.startswith("sym_kc"):
        # Sec. 6 control: fraction F of inner kernels accelerated, from the
        # name (sym_kc50 = half of them)
        p = tdg.Plan(n, n, n, L=L_BLOCK, W=W_PACK, dtype="f32", form="sym",
                     target_snr_db=TARGET_DB)
        p.set_kernel_control("fraction", int(form[6:] or "50") / 100.0)
    else:
        p = tdg.Plan(n, n, n, L=L_BLOCK, W=W_PACK, dtype="f32", form=form,
                     target_snr_db=TARGET_DB)
    C = torch.empty((n, n), device="cuda")
    for _ in range(3):
        p.run(A, B, C)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": form, "n": n, "info": p.info()}))
    p.close()


def sweep(out_path=None):
    """The distortion sweep at 4096^3: fp32/fp64 x Gaussian/Laplacian/uniform x
    sym/asym x W 2, 3 x targets 20..80 dB.  One JSON record per run: effective
    GFLOP/s of the whole path (mean of two timed runs after one warm-up), the W
    the planner chose, predicted and measured SNR against the fp64 product."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    n = N_SIZE
    flops = 2.0 * n ** 3
    recs = []
    for dtype, T, tt in (("f32", np.float32, torch.float32), ("f64", np.float64, torch.float64)):
        for kind in ("gaussian", "laplace", "uniform"):
            A = torch.from_numpy(synth.iid(kind, (n, n), 2001, T)).cuda()
            B = torch.from_numpy(synth.iid(kind, (n, n), 2002, T)).cuda()
            ref = torch.matmul(A.double(), B.double())
            C = torch.empty((n, n), dtype=tt, device="cuda")
            for form in ("sym", "asym"):
                for W in (2, 3):
                    for target in range(20, 81, 10):
                        p = tdg.Plan(n, n, n, L=L_BLOCK, W=W, dtype=dtype, form=form,
                                     target_snr_db=float(target))
                        t = _time(lambda: p.run(A, B, C), torch, reps=2)
                        info = p.info()
                        p.close()
                        rec = {"dtype": dtype, "source": kind, "form": form, "W_req": W,
                               "target_db": target, "W_used": info["W_used"],
                               "pred_snr_db": info["pred_snr_db"],
                               "snr_db": tdg.snr_db(C, ref), "ms": t * 1e3,
                               "gflops": flops / t / 1e9}
                        recs.append(rec)
                        print(json.dumps(rec), flush=True)
            del ref
    if out_path:
        with open(out_path, "w") as f:
            json.dump(recs, f)
    return recs


def kernel_control_sweep(out_path=None):
    """Throughput control over inner kernels (Sec. 6, Fig. 7's experiment):
    4096^3 fp32, inputs uniform on [-max_e, max_e] with max_e drawn per L x L
    block from {4, ..., 2048} (the paper's generic test matrices, L = 128
    here), symmetric packing planned for a 20 dB target, and the fraction of
    accelerated inner kernels raised from 0 to 1 in steps of 0.1.  One JSON
    record per point: effective GFLOP/s of the whole path (mean of three timed
    runs after one warm-up) and the SNR against the fp64 product."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    n = N_SIZE
    flops = 2.0 * n ** 3
    A = torch.from_numpy(synth.blockwise_range_uniform((n, n), 3001, L_BLOCK, np.float32)).cuda()
    B = torch.from_numpy(synth.blockwise_range_uniform((n, n), 3002, L_BLOCK, np.float32)).cuda()
    ref = torch.matmul(A.double(), B.double())
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    recs = []
    p = tdg.Plan(n, n, n, L=L_BLOCK, W=W_PACK, dtype="f32", form="sym", target_snr_db=TARGET_DB)
    t = _time(lambda: p.run(A, B, C), torch)
    recs.append({"control": "off", "ms": t * 1e3, "gflops": flops / t / 1e9,
                 "snr_db": tdg.snr_db(C, ref), "W_used": p.info()["W_used"]})
    print(json.dumps(recs[-1]), flush=True)
    for k in range(11):
        F = k / 10.0
        p.set_kernel_control("fraction", F)
        t = _time(lambda: p.run(A, B, C), torch)
        m = p.kernel_mask()
        recs.append({"control": "fraction", "F": F, "accelerated": int(m.sum()),
                     "kernels": int(m.size), "ms": t * 1e3, "gflops": flops / t / 1e9,
                     "snr_db": tdg.snr_db(C, ref)})
        print(json.dumps(recs[-1]), flush=True)
    p.close()
    if out_path:
        with open(out_path, "w") as f:
            json.dump(recs, f)
    return recs


def speedup_table(out_path=None) -> dict:
    """F_W of Sec. 5.B on this GPU: the GEMM step (tdgemm_gemm alone) of the
    inner-kernel-controlled symmetric product with every inner kernel
    conventional (fraction 0) against every inner kernel packed at W
    (fraction 1) -- the mixed launch that throughput control runs -- per
    (dtype, W, L).  Writes it in the package's f_table.json format."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    tables = {}
    for dtype, n, Ls, reps in (("f32", 4096, (128, 256), 5), ("f64", 2048, (64, 128), 3)):
        T = np.float32 if dtype == "f32" else np.float64
        A = torch.from_numpy(synth.uniform((n, n), 31, T)).cuda()
        B = torch.from_numpy(synth.uniform((n, n), 32, T)).cuda()
        C = torch.empty_like(A)
        for L in Ls:
            for W in (2, 3, 4):
                p = tdg.Plan(n, n, n, L=L, W=W, dtype=dtype, form="sym", bits=6,
                             rep_noise=None, speedup=None)
                t = {}
                for frac in (0.0, 1.0):
                    p.set_kernel_control("fraction", frac)
                    p.run(A, B, C)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        p.gemm(C)
                    e1.record()
                    torch.cuda.synchronize()
                    t[frac] = e0.elapsed_time(e1) / reps
                p.close()
                tables[f"{dtype}/sym/W{W}/L{L}"] = {"F": t[0.0] / t[1.0], "n": n,
                                                    "t_conventional_ms": t[0.0],
                                                    "t_packed_ms": t[1.0]}
    out = {"about": ("F_W (Sec. 5.B): GEMM-step time of the inner-kernel-controlled symmetric "
                     "product with all inner kernels conventional over all packed at W "
                     "(tdgemm_gemm, CUDA events; fixed 6-bit companders; M = N = K = n)"),
           "gpu": torch.cuda.get_device_name(), "tables": tables}
    if out_path:
        with open(out_path, "w") as f:
            json.dump(out, f, indent=1)
    print(json.dumps(out))
    return out


def fig6_study(out_path=None, ftab=None):
    """Throughput-distortion curves at 4096^3 on the paper's generic input
    family (uniform within 128 x 128 blocks, max_e per block drawn from
    {4, 5, ..., 2048}, Sec. 7):
      (a) distortion control (Fig. 6): the planner's SNR target 10..100 dB,
          sGEMM (W <= 2) and dGEMM (W <= 4), the planner choosing W;
      (b) throughput control (Sec. 6 (ii)): fp32 W = 2 plan at a 20 dB
          target with a required acceleration F (mode 3) from 1.0 to F_W.
    Each point: whole-path effective TFLOP/s = 2 M N K / t, its percentage of
    the measured FMA-pipe peak of the dtype, the measured SNR against the
    fp64 product, and (b) the number of inner kernels accelerated."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    n = N_SIZE
    pk = fma_peaks(tdg, torch)
    flops = 2.0 * n ** 3
    A32 = torch.from_numpy(synth.blockwise_range_uniform((n, n), 61, L_BLOCK, np.float32)).cuda()
    B32 = torch.from_numpy(synth.blockwise_range_uniform((n, n), 62, L_BLOCK, np.float32)).cuda()
    ref = torch.matmul(A32.double(), B32.double())
    recs = {"peaks": pk, "distortion": [], "throughput": []}
    for dtype, W in (("f32", 2), ("f64", 4)):
        A = A32 if dtype == "f32" else A32.double()
        B = B32 if dtype == "f32" else B32.double()
        C = torch.empty_like(A)
        reps = 3 if dtype == "f32" else 1
        for target in range(10, 101, 10):
            p = tdg.Plan(n, n, n, L=L_BLOCK, W=W, dtype=dtype, form="sym",
                         target_snr_db=float(target))
            t, tg = _time_split(p, A, B, C, torch, reps=reps)
            info = p.info()
            p.close()
            tf = flops / t / 1e12
            recs["distortion"].append({"dtype": dtype, "target_db": target, "W": info["W_used"],
                                       "tflops": tf, "pct_peak": 100 * tf / pk[f"{dtype}_tflops"],
                                       "snr_db": tdg.snr_db(C, ref),
                                       "pred_snr_db": info["pred_snr_db"], "gemm_ms": tg * 1e3})
    C = torch.empty_like(A32)
    ftab = ftab if ftab is not None else "package"
    p = tdg.Plan(n, n, n, L=L_BLOCK, W=2, dtype="f32", form="sym", target_snr_db=20.0,
                 speedup=ftab)
    fw = (ftab if isinstance(ftab, dict) else tdg.api.load_speedups()).get(
        f"f32/sym/W2/L{L_BLOCK}", {}).get("F")
    if fw:
        for F in sorted({F for F in (1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.6) if F < fw} | {fw}):
            p.set_kernel_control("throughput", F)
            t, tg = _time_split(p, A32, B32, C, torch, reps=3)
            mask = p.kernel_mask()
            tf = flops / t / 1e12
            recs["throughput"].append({"F_target": F, "F_W": fw, "accelerated": int(mask.sum()),
                                       "kernels": int(mask.size), "tflops": tf,
                                       "pct_peak": 100 * tf / pk["f32_tflops"],
                                       "snr_db": tdg.snr_db(C, ref), "gemm_ms": tg * 1e3})
    p.close()
    if out_path:
        with open(out_path, "w") as f:
            json.dump(recs, f, indent=1)
    print(json.dumps(recs))
    return recs


def pca2d_study(out_path=None):
    """Sec. 8.A's 2DPCA face recognition with every GEMM through the library
    (Table 1's rows): synthetic faces (15 persons x 11 images of 288 x 288,
    5 training and 6 test images each, d = 10), G = sum_j A_j A_j^T as one
    288 x 288 x 21600 GEMM, the projections of all 165 images as 21600 x 288 x 10
    and 25920 x 288 x 10 GEMMs.  For each method: recognition rate, W the
    planner chose per GEMM, SNR of each GEMM against fp64, and effective
    GFLOP/s over the three GEMMs (device-resident operands, CUDA events, mean of
    five runs after one warm-up).  These sizes fill only part of a GB300 (the G
    product has 9 output tiles of 128 x 128)."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    torch.backends.cuda.matmul.allow_tf32 = False
    faces = synth.faces_2dpca(15, 11, 288, 7)
    n, d, n_train = 288, 10, 5
    train = faces[:, :n_train].reshape(-1, n, n)
    test = faces[:, n_train:].reshape(-1, n, n)
    mean = train.mean(axis=0)
    tr = (train - mean).astype(np.float32)
    te = (test - mean).astype(np.float32)
    side = np.ascontiguousarray(np.concatenate(list(tr), axis=1))
    truth = np.repeat(np.arange(15), 6)

    def study(make):
        """make(M, N, K) -> callable(A, B) -> C on the device"""
        t_total, info = 0.0, {}
        flops = 0.0

        def mm(A, B, name):
            nonlocal t_total, flops
            M, K = A.shape
            N = B.shape[1]
            fn = make(M, N, K)
            dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
            dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
            C, extra = fn(dA, dB)
            for _ in range(3):                # warm-up (clocks, caches)
                fn(dA, dB, False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                C, _ = fn(dA, dB, False)     # no host read-back inside the timing
            e1.record()
            torch.cuda.synchronize()
            t_total += e0.elapsed_time(e1) / 1e3 / 5
            flops += 2.0 * M * N * K
            Cn = C.float().cpu().numpy()
            ref = A.astype(np.float64) @ B.astype(np.float64)
            err = np.sum((Cn - ref) ** 2)
            info[name] = dict(extra, snr_db=(math.inf if err == 0 else
                                             10 * math.log10(np.sum(ref ** 2) / err)))
            return Cn

        G = mm(side, np.ascontiguousarray(side.T), "G")
        w, V = np.linalg.eigh(G.astype(np.float64))
        X = np.ascontiguousarray(V[:, ::-1][:, :d]).astype(np.float32)
        Ytr = mm(np.ascontiguousarray(tr.reshape(-1, n)), X, "Ytrain").reshape(len(tr), n, d)
        Yte = mm(np.ascontiguousarray(te.reshape(-1, n)), X, "Ytest").reshape(len(te), n, d)
        dist = ((Yte[:, None].astype(np.float64) - Ytr[None]) ** 2).sum(axis=(2, 3))
        acc = float(((dist.argmin(axis=1) // n_train) == truth).mean())
        return {"recognition": acc, "gflops": flops / t_total / 1e9, "ms": t_total * 1e3,
                "gemms": info}

    def cublas(M, N, K):
        return lambda A, B, want_info=True: (torch.matmul(A, B), {})

    def plan_maker(**kw):
        manual = kw.pop("manual", None)

        def make(M, N, K):
            p = tdg.Plan(M, N, K, L=L_BLOCK, dtype="f32", **kw)
            if manual:
                p.set_manual(*manual)

            C = None

            def fn(A, B, want_info=True):
                nonlocal C
                if C is None:
                    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
                p.run(A, B, C)
                if not want_info:
                    return C, {}
                i = p.info()
                return C, {"W_used": i["W_used"], "pred_snr_db": i["pred_snr_db"]}
            return fn
        return make

    recs = {}
    recs["cuBLAS fp32"] = study(cublas)
    recs["plain fp32"] = study(plan_maker(W=1, form="plain"))
    recs["50 dB"] = study(plan_maker(W=2, form="sym", target_snr_db=50.0, noise_rms=True))
    recs["20 dB"] = study(plan_maker(W=2, form="sym", target_snr_db=20.0, noise_rms=True))
    q = (2 * 50000 + 50 - 1).bit_length()      # eq. 15 for R_max = 50000
    recs["ad-hoc (W = 2, R_max = 50000, c = 0.1)"] = study(
        plan_maker(W=2, form="sym", bits=8, manual=(q, 0.1, 0.1)))
    for k, v in recs.items():
        print(json.dumps({"method": k, **v}), flush=True)
    if out_path:
        with open(out_path, "w") as f:
            json.dump(recs, f)
    return recs


def mlp_study(out_path=None, steps=50):
    """The differentiation form: a 128-1024-1024-10 tanh MLP, batch
    4096, synthetic labels from a teacher MLP, cross-entropy, SGD lr 0.1.  Every
    GEMM (3 forward, 5 adjoint products per step) through the straight-through
    autograd form at a 20 dB target (RMS-scaled noise), beside the same
    training with torch fp32 matmuls (TF32 off).  Reports ms per step (CUDA
    events over the steps after two warm-up steps), the loss after `steps`
    steps, and the W the planner chose for each product."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    from paper_1110_5765_gb300 import autograd as ag
    torch.backends.cuda.matmul.allow_tf32 = False
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
    opts = dict(L=L_BLOCK, W=2, form="sym", target_snr_db=20.0, noise_rms=True)

    def train(use_tdg):
        ws = [w.clone().requires_grad_() for w in init]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        loss = None
        for it in range(steps + 2):
            if it == 2:
                torch.cuda.synchronize()
                e0.record()
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
        e1.record()
        torch.cuda.synchronize()
        return {"ms_per_step": e0.elapsed_time(e1) / steps, "loss": float(loss.detach())}

    def train_graph(use_tdg):
        """The same training with one step captured as a CUDA graph and replayed
        (no host work per step: what the GPU takes for the step's kernels)."""
        ws = [w.clone().requires_grad_() for w in init]

        def step():
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
            return loss

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            loss = step()
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        return {"ms_per_step": e0.elapsed_time(e1) / steps, "loss": float(loss.detach()),
                "steps_trained": steps + 4}

    ag.clear_plan_cache()
    out = {"torch fp32": train(False), "tdgemm 20 dB": train(True)}
    for name, use in (("torch fp32, CUDA graph", False), ("tdgemm 20 dB, CUDA graph", True)):
        try:
            out[name] = train_graph(use)
        except Exception as e:          # reported, not hidden
            out[name] = {"error": str(e)[:300]}
    out["tdgemm 20 dB"]["products"] = {
        f"{k[0]}x{k[1]}x{k[2]} {k[3]}{k[4]}": p.info()["W_used"] for k, p in ag._plans.items()}
    ag.clear_plan_cache()
    print(json.dumps(out), flush=True)
    if out_path:
        with open(out_path, "w") as f:
            json.dump(out, f)
    return out


def pair_exact_study(out_path=None):
    """Pair-exact companders (eq. 26 per subblock product) against the
    separable default at the same plan: effective GFLOP/s of the whole path
    and SNR against fp64, on the benchmark input (uniform), on blocks of unlike
    peak-to-RMS ratios (synth.blockwise_crest), fp32 at the 20 dB target and
    fp64 with 10-bit companders inside the error-free region."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    n = N_SIZE
    flops = 2.0 * n ** 3
    recs = []
    cases = [("f32 uniform[-1,1], 20 dB", "f32", 128, dict(target_snr_db=20.0),
              lambda s, T: synth.uniform((n, n), s, T)),
             ("f32 block crest, 20 dB", "f32", 128, dict(target_snr_db=20.0),
              lambda s, T: synth.blockwise_crest((n, n), s, 128, T)),
             ("f64 block crest, 10 bits", "f64", 64, dict(bits=10),
              lambda s, T: synth.blockwise_crest((n, n), s, 64, T))]
    for name, dtype, L, kw, gen in cases:
        T = np.float32 if dtype == "f32" else np.float64
        A = torch.from_numpy(gen(3101, T)).cuda()
        B = torch.from_numpy(gen(3102, T)).cuda()
        ref = torch.matmul(A.double(), B.double())
        C = torch.empty_like(A)
        for px in (False, True):
            p = tdg.Plan(n, n, n, L=L, W=2, dtype=dtype, form="sym", pair_exact=px, **kw)
            t = _time(lambda: p.run(A, B, C), torch, reps=1 if dtype == "f64" else 3)
            info = p.info()
            p.close()
            rec = {"case": name, "companders": "pair-exact" if px else "separable",
                   "W_used": info["W_used"], "gflops": flops / t / 1e9, "ms": t * 1e3,
                   "snr_db": tdg.snr_db(C, ref)}
            recs.append(rec)
            print(json.dumps(rec), flush=True)
        del ref
    if out_path:
        with open(out_path, "w") as f:
            json.dump(recs, f)
    return recs


def reuse_study(out_path=None):
    """A product repeated with a fixed right operand (inference with fixed
    weights): tdgemm_quantize_pack_a reuses B's statistics, companders and
    packed form, so each call companders and packs only A.  Whole-path time of
    a full pack + GEMM against an A-only pack + GEMM (L2 flushed before each
    call, median of 20), with the reused result checked bit for bit against
    the full one; at 4096^3 (uniform inputs) and for the forward pass of a
    128 -> 1024 -> 1024 -> 10 MLP (batch 4096, ReLU between layers) with fixed
    weights."""
    import torch
    from paper_1110_5765_gb300 import build as b
    b.build()
    import paper_1110_5765_gb300 as tdg
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def tmed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    recs = []
    forms = [("sym f32 W=2, 6-bit companders", dict(form="sym", W=2, bits=6)),
             ("plain f32", dict(form="plain", W=1)),
             ("tcgen05 integer, 8 bits", dict(form="tc_int", W=1, bits=8)),
             ("tcgen05 E4M3", dict(form="tc_fp8", W=1))]
    n = N_SIZE
    A = torch.from_numpy(synth.uniform((n, n), 4101, np.float32)).cuda()
    B = torch.from_numpy(synth.uniform((n, n), 4102, np.float32)).cuda()
    C1, C2 = torch.empty_like(A), torch.empty_like(A)
    for name, kw in forms:
        p = tdg.Plan(n, n, n, L=L_BLOCK, dtype="f32", **kw)
        full = tmed(lambda: (p.quantize_pack(A, B), p.gemm(C1)))
        p.quantize_pack(A, B)
        reuse = tmed(lambda: (p.quantize_pack(A), p.gemm(C2)))
        torch.cuda.synchronize()
        rec = {"case": f"{n}^3, {name}", "full_ms": full, "reuse_ms": reuse,
               "saving": 1.0 - reuse / full, "same_bits": bool(torch.equal(C1, C2))}
        recs.append(rec)
        print(json.dumps(rec), flush=True)
        p.close()
    del A, B, C1, C2
    batch, dims = 4096, (128, 1024, 1024, 10)
    X = torch.from_numpy(synth.gaussian((batch, dims[0]), 4103, np.float32)).cuda()
    Ws = [torch.from_numpy(synth.gaussian((dims[i], dims[i + 1]), 4104 + i, np.float32)).cuda()
          * (2.0 / dims[i]) ** 0.5 for i in range(3)]
    for name, kw in forms[0:1] + forms[3:4]:
        plans = [tdg.Plan(batch, dims[i + 1], dims[i], L=L_BLOCK, dtype="f32", **kw)
                 for i in range(3)]
        outs = [torch.empty((batch, dims[i + 1]), device="cuda") for i in range(3)]

        def fwd(reuse):
            h = X
            for i in range(3):
                if reuse:
                    plans[i].quantize_pack(h)
                else:
                    plans[i].quantize_pack(h, Ws[i])
                plans[i].gemm(outs[i])
                h = torch.relu(outs[i]) if i < 2 else outs[i]
            return h
        full = tmed(lambda: fwd(False))
        y1 = fwd(False).clone()
        reuse = tmed(lambda: fwd(True))
        y2 = fwd(True)
        torch.cuda.synchronize()
        rec = {"case": f"MLP forward, batch {batch}, {dims}, {name}", "full_ms": full,
               "reuse_ms": reuse, "saving": 1.0 - reuse / full,
               "same_bits": bool(torch.equal(y1, y2))}
        recs.append(rec)
        print(json.dumps(rec), flush=True)
        for p in plans:
            p.close()
    if out_path:
        with open(out_path, "w") as f:
            json.dump(recs, f)
    return recs


def measure_eigenface(tdg, torch) -> dict:
    """The eigenface-shaped workload: X = 10304 pixels x 4096 images, uniform
    integers 0..255 with the pixel mean removed; the covariance C = X^T X
    (4096 x 4096 x 10304, op(A) through the transpose flag) and the
    projection of the 4096 images onto 400 orthonormal columns (4096 x 400 x
    10304) at 30 and 50 dB: fp32 symmetric packing (W <= 2), fp64 symmetric
    packing (W <= 3) and the tensor-core integer form, beside cuBLAS fp32
    (TF32 off).  SNR against the fp64 product."""
    X = torch.from_numpy(synth.eigenface_pixels(10304, 4096, 7)).cuda()
    U = torch.from_numpy(np.linalg.qr(synth.rng(8).standard_normal((10304, 400)))[0]
                         .astype(np.float32)).cuda()
    X64 = X.double()
    out = {}
    torch.backends.cuda.matmul.allow_tf32 = False
    for what, Bop, n_out in (("cov", X, 4096), ("proj", U, 400)):
        flops = 2.0 * 4096 * n_out * 10304
        ref = torch.matmul(X64.t(), Bop.double())
        C = torch.empty((4096, n_out), device="cuda")
        t = _time(lambda: torch.matmul(X.t(), Bop, out=C), torch)
        out[f"eig_{what}_cublas_f32"] = {"gflops": flops / t / 1e9, "ms": t * 1e3,
                                         "snr_db": tdg.snr_db(C, ref)}
        B64 = X64 if what == "cov" else Bop.double()
        C64 = torch.empty((4096, n_out), dtype=torch.float64, device="cuda")
        for target in (30.0, 50.0):
            # fp32 packing (falls back to the conventional product at these
            # targets), fp64 packing (W <= 3) and the tensor-core integer form
            for name, kw, Aop, Bo, Co in (
                    ("sym_f32_W2", dict(dtype="f32", form="sym", W=2), X, Bop, C),
                    ("sym_f64_W3", dict(dtype="f64", form="sym", W=3), X64, B64, C64),
                    ("tc_int", dict(dtype="f32", form="tc_int", W=1), X, Bop, C)):
                p = tdg.Plan(4096, n_out, 10304, L=L_BLOCK, target_snr_db=target, transA="T",
                             lda=4096, **kw)
                reps = 1 if kw["dtype"] == "f64" else 3
                t = _time(lambda: p.run(Aop, Bo, Co), torch, reps=reps)
                info = p.info()
                p.close()
                out[f"eig_{what}_{name}_{int(target)}dB"] = {
                    "gflops": flops / t / 1e9, "ms": t * 1e3, "snr_db": tdg.snr_db(Co, ref),
                    "W_used": info["W_used"], "pred_snr_db": info["pred_snr_db"],
                    "status": info["device_status"]}
        del ref, C64
    return out


def measure_precision_form(tdg, torch) -> dict:
    """The precision-form workload: 8192^3 Laplacian(b = 1) fp32, L = 128,
    tensor-core forms and the packed CUDA-core forms at a 40 dB target, beside
    cuBLAS fp32 / fp64 on the same GPU."""
    n = 8192
    flops = 2.0 * n ** 3
    A = torch.from_numpy(synth.laplace((n, n), 5001, np.float32)).cuda()
    B = torch.from_numpy(synth.laplace((n, n), 5002, np.float32)).cuda()
    ref = torch.matmul(A.double(), B.double())
    out = {}
    C32 = torch.empty_like(A)
    torch.backends.cuda.matmul.allow_tf32 = False
    t = _time(lambda: torch.matmul(A, B, out=C32), torch)
    out["p8192_cublas_f32"] = {"gflops": flops / t / 1e9, "ms": t * 1e3, "snr_db": tdg.snr_db(C32, ref)}
    cases = [("p8192_tc_int_40dB", dict(form="tc_int", W=1, target_snr_db=40.0)),
             ("p8192_tc_int_8bit", dict(form="tc_int", W=1, bits=8)),
             ("p8192_tc_fp8", dict(form="tc_fp8", W=1)),
             ("p8192_sym_f32_W2_40dB", dict(form="sym", W=2, target_snr_db=40.0))]
    for name, kw in cases:
        try:
            p = tdg.Plan(n, n, n, L=L_BLOCK, dtype="f32", **kw)
            t, tg = _time_split(p, A, B, C32, torch)
            info = p.info()
            out[name] = {"gflops": flops / t / 1e9, "ms": t * 1e3, "snr_db": tdg.snr_db(C32, ref),
                         "W_used": info["W_used"], "pred_snr_db": info["pred_snr_db"],
                         "gamma_a": info["gamma_a"], "gamma_b": info["gamma_b"],
                         "gemm_ms": tg * 1e3}
            p.close()
        except Exception as e:
            out[name] = {"error": str(e)[:200]}
    A64, B64 = A.double(), B.double()
    C64 = torch.empty_like(A64)
    t = _time(lambda: torch.matmul(A64, B64, out=C64), torch, reps=1)
    out["p8192_cublas_f64"] = {"gflops": flops / t / 1e9, "ms": t * 1e3}
    for form in ("sym", "asym"):
        p = tdg.Plan(n, n, n, L=L_BLOCK, dtype="f64", form=form, W=3, target_snr_db=40.0)
        t, tg = _time_split(p, A64, B64, C64, torch, reps=1)
        info = p.info()
        out[f"p8192_{form}_f64_W3_40dB"] = {"gflops": flops / t / 1e9, "ms": t * 1e3,
                                           "snr_db": tdg.snr_db(C64, ref), "W_used": info["W_used"],
                                           "pred_snr_db": info["pred_snr_db"], "gemm_ms": tg * 1e3}
        p.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tdgemm", choices=["tdgemm", "reference"])
    ap.add_argument("--no-forms", dest="forms", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile-case", default=None,
                    help="plain|sym|asym|tc_int|tc_fp8|sym_kc<percent>: run one plan three "
                         "times for ncu")
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--sweep", default=None, metavar="OUT.json",
                    help="run the 4096^3 distortion sweep (168 runs) and write its records")
    ap.add_argument("--pairx", default=None, metavar="OUT.json",
                    help="pair-exact against separable companders at 4096^3")
    ap.add_argument("--mlp", default=None, metavar="OUT.json",
                    help="time training of a 128-1024-1024-10 MLP (batch 4096) through the "
                         "autograd form")
    ap.add_argument("--pca2d", default=None, metavar="OUT.json",
                    help="run the 2DPCA face-recognition study (Sec. 8.A, Table 1)")
    ap.add_argument("--reuse", default=None, metavar="OUT.json",
                    help="run the fixed-right-operand (packed B reuse) study")
    ap.add_argument("--fig7", default=None, metavar="OUT.json",
                    help="run the 4096^3 inner-kernel throughput-control sweep (Sec. 6)")
    ap.add_argument("--fw", default=None, metavar="OUT.json",
                    help="measure the F_W throughput-scaling table (Sec. 5.B)")
    ap.add_argument("--fig6", default=None, metavar="OUT.json",
                    help="throughput-distortion curves at 4096^3 (distortion and throughput "
                         "control, Sec. 6-7)")
    args = ap.parse_args()
    if args.fw:
        speedup_table(args.fw)
        return
    if args.fig6:
        fw = None
        if not os.path.exists(os.path.join(ROOT, "paper_1110_5765_gb300", "f_table.json")):
            fw = speedup_table()["tables"]
        fig6_study(args.fig6, fw)
        return
    if args.reuse:
        reuse_study(args.reuse)
        return
    if args.fig7:
        kernel_control_sweep(args.fig7)
        return
    if args.pca2d:
        pca2d_study(args.pca2d)
        return
    if args.mlp:
        mlp_study(args.mlp)
        return
    if args.pairx:
        pair_exact_study(args.pairx)
        return
    if args.sweep:
        sweep(args.sweep)
        return
    if args.profile_case:
        profile_case(args.profile_case, args.size)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
