#!/usr/bin/env python3
"""Benchmark: Bloch spectra per second of periodic (256,1,1) tubes on one GB300.

Workload (one step): a batch of B seeded variants of the tube_256 lattice (b = 2.8 bohr, two
Z = 1 nuclei per cell, m0 = 16 Gaussians of s and p type, n1 = 32768 x 256 x 256 grid, R = 32
sinc terms, K_sum = 256 images), each taken through the whole path in one batched pass:
basis samples -> potential factors -> weighted 1D Grams -> rank sum -> block DFT -> k-point
eigensolves.  One Bloch spectrum = all 256 x 16 = 4096 eigenvalues of one system.

value: systems/s with the system descriptors on the host and every intermediate on the device
       (device-timed with CUDA events on the launching stream; the per-step working set,
       ~13 MB per system, is far larger than L2).
e2e:   the same through lhf_bloch_spectra_host: descriptor upload and the copy of all
       eigenvalues back to host memory inside the timed region (wall clock, synchronised).
--impl reference: the CPU oracle as it stands (the plain FP64 C reference), on this host's
       cores, one system per core per step.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lhf_workloads as W  # noqa: E402

METRIC = "Bloch spectra/s at L=256, mixed vs FP64 GPU, at stated eigenvalue error (Ha)"
UNIT = "spectra/s"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------
# algorithmic work per system (roofline numerators)

def work_model(sizes: list[dict], sweeps: int, matrices: int) -> dict:
    """Algorithmic FLOPs / bytes per batch for the stages (roofline section)."""
    gram = 0.0
    dft_bytes = 0.0
    rank = 0.0
    eig = 0.0
    for s in sizes:
        m0, Rt = s["m0"], s["rank"]
        for l in range(3):
            gram += 2.0 * Rt * s["window"][l] * m0 * m0 * s["n_potential"][l]
        nwin = s["window"][0] * s["window"][1] * s["window"][2]
        rank += nwin * m0 * m0 * (4.0 * Rt + 12.0)
        dft_bytes += s["n_blocks"] * m0 * m0 * (2 * 8 + 2 * 16)
    if sizes:
        m = sizes[0]["m0"]
        eig = matrices * 9.33 * m ** 3 + sweeps * 20.0 * m * m * (m - 1 + (m & 1))
    return {"gram_flops": gram, "rank_flops": rank, "dft_bytes": dft_bytes, "eig_flops": eig}


def fp64_peak_tflops() -> float:
    # 152 SMs x 2 FP64 FMA / clk / SM x 2 FLOP x 2.07 GHz (nominal FP64 of the part: 1.25 TFLOP/s)
    return 152 * 2 * 2 * 2.07e9 / 1e12


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            pass
    return {}


# ----------------------------------------------------------------------------------------------
# CPU baseline / reference arm (the oracle as it stands)

def _oracle_one(seed: int, keep: bool = False):
    import oracle

    cfg = W.tube_256(seed)
    t0 = time.perf_counter()
    H, S = oracle.core_blocks(cfg)
    Hb, Sb = oracle.block_dft(H), oracle.block_dft(S)
    eig, st = oracle.k_point_eigenvalues(Hb, Sb)
    dt = time.perf_counter() - t0
    if keep:
        return dt, eig, st, (H, S, Hb, Sb)
    return dt, eig, st


def cpu_baseline(seed: int, procs: int = 1):
    """Time the oracle on `procs` systems in parallel (spawned workers, one system each)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    if procs <= 1:
        t0 = time.perf_counter()
        dt, eig, st, mats = _oracle_one(seed, keep=True)
        return {"wall": time.perf_counter() - t0, "systems": 1, "cores": 1, "eig": [eig], "status": [st],
                "mats": mats}
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_one, [seed + i for i in range(procs)])
    wall = time.perf_counter() - t0
    return {"wall": wall, "systems": procs, "cores": procs, "eig": [r[1] for r in res]}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = min(os.cpu_count() or 1, 16)
    for _ in range(args.warmup):
        cpu_baseline(3000, cores)
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        r = cpu_baseline(3000 + k * cores, cores)
        done += r["systems"]
    wall = time.perf_counter() - t0
    value = done / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded tube_256 variants)",
        "config": {"workload": "tube_256: periodic (256,1,1), m0=16, n=32768x256x256, R=32, K_sum=256",
                   "systems_per_step": cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{cores} systems per step, one per spawned process"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# GPU arm

def run_gpu(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("nccl")
    from paper_1408_3839_gb300 import lhf

    stream = torch.cuda.current_stream()
    ctx = lhf.Context(local, stream)
    precision = lhf.MIXED if args.precision == "mixed" else lhf.FP64
    B = args.batch
    cfgs = W.tube_256_batch(B, first_seed=3000 + rank * B)
    sizes = []
    for c in cfgs[:1]:
        ctx.setup(c)
        sizes.append(ctx.query_sizes())
    per_sys = sizes[0]["n_kpoints"] * sizes[0]["m0"]
    eig = torch.empty(B * per_sys, dtype=torch.float64, device="cuda")
    kst = torch.empty(B * sizes[0]["n_kpoints"], dtype=torch.int32, device="cuda")

    for _ in range(max(args.warmup, 0)):
        ctx.bloch_spectra(cfgs, eig, kst, precision)
    torch.cuda.synchronize()
    all_sizes = []
    for c in cfgs:
        ctx.setup(c)
        all_sizes.append(ctx.query_sizes())
    ctx.eig_counters()
    ctx.stage_times()
    ctx.set_profiling(True)

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        ctx.bloch_spectra(cfgs, eig, kst, precision)
    t_end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    ctx.set_profiling(False)
    stages = ctx.stage_times()
    sweeps, mats = ctx.eig_counters()
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    total_systems = B * args.steps * world
    value = total_systems / (ms / 1e3)
    bad_k = int((kst < 0).sum().item())

    # end to end through the host entry point
    host = np.empty(B * per_sys)
    hk = np.empty(B * sizes[0]["n_kpoints"], dtype=np.int32)
    ctx.bloch_spectra_host(cfgs, host, hk, precision)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.bloch_spectra_host(cfgs, host, hk, precision)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = total_systems / e2e_s

    # roofline of the dominant kernel (stage with the most device time)
    work = work_model(all_sizes, sweeps, mats)
    kernel_stages = ["basis", "potential", "gram", "ranksum", "dft", "eig"]
    dom = max(kernel_stages, key=lambda s: stages[s][0])
    dom_ms, dom_n = stages[dom]
    per_launch_s = dom_ms / 1e3 / max(dom_n, 1)
    peaks = measured_peaks()
    if dom == "dft":
        achieved = work["dft_bytes"] / per_launch_s / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    else:
        flops = {"gram": work["gram_flops"], "eig": work["eig_flops"] / max(args.steps, 1),
                 "ranksum": work["rank_flops"]}.get(dom, float("nan"))
        achieved = flops / per_launch_s / 1e12
        peak = fp64_peak_tflops()
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    stage_summary = {k: {"ms_per_step": v[0] / args.steps, "launches": v[1]} for k, v in stages.items()}
    gpu_launches = sum(stages[s][1] for s in kernel_stages)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "precision": args.precision, "data": "synthetic (seeded tube_256 variants)",
        "config": {"workload": "tube_256: periodic (256,1,1), b=2.8, M0=2, m0=16, n=32768x256x256, R=32, K_sum=256",
                   "systems_per_step_per_gpu": B, "l2": "working set per step >> L2 (no flush needed)",
                   "parallelism": f"replicas x{world} (independent systems per GPU)"},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": B * per_sys * 8 + hk.nbytes},
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "stages": stage_summary,
        "eig_sweeps_per_matrix": sweeps / max(mats, 1),
        "bad_kpoints": bad_k,
        "clocks": ck,
    }
    if rank == 0 and not args.no_cpu_baseline:
        from tests._numerics import check_eigenvalues

        cb = cpu_baseline(3000, 1)
        ref = cb["eig"][0]
        got = eig[:per_sys].cpu().numpy().reshape(ref.shape)
        H, S, Hb, Sb = cb["mats"]
        worst, ratio = check_eigenvalues(got, ref, Hb, Sb, H, S, status=cb["status"][0])
        fin = np.isfinite(ref) & np.isfinite(got)
        line["eig_error_vs_oracle"] = {
            "system": "tube_256 seed 3000", "max_abs_ha": worst, "ratio_to_tolerance": ratio,
            "removed_functions": int(cb["status"][0].clip(min=0).sum()),
            "median_abs_ha": float(np.median(np.abs(got[fin] - ref[fin]))),
            "k_status_match": bool(np.array_equal(kst[:ref.shape[0]].cpu().numpy(), cb["status"][0]))}
        line["cpu_baseline"] = {"value": cb["systems"] / cb["wall"], "unit": UNIT, "cores": cb["cores"],
                                "kind": "oracle", "sample": "1 tube_256 system (seed 3000), single process"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
