#!/usr/bin/env python3
"""Benchmark: Bloch spectra per second of periodic (256,1,1) tubes on one GB300.

Workload (one step): a batch of B seeded variants of the tube_256 lattice (b = 2.8 bohr, two
Z = 1 nuclei per cell, m0 = 16 Gaussians of s and p type, n1 = 32768 x 256 x 256 grid, R = 32
sinc terms, K_sum = 256 images), each taken through the whole path in one batched pass:
basis samples -> potential factors -> weighted 1D Grams -> rank sum -> block DFT -> k-point
eigensolves.  One Bloch spectrum = all 256 x 16 = 4096 eigenvalues of one system.

value: systems/s with the system descriptors on the host and every intermediate on the device
       (device-timed with CUDA events on the launching stream; the per-step working set,
       ~13 MB per system, is far larger than L2), for --precision (default mixed: the Gram
       contractions on tensor cores through exact BF16 digit slices); the other route (FP64
       CUDA-core Grams) is timed beside it and reported with the ratio of the two.
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

def work_model(sizes: list[dict], passes: int, matrices: int) -> dict:
    """Algorithmic FLOPs / bytes per batch for the stages (the roofline numerators).

    gram: 2 R_tot J m0^2 n_v per direction (the weighted-Gram contraction, counted over the whole
    window although the mirrored half is copied); gram_tc: the same contraction as 28 exact BF16
    digit-pair products (7 digits per operand, pairs a + b <= 6); rank: (4 R_tot + 12) per window
    entry; dft: read 2 real blocks, write 2 complex blocks; eig: per solved matrix 9.33 m^3
    (Cholesky and two triangular solves, complex) + 8 m^3 (Householder reduction to tridiagonal
    form: per column a complex matrix-vector product and a rank-2 update of the trailing block),
    plus 8 m flops per FP64 characteristic-polynomial pass of the tridiagonal stage (the
    minors and their derivatives; its FP32 bisection is not counted)."""
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
        eig = matrices * 17.33 * m ** 3 + passes * 8.0 * m
    return {"gram_flops": gram, "gram_tc_flops": 28.0 * gram, "rank_flops": rank, "dft_bytes": dft_bytes,
            "eig_flops": eig}


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

def replica_seeds(rank: int, batch: int, first: int = 3000) -> list[int]:
    """Seeds of the tube_256 variants that replica `rank` solves per step (disjoint per rank)."""
    return list(range(first + rank * batch, first + (rank + 1) * batch))


def max_over_ranks(x: float, dist, device) -> float:
    """Maximum of a per-rank scalar over the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(ctx, cfgs, eig, kst, precision, steps, stream, dist, clocks=None):
    """Device time (ms, max over ranks) of `steps` batched passes, with live stage times."""
    import torch

    ctx.eig_counters()
    ctx.stage_times()
    ctx.set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(steps):
        ctx.bloch_spectra(cfgs, eig, kst, precision)
    t_end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    ms = t_start.elapsed_time(t_end)
    ctx.set_profiling(False)
    stages = ctx.stage_times()
    passes, mats = ctx.eig_counters()
    return max_over_ranks(ms, dist, "cuda"), stages, passes, mats, ck


def _device_time_ms(fn, steps, stream):
    import torch

    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def run_extras(ctx, lhf, stream, steps: int, warmup: int) -> dict:
    """The other workloads of the path, each timed on the device (not part of the headline):
    the heterogeneous batch of 64 tubes and slabs as one captured CUDA graph (mixed route), the
    open (64,1,1) box (dense matrices and dense eigensolve, FP64) and the periodic (32,32,32)
    cube (three-level block DFT, 16 385 k-point solves; mixed route)."""
    import torch

    out = {}
    # heterogeneous batch through a graph
    try:
        cfgs = W.hetero_batch()
        ne = nk = 0
        for c in cfgs:
            ctx.setup(c)
            sz = ctx.query_sizes()
            ne += sz["n_kpoints"] * sz["m0"]
            nk += sz["n_kpoints"]
        eig = torch.empty(ne, dtype=torch.float64, device="cuda")
        ks = torch.empty(nk, dtype=torch.int32, device="cuda")
        g = ctx.graph_create(cfgs, eig, ks, lhf.MIXED)
        for _ in range(warmup):
            g.launch()
        ms_graph = _device_time_ms(g.launch, steps, stream)
        for _ in range(warmup):
            ctx.bloch_spectra(cfgs, eig, ks, lhf.MIXED)
        ms_direct = _device_time_ms(lambda: ctx.bloch_spectra(cfgs, eig, ks, lhf.MIXED), steps, stream)
        g.close()
        out["hetero_64"] = {
            "workload": "64 seeded tubes (L in [16, 512]) and slabs (L x L, L in [4, 32]), m0 in {4, 8, 16}, "
                        "h in {0.05, 0.0625, 0.08}, R in {24, 32}, b = 2.0; mixed route",
            "graph": {"value": len(cfgs) * steps / (ms_graph / 1e3), "unit": UNIT, "ms_per_step": ms_graph / steps},
            "direct": {"value": len(cfgs) * steps / (ms_direct / 1e3), "unit": UNIT, "ms_per_step": ms_direct / steps},
            "eigenvalues_per_step": ne, "bad_kpoints": int((ks < 0).sum().item())}
    except Exception as e:  # reported, not hidden
        out["hetero_64"] = {"error": str(e)}
    # open box (64,1,1)
    try:
        box = W.box_64()
        ctx.setup(box)
        N = ctx.query_sizes()["n_basis"]
        eig = torch.empty(N, dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            ctx.bloch_spectra([box], eig)
        ctx.stage_times()
        ctx.set_profiling(True)
        ms = _device_time_ms(lambda: ctx.bloch_spectra([box], eig), steps, stream)
        ctx.set_profiling(False)
        st = ctx.stage_times()
        out["box_64"] = {
            "workload": "open (64,1,1) box, N_b = 512, n1 = 3712, n2 = n3 = 320, R = 32, FP64",
            "value": steps / (ms / 1e3), "unit": "spectra/s", "ms_per_step": ms / steps,
            "stages_ms": {k: v[0] / steps for k, v in st.items() if v[1]}}
    except Exception as e:
        out["box_64"] = {"error": str(e)}
    # periodic cube (32,32,32)
    try:
        cube = W.cubic_32()
        ctx.setup(cube)
        sz = ctx.query_sizes()
        eig = torch.empty(sz["n_kpoints"] * sz["m0"], dtype=torch.float64, device="cuda")
        ks = torch.empty(sz["n_kpoints"], dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            ctx.bloch_spectra([cube], eig, ks, lhf.MIXED)
        ctx.stage_times()
        ctx.set_profiling(True)
        ms = _device_time_ms(lambda: ctx.bloch_spectra([cube], eig, ks, lhf.MIXED), steps, stream)
        ctx.set_profiling(False)
        st = ctx.stage_times()
        out["cubic_32"] = {
            "workload": "periodic (32,32,32), b = 2.0, m0 = 16, n_cell = 64 per direction, R = 32, mixed route",
            "value": steps / (ms / 1e3), "unit": "spectra/s", "ms_per_step": ms / steps,
            "kpoints": sz["n_kpoints"], "removed_slots": int(ks.clamp(min=0).sum().item()),
            "stages_ms": {k: v[0] / steps for k, v in st.items() if v[1]}}
    except Exception as e:
        out["cubic_32"] = {"error": str(e)}
    return out


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
    cfgs = [W.tube_256(seed) for seed in replica_seeds(rank, B)]
    ctx.setup(cfgs[0])
    sizes = [ctx.query_sizes()]
    per_sys = sizes[0]["n_kpoints"] * sizes[0]["m0"]
    eig = torch.empty(B * per_sys, dtype=torch.float64, device="cuda")
    kst = torch.empty(B * sizes[0]["n_kpoints"], dtype=torch.int32, device="cuda")
    all_sizes = []
    for c in cfgs:
        ctx.setup(c)
        all_sizes.append(ctx.query_sizes())

    # FP64 route beside the mixed one (the metric compares the two); the main line is
    # args.precision, timed last
    other = lhf.FP64 if precision == lhf.MIXED else lhf.MIXED
    for prec in (other, precision):
        for _ in range(max(args.warmup, 0)):
            ctx.bloch_spectra(cfgs, eig, kst, prec)
    torch.cuda.synchronize()
    ms_other, stages_other, _, _, _ = timed_steps(ctx, cfgs, eig, kst, other, args.steps, stream, dist)
    clocks = ClockSampler(local)
    ms, stages, passes, mats, ck = timed_steps(ctx, cfgs, eig, kst, precision, args.steps, stream, dist, clocks)
    total_systems = B * args.steps * world
    value = total_systems / (ms / 1e3)
    value_other = total_systems / (ms_other / 1e3)
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
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = total_systems / e2e_s

    # rooflines per stage and of the dominant one (the stage with the most device time)
    work = work_model(all_sizes, passes, mats)
    kernel_stages = ["basis", "potential", "gram", "gram_tc", "ranksum", "dft", "eig"]
    peaks = measured_peaks()
    rooflines = {}
    for st_name in kernel_stages:
        st_ms, st_n = stages[st_name]
        if st_n == 0 or st_ms <= 0:
            continue
        per_launch_s = st_ms / 1e3 / st_n
        if st_name == "dft":
            achieved = work["dft_bytes"] / per_launch_s / 1e9
            peak = float(peaks.get("hbm_gbs", 6800.0))
            rooflines[st_name] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak,
                                  "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
        elif st_name == "gram_tc":
            achieved = work["gram_tc_flops"] / per_launch_s / 1e12
            peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
            rooflines[st_name] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                  "frac": achieved / peak,
                                  "peak_source": "measured bf16 sustained" if "bf16_tflops_sustained" in peaks
                                  else "fallback"}
        elif st_name in ("gram", "ranksum", "eig") and not (st_name == "gram" and args.precision == "mixed"):
            flops = {"gram": work["gram_flops"], "ranksum": work["rank_flops"],
                     "eig": work["eig_flops"] / max(args.steps, 1)}[st_name]
            achieved = flops / per_launch_s / 1e12
            peak = fp64_peak_tflops()
            rooflines[st_name] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                  "frac": achieved / peak, "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    dom = max(kernel_stages, key=lambda s: stages[s][0])
    roof = dict(rooflines.get(dom, {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None}))
    roof["traffic"] = None
    roof["kernel"] = dom
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
                "h2d_bytes_per_step": B * sizes[0]["desc_bytes"], "d2h_bytes_per_step": B * per_sys * 8 + hk.nbytes},
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "stage_rooflines": rooflines,
        ("fp64" if other == lhf.FP64 else "mixed"): {
            "value": value_other, "unit": UNIT, "ms_per_step": ms_other / args.steps,
            "stages": {k: {"ms_per_step": v[0] / args.steps, "launches": v[1]} for k, v in stages_other.items()}},
        "mixed_over_fp64": (value / value_other) if precision == lhf.MIXED else (value_other / value),
        "stages": stage_summary,
        "eig_tridiag_passes_per_matrix": passes / max(mats, 1),
        "bad_kpoints": bad_k,
        "clocks": ck,
    }
    if rank == 0 and not args.no_extras:
        line["extra"] = run_extras(ctx, lhf, stream, max(args.steps // 2, 2), 2)
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
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads (box, cube, batch)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
