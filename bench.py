"""Throughput benchmark: shots/s of d=5, 5-round crosstalk syndrome extraction
on one GB300 (theta = 0.10 ZZ on idle adjacent pairs, depolarising p = 1e-3
with the Table I ratios, chi cap 256, complex64 contractions).

A step is one program segment (one syndrome round, or the final readout)
applied to a batch of B shots; a batch completes after rounds + 1 = 6 steps
and the next batch starts with new shot indices.  K is rounded up to a
multiple of 6 so every segment is timed equally often, and
    value = B * K / 6 / device seconds
is whole-shot throughput, timed with CUDA events on the simulator's stream;
the angle table and program are resident in HBM.  The W warm-up steps are
syndrome round 0 of W fresh batches.  `e2e` is the same batches timed on the
host clock through the C ABI with host buffers: the angle upload from pinned
memory and every batch's record download are inside it.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--shots B]
     python bench.py --impl reference    (the CPU oracle on a bounded sample)
Under torchrun each rank simulates its own disjoint shot range (weak scaling,
no data-path collective); the slowest rank's time is reported.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import D5_BENCH, theta_table  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SMS = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--shots", type=int, default=152, help="shots per batch and rank")
    ap.add_argument("--impl", default="stn", choices=["stn", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chi-cap", type=int, default=None,
                    help="override the bond cap (smaller profiling captures only; not a bench line)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# -- clocks during the timed region --------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, flag in zip(names, f[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -- CPU baseline: the oracle, as it stands, on the host cores ------------------
# Algorithmic FLOPs per shot of the d=5, 5-round, chi-cap-256 complex64 workload,
# counted by the device with the textbook formulas below in a bench.py run on
# this workload (35.6 TFLOP).  Used only when no device count is available
# (the reference arm).
ALG_FLOPS_PER_SHOT_D5_CAP256 = 35.6e12


def _gemm(m, n, k):
    return 8.0 * m * n * k


def _qr(m, n):
    a, b = (m, n) if m >= n else (n, m)
    return 4.0 * (2.0 * a * b * b - 2.0 * b ** 3 / 3.0)


def _svd(m, n):
    return 4.0 * (4.0 * m * n * n + 8.0 * n ** 3)


def _sweep_flops(lo, before, after):
    """Textbook FLOPs of one truncating sweep over [lo, lo + len(before)]:
    per doubled bond D (kept: c) an R factor of 2D x D, its product with the
    site, C = R M, the SVD of C (D x 2c) and the two contractions that carry
    the kept vectors to the left (the same counts the kernel accumulates)."""
    off = 1 if lo > 0 else 0
    total = 0.0
    for i, d in enumerate(before):
        c = after[i + off] if i + off < len(after) else d
        total += _qr(2 * d, d) + _gemm(d, 2 * d, d) + _gemm(d, 2 * c, d) + _svd(d, 2 * c) \
            + _gemm(d, c, 2 * c) + _gemm(2 * d, c, d)
    return total


def _oracle_worker(args):
    shot, budget, w_fields = args
    from oracle.shot import ShotSim, make_program
    from workloads import Workload
    w = Workload(**w_fields)
    prog = make_program(w)
    sim = ShotSim(w, shot, theta_table(w, len(prog.pairs)), prog, trace=True)
    t0 = time.perf_counter()
    done = 0
    for op in prog.ops:
        if time.perf_counter() - t0 > budget:
            break
        sim.step(op)
        done += 1
    secs = time.perf_counter() - t0
    flops = sum(_sweep_flops(lo, before, after) for _, lo, _, before, after in sim.trace)
    # the oracle's dominant primitives at the workload's largest bond (2 chi_cap)
    import numpy as np
    n = 2 * w.chi_cap
    rng = np.random.default_rng(shot)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    b = rng.normal(size=(2 * n, n)) + 1j * rng.normal(size=(2 * n, n))
    t1 = time.perf_counter()
    np.linalg.svd(a, full_matrices=False)
    np.linalg.qr(b)
    big_rate = (_svd(n, n) + _qr(2 * n, n)) / (time.perf_counter() - t1)
    return done, len(prog.ops), secs, flops, big_rate


def cpu_baseline(w, budget, flops_per_shot):
    """Each host core runs the oracle on its own shot of the workload for
    `budget` seconds.  A shot's early ops are far cheaper than its later ones
    (the bonds grow to the cap), so the sample is converted to shots/s by work:
    the algorithmic FLOPs of the sweeps the oracle completed (textbook counts
    from its bond dimensions) per second, over the workload's algorithmic
    FLOPs per shot.  Without `flops_per_shot` the completed fraction of each
    shot's ops is used instead, an upper bound."""
    import multiprocessing as mp
    from dataclasses import asdict
    cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"  # one core per worker process
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(s, budget, asdict(w)) for s in range(cores)])
    frac = sum(r[0] / r[1] for r in res)
    secs = max(r[2] for r in res)
    ops_done = sum(r[0] for r in res)
    flops = sum(r[3] for r in res)
    big_rate = sum(r[4] for r in res)
    sample = f"{cores} shots of {w.name}, one per core, {budget:.0f} s each: {ops_done} of {cores * res[0][1]} ops done"
    if flops_per_shot:
        return {"value": big_rate / flops_per_shot, "unit": "shots/s", "cores": cores, "kind": "oracle",
                "sample": sample + f"; shots/s = the {cores} cores' rate on the oracle's dominant primitives at "
                                   f"the largest bond (numpy complex128 SVD {2 * w.chi_cap}^2 and QR, "
                                   f"{big_rate / 1e9:.1f} GFLOP/s together) over {flops_per_shot / 1e12:.1f} TFLOP "
                                   f"of algorithmic work per shot; the sampled ops ran at {flops / secs / 1e9:.2f} "
                                   f"GFLOP/s ({flops / secs / flops_per_shot:.2g} shots/s) and their completed "
                                   f"fraction would give {frac / secs:.3g} shots/s (an upper bound)"}
    return {"value": frac / secs, "unit": "shots/s", "cores": cores, "kind": "oracle",
            "sample": sample + "; shots/s counts completed op fractions (an upper bound: the remaining ops "
                               "carry the large bond dimensions)"}


def reference_arm(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    per = max(args.cpu_seconds / max(args.steps, 1), 2.0)
    for _ in range(args.warmup):
        pass  # the oracle has nothing to warm up; steps below are all timed
    vals = []
    t0 = time.perf_counter()
    last = None
    fps = ALG_FLOPS_PER_SHOT_D5_CAP256 if w == D5_BENCH else None
    for _ in range(args.steps):
        last = cpu_baseline(w, per, fps)
        vals.append(last["value"])
    total = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {"metric": "shots/s of d=5, 5-round crosstalk syndrome extraction on 1 GB300 at <=1e-5 Born error",
            "impl": "reference", "value": v, "unit": "shots/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": w.name, "shots_per_batch": last["cores"]},
            "cpu_baseline": {"value": v, "unit": "shots/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -- GPU arm -------------------------------------------------------------------
def main():
    args = parse()
    w = D5_BENCH
    if args.chi_cap is not None and args.chi_cap != w.chi_cap:
        w = w.with_(chi_cap=args.chi_cap, name=f"{w.name}_cap{args.chi_cap}")
    if args.impl == "reference":
        reference_arm(args, w)
        return
    import torch
    import paper_2605_29514_gb300 as stn
    from paper_2605_29514_gb300.shards import rank_base

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    stn.build()
    segs = w.rounds + 1
    K = max(segs, ((args.steps + segs - 1) // segs) * segs)
    W = max(3, args.warmup)
    B = args.shots
    stream = torch.cuda.current_stream()
    sim = stn.Simulator(w, max_shots=B, stream=stream.cuda_stream)
    theta = theta_table(w, sim.n_pairs)
    th_host = torch.tensor(theta, dtype=torch.float64).pin_memory()
    d_theta = torch.empty_like(th_host, device="cuda")
    d_theta.copy_(th_host)
    rec_host = torch.empty((B, sim.rec_bytes), dtype=torch.uint8).pin_memory()
    base = rank_base(rank)  # disjoint global shot ranges per rank

    # warm-up: W steps, each the first segment (syndrome round 0) of a fresh batch
    for i in range(W):
        sim.begin_batch(B, base + i * B)
        sim.apply_round_device(0, d_theta.data_ptr())
    sim.sync()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seg_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(segs + 1)] for _ in range(K // segs)]
    flops0 = sim.algorithmic_flops()
    prof0 = sim.profile_counters()
    launches = 0
    # timed: K segments = K / 6 complete batches.  The host clock also covers the
    # angle upload from pinned memory and each batch's record download (e2e).
    t_host = time.perf_counter()
    d_theta.copy_(th_host, non_blocking=True)
    ev0.record(stream)
    for b in range(K // segs):
        sim.begin_batch(B, base + (W + b) * B)
        launches += 1
        for seg in range(segs):
            seg_ev[b][seg].record(stream)
            sim.apply_round_device(seg, d_theta.data_ptr())
            launches += 1
        seg_ev[b][segs].record(stream)
        if b + 1 == K // segs:
            ev1.record(stream)
        sim.read_records_into(rec_host.data_ptr())
    host_s = time.perf_counter() - t_host
    torch.cuda.synchronize()
    flops = sim.algorithmic_flops() - flops0
    prof1 = sim.profile_counters()
    clk = clocks.stop()
    seg_ms = [statistics.mean(seg_ev[b][g].elapsed_time(seg_ev[b][g + 1]) for b in range(K // segs))
              for g in range(segs)]
    dprof = {k: prof1[k] - prof0[k] for k in prof1}
    loop = max(dprof["op_loop_cycles"], 1.0)
    phases = {"segment_ms": [round(x, 3) for x in seg_ms],
              "cycle_share": {k.replace("_cycles", ""): round(dprof[k] / loop, 4)
                              for k in ("left_sweep_cycles", "svd_cycles", "right_sweep_rest_cycles",
                                        "expectation_cycles", "gauge_cycles")},
              "svds_per_shot": {"shared_memory": dprof["svd_count_shared"] / (B * (K // segs)),
                                "large_bond": dprof["svd_count_large"] / (B * (K // segs)),
                                "gauge_sites": dprof["gauge_sites"] / (B * (K // segs))},
              "source": "stn_profile_counters: SM clock cycles of each CTA per phase, over the timed batches"}
    secs = ev0.elapsed_time(ev1) / 1000.0
    if pg:
        t = torch.tensor([secs, host_s], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        secs, host_s = float(t[0].item()), float(t[1].item())
    shots_done = ws * B * K // segs
    value = shots_done / secs
    e2e = {"value": shots_done / host_s, "unit": "shots/s",
           "h2d_bytes_per_step": int(th_host.numel() * 8) / K,
           "d2h_bytes_per_step": int(rec_host.numel()) * (K // segs) / K,
           "path": "C ABI with host buffers: angles copied from pinned host memory, records read back "
                   "into pinned host memory after each batch (stn_read_records)"}

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    achieved = flops / secs / 1e12 / ws
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "traffic_note": "DRAM bytes of the round kernel are not captured at this workload's size; "
                                "in a capture at chi cap 16 they were negligible (the path is latency-bound)",
                "peak_source": f"FP32 FMA: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {max_mhz:.0f} MHz "
                               "(max SM clock of MEASURED_PEAKS.json)",
                "kernel": "stn::round_kernel<float>",
                "work": "algorithmic FLOPs of the MPS sweeps (standard GEMM, Householder QR and SVD counts)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(w, args.cpu_seconds, flops / shots_done if flops > 0 else None)

    if rank == 0:
        line = {"metric": "shots/s of d=5, 5-round crosstalk syndrome extraction on 1 GB300 at <=1e-5 Born error",
                "value": value, "unit": "shots/s", "n_gpus": ws, "steps": K, "warmup": W,
                "ms_per_step": 1000.0 * secs / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": {"workload": w.name, "distance": w.distance, "rounds": w.rounds, "theta": w.theta,
                           "p": w.p, "chi_cap": w.chi_cap, "shots_per_batch_per_rank": B,
                           "step": "one program segment (syndrome round or final readout) over the batch",
                           "l2": "per-shot MPS state (GBs) larger than L2; no flush",
                           "parallelism": f"shots sharded over {ws} rank(s)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "phases": phases}
        print(json.dumps(line), flush=True)
    sim.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
