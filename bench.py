"""Benchmark of the hybrid fluid-kinetic step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One "step" is one pass of the whole step (every phase the workload enables)
over the workload's resident state.  Prints ONE JSON line (rank 0):
value = steps/s of the whole job (all ranks; independent replicas, weak
scaling), particle-pushes/s and cell-updates/s beside it, the roofline of the
dominant kernel (push + gather + deposit, HBM-bound) measured with CUDA events
captured in the step graph, the end-to-end rate through the C ABI with host
buffers, and the FP64 oracle timed on the host cores on a bounded sample.

--impl reference times the FP64 oracle (the only reference this method has:
the paper ships no code) on the same workload, rank 0 only.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hybrid steps/s & particle-pushes/s vs full-PIC on 1 GB300; % HBM roofline"
L2_BYTES = 129 * 2 ** 20
# algorithmic bytes of the push + gather + deposit kernel: per particle read
# x,y,z,ux,uy,uz,w (28 B) + write x,y,z,ux,uy,uz (24 B); per cell read E,B
# (24 B) + write J (12 B)
PUSH_BYTES_PER_PARTICLE = 52
PUSH_BYTES_PER_CELL = 36


def workloads():
    from paper_2510_11174_gb300 import inputs
    return {
        # plain full PIC: periodic 32^3, lambda/16, e-/p+ 0.1 n_c, 8 ppc, 1 keV, a0 = 1
        "periodic_plasma_32": lambda seed: inputs.periodic_plasma(n=32, ppc=8, seed=seed),
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench_%d.csv" % os.getpid())
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_sim(P, inp, stream=None):
    g = inp["grid"]
    sim = P.Simulation(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"],
                       laser=inp.get("laser"), stream=stream)
    for sp in inp["species"]:
        sim.load_species(**sp)
    if "E" in inp:
        sim.set_fields(inp["E"], inp["B"])
    return sim


def count_particles(inp):
    return sum(len(sp["x"]) for sp in inp["species"])


def run_ours(args, rank, world):
    import torch
    import paper_2510_11174_gb300 as P
    from paper_2510_11174_gb300 import build
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    # a capturable (non-default) stream shared by the library, the L2 flush and the events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    inp = workloads()[args.workload](1 + rank)
    g = inp["grid"]
    cells = g["nx"] * g["ny"] * g["nz"]
    npart = count_particles(inp)
    sim = make_sim(P, inp, stream.cuda_stream)
    sim.set_profiling(True)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    sim.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    push_ms, phases = [], []
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the event pair)
        ev0[k].record(stream)
        sim.step(1)
        ev1[k].record(stream)
        pt = sim.phase_times()  # synchronises
        phases.append(pt)
        push_ms.append(pt.get("push", 0.0))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = sum(step_ms)
    diag = sim.diagnostics()
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    steps_per_s = world * args.steps / (total_ms * 1e-3)
    mean_push_ms = statistics.mean(push_ms)
    peak, peak_kind = measured_peaks()
    push_bytes = PUSH_BYTES_PER_PARTICLE * npart + PUSH_BYTES_PER_CELL * cells
    achieved = push_bytes / (mean_push_ms * 1e-3) / 1e9
    phase_mean = {k: statistics.mean(p.get(k, 0.0) for p in phases) for k in phases[-1]}
    launches = diag["launches_per_step"] * args.steps
    sim.close()

    e2e = run_e2e(P, inp, args.steps, stream) if rank == 0 else None
    out = {
        "metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "grid": [g["nx"], g["ny"], g["nz"]], "particles": npart,
                   "species": len(inp["species"]), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between timed steps (256 MiB write outside the events)"},
        "particle_pushes_per_s": world * npart * args.steps / (total_ms * 1e-3),
        "cell_updates_per_s": world * cells * args.steps / (total_ms * 1e-3),
        "phase_ms": phase_mean,
        "roofline": {"kernel": "k_push_deposit", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "algorithmic_bytes_per_launch": push_bytes,
                     "mean_launch_ms": mean_push_ms},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    return out


def run_e2e(P, inp, steps, stream):
    """Whole job through the C ABI from pinned host buffers: create the context,
    upload particles and fields, then per step advance and read the FP64
    diagnostics back to the host."""
    import torch

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy(), t

    keep = []
    pin = {"grid": inp["grid"], "species": []}
    h2d = 0
    for sp in inp["species"]:
        d = {"q": sp["q"], "m": sp["m"]}
        for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
            arr, t = pinned(sp[k])
            keep.append(t)
            d[k] = arr
            h2d += arr.nbytes
        pin["species"].append(d)
    if "E" in inp:
        for k in ("E", "B"):
            arr, t = pinned(inp[k])
            keep.append(t)
            pin[k] = arr
            h2d += arr.nbytes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = make_sim(P, pin, stream.cuda_stream)
    d2h = 0
    for _ in range(steps):
        sim.step(1)
        sim.diagnostics()
        d2h += 8 * (3 + 2 * len(inp["species"]))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    sim.close()
    return {"value": steps / dt, "unit": "steps/s", "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps,
            "note": "context creation + host upload amortised over the steps; per-step FP64 diagnostics read"}


def run_oracle_sample(workload, budget_s=15.0, max_steps=None):
    """Time the FP64 oracle (as it stands) on the workload for about budget_s."""
    import oracle.sim as S
    inp = workloads()[workload](1)
    g = inp["grid"]
    o = S.OracleSim(g["nx"], g["ny"], g["nz"], g["dx"], cfl_frac=g["cfl_frac"], bc=g["bc"],
                    laser=inp.get("laser"))
    for sp in inp["species"]:
        o.load_species(**sp)
    if "E" in inp:
        o.set_fields(inp["E"], inp["B"])
    npart = count_particles(inp)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < budget_s and (max_steps is None or n < max_steps):
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d full steps of the %s workload (%d particles), single-threaded FP64 C" % (n, workload, npart),
            "particle_pushes_per_s": n * npart / dt}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import build as OB
    OB.build()
    for _ in range(args.warmup):
        pass
    samples = []
    per = max(5.0, 60.0 / max(1, args.steps))
    for _ in range(max(1, args.steps)):
        samples.append(run_oracle_sample(args.workload, budget_s=min(per, 20.0))["value"])
        if sum(1.0 / s for s in samples) > 150:
            break
    cb = run_oracle_sample(args.workload, budget_s=5.0)
    v = statistics.mean(samples)
    inp = workloads()[args.workload](1)
    g = inp["grid"]
    return {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
            "config": {"workload": args.workload, "grid": [g["nx"], g["ny"], g["nz"]],
                       "particles": count_particles(inp)},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="periodic_plasma_32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cb = run_oracle_sample(args.workload, budget_s=15.0)
            out["cpu_baseline"] = cb
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
